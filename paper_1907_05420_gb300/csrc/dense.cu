// (c) Dense LDL^T of the Schur complement, S = L_s D_s L_s^T, and the solve
// S x_g = t (Algorithm 1; eqs. SCform and SCsolve).
//
// S is n x n, column-major, lower triangle.  Blocked right-looking, block
// width kDenseNB = 64, per block column k0:
//   diagonal block: LDL^T of the 64 x 64 block with rows in registers, and
//   panel: L21 = A21 L11^{-T} D1^{-1}, Y = L21 D1 kept for the update
//     (k_dense_diag_t / k_dense_panel_t in dense_kernels.cuh, shared with the
//     tensor-core modes and the dense tail of the block factors);
//   k_dense_update: A22 -= Y L21^T on the lower-triangle 64 x 64 tiles (FP64).
// No pivoting: S is positive definite when the blocks are quasidefinite and C
// is positive definite; a zero pivot is counted and reported.
#include "dense_kernels.cuh"

namespace kkt {

namespace {

constexpr int NB = kDenseNB;

// forward substitution with unit lower L: diagonal block of one block column
__global__ void k_dense_fwd_diag(const double* __restrict__ S, double* __restrict__ x, int n, int k0) {
  const int kb = min(NB, n - k0);
  if (threadIdx.x != 0) return;
  for (int c = 0; c < kb; c++) {
    double v = x[k0 + c];
    for (int c2 = 0; c2 < c; c2++) v -= S[(k0 + c) + (int64_t)(k0 + c2) * n] * x[k0 + c2];
    x[k0 + c] = v;
  }
}

// x[i] -= sum_{c in block} L[i][c] x[c] for rows below the block
__global__ void k_dense_fwd_update(const double* __restrict__ S, double* __restrict__ x, int n, int k0) {
  const int kb = min(NB, n - k0);
  const int i = k0 + kb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int c = 0; c < kb; c++) acc += S[i + (int64_t)(k0 + c) * n] * x[k0 + c];
  x[i] -= acc;
}

__global__ void k_dense_diag_scale(const double* __restrict__ S, double* __restrict__ x, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x[i] /= S[i + (int64_t)i * n];
}

// dot[c] = sum_{i >= k0+kb} L[i][k0+c] x[i]
__global__ void k_dense_bwd_dot(const double* __restrict__ S, const double* __restrict__ x,
                                double* __restrict__ dot, int n, int k0) {
  const int kb = min(NB, n - k0);
  const int c = blockIdx.x;
  if (c >= kb) return;
  __shared__ double red[256];
  double acc = 0.0;
  const double* col = S + (int64_t)(k0 + c) * n;
  for (int i = k0 + kb + threadIdx.x; i < n; i += blockDim.x) acc += col[i] * x[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) dot[c] = red[0];
}

__global__ void k_dense_bwd_diag(const double* __restrict__ S, double* __restrict__ x,
                                 const double* __restrict__ dot, int n, int k0) {
  const int kb = min(NB, n - k0);
  if (threadIdx.x != 0) return;
  for (int c = kb - 1; c >= 0; c--) {
    double v = x[k0 + c] - dot[c];
    for (int c2 = c + 1; c2 < kb; c2++) v -= S[(k0 + c2) + (int64_t)(k0 + c) * n] * x[k0 + c2];
    x[k0 + c] = v;
  }
}

// ---- pipelined triangular solves with the dense factor ----
//
// One launch per direction.  CTAs take 64-row blocks in the order of an atomic
// ticket, so a CTA only ever waits for blocks owned by CTAs that started
// before it.  A finished block publishes its solution, then its flag
// (threadfence + volatile store); waiting CTAs poll the flag with a bounded
// budget and record a timeout instead of spinning forever.

constexpr long long kSpinBudgetCycles = 4000000000LL;  // about 2 s at 2 GHz

__device__ __forceinline__ bool wait_flag(const int* flag, int epoch, int* err) {
  const long long t0 = clock64();
  while (*((volatile const int*)flag) < epoch) {
    __nanosleep(32);
    if (clock64() - t0 > kSpinBudgetCycles) {
      atomicExch(err, 1);
      return false;
    }
  }
  __threadfence();
  return true;
}

// Inverses X_t = L_tt^{-1} of the unit lower 64 x 64 diagonal blocks of a
// factor (row-major per block, zero above the diagonal and outside the
// matrix) and the reciprocal pivots 1 / D.  With them each step of the block
// triangular solves applies its diagonal block as a product instead of a
// 64-step substitution.  Row i of X is e_i - sum_{k<i} L_ik X_k (right-looking
// over k, one barrier per k).
// Batched over blockIdx.y (matrix b at L0 + b * bstride with leading dimension
// ld, its inverses at X0 + b * xstride); dinv may be null.
template <class T>
__global__ void __launch_bounds__(256) k_diag_inverse(const T* __restrict__ L0, int n, int ld, int64_t bstride,
                                                      double* __restrict__ X0, int64_t xstride,
                                                      double* __restrict__ dinv) {
  extern __shared__ double dsm[];
  double(*Ls)[65] = reinterpret_cast<double(*)[65]>(dsm);
  double(*Xs)[65] = reinterpret_cast<double(*)[65]>(dsm + 64 * 65);
  const T* L = L0 + (int64_t)blockIdx.y * bstride;
  double* X = X0 + (int64_t)blockIdx.y * xstride;
  const int t = blockIdx.x, r0 = t * 64, rows = min(64, n - r0), tid = threadIdx.x;
  for (int q = tid; q < 64 * 64; q += blockDim.x) {
    const int c = q / 64, i = q - c * 64;
    Ls[i][c] = (i > c && i < rows) ? (double)L[(int64_t)(r0 + i) + (int64_t)(r0 + c) * ld] : 0.0;
    Xs[i][c] = (i == c && i < rows) ? 1.0 : 0.0;
  }
  if (dinv && tid < rows) dinv[r0 + tid] = 1.0 / (double)L[(int64_t)(r0 + tid) * (ld + 1)];
  __syncthreads();
  for (int k = 0; k + 1 < rows; k++) {
    const int cnt = (rows - 1 - k) * (k + 1);
    for (int q = tid; q < cnt; q += blockDim.x) {
      const int i = k + 1 + q / (k + 1), j = q % (k + 1);
      Xs[i][j] -= Ls[i][k] * Xs[k][j];
    }
    __syncthreads();
  }
  for (int q = tid; q < 64 * 64; q += blockDim.x) X[(int64_t)t * 4096 + q] = Xs[q / 64][q % 64];
}

// L y = b in place (unit lower L, column-major n x n, leading dimension n).
// One CTA per 64-row block, taken in ticket order; block t adds the products
// of the finished blocks j < t (each awaited on its flag), then applies X_t.
// For an FP32 factor (the TF32 and BF16 modes) the products of each 64 x 64
// block are formed in FP32 (x_j rounded to FP32, 16 FMAs per thread) and added
// to the FP64 row sums once per block: the FP32 factor's own error is some
// 1e-4 relative, far above the 1e-7 of these products, and the conversions
// and FMAs stay off this GPU's narrow FP64 pipe.  The FP64 factor keeps FP64
// products.
template <class T>
__global__ void __launch_bounds__(256) k_trsv_lower(const T* __restrict__ L, int n, double* x,
                                                    int* flags, unsigned* ticket, int epoch, int* err,
                                                    const int* __restrict__ jlo, const double* __restrict__ X) {
  __shared__ int s_blk, s_ok;
  __shared__ double yj[64];
  __shared__ T yjt[64];  // x_j in the factor's type, for the products
  __shared__ double part[4][64];
  __shared__ double Xs[64][65];
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_blk = (int)atomicAdd(ticket, 1u);
    s_ok = 1;
  }
  __syncthreads();
  const int t = s_blk, r0 = t * 64, rows = min(64, n - r0);
  const int r = tid & 63, pid = tid >> 6;
  for (int q = tid; q < 64 * 64; q += 256) Xs[q / 64][q % 64] = X[(int64_t)t * 4096 + q];
  double acc = 0.0;
  for (int j = jlo ? jlo[t] : 0; j < t; j++) {  // blocks left of the row envelope are zero
    if (tid == 0 && !wait_flag(flags + j, epoch, err)) s_ok = 0;
    __syncthreads();
    if (!s_ok) break;
    if (tid < 64) yjt[tid] = (T)__ldcg(x + j * 64 + tid);
    __syncthreads();
    if (r < rows) {
      const T* col = L + (int64_t)(r0 + r) + (int64_t)(j * 64 + pid * 16) * n;
      if constexpr (sizeof(T) == 8) {
#pragma unroll 4
        for (int c = 0; c < 16; c++) acc += col[(int64_t)c * n] * yjt[pid * 16 + c];
      } else {
        T a = T(0);
#pragma unroll 4
        for (int c = 0; c < 16; c++) a += col[(int64_t)c * n] * yjt[pid * 16 + c];
        acc += (double)a;
      }
    }
    __syncthreads();
  }
  part[pid][r] = acc;
  __syncthreads();
  if (tid < 64) yj[tid] = tid < rows ? __ldcg(x + r0 + tid) - (part[0][tid] + part[1][tid] + part[2][tid] + part[3][tid]) : 0.0;
  __syncthreads();
  double y = 0.0;
#pragma unroll
  for (int c = 0; c < 16; c++) y += Xs[r][pid * 16 + c] * yj[pid * 16 + c];
  part[pid][r] = y;
  __syncthreads();
  if (tid < rows) {
    x[r0 + tid] = part[0][tid] + part[1][tid] + part[2][tid] + part[3][tid];
    __threadfence();  // publish this block's solution before its flag
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    *((volatile int*)(flags + t)) = epoch;
  }
}

// L^T x = D^{-1} y in place (blocks from the bottom up; the pivots' scaling
// is applied to the block's own right-hand side), then X_t^T.
template <class T>
__global__ void __launch_bounds__(256) k_trsv_upper(const T* __restrict__ L, int n, double* x,
                                                    int* flags, unsigned* ticket, int epoch, int* err,
                                                    const int* __restrict__ jhi, const double* __restrict__ X,
                                                    const double* __restrict__ dinv) {
  __shared__ int s_blk, s_ok;
  __shared__ double xj[64];
  __shared__ T xjt[64];  // x_j in the factor's type, for the products
  __shared__ double accs[64];
  __shared__ double part[4][64];
  __shared__ double Xs[64][65];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (n + 63) / 64;
  if (tid == 0) {
    s_blk = nb - 1 - (int)atomicAdd(ticket, 1u);
    s_ok = 1;
  }
  if (tid < 64) accs[tid] = 0.0;
  __syncthreads();
  const int b = s_blk, r0 = b * 64, rows = min(64, n - r0);
  for (int q = tid; q < 64 * 64; q += 256) Xs[q / 64][q % 64] = X[(int64_t)b * 4096 + q];
  for (int j = (jhi ? jhi[b] : nb) - 1; j > b; j--) {  // blocks below the envelope are zero
    if (tid == 0 && !wait_flag(flags + j, epoch, err)) s_ok = 0;
    __syncthreads();
    if (!s_ok) break;
    const int c0 = j * 64, cols = min(64, n - c0);
    if (tid < 64) xjt[tid] = tid < cols ? (T)__ldcg(x + c0 + tid) : T(0);
    __syncthreads();
    // warp w handles rows 8w..8w+7 of this block; lanes run along the column
    for (int rr = warp * 8; rr < warp * 8 + 8; rr++) {
      if (rr >= rows) break;
      const T* col = L + (int64_t)(r0 + rr) * n + c0;
      T v = T(0);
      if (lane < cols) v += col[lane] * xjt[lane];
      if (lane + 32 < cols) v += col[lane + 32] * xjt[lane + 32];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) accs[rr] += (double)v;
    }
    __syncthreads();
  }
  if (tid < 64) xj[tid] = tid < rows ? __ldcg(x + r0 + tid) * dinv[r0 + tid] - accs[tid] : 0.0;
  __syncthreads();
  const int c = tid & 63, pid = tid >> 6;
  double v = 0.0;
#pragma unroll
  for (int q = 0; q < 16; q++) v += Xs[pid * 16 + q][c] * xj[pid * 16 + q];
  part[pid][c] = v;
  __syncthreads();
  if (tid < rows) {
    x[r0 + tid] = part[0][tid] + part[1][tid] + part[2][tid] + part[3][tid];
    __threadfence();  // publish this block's solution before its flag
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    *((volatile int*)(flags + b)) = epoch;
  }
}

}  // namespace

// The epochs the two triangular solves of one application wait for (a block's
// flag holds the epoch of the last solve that finished it; a wait ends once it
// is at least the solve's own).  Launched directly, each solve takes new,
// growing ones, starting above kGraphEpoch; inside the solve graph, whose
// launches replay their captured arguments, the flags are cleared first and
// the fixed kGraphEpoch is used, which leaves flags below every later direct
// epoch.
constexpr int kGraphEpoch = 1;

static cudaError_t trsv_epochs(Handle& h, int nb, int& ep_f, int& ep_b, cudaStream_t st) {
  if (h.solve_capturing) {
    ep_f = ep_b = kGraphEpoch;
    return cudaMemsetAsync(h.trsv_flags, 0, sizeof(int) * 2 * (size_t)nb, st);
  }
  ep_f = ++h.trsv_epoch;
  ep_b = ++h.trsv_epoch;
  return cudaSuccess;
}

cudaError_t launch_dense_ldlt(Handle& h, unsigned long long* counters, cudaStream_t st) {
  const int n = h.nC;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = std::min(NB, n - k0);
    const int rend = h.panel_rend.empty() ? n : h.panel_rend[k0 / NB];
    // diagonal block (rows in registers) and panel (warp per row), FP64
    cudaError_t e = launch_dense_diag_panel_f64(h, k0, kb, rend, counters, st);
    if (e != cudaSuccess) return e;
    const int rest = rend - k0 - kb;
    if (rest > 0) {
      const int T = (rest + 63) / 64;
      const int kt = kt_begin(h, kFamDenseF64, update_flops(rest, 0, rest, kb), st);
      k_dense_update<<<T * (T + 1) / 2, 256, 0, st>>>(h.S, h.Ypanel, n, k0, kb, rend, 0, 0);
      kt_end(h, kt, st);
      h.launches++;
    }
  }
  cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : launch_diag_inverse(h, false, st);
}

cudaError_t launch_dense_solve(Handle& h, const double* t, double* x, cudaStream_t st) {
  const int n = h.nC;
  if (n == 0) return cudaSuccess;
  const int nb = (n + NB - 1) / NB;
  cudaError_t e = cudaMemcpyAsync(x, t, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h.trsv_ticket, 0, sizeof(unsigned) * 2, st);
  if (e != cudaSuccess) return e;
  // flags hold the epoch of the last solve that finished each block; two per solve
  int ep_f, ep_b;
  e = trsv_epochs(h, nb, ep_f, ep_b, st);
  if (e != cudaSuccess) return e;
  k_trsv_lower<double><<<nb, 256, 0, st>>>(h.S, n, x, h.trsv_flags, h.trsv_ticket, ep_f, h.dev_err,
                                           h.d.trsv_jlo, h.Xinv);
  k_trsv_upper<double><<<nb, 256, 0, st>>>(h.S, n, x, h.trsv_flags + nb, h.trsv_ticket + 1, ep_b,
                                           h.dev_err, h.d.trsv_jhi, h.Xinv, h.Sdinv);
  h.launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_dense_solve_ws(Handle& h, const double* t, double* x, double* dot,
                                  cudaStream_t st) {
  const int n = h.nC;
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(x, t, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = std::min(NB, n - k0);
    k_dense_fwd_diag<<<1, 32, 0, st>>>(h.S, x, n, k0);
    h.launches++;
    const int rest = n - k0 - kb;
    if (rest > 0) {
      k_dense_fwd_update<<<(rest + 255) / 256, 256, 0, st>>>(h.S, x, n, k0);
      h.launches++;
    }
  }
  k_dense_diag_scale<<<(n + 255) / 256, 256, 0, st>>>(h.S, x, n);
  h.launches++;
  const int last = ((n - 1) / NB) * NB;
  for (int k0 = last; k0 >= 0; k0 -= NB) {
    k_dense_bwd_dot<<<NB, 256, 0, st>>>(h.S, x, dot, n, k0);
    k_dense_bwd_diag<<<1, 32, 0, st>>>(h.S, x, dot, n, k0);
    h.launches += 2;
  }
  return cudaGetLastError();
}

// The diagonal-block inverses and reciprocal pivots of the current factor of S
// (FP64 in S, or FP32 in S32), for the block triangular solves.
constexpr int kInvSmem = 2 * 64 * 65 * (int)sizeof(double);

// Kernel attributes set once (before any launch, outside stream capture).
cudaError_t dense_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_diag_inverse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kInvSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_diag_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kInvSmem);
  return e;
}

cudaError_t launch_diag_inverse(Handle& h, bool f32, cudaStream_t st) {
  const int n = h.nC;
  if (n == 0) return cudaSuccess;
  const int nb = (n + NB - 1) / NB;
  const int smem = kInvSmem;
  if (f32) k_diag_inverse<float><<<nb, 256, smem, st>>>(h.S32, n, n, 0, h.Xinv, 0, h.Sdinv);
  else k_diag_inverse<double><<<nb, 256, smem, st>>>(h.S, n, n, 0, h.Xinv, 0, h.Sdinv);
  h.launches++;
  return cudaGetLastError();
}

// The diagonal-block inverses of the N dense tails (order nT, leading
// dimension nTa), for the tail's block triangular solves.
cudaError_t launch_tail_inverse(Handle& h, cudaStream_t st) {
  const int nbT = (h.nT + NB - 1) / NB;
  const int smem = kInvSmem;
  k_diag_inverse<double><<<dim3(nbT, h.N), 256, smem, st>>>(h.Tt, h.nT, h.nTa, (int64_t)h.nTa * h.nTa, h.Xtail,
                                                           (int64_t)nbT * 4096, nullptr);
  h.launches++;
  return cudaGetLastError();
}

// x = S32^{-1} t with the FP32 factor of the TF32/BF16 modes (FP64 accumulation)
cudaError_t launch_dense_solve_f32(Handle& h, const double* t, double* x, cudaStream_t st) {
  const int n = h.nC;
  if (n == 0) return cudaSuccess;
  const int nb = (n + NB - 1) / NB;
  cudaError_t e = cudaMemcpyAsync(x, t, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h.trsv_ticket, 0, sizeof(unsigned) * 2, st);
  if (e != cudaSuccess) return e;
  int ep_f, ep_b;
  e = trsv_epochs(h, nb, ep_f, ep_b, st);
  if (e != cudaSuccess) return e;
  k_trsv_lower<float><<<nb, 256, 0, st>>>(h.S32, n, x, h.trsv_flags, h.trsv_ticket, ep_f, h.dev_err,
                                          h.d.trsv_jlo, h.Xinv);
  k_trsv_upper<float><<<nb, 256, 0, st>>>(h.S32, n, x, h.trsv_flags + nb, h.trsv_ticket + 1, ep_b,
                                          h.dev_err, h.d.trsv_jhi, h.Xinv, h.Sdinv);
  h.launches += 2;
  return cudaGetLastError();
}

}  // namespace kkt
