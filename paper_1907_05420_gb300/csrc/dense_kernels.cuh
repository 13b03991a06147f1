// Building blocks of the blocked right-looking dense LDL^T (panel width
// kDenseNB = 64), shared by the factor of the Schur complement S (one matrix)
// and by the dense tail of the block factors (one matrix per block, batched
// over blockIdx with a stride).  Matrices are column-major with leading
// dimension n; only the lower triangle is read or written.  A panel k0 has
// kb pivot columns (kb < 64 for a last ragged panel; the rows below the
// pivots may extend past the last pivot column: the tail's augmented rows).
// Per panel:
//   k_dense_diag_t:   LDL^T of the kb x kb diagonal block;
//   k_dense_panel_t:  L21 = A21 L11^{-T} D1^{-1} and Y = L21 D1 (rows below);
//   k_dense_update:   A22 -= Y L21^T on the lower 64 x 64 tiles (FP64).
// A division by a pivot is a multiplication by its reciprocal.
// Included by the translation units that launch them (internal linkage).
#pragma once
#include "handle.h"
#include "pivot.cuh"

namespace kkt {

namespace {

constexpr int kPanelW = kDenseNB;

// Static-pivot rule of the block factors: a pivot with |d| < pivot_eps *
// max|A_b| is replaced by +-pivot_eps * max|A_b|, with the sign the inertia of
// a quasidefinite block gives its column (+ primal, - multiplier).  A null
// anorm turns the rule off (the factor of S).
struct PivotRule {
  const double* anorm = nullptr;   // per matrix of the batch
  double pivot_eps = 0.0;
  const int32_t* primal = nullptr; // per column of the matrix: 1 if primal
};

// Pairs (i, j) with 1 <= j <= i < 64 ordered by j descending, then i: the
// pairs with j >= r0 are the first (64 - r0)(65 - r0) / 2 entries, so a
// trailing triangle of the diagonal block spreads evenly over the threads.
constexpr int kDiagPairs = (kPanelW - 1) * kPanelW / 2;

__device__ __forceinline__ void diag_pair(int p, int& i, int& j) {
  // group t = 64 - j holds pairs [t(t-1)/2, t(t+1)/2)
  int t = (int)((sqrtf(8.0f * p + 1.0f) + 1.0f) * 0.5f);
  while (t * (t - 1) / 2 > p) t--;
  while (t * (t + 1) / 2 <= p) t++;
  j = kPanelW - t;
  i = j + (p - t * (t - 1) / 2);
}

// LDL^T of the diagonal block at (k0, k0) of matrix blockIdx.x, in shared
// memory, in sub-panels of kSub = 16 columns:
//   (1) the 16 x 16 diagonal sub-block, one thread per entry, a barrier pair
//       per column (thread 0 applies the pivot rule and forms 1/d; the
//       trailing entries take -l_i u_j; the column is scaled one step late,
//       after its unscaled values have been used);
//   (2) the rows below it in the block solve y L11^T = a, one thread per row
//       (Y = y kept unscaled, L = y D^{-1});
//   (3) the trailing triangle of the block takes A[i][j] -= sum_c L[i][c] Y[j][c]
//       over the sub-panel, spread over all threads through the pair table.
constexpr int kSub = 16;

template <class T>
__global__ void __launch_bounds__(256, 1) k_dense_diag_t(T* __restrict__ S0, int n, int k0, int kb,
                                                      int64_t bstride, PivotRule rule,
                                                      unsigned long long* __restrict__ counters) {
  __shared__ T A[kPanelW][kPanelW + 1];
  __shared__ T Ys[kPanelW][kSub + 1];
  __shared__ T Dinv[kSub];
  __shared__ uint16_t pairs[kDiagPairs];
  __shared__ int pert;
  T* S = S0 + (int64_t)blockIdx.x * bstride;
  const int tid = threadIdx.x;
  {
    // 16 loads per thread issued together, then stored
    T v[16];
#pragma unroll
    for (int u = 0; u < 16; u++) {
      const int q = tid + u * 256, c = q >> 6, r = q & 63;
      v[u] = (r >= c && r < kb && c < kb) ? S[(int64_t)(k0 + r) + (int64_t)(k0 + c) * n] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 16; u++) {
      const int q = tid + u * 256, c = q >> 6, r = q & 63;
      A[r][c] = v[u];
    }
  }
  for (int p = tid; p < kDiagPairs; p += blockDim.x) {
    int i, j;
    diag_pair(p, i, j);
    pairs[p] = (uint16_t)(i | (j << 8));
  }
  if (tid == 0) pert = 0;
  __syncthreads();
  const double thr = rule.anorm ? rule.pivot_eps * rule.anorm[blockIdx.x] : 0.0;
  const int si = tid >> 4, sj = tid & 15;  // this thread's entry of a 16 x 16 sub-block
  for (int c0 = 0; c0 < kb; c0 += kSub) {
    const int cb = min(kSub, kb - c0);
    for (int c = 0; c < cb; c++) {  // (1)
      if (tid == 0) {
        T d = A[c0 + c][c0 + c];
        if (thr > 0.0 && fabs((double)d) < thr) {
          d = (T)(rule.primal[k0 + c0 + c] ? thr : -thr);
          A[c0 + c][c0 + c] = d;
          pert++;
        }
        Dinv[c] = pivot_recip(d);
      }
      if (c > 0 && sj == c - 1 && si > c - 1 && si < cb) A[c0 + si][c0 + c - 1] *= Dinv[c - 1];
      __syncthreads();
      if (si > c && sj > c && sj <= si && si < cb)
        A[c0 + si][c0 + sj] -= A[c0 + si][c0 + c] * Dinv[c] * A[c0 + sj][c0 + c];
      __syncthreads();
    }
    if (sj == cb - 1 && si > cb - 1 && si < cb) A[c0 + si][c0 + cb - 1] *= Dinv[cb - 1];
    __syncthreads();
    const int r0 = c0 + cb;
    for (int row = r0 + tid; row < kb; row += blockDim.x) {  // (2)
      T y[kSub];
#pragma unroll
      for (int c = 0; c < kSub; c++) {
        if (c < cb) {
          T acc = A[row][c0 + c];
#pragma unroll
          for (int c2 = 0; c2 < c; c2++) acc -= y[c2] * A[c0 + c][c0 + c2];
          y[c] = acc;
        }
      }
#pragma unroll
      for (int c = 0; c < kSub; c++)
        if (c < cb) {
          Ys[row][c] = y[c];
          A[row][c0 + c] = y[c] * Dinv[c];
        }
    }
    __syncthreads();
    if (r0 < kb) {  // (3): pairs with j >= r0
      const int npairs = (kPanelW - r0) * (kPanelW - r0 + 1) / 2;
      for (int p = tid; p < npairs; p += blockDim.x) {
        const int ij = pairs[p], i = ij & 0xFF, j = ij >> 8;
        if (i < kb) {
          T acc = T(0);
#pragma unroll
          for (int c = 0; c < kSub; c++)
            if (c < cb) acc += A[i][c0 + c] * Ys[j][c];
          A[i][j] -= acc;
        }
      }
    }
    __syncthreads();
  }
  {
#pragma unroll
    for (int u = 0; u < 16; u++) {
      const int q = tid + u * 256, c = q >> 6, r = q & 63;
      if (r >= c && r < kb && c < kb) S[(int64_t)(k0 + r) + (int64_t)(k0 + c) * n] = A[r][c];
    }
  }
  const T dd = tid < kb ? A[tid][tid] : T(0);
  const int pos = __syncthreads_count(dd > T(0));
  const int neg = __syncthreads_count(dd < T(0));
  if (tid == 0) {
    atomicAdd(&counters[kPos], (unsigned long long)pos);
    atomicAdd(&counters[kNeg], (unsigned long long)neg);
    if (kb - pos - neg) atomicAdd(&counters[kZero], (unsigned long long)(kb - pos - neg));
    if (pert) atomicAdd(&counters[kPerturbed], (unsigned long long)pert);
  }
}

// TF32 operand images of the trailing update, written by the panel kernels
// themselves (FP32 only): the shared-memory layout of the tensor-core update's
// 128-row A blocks (Y) and 64-row B blocks (L21), K-major 8-row x 16-byte core
// matrices, 16 cores along K.  Rows are counted from the first trailing row;
// columns at or past kb are zero.  A null A skips the images.
struct Tf32Images {
  uint8_t* A = nullptr;
  uint8_t* B = nullptr;
};

__device__ __forceinline__ int64_t tf32_img_off(int rho, int c, int rows_blk) {
  const int blk = rho / rows_blk, rr = rho - blk * rows_blk;
  return (int64_t)blk * (rows_blk / 8) * 16 * 128 + ((rr >> 3) * 16 + (c >> 2)) * 128 + (rr & 7) * 16 + (c & 3) * 4;
}

// Rows k0+kb .. rend-1 of matrix blockIdx.y, one thread per row (ROWS rows
// per CTA): solve y L11^T = a with y in registers and L11 in shared memory
// (every thread of a warp reads the same L11 entry), then Y = y and
// L21 = y D1^{-1}.  Y has the matrix's leading dimension n and its rows.
template <class T, int ROWS>
__global__ void __launch_bounds__(ROWS) k_dense_panel_t(T* __restrict__ S0, T* __restrict__ Y0, int n,
                                                        int k0, int kb, int rend, int64_t bstride,
                                                        int64_t ystride, Tf32Images img) {
  __shared__ T L11[kPanelW][kPanelW];  // [j][c], zero outside the strict lower triangle
  __shared__ T dinv[kPanelW];
  T* S = S0 + (int64_t)blockIdx.y * bstride;
  T* Y = Y0 + (int64_t)blockIdx.y * ystride;
  for (int q = threadIdx.x; q < kPanelW * kPanelW; q += blockDim.x) {
    const int c = q / kPanelW, j = q - c * kPanelW;
    L11[j][c] = (j > c && j < kb) ? S[(int64_t)(k0 + j) + (int64_t)(k0 + c) * n] : T(0);
  }
  for (int c = threadIdx.x; c < kPanelW; c += blockDim.x)
    dinv[c] = c < kb ? T(1) / S[(int64_t)(k0 + c) + (int64_t)(k0 + c) * n] : T(0);
  __syncthreads();
  const int row = k0 + kb + blockIdx.x * ROWS + threadIdx.x;
  if (row >= rend) return;
  T y[kPanelW];
#pragma unroll
  for (int c = 0; c < kPanelW; c++) y[c] = c < kb ? S[row + (int64_t)(k0 + c) * n] : T(0);
  // y_j = a_j - sum_{c<j} y_c L_jc, subtracted in increasing c
#pragma unroll
  for (int j = 1; j < kPanelW; j++) {
    T acc = y[j];
#pragma unroll
    for (int c = 0; c < j; c++) acc -= y[c] * L11[j][c];
    y[j] = acc;
  }
#pragma unroll
  for (int c = 0; c < kPanelW; c++)
    if (c < kb) {
      Y[row + (int64_t)c * n] = y[c];
      S[row + (int64_t)(k0 + c) * n] = y[c] * dinv[c];
    }
  if constexpr (sizeof(T) == 4) {
    if (img.A) {
      const int rho = row - (k0 + kb);
#pragma unroll
      for (int kq = 0; kq < kPanelW / 4; kq++) {
        float4 a, l;
        a.x = y[4 * kq];
        a.y = y[4 * kq + 1];
        a.z = y[4 * kq + 2];
        a.w = y[4 * kq + 3];
        l.x = y[4 * kq] * dinv[4 * kq];
        l.y = y[4 * kq + 1] * dinv[4 * kq + 1];
        l.z = y[4 * kq + 2] * dinv[4 * kq + 2];
        l.w = y[4 * kq + 3] * dinv[4 * kq + 3];
        *reinterpret_cast<float4*>(img.A + tf32_img_off(rho, 4 * kq, 128)) = a;
        *reinterpret_cast<float4*>(img.B + tf32_img_off(rho, 4 * kq, 64)) = l;
      }
    }
  }
}

// The same solve with one warp per row: lane l holds y_l and y_{l+32}, and
// column c's value reaches the other lanes by shuffle.  The dependency chain
// of a row is 64 steps long instead of 2016 multiply-adds, which is what counts
// for few rows (and in FP64, whose dependent multiply-add latency is long).
template <class T>
__global__ void __launch_bounds__(256) k_dense_panel_w(T* __restrict__ S0, T* __restrict__ Y0, int n, int k0,
                                                       int kb, int rend, int64_t bstride, int64_t ystride,
                                                       Tf32Images img) {
  __shared__ T L11[kPanelW][kPanelW + 1];
  __shared__ T dinv[kPanelW];
  T* S = S0 + (int64_t)blockIdx.y * bstride;
  T* Y = Y0 + (int64_t)blockIdx.y * ystride;
  for (int q = threadIdx.x; q < kb * kb; q += blockDim.x) {
    const int j = q / kb, i = q - j * kb;
    L11[i][j] = S[(int64_t)(k0 + i) + (int64_t)(k0 + j) * n];
  }
  for (int c = threadIdx.x; c < kb; c += blockDim.x) dinv[c] = T(1) / S[(int64_t)(k0 + c) + (int64_t)(k0 + c) * n];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int row = k0 + kb + blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (row >= rend) return;
  T y0 = lane < kb ? S[row + (int64_t)(k0 + lane) * n] : T(0);
  T y1 = lane + 32 < kb ? S[row + (int64_t)(k0 + lane + 32) * n] : T(0);
  for (int c = 0; c < kb; c++) {
    const T yc = __shfl_sync(0xffffffffu, c < 32 ? y0 : y1, c & 31);
    if (lane > c && lane < kb) y0 -= yc * L11[lane][c];
    if (lane + 32 > c && lane + 32 < kb) y1 -= yc * L11[lane + 32][c];
  }
  if (lane < kb) {
    Y[row + (int64_t)lane * n] = y0;
    S[row + (int64_t)(k0 + lane) * n] = y0 * dinv[lane];
  }
  if (lane + 32 < kb) {
    Y[row + (int64_t)(lane + 32) * n] = y1;
    S[row + (int64_t)(k0 + lane + 32) * n] = y1 * dinv[lane + 32];
  }
  if constexpr (sizeof(T) == 4) {
    if (img.A) {
      const int rho = row - (k0 + kb);
      const float l0 = lane < kb ? y0 * dinv[lane] : 0.f, l1 = lane + 32 < kb ? y1 * dinv[lane + 32] : 0.f;
      *reinterpret_cast<float*>(img.A + tf32_img_off(rho, lane, 128)) = y0;
      *reinterpret_cast<float*>(img.A + tf32_img_off(rho, lane + 32, 128)) = y1;
      *reinterpret_cast<float*>(img.B + tf32_img_off(rho, lane, 64)) = l0;
      *reinterpret_cast<float*>(img.B + tf32_img_off(rho, lane + 32, 64)) = l1;
    }
  }
}

// A launch with a scheduling priority (a launch attribute, so that it also
// holds for the kernel node when the launch is captured in a graph).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_prio(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                               int prio, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = prio;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Rows below the diagonal block of nb matrices.  A thread per row issues the
// fewest instructions (no idle lanes) but its dependency chain is long; a
// warp per row has a 64-step chain.  FP32 takes a thread per row from 2048
// rows on.  In FP64 a warp issues one multiply-add per 64 cycles, so a thread
// per row pays off once there are enough rows (m * nb >= 32768, over 1000
// warps) to keep every sub-partition's FP64 pipe busy.
template <class T>
inline void launch_dense_panel(T* S, T* Y, int n, int k0, int kb, int rend, int nb, int64_t bstride,
                               int64_t ystride, cudaStream_t st, int prio = 0, Tf32Images img = Tf32Images{}) {
  const int m = rend - k0 - kb;
  if (m <= 0) return;
  if constexpr (sizeof(T) == 4) {
    if (m > 2048) {
      launch_prio(k_dense_panel_t<T, 128>, dim3((m + 127) / 128, nb), dim3(128), 0, st, prio, S, Y, n, k0, kb,
                  rend, bstride, ystride, img);
      return;
    }
  } else {
    if ((int64_t)m * nb >= 32768) {
      launch_prio(k_dense_panel_t<T, 32>, dim3((m + 31) / 32, nb), dim3(32), 0, st, prio, S, Y, n, k0, kb, rend,
                  bstride, ystride, img);
      return;
    }
  }
  launch_prio(k_dense_panel_w<T>, dim3((m + 7) / 8, nb), dim3(256), 0, st, prio, S, Y, n, k0, kb, rend, bstride,
              ystride, img);
}

// Trailing update of matrix blockIdx.y on the lower 64 x 64 tiles below the
// panel: A[i][j] -= sum_c Y[i][c] L[j][c] for k0+kb <= j <= i < rend.
__global__ void __launch_bounds__(256) k_dense_update(double* __restrict__ S0, const double* __restrict__ Y0,
                                                      int n, int k0, int kb, int rend, int64_t bstride,
                                                      int64_t ystride) {
  double* S = S0 + (int64_t)blockIdx.y * bstride;
  const double* Y = Y0 + (int64_t)blockIdx.y * ystride;
  const int base = k0 + kb;
  int tile = blockIdx.x, ti = 0;
  while (tile > ti) {
    tile -= ti + 1;
    ti++;
  }
  const int tj = tile;
  const int i0 = base + ti * 64, j0 = base + tj * 64;
  constexpr int KC = 32;              // columns staged per pass
  __shared__ double Ys[KC][64 + 1];  // [c][i]
  __shared__ double Ls[KC][64 + 1];  // [c][j]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16, 4x4 outputs each
  double acc[4][4] = {};
  for (int cb = 0; cb < kb; cb += KC) {
    const int kc = min(KC, kb - cb);
    __syncthreads();
    for (int q = threadIdx.x; q < kc * 64; q += 256) {
      const int c = q / 64, r = q % 64;
      Ys[c][r] = (i0 + r < rend) ? Y[(i0 + r) + (int64_t)(cb + c) * n] : 0.0;
      Ls[c][r] = (j0 + r < rend) ? S[(j0 + r) + (int64_t)(k0 + cb + c) * n] : 0.0;
    }
    __syncthreads();
    for (int c = 0; c < kc; c++) {
      double a[4], bb[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        a[u] = Ys[c][ty + 16 * u];
        bb[u] = Ls[c][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 4; v++) acc[u][v] += a[u] * bb[v];
    }
  }
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < rend && j < rend && i >= j) S[i + (int64_t)j * n] -= acc[u][v];
    }
}

}  // namespace

}  // namespace kkt
