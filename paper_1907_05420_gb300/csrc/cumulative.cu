// The structured Schur complement of the cumulative MPOPF coupling (Sec. 4.3,
// eqs. LocalSchurBs, LocalSchurBs3, GlobalSchur; kkt_options.structured_s = 2).
//
// The coupling variables are ordered by period, ns per period (nC = N ns).  In
// block i the coupling columns of period m are zero for m < i, Y_i for m = i
// (the paper's C_1) and one and the same Z_i for every m > i (C_0).  With
// E^T A_i^{-1} E = G_i (the contraction every mode computes), the three
// distinct blocks of S_i (eq. LocalSchurBs3) are -H11_i, -H10_i, -H00_i with
//
//   H11_i = Y_i^T G_i Y_i,  H10_i = Z_i^T G_i Y_i,  H00_i = Z_i^T G_i Z_i
//
// (Y_i, Z_i here the k x ns coefficient matrices of B_i = E [.. Y_i Z_i ..]),
// and S (eq. GlobalSchur) is kept as the two block vectors
//
//   S_d[j] = C_j - H11_j - sum_{i<j} H00_i,   S_o[j] = -H10_j - sum_{i<j} H00_i.
//
// Factor: a block LDL^T of S without pivoting.  All blocks below the diagonal
// in a block column are equal, so eliminating that column lowers every trailing
// block by the same matrix; step j is the partial LDL^T (ns pivots) of the
// order-2ns matrix
//
//   Q_j = [ S_d[j] + V_j     .  ]      V_0 = 0,
//         [ S_o[j] + V_j    V_j ]      V_{j+1} = the trailing block of Q_j after its pivots,
//
// which leaves L_j, D_j (Delta_j = S_d[j] - U_j = L_j D_j L_j^T, U_j = -V_j)
// and L21_j (the block in every row m > j) in its first ns columns.  These N
// steps are the only sequential part (N ns^3 7/3 flops instead of nC^3/3).
// In the TF32 and BF16 modes these steps, the inversion and the solve's
// products run in FP32 (like the dense factor of S there), with FP64
// refinement on K and the FP64 steps as the fallback.
// Then, for all periods at once, Z L_j = [I; L21_j] gives Linv_j = L_j^{-1}
// and M_j = L21_j L_j^{-1}, and a solve S x = t is two chains of one ns x ns
// matrix-vector product per period,
//
//   forward:   w_j = t_j - R_j,            R_{j+1} = R_j + M_j w_j     (R_0 = 0)
//   diagonal:  a_j = Linv_j^T D_j^{-1} Linv_j w_j                     (all j at once)
//   backward:  x_j = a_j - M_j^T Q_j,      Q_{j-1} = Q_j + x_j         (Q_{N-1} = 0)
//
// run by a cluster of CTAs that exchange the vector through distributed
// shared memory, one cluster barrier per period.
#include <cooperative_groups.h>

#include <algorithm>
#include <string>
#include <vector>

#include "dense_kernels.cuh"
#include "handle.h"

namespace kkt {
namespace {

namespace cg = cooperative_groups;

constexpr int kCumCluster = 8;    // CTAs of the solve's cluster
constexpr int kCumThreads = 256;  // threads per CTA of the chains
constexpr int kCumErrValues = 1;  // cum_err: B's values do not repeat over the later periods

inline int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

// Entries that must repeat (B's values of period m > i + 1 against period i + 1).
__global__ void k_cum_check(const int32_t* __restrict__ pairs, int64_t npairs, const double* __restrict__ b_vals,
                            int* __restrict__ err) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npairs; q += (int64_t)gridDim.x * blockDim.x) {
    const double v = b_vals[pairs[2 * q]], w = b_vals[pairs[2 * q + 1]];
    if (v != w && !(v != v && w != w)) atomicExch(err, kCumErrValues);
  }
}

// H11, H10, H00 of every block, one thread per entry (row a, column c); the
// column lists hold (index t into E, B entry) per storage unit.
__global__ void k_cum_local(const int32_t* __restrict__ y_ptr, const int32_t* __restrict__ y_t,
                            const int32_t* __restrict__ y_e, const int32_t* __restrict__ z_ptr,
                            const int32_t* __restrict__ z_t, const int32_t* __restrict__ z_e,
                            const double* __restrict__ b_vals, const double* __restrict__ G, int k, int ns,
                            int N, double* __restrict__ H) {
  const int64_t nn = (int64_t)ns * ns, total = (int64_t)N * 3 * nn;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t bw = q / nn;  // block * 3 + which
    const int b = (int)(bw / 3), which = (int)(bw - (int64_t)b * 3);
    const int64_t rc = q - bw * nn;
    const int c = (int)(rc / ns), a = (int)(rc - (int64_t)c * ns);
    const int32_t* lp = which == 0 ? y_ptr : z_ptr;  // left factor: Y (H11) or Z (H10, H00)
    const int32_t* lt = which == 0 ? y_t : z_t;
    const int32_t* le = which == 0 ? y_e : z_e;
    const int32_t* rp = which == 2 ? z_ptr : y_ptr;  // right factor: Y (H11, H10) or Z (H00)
    const int32_t* rt = which == 2 ? z_t : y_t;
    const int32_t* re = which == 2 ? z_e : y_e;
    const int64_t base = (int64_t)b * (ns + 1);
    const double* Gb = G + (int64_t)b * k * k;
    double acc = 0.0;
    for (int p = lp[base + a]; p < lp[base + a + 1]; p++) {
      const double* Grow = Gb + (int64_t)lt[p] * k;
      double inner = 0.0;
      for (int r = rp[base + c]; r < rp[base + c + 1]; r++) inner += Grow[rt[r]] * b_vals[re[r]];
      acc += b_vals[le[p]] * inner;
    }
    H[q] = acc;
  }
}

// S_d and S_o (eq. GlobalSchur): one thread per entry, the sum over earlier
// periods carried along the periods in order.
__global__ void k_cum_prefix(const double* __restrict__ H, const double* __restrict__ c_vals, int ns, int N,
                             double* __restrict__ Sd, double* __restrict__ So) {
  const int64_t nn = (int64_t)ns * ns;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nn; q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q / ns), a = (int)(q - (int64_t)c * ns);
    double acc = 0.0;  // sum_{i<j} S00_i = -sum_{i<j} H00_i
    for (int j = 0; j < N; j++) {
      const double* Hj = H + (int64_t)j * 3 * nn;
      const double cj = a == c ? c_vals[(int64_t)j * ns + a] : 0.0;
      Sd[(int64_t)j * nn + q] = (cj - Hj[q]) + acc;
      if (j + 1 < N) {
        So[(int64_t)j * nn + q] = -Hj[nn + q] + acc;
        acc -= Hj[2 * nn + q];
      }
    }
  }
}

// Q_j (column-major, leading dimension 2ns, lower triangle) from S_d[j],
// S_o[j] and the trailing block V of Q_{j-1}; the last period has no rows below.
// T: the type of the period factors (FP32 in the TF32 and BF16 modes).
template <class T>
__global__ void k_cum_build(const double* __restrict__ Sd, const double* __restrict__ So,
                            const T* __restrict__ Qprev, T* __restrict__ Q, int ns, int j, int last) {
  const int n2 = 2 * ns;
  const int64_t nn = (int64_t)ns * ns, total = (int64_t)n2 * n2;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q / n2), r = (int)(q - (int64_t)c * n2);
    if (r < c) continue;
    auto V = [&](int r1, int c1) -> double {
      if (!Qprev) return 0.0;
      const int hi = max(r1, c1), lo = min(r1, c1);
      return (double)Qprev[(ns + hi) + (int64_t)(ns + lo) * n2];
    };
    double v;
    if (c < ns && r < ns) {
      v = Sd[(int64_t)j * nn + r + (int64_t)c * ns] + V(r, c);
    } else if (last) {
      v = 0.0;
    } else if (c < ns) {
      v = So[(int64_t)j * nn + (r - ns) + (int64_t)c * ns] + V(r - ns, c);
    } else {
      v = V(r - ns, c - ns);
    }
    Q[q] = (T)v;
  }
}

// Trailing update of one period's partial factor, A[i][j] -= sum_c Y[i][c]
// L[j][c] for base <= j <= i < rend: a 16 x 16 tile of the lower triangle per
// CTA, one entry per thread.  The trailing matrices here are small (2 n_s
// rows), so small tiles spread each update over many SMs.
constexpr int kCumTile = 16;
constexpr int kCumPanel = 32;  // pivot columns per panel of the period factors

template <class T>
__global__ void __launch_bounds__(kCumTile * kCumTile) k_cum_update(T* __restrict__ S, const T* __restrict__ Y, int n,
                                                                   int k0, int kb, int rend) {
  const int base = k0 + kb;
  int tile = blockIdx.x, ti = 0;
  while (tile > ti) {
    tile -= ti + 1;
    ti++;
  }
  const int i0 = base + ti * kCumTile, j0 = base + tile * kCumTile;
  __shared__ T Ys[kCumPanel][kCumTile + 1];
  __shared__ T Ls[kCumPanel][kCumTile + 1];
  const int tx = threadIdx.x % kCumTile, ty = threadIdx.x / kCumTile;
  for (int q = threadIdx.x; q < kb * kCumTile; q += blockDim.x) {
    const int c = q / kCumTile, r = q % kCumTile;
    Ys[c][r] = i0 + r < rend ? Y[(i0 + r) + (int64_t)c * n] : T(0);
    Ls[c][r] = j0 + r < rend ? S[(j0 + r) + (int64_t)(k0 + c) * n] : T(0);
  }
  __syncthreads();
  T acc = T(0);
  for (int c = 0; c < kb; c++) acc += Ys[c][ty] * Ls[c][tx];
  const int i = i0 + ty, j = j0 + tx;
  if (i < rend && j <= i) S[i + (int64_t)j * n] -= acc;
}

// Z L_j = [I; L21_j] for the rows of Z: rows < ns give Linv_j = L_j^{-1}, the
// others M_j = L21_j L_j^{-1} (stored also transposed); D_j is copied out.
// One thread per row of Z, its row in shared memory; the columns are swept
// from the last, z_c = b_c - sum_{k>c} z_k L(k, c).
template <class T>
__global__ void k_cum_inverse(const T* __restrict__ Qall, int ns, int N, int rows_per_cta, int ld,
                              T* __restrict__ Linv, T* __restrict__ M, T* __restrict__ Mt, T* __restrict__ D) {
  extern __shared__ __align__(16) unsigned char zraw[];
  T* zs = reinterpret_cast<T*>(zraw);  // rows_per_cta x ld
  const int j = blockIdx.y;
  const int n2 = 2 * ns;
  const int rows = j + 1 < N ? n2 : ns;
  const int r = blockIdx.x * rows_per_cta + threadIdx.x;
  if (threadIdx.x >= rows_per_cta || r >= rows) return;  // no barrier below: each thread works alone
  const T* Q = Qall + (int64_t)j * n2 * n2;
  T* z = zs + (int64_t)threadIdx.x * ld;
  const int64_t nn = (int64_t)ns * ns;
  const int cstart = r < ns ? r : ns - 1;  // L^{-1} is lower triangular
  for (int c = cstart + 1; c < ns; c++) z[c] = T(0);
  for (int c = cstart; c >= 0; c--) {
    T v = r < ns ? (r == c ? T(1) : T(0)) : Q[r + (int64_t)c * n2];
    for (int kk = c + 1; kk <= cstart; kk++) v -= z[kk] * Q[kk + (int64_t)c * n2];
    z[c] = v;
  }
  if (r < ns) {
    for (int c = 0; c < ns; c++) Linv[(int64_t)j * nn + r + (int64_t)c * ns] = z[c];
    D[(int64_t)j * ns + r] = Q[r + (int64_t)r * n2];
  } else {
    const int a = r - ns;
    for (int c = 0; c < ns; c++) {
      M[(int64_t)j * nn + a + (int64_t)c * ns] = z[c];
      Mt[(int64_t)j * nn + c + (int64_t)a * ns] = z[c];
    }
  }
}

// Rows [r0, r1) of y = A v for a column-major ns x ns A, v in shared memory:
// tpr threads per row (a power of two, 32 at most), each a stride of the
// columns, reduced with shuffles.  Every thread runs the same number of
// iterations, so whole warps take part in the shuffles.
template <class T>
__device__ __forceinline__ void rows_matvec(const T* __restrict__ A, const T* v, int ns, int r0, int r1, int tpr,
                                            double* out) {
  const int tid = threadIdx.x, part = tid % tpr, per_it = kCumThreads / tpr;
  const int iters = (r1 - r0 + per_it - 1) / per_it;
  for (int it = 0; it < iters; it++) {
    const int a = r0 + it * per_it + tid / tpr;
    const bool live = a < r1;
    T s = T(0);
    if (live)
      for (int c = part; c < ns; c += tpr) s += A[a + (int64_t)c * ns] * v[c];
    for (int off = tpr / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (live && part == 0) out[a - r0] = (double)s;
  }
}

// The forward (FORWARD) or backward chain of the solve over the periods, by a
// cluster of kCumCluster CTAs; CTA `rank` owns rows [r0, r1) of the vectors.
//   forward:  x_j := w_j = t_j - R_j, R += M_j w_j
//   backward: x_j := a_j - Mt_j Q, Q += x_j (x holds a_j on entry)
// The running sums and x stay FP64; with an FP32 factor (T float) the
// exchanged vector and the products are FP32, each product row added to the
// FP64 sum.
template <bool FORWARD, class T>
__global__ void __cluster_dims__(kCumCluster, 1, 1) __launch_bounds__(kCumThreads)
    k_cum_chain(const T* __restrict__ Mall, int ns, int N, int tpr, double* __restrict__ x) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* state = reinterpret_cast<double*>(smraw);  // own rows of R (forward) or Q (backward)
  double* part = state + ns;                          // own rows of the product
  T* vbuf = reinterpret_cast<T*>(part + ns);          // 2 x ns: the exchanged vector, double-buffered
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int per = (ns + kCumCluster - 1) / kCumCluster;
  const int r0 = min(ns, rank * per), r1 = min(ns, r0 + per);
  const int64_t nn = (int64_t)ns * ns;
  for (int a = threadIdx.x; a < r1 - r0; a += blockDim.x) state[a] = 0.0;
  cluster.sync();  // every CTA of the cluster runs before any writes into its shared memory
  for (int s = 0; s < N; s++) {
    const int j = FORWARD ? s : N - 1 - s;
    T* vb = vbuf + (s & 1) * ns;
    double* xj = x + (int64_t)j * ns;
    if (FORWARD) {
      // w_j = t_j - R_j on own rows, to every CTA's buffer
      for (int a = threadIdx.x; a < r1 - r0; a += blockDim.x) {
        const double w = xj[r0 + a] - state[a];
        xj[r0 + a] = w;
        for (int q = 0; q < kCumCluster; q++) cluster.map_shared_rank(vb, q)[r0 + a] = (T)w;
      }
    } else {
      for (int a = threadIdx.x; a < r1 - r0; a += blockDim.x)
        for (int q = 0; q < kCumCluster; q++) cluster.map_shared_rank(vb, q)[r0 + a] = (T)state[a];
    }
    cluster.sync();  // the full vector is in vb on every CTA
    if (FORWARD && j == N - 1) break;
    rows_matvec(Mall + (int64_t)j * nn, vb, ns, r0, r1, tpr, part);
    __syncthreads();
    for (int a = threadIdx.x; a < r1 - r0; a += blockDim.x) {
      if (FORWARD) {
        state[a] += part[a];
      } else {
        const double xv = xj[r0 + a] - part[a];
        xj[r0 + a] = xv;
        state[a] += xv;
      }
    }
    __syncthreads();
  }
  cluster.sync();  // no CTA leaves while another may still write into its buffer
}

// a_j = Linv_j^T D_j^{-1} Linv_j w_j for every period (one CTA each), in place
// in x (in the factor's type T).
template <class T>
__global__ void __launch_bounds__(kCumThreads) k_cum_diag(const T* __restrict__ Linv, const T* __restrict__ D,
                                                          int ns, double* __restrict__ x) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* w = reinterpret_cast<T*>(smraw);  // ns
  T* z = w + ns;                       // ns
  const int j = blockIdx.x;
  const int64_t nn = (int64_t)ns * ns;
  const T* Lj = Linv + (int64_t)j * nn;
  double* xj = x + (int64_t)j * ns;
  for (int a = threadIdx.x; a < ns; a += blockDim.x) w[a] = (T)xj[a];
  __syncthreads();
  for (int a = threadIdx.x; a < ns; a += blockDim.x) {  // y = Linv w (lower), z = y / d
    T s = T(0);
    for (int c = 0; c <= a; c++) s += Lj[a + (int64_t)c * ns] * w[c];
    z[a] = s / D[(int64_t)j * ns + a];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ns; c += blockDim.x) {  // a = Linv^T z
    T s = T(0);
    for (int a = c; a < ns; a++) s += Lj[a + (int64_t)c * ns] * z[a];
    xj[c] = (double)s;
  }
}

int threads_per_row(int ns) {
  const int per = (ns + kCumCluster - 1) / kCumCluster;
  int tpr = 32;
  while (tpr > 1 && tpr * per > kCumThreads) tpr >>= 1;
  return tpr;
}

}  // namespace

// ---- analysis ----

std::string analyze_cumulative(const kkt_pattern* pat, const Coupling& C, CumPattern& out) {
  out = CumPattern();
  const int32_t N = pat->N, nC = pat->nC;
  if (pat->c_kind != 0) return "structured_s = 2 needs a diagonal C (c_kind 0)";
  if (nC <= 0 || nC % N != 0) return "structured_s = 2 needs nC a positive multiple of N";
  const int32_t ns = nC / N;
  if (ns > kCumMaxStor) return "structured_s = 2: more than 4096 coupling variables per period";
  out.ns = ns;
  out.y_ptr.assign((size_t)N * (ns + 1), 0);
  out.z_ptr.assign((size_t)N * (ns + 1), 0);
  struct Ent {
    int32_t row, s, e;
  };
  std::vector<std::vector<Ent>> groups(N);
  for (int32_t i = 0; i < N; i++) {
    for (auto& g : groups) g.clear();
    for (int32_t e = pat->b_blockptr[i]; e < pat->b_blockptr[i + 1]; e++) {
      const int32_t m = pat->b_col[e] / ns, s = pat->b_col[e] - m * ns;
      if (m < i)
        return "structured_s = 2: block " + std::to_string(i) + " has a coupling entry in the earlier period " +
               std::to_string(m);
      groups[m].push_back({pat->b_row[e], s, e});
    }
    const std::vector<Ent>& ref = i + 1 < N ? groups[i + 1] : groups[i];
    for (int32_t m = i + 2; m < N; m++) {
      const std::vector<Ent>& g = groups[m];
      bool same = g.size() == ref.size();
      for (size_t q = 0; same && q < g.size(); q++) same = g[q].row == ref[q].row && g[q].s == ref[q].s;
      if (!same)
        return "structured_s = 2: in block " + std::to_string(i) + " the coupling pattern of period " +
               std::to_string(m) + " differs from that of period " + std::to_string(i + 1);
      for (size_t q = 0; q < g.size(); q++) {
        out.check.push_back(g[q].e);
        out.check.push_back(ref[q].e);
      }
    }
    // per storage unit: the (t, entry) lists of Y_i (period i) and Z_i (period i + 1)
    auto lists = [&](const std::vector<Ent>& g, std::vector<int32_t>& ptr, std::vector<int32_t>& t,
                     std::vector<int32_t>& ent) {
      int32_t* p = ptr.data() + (size_t)i * (ns + 1);
      std::vector<int32_t> cnt(ns, 0);
      for (const Ent& x : g) cnt[x.s]++;
      p[0] = (int32_t)t.size();
      for (int32_t s = 0; s < ns; s++) p[s + 1] = p[s] + cnt[s];
      t.resize(p[ns]);
      ent.resize(p[ns]);
      std::vector<int32_t> fill(p, p + ns);
      for (const Ent& x : g) {
        t[fill[x.s]] = C.e_t[x.e];
        ent[fill[x.s]++] = x.e;
      }
    };
    lists(groups[i], out.y_ptr, out.y_t, out.y_e);
    static const std::vector<Ent> none;
    lists(i + 1 < N ? groups[i + 1] : none, out.z_ptr, out.z_t, out.z_e);
  }
  return std::string();
}

int cum_inverse_rows(int ns) {
  const int ld = ns % 2 ? ns : ns + 1;
  int rows = 32;
  while (rows > 1 && (int64_t)rows * ld * 8 > kCumInverseSmem) rows >>= 1;
  return rows;
}

cudaError_t cum_prepare() {
  const int chain = (4 * kCumMaxStor) * 8;
  cudaError_t e = cudaFuncSetAttribute(k_cum_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kCumInverseSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cum_inverse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCumInverseSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cum_chain<true, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, chain);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cum_chain<false, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, chain);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cum_chain<true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, chain);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cum_chain<false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, chain);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cum_diag<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kCumMaxStor * 8);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cum_diag<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kCumMaxStor * 8);
  return e;
}

// ---- factor ----

cudaError_t launch_cum_assemble(Handle& h, cudaStream_t st) {
  const int ns = h.cum_ns, N = h.N, k = h.cpl.k;
  const int64_t nn = (int64_t)ns * ns;
  cudaError_t e = cudaMemsetAsync(h.cum_err, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (h.cum_npairs > 0) {
    k_cum_check<<<grid_of(h.cum_npairs), 256, 0, st>>>(h.d.cum_check, h.cum_npairs, h.b_vals, h.cum_err);
    h.launches++;
  }
  k_cum_local<<<grid_of((int64_t)N * 3 * nn), 256, 0, st>>>(h.d.cum_y_ptr, h.d.cum_y_t, h.d.cum_y_e, h.d.cum_z_ptr,
                                                            h.d.cum_z_t, h.d.cum_z_e, h.b_vals, h.G, k, ns, N,
                                                            h.cum_H);
  k_cum_prefix<<<grid_of(nn), 256, 0, st>>>(h.cum_H, h.c_vals, ns, N, h.cum_Sd, h.cum_So);
  h.launches += 2;
  return cudaGetLastError();
}

namespace {

// The N period steps and the batched inversion in type T, on the buffers of
// that type (Q, its panel scratch, L^{-1}, M, M^T, D).
template <class T>
cudaError_t cum_factor_in(Handle& h, unsigned long long* counters, cudaStream_t st, T* Qall, T* QY, T* Linv, T* M,
                          T* Mt, T* D) {
  const int ns = h.cum_ns, N = h.N, n2 = 2 * ns;
  const int64_t q2 = (int64_t)n2 * n2;
  for (int j = 0; j < N; j++) {
    T* Q = Qall + (int64_t)j * q2;
    const int last = j + 1 == N;
    k_cum_build<T><<<grid_of(q2), 256, 0, st>>>(h.cum_Sd, h.cum_So, j ? Q - q2 : nullptr, Q, ns, j, last);
    h.launches++;
    const int rend = last ? ns : n2;
    for (int k0 = 0; k0 < ns; k0 += kCumPanel) {
      const int kb = std::min(kCumPanel, ns - k0);
      const int kd = kt_begin(h, kFamDiag, (2.0 / 3.0) * kb * kb * kb, st);
      k_dense_diag_t<T><<<1, 256, 0, st>>>(Q, n2, k0, kb, 0, PivotRule{}, counters);
      kt_end(h, kd, st);
      h.launches++;
      const int rest = rend - k0 - kb;
      if (rest > 0) {
        launch_dense_panel<T>(Q, QY, n2, k0, kb, rend, 1, 0, 0, st);
        const int tiles = (rest + kCumTile - 1) / kCumTile;
        const int kt = kt_begin(h, kFamDenseF64, update_flops(rest, 0, rest, kb), st);
        k_cum_update<T><<<tiles * (tiles + 1) / 2, kCumTile * kCumTile, 0, st>>>(Q, QY, n2, k0, kb, rend);
        kt_end(h, kt, st);
        h.launches += 2;
      }
    }
  }
  const int rows = cum_inverse_rows(ns), ld = ns % 2 ? ns : ns + 1;
  k_cum_inverse<T><<<dim3((n2 + rows - 1) / rows, N), rows, (size_t)rows * ld * sizeof(T), st>>>(Qall, ns, N, rows,
                                                                                                ld, Linv, M, Mt, D);
  h.launches++;
  return cudaGetLastError();
}

template <class T>
cudaError_t cum_solve_in(Handle& h, double* x, cudaStream_t st, const T* Linv, const T* M, const T* Mt,
                         const T* D) {
  const int ns = h.cum_ns, N = h.N;
  const int tpr = threads_per_row(ns);
  const size_t chain_smem = (size_t)2 * ns * sizeof(double) + (size_t)2 * ns * sizeof(T);
  k_cum_chain<true, T><<<kCumCluster, kCumThreads, chain_smem, st>>>(M, ns, N, tpr, x);
  k_cum_diag<T><<<N, kCumThreads, (size_t)2 * ns * sizeof(T), st>>>(Linv, D, ns, x);
  k_cum_chain<false, T><<<kCumCluster, kCumThreads, chain_smem, st>>>(Mt, ns, N, tpr, x);
  h.launches += 3;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cum_factor(Handle& h, unsigned long long* counters, cudaStream_t st, bool f32) {
  if (f32)
    return cum_factor_in<float>(h, counters, st, h.cum_Q32, h.cum_QY32, h.cum_Linv32, h.cum_M32, h.cum_Mt32,
                                h.cum_D32);
  return cum_factor_in<double>(h, counters, st, h.cum_Q, h.cum_QY, h.cum_Linv, h.cum_M, h.cum_Mt, h.cum_D);
}

// ---- solve: x = S^{-1} t (x and t may be the same array) ----

cudaError_t launch_cum_solve(Handle& h, const double* t, double* x, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (x != t) e = cudaMemcpyAsync(x, t, sizeof(double) * (size_t)h.nC, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  if (h.s_factor == 1) return cum_solve_in<float>(h, x, st, h.cum_Linv32, h.cum_M32, h.cum_Mt32, h.cum_D32);
  return cum_solve_in<double>(h, x, st, h.cum_Linv, h.cum_M, h.cum_Mt, h.cum_D);
}

}  // namespace kkt

using namespace kkt;

extern "C" kkt_status kkt_schur_blocks(kkt_handle* hh, double* Sd, double* So, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !Sd || (!So && h->N > 1)) {
    set_error("kkt_schur_blocks: null argument");
    return KKT_ERR_INVALID;
  }
  if (!h->cum) {
    set_error("kkt_schur_blocks: the handle has no structured S (structured_s = 2)");
    return KKT_ERR_INVALID;
  }
  if (!h->factored) {
    set_error("kkt_schur_blocks: no factorization");
    return KKT_ERR_STATE;
  }
  const size_t nn = (size_t)h->cum_ns * h->cum_ns;
  cudaStream_t st = (cudaStream_t)stream;
  KKT_CUDA(cudaMemcpyAsync(Sd, h->cum_Sd, sizeof(double) * nn * h->N, cudaMemcpyDeviceToDevice, st));
  if (h->N > 1)
    KKT_CUDA(cudaMemcpyAsync(So, h->cum_So, sizeof(double) * nn * (h->N - 1), cudaMemcpyDeviceToDevice, st));
  return KKT_OK;
}
