// (d) Local solves and the right-hand-side reduction (eqs. SCsolve and
// SCsolve1; Algorithm 1), plus the FP64 residual of the
// iterative refinement on the full K.
//
// One application of the factored K^{-1} to r = [r_0..r_{N-1}; r_g]:
//   z_i = L_i^{-1} P^T r_i                       (k_fsolve_level, level by level)
//   u_i = W_i^T D_i^{-1} z_i                     (k_reduce_u: E^T A_i^{-1} r_i)
//   t   = r_g - sum_i M_i^T u_i                  (k_reduce_t, block order)
//   x_g = S^{-1} t                               (dense solve)
//   z_i -= W_i (M_i x_g)                         (k_apply_xg: L^{-1} P^T B_i x_g)
//   x_i = P L_i^{-T} D_i^{-1} z_i                (k_diag_scale, k_bsolve_level)
// which is x_i = A_i^{-1} (r_i - B_i x_g).  Every output is summed by one thread
// or one warp in a fixed order.
#include "handle.h"

namespace kkt {

namespace {

__global__ void k_permute_in(const double* __restrict__ r, const int32_t* __restrict__ perm,
                             double* __restrict__ z, int nA, int N) {
  const int64_t total = (int64_t)nA * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = q / nA, kk = q - b * nA;
    z[q] = r[b * nA + perm[kk]];
  }
}

__global__ void k_permute_out(const double* __restrict__ z, const int32_t* __restrict__ perm,
                              double* __restrict__ x, int nA, int N) {
  const int64_t total = (int64_t)nA * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = q / nA, kk = q - b * nA;
    x[b * nA + perm[kk]] = z[q];
  }
}

// one warp per (supernode, block): z[cols(s)] -= sum_d L_d[rows in s] z[cols(d)];
// then the unit-lower solve with the diagonal block.
__global__ void __launch_bounds__(128) k_fsolve_level(const int32_t* __restrict__ sn_list, int nsn,
                                                      DevSym d, const double* __restrict__ Lx,
                                                      int64_t pt, double* __restrict__ z, int nA,
                                                      int N) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nsn * N) return;
  const int si = warp % nsn, b = warp / nsn;
  const int s = sn_list[si];
  const int m = (int)(d.sn_rowptr[s + 1] - d.sn_rowptr[s]);
  const int f = d.sn_first[s], w = d.sn_first[s + 1] - f;
  const double* P = Lx + b * pt + d.sn_valoff[s];
  double* zb = z + (int64_t)b * nA;
  for (int64_t u = d.upd_ptr[s]; u < d.upd_ptr[s + 1]; u++) {
    const int dd = d.upd_src[u];
    const int r0 = d.upd_r0[u], r1 = d.upd_r1[u];
    const int md = (int)(d.sn_rowptr[dd + 1] - d.sn_rowptr[dd]);
    const int fd = d.sn_first[dd], wd = d.sn_first[dd + 1] - fd;
    const double* Pd = Lx + b * pt + d.sn_valoff[dd];
    const int32_t* Rd = d.sn_rows + d.sn_rowptr[dd];
    const int j = r0 + lane;  // r1 - r0 <= w <= 32
    if (j < r1) {
      double acc = 0.0;
      for (int kk = 0; kk < wd; kk++) acc += Pd[(int64_t)kk * md + j] * zb[fd + kk];
      zb[Rd[j]] -= acc;
    }
    __syncwarp();
  }
  double zc = lane < w ? zb[f + lane] : 0.0;
  for (int c = 0; c + 1 < w; c++) {
    const double zcc = __shfl_sync(0xffffffffu, zc, c);
    if (lane > c && lane < w) zc -= P[(int64_t)c * m + lane] * zcc;
  }
  if (lane < w) zb[f + lane] = zc;
}

// Narrow levels (few supernodes x blocks): one CTA of kSolveWarps warps per
// (supernode, block).  Forward: warp w accumulates the updates u with
// u % kSolveWarps == w into its own partial vector; the partials are summed in
// warp order.  Backward: warp w owns the columns c with c % kSolveWarps == w.
constexpr int kSolveWarps = 8;
constexpr int kWideLevelWarps = 152 * 32;  // levels with fewer (supernode, block) pairs use a CTA per pair

__global__ void __launch_bounds__(kSolveWarps * 32) k_fsolve_level_wide(
    const int32_t* __restrict__ sn_list, DevSym d, const double* __restrict__ Lx, int64_t pt,
    double* __restrict__ z, int nA) {
  __shared__ double part[kSolveWarps][32];
  const int s = sn_list[blockIdx.x], b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = (int)(d.sn_rowptr[s + 1] - d.sn_rowptr[s]);
  const int f = d.sn_first[s], w = d.sn_first[s + 1] - f;
  const double* P = Lx + b * pt + d.sn_valoff[s];
  double* zb = z + (int64_t)b * nA;
  double mine = 0.0;  // partial for row f + lane of this warp's updates
  for (int64_t u = d.upd_ptr[s] + warp; u < d.upd_ptr[s + 1]; u += kSolveWarps) {
    const int dd = d.upd_src[u];
    const int r0 = d.upd_r0[u], r1 = d.upd_r1[u];
    const int md = (int)(d.sn_rowptr[dd + 1] - d.sn_rowptr[dd]);
    const int fd = d.sn_first[dd], wd = d.sn_first[dd + 1] - fd;
    const double* Pd = Lx + b * pt + d.sn_valoff[dd];
    const int32_t* Rd = d.sn_rows + d.sn_rowptr[dd];
    // lane j handles row r0 + j of d; its target is row Rd[r0 + j] - f of s
    double acc = 0.0;
    const int j = r0 + lane;
    if (j < r1)
      for (int kk = 0; kk < wd; kk++) acc += Pd[(int64_t)kk * md + j] * zb[fd + kk];
    const int tgt = j < r1 ? Rd[j] - f : -1;
    // route acc to the lane owning its target row (targets are distinct within an update)
    for (int src = 0; src < r1 - r0; src++) {
      const double v = __shfl_sync(0xffffffffu, acc, src);
      const int tg = __shfl_sync(0xffffffffu, tgt, src);
      if (lane == tg) mine += v;
    }
  }
  part[warp][lane] = mine;
  __syncthreads();
  if (warp == 0) {
    double zc = 0.0;
    if (lane < w) {
      double sum = 0.0;
      for (int q = 0; q < kSolveWarps; q++) sum += part[q][lane];
      zc = zb[f + lane] - sum;
    }
    for (int c = 0; c + 1 < w; c++) {
      const double zcc = __shfl_sync(0xffffffffu, zc, c);
      if (lane > c && lane < w) zc -= P[(int64_t)c * m + lane] * zcc;
    }
    if (lane < w) zb[f + lane] = zc;
  }
}

__global__ void __launch_bounds__(kSolveWarps * 32) k_bsolve_level_wide(
    const int32_t* __restrict__ sn_list, DevSym d, const double* __restrict__ Lx, int64_t pt,
    double* __restrict__ z, int nA) {
  __shared__ double dots[32];
  const int s = sn_list[blockIdx.x], b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = (int)(d.sn_rowptr[s + 1] - d.sn_rowptr[s]);
  const int f = d.sn_first[s], w = d.sn_first[s + 1] - f;
  const double* P = Lx + b * pt + d.sn_valoff[s];
  const int32_t* R = d.sn_rows + d.sn_rowptr[s];
  double* zb = z + (int64_t)b * nA;
  for (int c = warp; c < w; c += kSolveWarps) {
    const double* col = P + (int64_t)c * m;
    double acc = 0.0;
    for (int r = w + lane; r < m; r += 32) acc += col[r] * zb[R[r]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) dots[c] = acc;
  }
  __syncthreads();
  if (warp == 0) {
    double mine = lane < w ? zb[f + lane] - dots[lane] : 0.0;
    for (int c = w - 1; c >= 0; c--) {
      const double xc = __shfl_sync(0xffffffffu, mine, c);
      if (lane < c) mine -= P[(int64_t)lane * m + c] * xc;
    }
    if (lane < w) zb[f + lane] = mine;
  }
}

// z /= D (D from the panel diagonals)
__global__ void k_diag_scale(const int64_t* __restrict__ col_dpos, const double* __restrict__ Lx,
                             int64_t pt, double* __restrict__ z, int nA, int N) {
  const int64_t total = (int64_t)nA * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = q / nA, j = q - b * nA;
    z[q] /= Lx[b * pt + col_dpos[j]];
  }
}

// one warp per (supernode, block), top-down:
// x[cols(s)] = L_ss^{-T} (y[cols(s)] - L_off^T x[offrows(s)])
__global__ void __launch_bounds__(128) k_bsolve_level(const int32_t* __restrict__ sn_list, int nsn,
                                                      DevSym d, const double* __restrict__ Lx,
                                                      int64_t pt, double* __restrict__ z, int nA,
                                                      int N) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nsn * N) return;
  const int si = warp % nsn, b = warp / nsn;
  const int s = sn_list[si];
  const int m = (int)(d.sn_rowptr[s + 1] - d.sn_rowptr[s]);
  const int f = d.sn_first[s], w = d.sn_first[s + 1] - f;
  const double* P = Lx + b * pt + d.sn_valoff[s];
  const int32_t* R = d.sn_rows + d.sn_rowptr[s];
  double* zb = z + (int64_t)b * nA;
  double mine = lane < w ? zb[f + lane] : 0.0;
  for (int c = 0; c < w; c++) {
    const double* col = P + (int64_t)c * m;
    double acc = 0.0;
    for (int r = w + lane; r < m; r += 32) acc += col[r] * zb[R[r]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == c) mine -= acc;
  }
  for (int c = w - 1; c >= 0; c--) {
    const double xc = __shfl_sync(0xffffffffu, mine, c);
    if (lane < c) mine -= P[(int64_t)lane * m + c] * xc;
  }
  if (lane < w) zb[f + lane] = mine;
}

// u_b[t] = sum_rho W_b[rho][t] z_b[w_col[rho]] / D[rho]; one CTA per (block,
// 32 columns): warp w sums the rows rho = w mod 8, the 8 partials are added in
// warp order.
__global__ void __launch_bounds__(256) k_reduce_u(const double* __restrict__ W, const double* __restrict__ z,
                                                  const double* __restrict__ wdinv,
                                                  const int32_t* __restrict__ w_col, int nw, int k, int nA,
                                                  double* __restrict__ u) {
  __shared__ double part[8][32];
  const int b = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 32 + lane;
  const double* Wb = W + (int64_t)b * nw * k;
  const double* zb = z + (int64_t)b * nA;
  const double* db = wdinv + (int64_t)b * nw;
  double acc = 0.0;
  if (t < k)
    for (int rho = warp; rho < nw; rho += 8) acc += Wb[(int64_t)rho * k + t] * (zb[w_col[rho]] * db[rho]);
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && t < k) {
    double sum = 0.0;
    for (int q = 0; q < 8; q++) sum += part[q][lane];
    u[(int64_t)b * k + t] = sum;
  }
}

// t[c] = r_g[c] - sum_{e in column c} b[e] u[block(e)][t(e)]
__global__ void k_reduce_t(const double* __restrict__ rg, const int32_t* __restrict__ t_ptr,
                           const int32_t* __restrict__ t_e, const int32_t* __restrict__ e_t,
                           const int32_t* __restrict__ e_block, const double* __restrict__ b_vals,
                           const double* __restrict__ u, int k, int nC, double* __restrict__ tg) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nC) return;
  double acc = rg[c];
  for (int q = t_ptr[c]; q < t_ptr[c + 1]; q++) {
    const int e = t_e[q];
    acc -= b_vals[e] * u[(int64_t)e_block[e] * k + e_t[e]];
  }
  tg[c] = acc;
}

// v_b[t] = sum_{e in block b, index t} b[e] x_g[col(e)]
__global__ void k_mx(const int32_t* __restrict__ bt_ptr, const int32_t* __restrict__ b_col,
                     const double* __restrict__ b_vals, const double* __restrict__ xg, int k, int N,
                     double* __restrict__ v) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= k * N) return;
  const int b = q / k, t = q - b * k;
  const int32_t* bp = bt_ptr + (int64_t)b * (k + 1);
  double acc = 0.0;
  for (int e = bp[t]; e < bp[t + 1]; e++) acc += b_vals[e] * xg[b_col[e]];
  v[q] = acc;
}

// z_b[w_col[rho]] -= sum_t W_b[rho][t] v_b[t]
__global__ void k_apply_xg(const double* __restrict__ W, const double* __restrict__ v,
                           const int32_t* __restrict__ w_col, int nw, int k, int nA, int N,
                           double* __restrict__ z) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= (int64_t)nw * N) return;
  const int b = (int)(q / nw), rho = (int)(q - (int64_t)b * nw);
  const double* Wr = W + ((int64_t)b * nw + rho) * k;
  const double* vb = v + (int64_t)b * k;
  double acc = 0.0;
  for (int t = 0; t < k; t++) acc += Wr[t] * vb[t];
  z[(int64_t)b * nA + w_col[rho]] -= acc;
}

// ---- residual rho = r - K x ----

__global__ void k_resid_blocks(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ src, const double* __restrict__ a_vals,
                               int64_t nnzA, const double* __restrict__ r, const double* __restrict__ x,
                               double* __restrict__ rho, int nA, int N) {
  const int64_t total = (int64_t)nA * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = q / nA;
    const int row = (int)(q - b * nA);
    const double* a = a_vals + b * nnzA;
    const double* xb = x + b * nA;
    double acc = 0.0;
    for (int p = rowptr[row]; p < rowptr[row + 1]; p++) acc += a[src[p]] * xb[col[p]];
    rho[q] = r[q] - acc;
  }
}

// rows of E: subtract B_i x_g
__global__ void k_resid_b(const int32_t* __restrict__ bt_ptr, const int32_t* __restrict__ b_row,
                          const int32_t* __restrict__ b_col, const double* __restrict__ b_vals,
                          const double* __restrict__ xg, int k, int nA, int N,
                          double* __restrict__ rho) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= k * N) return;
  const int b = q / k, t = q - b * k;
  const int32_t* bp = bt_ptr + (int64_t)b * (k + 1);
  if (bp[t] == bp[t + 1]) return;
  double acc = 0.0;
  for (int e = bp[t]; e < bp[t + 1]; e++) acc += b_vals[e] * xg[b_col[e]];
  rho[(int64_t)b * nA + b_row[bp[t]]] -= acc;
}

// coupling rows: rho_g = r_g - sum_i B_i^T x_i - C x_g
__global__ void k_resid_g(const int32_t* __restrict__ t_ptr, const int32_t* __restrict__ t_e,
                          const int32_t* __restrict__ e_block, const int32_t* __restrict__ b_row,
                          const double* __restrict__ b_vals, const double* __restrict__ c_vals,
                          int c_kind, const double* __restrict__ r, const double* __restrict__ x,
                          int nA, int N, int nC, double* __restrict__ rho) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nC) return;
  const int64_t g = (int64_t)N * nA;
  double acc = 0.0;
  for (int q = t_ptr[c]; q < t_ptr[c + 1]; q++) {
    const int e = t_e[q];
    acc += b_vals[e] * x[(int64_t)e_block[e] * nA + b_row[e]];
  }
  if (c_kind == 0) {
    acc += c_vals[c] * x[g + c];
  } else {
    for (int c2 = 0; c2 < nC; c2++) {
      const double cv = c2 <= c ? c_vals[(int64_t)c * nC + c2] : c_vals[(int64_t)c2 * nC + c];
      acc += cv * x[g + c2];
    }
  }
  rho[g + c] = r[g + c] - acc;
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns; a NaN with a clear
  // sign bit orders above +Inf, so it survives the maximum
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// max(a, b) that keeps a NaN of either argument (fmax drops it), so that a
// non-finite entry reaches the norm and the convergence test sees it
__device__ __forceinline__ double max_keep_nan(double a, double b) { return (a > b || a != a) ? a : b; }

// red[0] = ||a||_inf, red[1] = ||b||_inf, red[2] = ||c||_inf; NaN if an entry is NaN
__global__ void k_norms3(const double* __restrict__ a, const double* __restrict__ b,
                         const double* __restrict__ c, int64_t n, double* __restrict__ red) {
  __shared__ double sh[3][256];
  double m0 = 0, m1 = 0, m2 = 0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    m0 = max_keep_nan(m0, fabs(a[q]));
    m1 = max_keep_nan(m1, fabs(b[q]));
    m2 = max_keep_nan(m2, fabs(c[q]));
  }
  sh[0][threadIdx.x] = m0;
  sh[1][threadIdx.x] = m1;
  sh[2][threadIdx.x] = m2;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 3; k++) sh[k][threadIdx.x] = max_keep_nan(sh[k][threadIdx.x], sh[k][threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; k++) atomic_max_nonneg(&red[k], sh[k][0]);
}

// ||K||_inf: row sums of |K| (NaN if an entry of A or B is NaN)
__global__ void k_knorm_blocks(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ src,
                               const double* __restrict__ a_vals, int64_t nnzA,
                               const int32_t* __restrict__ bt_ptr, const int32_t* __restrict__ b_row,
                               const double* __restrict__ b_vals, const int32_t* __restrict__ E,
                               int k, int nA, int N, double* __restrict__ out) {
  const int64_t total = (int64_t)nA * N;
  double m = 0.0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = q / nA;
    const int row = (int)(q - b * nA);
    const double* a = a_vals + b * nnzA;
    double acc = 0.0;
    for (int p = rowptr[row]; p < rowptr[row + 1]; p++) acc += fabs(a[src[p]]);
    m = max_keep_nan(m, acc);
  }
  // rows of E also carry B's entries
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)k * N;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(q / k), t = (int)(q - (int64_t)b * k);
    const int32_t* bp = bt_ptr + (int64_t)b * (k + 1);
    if (bp[t] == bp[t + 1]) continue;
    const double* a = a_vals + (int64_t)b * nnzA;
    const int row = E[t];
    double acc = 0.0;
    for (int p = rowptr[row]; p < rowptr[row + 1]; p++) acc += fabs(a[src[p]]);
    for (int e = bp[t]; e < bp[t + 1]; e++) acc += fabs(b_vals[e]);
    m = max_keep_nan(m, acc);
  }
  atomic_max_nonneg(out, m);
}

__global__ void k_knorm_g(const int32_t* __restrict__ t_ptr, const int32_t* __restrict__ t_e,
                          const double* __restrict__ b_vals, const double* __restrict__ c_vals,
                          int c_kind, int nC, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nC) return;
  double acc = 0.0;
  for (int q = t_ptr[c]; q < t_ptr[c + 1]; q++) acc += fabs(b_vals[t_e[q]]);
  if (c_kind == 0) {
    acc += fabs(c_vals[c]);
  } else {
    for (int c2 = 0; c2 < nC; c2++)
      acc += fabs(c2 <= c ? c_vals[(int64_t)c * nC + c2] : c_vals[(int64_t)c2 * nC + c]);
  }
  atomic_max_nonneg(out, acc);
}

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    y[q] += x[q];
}

// Deterministic dot products (a fixed reduction order for a given n): each
// of kDotBlocks CTAs sums a strided part of the vectors in a fixed order and
// reduces it by a tree; one CTA adds the partial sums by a tree.
constexpr int kDotBlocks = 512;

__global__ void __launch_bounds__(256) k_dot_partial(const double* __restrict__ a, const double* __restrict__ b,
                                                     int64_t n, double* __restrict__ partial) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    acc += a[q] * b[q];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kDotBlocks) k_dot_final(const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sh[kDotBlocks];
  sh[threadIdx.x] = partial[threadIdx.x];
  __syncthreads();
  for (int s = kDotBlocks / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

// y += a x
__global__ void k_axpby(double* __restrict__ y, double a, const double* __restrict__ x, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    y[q] += a * x[q];
}

// y = a x
__global__ void k_scale_into(double* __restrict__ y, double a, const double* __restrict__ x, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    y[q] = a * x[q];
}

inline int grid_for(int64_t n, int bs = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + bs - 1) / bs, 152 * 16));
}

}  // namespace

// The application is split where it first needs the factor of S: the front
// (forward block solves and right-hand-side reduction) needs only the block
// factors and W; the back does the rest.
cudaError_t launch_apply_front(Handle& h, const double* r, cudaStream_t st) {
  const int nA = h.nA, N = h.N, k = h.cpl.k, nw = h.cpl.nw;
  const int64_t pt = h.sym.panel_total;
  const int64_t nb = (int64_t)nA * N;
  {
    k_permute_in<<<grid_for(nb), 256, 0, st>>>(r, h.d.perm, h.z, nA, N);
    h.launches++;
  }
  // with a dense tail, the levels cover the supernodes outside it and the
  // tail's triangular solves are dense (the tail factor's triangles)
  const bool tail = h.nT > 0;
  const std::vector<int32_t>& lptr = tail ? h.flvl_ptr : h.lvl_ptr;
  const int32_t* lsn = tail ? h.d.flvl_sn : h.d.lvl_sn;
  for (int l = 0; l < h.sym.nlevels; l++) {
    const int s0 = lptr[l], nsn = lptr[l + 1] - s0;
    if (nsn == 0) continue;
    const int warps = nsn * N;
    if (warps < kWideLevelWarps) {
      k_fsolve_level_wide<<<dim3(nsn, N), kSolveWarps * 32, 0, st>>>(lsn + s0, h.d, h.Lx, pt, h.z, nA);
    } else {
      k_fsolve_level<<<(warps + 3) / 4, 128, 0, st>>>(lsn + s0, nsn, h.d, h.Lx, pt, h.z, nA, N);
    }
    h.launches++;
  }
  if (tail) {
    cudaError_t e = launch_tail_fsolve(h, h.z, st);
    if (e != cudaSuccess) return e;
  }
  if (h.nC > 0) {
    if (k > 0 && nw > 0) {
      dim3 g((k + 31) / 32, N);
      {
    k_reduce_u<<<g, 256, 0, st>>>(h.W, h.z, h.wdinv, h.d.w_col, nw, k, nA, h.u);
    h.launches++;
  }
    } else if (k > 0) {
      cudaMemsetAsync(h.u, 0, sizeof(double) * (size_t)k * N, st);
    }
    {
    k_reduce_t<<<(h.nC + 255) / 256, 256, 0, st>>>(r + nb, h.d.t_ptr, h.d.t_e, h.d.e_t, h.d.e_block,
                                                   h.b_vals, h.u, k, h.nC, h.tg);
    h.launches++;
  }
  }
  return cudaGetLastError();
}

cudaError_t launch_apply_back(Handle& h, double* out, cudaStream_t st, bool solve_s) {
  const int nA = h.nA, N = h.N, k = h.cpl.k, nw = h.cpl.nw;
  const int64_t pt = h.sym.panel_total;
  const int64_t nb = (int64_t)nA * N;
  const bool tail = h.nT > 0;
  const std::vector<int32_t>& lptr = tail ? h.flvl_ptr : h.lvl_ptr;
  const int32_t* lsn = tail ? h.d.flvl_sn : h.d.lvl_sn;
  if (h.nC > 0) {
    // without solve_s, h.xg already holds x_g (a sharded solve's broadcast)
    cudaError_t e = !solve_s ? cudaSuccess
                    : h.cum     ? launch_cum_solve(h, h.tg, h.xg, st)
                    : (h.s_factor == 1 ? launch_dense_solve_f32(h, h.tg, h.xg, st)
                                       : launch_dense_solve(h, h.tg, h.xg, st));
    if (e != cudaSuccess) return e;
    if (k > 0 && nw > 0) {
      {
    k_mx<<<(k * N + 255) / 256, 256, 0, st>>>(h.d.bt_ptr, h.d.b_col, h.b_vals, h.xg, k, N, h.v);
    h.launches++;
  }
      {
    k_apply_xg<<<grid_for((int64_t)nw * N), 256, 0, st>>>(h.W, h.v, h.d.w_col, nw, k, nA, N, h.z);
    h.launches++;
  }
    }
  }
  {
    k_diag_scale<<<grid_for(nb), 256, 0, st>>>(h.d.col_dpos, h.Lx, pt, h.z, nA, N);
    h.launches++;
  }
  if (tail) {
    cudaError_t e = launch_tail_bsolve(h, h.z, st);
    if (e != cudaSuccess) return e;
  }
  for (int l = h.sym.nlevels - 1; l >= 0; l--) {
    const int s0 = lptr[l], nsn = lptr[l + 1] - s0;
    if (nsn == 0) continue;
    const int warps = nsn * N;
    if (warps < kWideLevelWarps) {
      k_bsolve_level_wide<<<dim3(nsn, N), kSolveWarps * 32, 0, st>>>(lsn + s0, h.d, h.Lx, pt, h.z, nA);
    } else {
      k_bsolve_level<<<(warps + 3) / 4, 128, 0, st>>>(lsn + s0, nsn, h.d, h.Lx, pt, h.z, nA, N);
    }
    h.launches++;
  }
  {
    k_permute_out<<<grid_for(nb), 256, 0, st>>>(h.z, h.d.perm, out, nA, N);
    h.launches++;
  }
  if (h.nC > 0)
    cudaMemcpyAsync(out + nb, h.xg, sizeof(double) * h.nC, cudaMemcpyDeviceToDevice, st);
  return cudaGetLastError();
}

cudaError_t launch_apply_inverse(Handle& h, const double* r, double* out, cudaStream_t st) {
  cudaError_t e = launch_apply_front(h, r, st);
  return e != cudaSuccess ? e : launch_apply_back(h, out, st);
}

cudaError_t launch_residual(Handle& h, const double* r, const double* x, double* rho, cudaStream_t st) {
  const int nA = h.nA, N = h.N, k = h.cpl.k;
  const int64_t nb = (int64_t)nA * N;
  {
    k_resid_blocks<<<grid_for(nb), 256, 0, st>>>(h.d.full_rowptr, h.d.full_col, h.d.full_src, h.a_vals,
                                               h.nnzA, r, x, rho, nA, N);
    h.launches++;
  }
  if (h.nC > 0) {
    if (k > 0)
      {
    k_resid_b<<<(k * N + 255) / 256, 256, 0, st>>>(h.d.bt_ptr, h.d.b_row, h.d.b_col, h.b_vals,
                                                     x + nb, k, nA, N, rho);
    h.launches++;
  }
    {
    k_resid_g<<<(h.nC + 255) / 256, 256, 0, st>>>(h.d.t_ptr, h.d.t_e, h.d.e_block, h.d.b_row, h.b_vals,
                                                  h.c_vals, h.c_kind, r, x, nA, N, h.nC, rho);
    h.launches++;
  }
  }
  return cudaGetLastError();
}

cudaError_t launch_knorm(Handle& h, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(h.knorm, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  const int64_t nb = (int64_t)h.nA * h.N;
  {
    k_knorm_blocks<<<grid_for(nb), 256, 0, st>>>(h.d.full_rowptr, h.d.full_src, h.a_vals, h.nnzA,
                                               h.d.bt_ptr, h.d.b_row, h.b_vals, h.d.E, h.cpl.k,
                                               h.nA, h.N, h.knorm);
    h.launches++;
  }
  if (h.nC > 0)
    {
    k_knorm_g<<<(h.nC + 255) / 256, 256, 0, st>>>(h.d.t_ptr, h.d.t_e, h.b_vals, h.c_vals, h.c_kind,
                                                  h.nC, h.knorm);
    h.launches++;
  }
  return cudaGetLastError();
}

cudaError_t launch_axpy(Handle& h, double* y, const double* x, int64_t n, cudaStream_t st) {
  {
    k_axpy<<<grid_for(n), 256, 0, st>>>(y, x, n);
    h.launches++;
  }
  return cudaGetLastError();
}

cudaError_t launch_norms(Handle& h, const double* rho, const double* x, const double* rhs,
                         cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(h.red, 0, sizeof(double) * 3, st);
  if (e != cudaSuccess) return e;
  const int64_t nK = (int64_t)h.nA * h.N + h.nC;
  {
    k_norms3<<<grid_for(nK), 256, 0, st>>>(rho, x, rhs, nK, h.red);
    h.launches++;
  }
  return cudaGetLastError();
}

cudaError_t launch_dot(Handle& h, const double* a, const double* b, int64_t n, double* out, cudaStream_t st) {
  k_dot_partial<<<kDotBlocks, 256, 0, st>>>(a, b, n, h.red + 16);
  k_dot_final<<<1, kDotBlocks, 0, st>>>(h.red + 16, out);
  h.launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_axpby(Handle& h, double* y, double a, const double* x, int64_t n, cudaStream_t st) {
  k_axpby<<<grid_for(n), 256, 0, st>>>(y, a, x, n);
  h.launches++;
  return cudaGetLastError();
}

cudaError_t launch_scale_into(Handle& h, double* y, double a, const double* x, int64_t n, cudaStream_t st) {
  k_scale_into<<<grid_for(n), 256, 0, st>>>(y, a, x, n);
  h.launches++;
  return cudaGetLastError();
}

cudaError_t launch_apply_inverse_ws(Handle& h, const double* r, double* out,
                                    const SolveWorkspace& ws, cudaStream_t st) {
  const int nA = h.nA, N = h.N, k = h.cpl.k, nw = h.cpl.nw;
  const int64_t pt = h.sym.panel_total;
  const int64_t nb = (int64_t)nA * N;
  k_permute_in<<<grid_for(nb), 256, 0, st>>>(r, h.d.perm, ws.z, nA, N);
  h.launches++;
  for (int l = 0; l < h.sym.nlevels; l++) {
    const int s0 = h.lvl_ptr[l], nsn = h.lvl_ptr[l + 1] - s0;
    const int warps = nsn * N;
    k_fsolve_level<<<(warps + 3) / 4, 128, 0, st>>>(h.d.lvl_sn + s0, nsn, h.d, h.Lx, pt, ws.z, nA, N);
    h.launches++;
  }
  if (h.nC > 0) {
    if (k > 0 && nw > 0) {
      dim3 g((k + 31) / 32, N);
      k_reduce_u<<<g, 256, 0, st>>>(h.W, ws.z, h.wdinv, h.d.w_col, nw, k, nA, ws.u);
      h.launches++;
    } else if (k > 0) {
      cudaError_t e = cudaMemsetAsync(ws.u, 0, sizeof(double) * (size_t)k * N, st);
      if (e != cudaSuccess) return e;
    }
    k_reduce_t<<<(h.nC + 255) / 256, 256, 0, st>>>(r + nb, h.d.t_ptr, h.d.t_e, h.d.e_t, h.d.e_block,
                                                   h.b_vals, ws.u, k, h.nC, ws.tg);
    h.launches++;
    cudaError_t e = h.cum ? launch_cum_solve(h, ws.tg, ws.xg, st) : launch_dense_solve_ws(h, ws.tg, ws.xg, ws.dot, st);
    if (e != cudaSuccess) return e;
    if (k > 0 && nw > 0) {
      k_mx<<<(k * N + 255) / 256, 256, 0, st>>>(h.d.bt_ptr, h.d.b_col, h.b_vals, ws.xg, k, N, ws.v);
      k_apply_xg<<<grid_for((int64_t)nw * N), 256, 0, st>>>(h.W, ws.v, h.d.w_col, nw, k, nA, N, ws.z);
      h.launches += 2;
    }
  }
  k_diag_scale<<<grid_for(nb), 256, 0, st>>>(h.d.col_dpos, h.Lx, pt, ws.z, nA, N);
  h.launches++;
  for (int l = h.sym.nlevels - 1; l >= 0; l--) {
    const int s0 = h.lvl_ptr[l], nsn = h.lvl_ptr[l + 1] - s0;
    const int warps = nsn * N;
    k_bsolve_level<<<(warps + 3) / 4, 128, 0, st>>>(h.d.lvl_sn + s0, nsn, h.d, h.Lx, pt, ws.z, nA, N);
    h.launches++;
  }
  k_permute_out<<<grid_for(nb), 256, 0, st>>>(ws.z, h.d.perm, out, nA, N);
  h.launches++;
  if (h.nC > 0) {
    cudaError_t e = cudaMemcpyAsync(out + nb, ws.xg, sizeof(double) * h.nC, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace kkt
