// (a) Dense tail of the block factors.
//
// The last supernodes of the postorder (the top of the elimination tree) have
// row sets inside the tail columns [c_T, n) and are nearly dense there, so the
// tail of every block is factored as one dense nT x nT lower triangle
// (nT = n - c_T) instead of supernode by supernode: the work is the same
// LDL^T (Algorithm 1's block factorization) with the explicit zeros of the
// tail included, done by the blocked dense kernels that factor S
// (dense_kernels.cuh), batched over the N blocks.
//
// Per factor: the tail panels (A's values plus the updates from outside the
// tail, applied by the level loop) are gathered into the zeroed dense
// triangles; each 64-wide panel step factors the diagonal blocks of all N
// triangles (with the static-pivot rule and the inertia counts of the sparse
// panels), forms L21 and Y = L21 D, and updates the trailing triangles, in
// FP64 on the CUDA cores (tail mode 1) or in emulated FP64 on the tensor cores
// (tail mode 2, the update of dense_tc.cu: 7 base-256 digit slices per
// operand); the factor is scattered back into the supernodal panels, which
// the solves use.
// Entries of the triangles outside the supernodal structure stay exact zeros
// (every product that reaches them has a zero factor).
//
// Augmented tail: each triangle gets k more rows, Z^T, where Z holds the
// tail's rows of P^T E - L_{T,rest} W_rest (the right-hand sides of W after
// the updates from outside the tail; zero rows for tail columns outside the
// reach of E).  Factoring only the nT tail pivots of [T Z; Z^T 0] is the
// incomplete factorization of Sec. 4.2 (eq. augmented) restricted to the tail:
// the augmented rows become W_T^T D_T^{-1} with W_T = L_T^{-1} Z, and the
// trailing k x k block becomes -W_T^T D_T^{-1} W_T, the tail's share of G.  So
// the tail's W solve and contraction run inside the tail factor.
#include <cooperative_groups.h>

#include "dense_kernels.cuh"

namespace kkt {

namespace cg = cooperative_groups;

namespace {

// panels of the tail supernodes <-> dense triangles (order nTa, the first nT
// columns), lower part only
template <bool TO_DENSE>
__global__ void __launch_bounds__(256) k_tail_move(DevSym d, double* __restrict__ Lx, int64_t pt,
                                                   double* __restrict__ T, int nTa, int tail_col,
                                                   int tail_sn) {
  const int s = tail_sn + blockIdx.x, b = blockIdx.y;
  const int m = (int)(d.sn_rowptr[s + 1] - d.sn_rowptr[s]);
  const int f = d.sn_first[s], w = d.sn_first[s + 1] - f;
  double* P = Lx + b * pt + d.sn_valoff[s];
  const int32_t* R = d.sn_rows + d.sn_rowptr[s];
  double* Tb = T + (int64_t)b * nTa * nTa;
  for (int q = threadIdx.x; q < m * w; q += blockDim.x) {
    const int c = q / m, i = q - c * m;
    const int row = R[i], col = f + c;
    if (row < col) continue;  // strictly upper part of the diagonal block: unused
    double* t = Tb + (int64_t)(row - tail_col) + (int64_t)(col - tail_col) * nTa;
    if (TO_DENSE) *t = P[q];
    else P[q] = *t;
  }
}

// Augmented rows: T_b[nT + t][j] = Z_b[j][t] (tail column j's W row before
// the tail solve; zero for a column outside the reach of E), and after the
// factor the tail's W rows from them: row nT + t of the factor holds
// (W_T^T D_T^{-1})[t][j], so W_b[row(j)][t] = T_b[nT + t][j] * D_j.
template <bool TO_DENSE>
__global__ void k_tail_aug_rows(double* __restrict__ W, int nw, int k, double* __restrict__ T, int nT,
                                int nTa, const int32_t* __restrict__ wrow) {
  const int b = blockIdx.y;
  double* Tb = T + (int64_t)b * nTa * nTa;
  double* Wb = W + (int64_t)b * nw * k;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nT * k; q += gridDim.x * blockDim.x) {
    const int j = q / k, t = q - j * k;
    const int r = wrow[j];
    if (r < 0) continue;
    double* a = Tb + (int64_t)(nT + t) + (int64_t)j * nTa;
    if (TO_DENSE) *a = Wb[(int64_t)r * k + t];
    else Wb[(int64_t)r * k + t] = *a * Tb[(int64_t)j + (int64_t)j * nTa];
  }
}

// Forward solve, the tail's share: z[cols(s)] -= sum over descendants d
// outside the tail of L_d[rows in s] z[cols(d)], for every tail supernode s
// (independent of one another; the triangular solve is the dense tail's).
// One CTA of 8 warps per (tail supernode, block), warp w taking the updates
// u = w mod 8, the partials added in warp order.
__global__ void __launch_bounds__(256) k_tail_fgather(DevSym d, const double* __restrict__ Lx, int64_t pt,
                                                      double* __restrict__ z, int nA, int tail_sn) {
  __shared__ double part[8][32];
  const int s = tail_sn + blockIdx.x, b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f = d.sn_first[s], w = d.sn_first[s + 1] - f;
  double* zb = z + (int64_t)b * nA;
  double mine = 0.0;
  const int64_t u0 = d.upd_ptr[s], u1 = u0 + d.upd_ntail[s];
  for (int64_t u = u0 + warp; u < u1; u += 8) {
    const int dd = d.upd_src[u];
    const int r0 = d.upd_r0[u], r1 = d.upd_r1[u];
    const int md = (int)(d.sn_rowptr[dd + 1] - d.sn_rowptr[dd]);
    const int fd = d.sn_first[dd], wd = d.sn_first[dd + 1] - fd;
    const double* Pd = Lx + b * pt + d.sn_valoff[dd];
    const int32_t* Rd = d.sn_rows + d.sn_rowptr[dd];
    double acc = 0.0;
    const int j = r0 + lane;
    if (j < r1)
      for (int kk = 0; kk < wd; kk++) acc += Pd[(int64_t)kk * md + j] * zb[fd + kk];
    const int tgt = j < r1 ? Rd[j] - f : -1;
    for (int src = 0; src < r1 - r0; src++) {  // targets are distinct within an update
      const double v = __shfl_sync(0xffffffffu, acc, src);
      const int tg = __shfl_sync(0xffffffffu, tgt, src);
      if (lane == tg) mine += v;
    }
  }
  part[warp][lane] = mine;
  __syncthreads();
  if (warp == 0 && lane < w) {
    double sum = 0.0;
    for (int q = 0; q < 8; q++) sum += part[q][lane];
    zb[f + lane] -= sum;
  }
}

// Dense triangular solves of the tails in 64-row steps with the
// diagonal-block inverses X_t.  Forward (L_T y = z): y_t = X_t z_t, then the
// rows below take z_i -= L_it y_t.  Backward (L_T^T x = y): x_t = X_t^T y_t,
// then the rows above take y_i -= L_ti^T x_t.  zt points at the tail's first
// entry of block 0 (blocks nA apart).
//
// A cluster of kTrsvCluster CTAs per block: the 64-row blocks of the tail are
// owned cyclically (block u by CTA u mod kTrsvCluster), each CTA updates only
// its own rows, and the CTAs meet at one hardware cluster barrier per step,
// after which the owner's z_t is complete; every CTA reads it from L2 and
// forms X_t z_t itself.  The owner keeps that solution block and stores it
// after the next barrier, when every CTA has read z_t.  The FP64 work of a tail
// thus spreads over several SMs, and a batch of N tails over N x kTrsvCluster
// CTAs, which also evens out N tails on 152 SMs.
constexpr int kTrsvCluster = 4;

template <bool FORWARD>
__global__ void __cluster_dims__(kTrsvCluster, 1, 1) __launch_bounds__(256)
    k_tail_trsv(const double* __restrict__ T, int nT, int nTa, const double* __restrict__ X,
                double* __restrict__ zt, int nA) {
  __shared__ double v[64];
  __shared__ double pend[64];  // the solution of the block this CTA owns, stored a step later
  __shared__ double part[4][64];
  cg::cluster_group cluster = cg::this_cluster();
  int pend_r0 = -1, pend_rows = 0;
  const int q = (int)cluster.block_rank();
  const int b = blockIdx.x / kTrsvCluster, tid = threadIdx.x, r = tid & 63, pid = tid >> 6;
  const int nbT = (nT + 63) / 64;
  const double* Tb = T + (int64_t)b * nTa * nTa;
  const double* Xb = X + (int64_t)b * nbT * 4096;
  double* z = zt + (int64_t)b * nA;
  for (int step = 0; step < nbT; step++) {
    const int t = FORWARD ? step : nbT - 1 - step;
    const int r0 = t * 64, rows = min(64, nT - r0);
    cluster.sync();  // the owner's updates of z_t (its own rows) are done and visible
    if (pend_r0 >= 0 && tid < pend_rows) z[pend_r0 + tid] = pend[tid];  // every CTA has read that block
    pend_r0 = -1;
    if (tid < 64) v[tid] = tid < rows ? __ldcg(z + r0 + tid) : 0.0;
    __syncthreads();
    // X_t v (forward) or X_t^T v (backward), 4 partial sums per output
    double acc = 0.0;
    const double* Xt = Xb + (int64_t)t * 4096;
#pragma unroll
    for (int c = 0; c < 16; c++)
      acc += (FORWARD ? Xt[r * 64 + pid * 16 + c] : Xt[(pid * 16 + c) * 64 + r]) * v[pid * 16 + c];
    part[pid][r] = acc;
    __syncthreads();
    if (tid < 64) {
      const double y = part[0][tid] + part[1][tid] + part[2][tid] + part[3][tid];
      v[tid] = y;
      pend[tid] = y;
    }
    if (t % kTrsvCluster == q) {
      pend_r0 = r0;
      pend_rows = rows;
    }
    __syncthreads();
    // this CTA's rows after (forward) or before (backward) block t: its blocks
    // u = q, q + kTrsvCluster, ... four at a time over the 256 threads
    const int ub = FORWARD ? t + 1 : 0, ue = FORWARD ? nbT : t;
    const int u0 = ub + ((q - ub) % kTrsvCluster + kTrsvCluster) % kTrsvCluster;
    for (int u = u0 + (tid >> 6) * kTrsvCluster; u < ue; u += 4 * kTrsvCluster) {
      const int i = u * 64 + r;
      if (i >= nT) continue;
      double a = 0.0;
      if (FORWARD) {
        for (int c = 0; c < rows; c++) a += Tb[(int64_t)i + (int64_t)(r0 + c) * nTa] * v[c];
      } else {
        for (int c = 0; c < rows; c++) a += Tb[(int64_t)(r0 + c) + (int64_t)i * nTa] * v[c];
      }
      z[i] -= a;
    }
  }
  cluster.sync();
  if (pend_r0 >= 0 && tid < pend_rows) z[pend_r0 + tid] = pend[tid];
}

}  // namespace

cudaError_t launch_tail_fsolve(Handle& h, double* z, cudaStream_t st) {
  const int nts = h.sym.nsuper - h.sym.tail_sn;
  k_tail_fgather<<<dim3(nts, h.N), 256, 0, st>>>(h.d, h.Lx, h.sym.panel_total, z, h.nA, h.sym.tail_sn);
  k_tail_trsv<true><<<h.N * kTrsvCluster, 256, 0, st>>>(h.Tt, h.nT, h.nTa, h.Xtail, z + h.sym.tail_col, h.nA);
  h.launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_tail_bsolve(Handle& h, double* z, cudaStream_t st) {
  k_tail_trsv<false><<<h.N * kTrsvCluster, 256, 0, st>>>(h.Tt, h.nT, h.nTa, h.Xtail, z + h.sym.tail_col, h.nA);
  h.launches++;
  return cudaGetLastError();
}

cudaError_t launch_dense_tail(Handle& h, cudaStream_t st) {
  const int nT = h.nT, nTa = h.nTa, N = h.N;
  const int tail_sn = h.sym.tail_sn, tail_col = h.sym.tail_col;
  const int nsn = h.sym.nsuper - tail_sn;
  const int64_t pt = h.sym.panel_total, t2 = (int64_t)nTa * nTa, ys = (int64_t)nTa * kPanelW;
  const int k = h.cpl.k, nw = h.cpl.nw;
  const dim3 agrid((int)std::min<int64_t>(((int64_t)nT * k + 255) / 256, 64), N);
  cudaError_t e = cudaMemsetAsync(h.Tt, 0, sizeof(double) * t2 * N, st);
  if (e != cudaSuccess) return e;
  k_tail_move<true><<<dim3(nsn, N), 256, 0, st>>>(h.d, h.Lx, pt, h.Tt, nTa, tail_col, tail_sn);
  h.launches++;
  if (h.tail_aug) {
    k_tail_aug_rows<true><<<agrid, 256, 0, st>>>(h.W, nw, k, h.Tt, nT, nTa, h.d.tail_wrow);
    h.launches++;
  }
  if (h.tail_mode == 2) {
    e = launch_tail_factor_emulated(h, st);
    if (e != cudaSuccess) return e;
  }
  const PivotRule rule{h.anorm, h.opt.pivot_eps, h.d.col_primal + tail_col};
  for (int k0 = 0; h.tail_mode == 1 && k0 < nT; k0 += kPanelW) {
    const int kb = std::min(kPanelW, nT - k0);
    const int kd = kt_begin(h, kFamDiag, N * (2.0 / 3.0) * kb * kb * kb, st);
    k_dense_diag_t<double><<<N, 256, 0, st>>>(h.Tt, nTa, k0, kb, t2, rule, h.counters);
    kt_end(h, kd, st);
    h.launches++;
    const int rest = nTa - k0 - kb;
    if (rest > 0) {
      launch_dense_panel<double>(h.Tt, h.TY, nTa, k0, kb, nTa, N, t2, ys, st);
      const int tiles = (rest + 63) / 64;
      const int kt = kt_begin(h, kFamDenseF64, N * update_flops(rest, 0, rest, kb), st);
      k_dense_update<<<dim3(tiles * (tiles + 1) / 2, N), 256, 0, st>>>(h.Tt, h.TY, nTa, k0, kb, nTa, t2, ys);
      kt_end(h, kt, st);
      h.launches += 2;
    }
  }
  k_tail_move<false><<<dim3(nsn, N), 256, 0, st>>>(h.d, h.Lx, pt, h.Tt, nTa, tail_col, tail_sn);
  h.launches++;
  if (h.tail_aug) {
    k_tail_aug_rows<false><<<agrid, 256, 0, st>>>(h.W, nw, k, h.Tt, nT, nTa, h.d.tail_wrow);
    h.launches++;
  }
  e = cudaGetLastError();
  return e != cudaSuccess ? e : launch_tail_inverse(h, st);
}

}  // namespace kkt
