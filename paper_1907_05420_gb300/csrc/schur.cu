// (b) Schur-complement assembly S = C - sum_i B_i^T A_i^{-1} B_i
// (eq. SCform; the Schur-complement accumulation of Algorithm 1).
//
// With E the k rows of A that carry a nonzero of some B_i, B_i = E M_i and
//     B_i^T A_i^{-1} B_i = M_i^T G_i M_i,   G_i = W_i^T D_i^{-1} W_i,
//     W_i = L_i^{-1} P^T E.
// This is the (2,2) block that the incomplete factorization of the augmented
// matrix [A_i B_i; B_i^T 0] leaves behind after A_i's last pivot (Sec. 4.2,
// eq. augmented), computed as
//   1. k_w_solve:     multi-RHS sparse forward solve, restricted to the
//                     elimination-tree reach of E (left-looking, level by level);
//   2. k_contract_g:  the contraction G_i = W_i^T D_i^{-1} W_i;
//   3. k_assemble_s:  S = C - sum_i M_i^T G_i M_i, each entry of S summed by one
//                     thread over its contributions in block order (no atomics).
#include "handle.h"

namespace kkt {

namespace {

// Column t of W is L^{-1} P^T e_{E_t}, nonzero only on the supernodes of the
// path from E_t's supernode to the root.  One CTA per (reach supernode s,
// block, chunk of 32 of s's columns T_s): s computes only those columns (its
// other entries stay zero from the clearing at analysis), and the update from
// a descendant d touches only d's columns T_d, a subset of T_s.
// TAIL_INIT: for a supernode of the augmented tail, all k columns of the
// right-hand side minus the updates from outside the tail (the rows Z the tail
// factor is augmented with); its triangular solve is the tail factor's.
constexpr int kWChunk = 32;

template <bool TAIL_INIT>
__global__ void __launch_bounds__(128) k_w_solve(const int32_t* __restrict__ sn_list, DevSym d,
                                                 const double* __restrict__ Lx, int64_t pt,
                                                 double* __restrict__ W, int nw, int k) {
  const int s = sn_list[blockIdx.x], b = blockIdx.y;
  const int32_t* Ts = d.wt_idx + d.wt_ptr[s];
  const int nts = d.wt_ptr[s + 1] - d.wt_ptr[s];
  const int c0 = blockIdx.z * kWChunk;
  if (!TAIL_INIT && c0 >= nts) return;
  const int nt = TAIL_INIT ? k : min(kWChunk, nts - c0);
  const int32_t* tc = Ts + c0;                       // this chunk's columns (sorted)
  const int lo = TAIL_INIT ? 0 : tc[0], hi = TAIL_INIT ? k - 1 : tc[nt - 1];
  const int m = (int)(d.sn_rowptr[s + 1] - d.sn_rowptr[s]);
  const int f = d.sn_first[s], w = d.sn_first[s + 1] - f;
  const int ws = d.sn_wrow[s];
  const double* P = Lx + b * pt + d.sn_valoff[s];
  double* Wb = W + (int64_t)b * nw * k;
  for (int q = threadIdx.x; q < w * nt; q += blockDim.x) {
    const int c = q / nt, jt = q - c * nt;
    const int t = TAIL_INIT ? jt : tc[jt];
    Wb[(int64_t)(ws + c) * k + t] = d.wpos[t] == ws + c ? 1.0 : 0.0;
  }
  __syncthreads();
  const int64_t u_end = TAIL_INIT ? d.upd_ptr[s] + d.upd_ntail[s] : d.upd_ptr[s + 1];
  for (int64_t u = d.upd_ptr[s]; u < u_end; u++) {
    const int dd = d.upd_src[u];
    const int wrd = d.sn_wrow[dd];
    if (wrd < 0) continue;  // descendant outside the reach: its W rows are zero
    const int32_t* Td = d.wt_idx + d.wt_ptr[dd];
    const int ntd = d.wt_ptr[dd + 1] - d.wt_ptr[dd];
    const int r0 = d.upd_r0[u], r1 = d.upd_r1[u];
    const int md = (int)(d.sn_rowptr[dd + 1] - d.sn_rowptr[dd]);
    const int wd = d.sn_first[dd + 1] - d.sn_first[dd];
    const double* Pd = Lx + b * pt + d.sn_valoff[dd];
    const int32_t* Rd = d.sn_rows + d.sn_rowptr[dd];
    const int total = (r1 - r0) * ntd;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
      const int j = r0 + q / ntd, t = Td[q % ntd];
      if (t < lo || t > hi) continue;  // a column of another chunk
      double acc = 0.0;
      for (int kk = 0; kk < wd; kk++) acc += Pd[(int64_t)kk * md + j] * Wb[(int64_t)(wrd + kk) * k + t];
      Wb[(int64_t)(ws + Rd[j] - f) * k + t] -= acc;
    }
    __syncthreads();
  }
  if (TAIL_INIT) return;
  for (int c = 0; c + 1 < w; c++) {
    const int total = (w - 1 - c) * nt;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
      const int c2 = c + 1 + q / nt, t = tc[q % nt];
      Wb[(int64_t)(ws + c2) * k + t] -= P[(int64_t)c * m + c2] * Wb[(int64_t)(ws + c) * k + t];
    }
    __syncthreads();
  }
}

// G_b = W_b^T D_b^{-1} W_b over the rows outside the tail, by structure: one
// thread per (nonzero entry t1 >= t2 of G, block) sums its rows in order
// (every other product is an exact zero).
__global__ void k_contract_g_sparse(const int32_t* __restrict__ g_key, const int64_t* __restrict__ g_ptr,
                                    const int32_t* __restrict__ g_row, int64_t nkeys,
                                    const double* __restrict__ W, const double* __restrict__ wdinv, int nw,
                                    int k, int N, double* __restrict__ G) {
  const int64_t total = nkeys * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = q / nkeys, e = q - b * nkeys;
    const int key = g_key[e], t1 = key / k, t2 = key - t1 * k;
    const double* Wb = W + b * nw * k;
    const double* db = wdinv + b * nw;
    double acc = 0.0;
    for (int64_t r = g_ptr[e]; r < g_ptr[e + 1]; r++) {
      const int row = g_row[r];
      acc += Wb[(int64_t)row * k + t1] * db[row] * Wb[(int64_t)row * k + t2];
    }
    double* Gb = G + b * k * k;
    Gb[(int64_t)t1 * k + t2] = acc;
    Gb[(int64_t)t2 * k + t1] = acc;
  }
}

// G_b = W_b^T D_b^{-1} W_b in FP64, one 32x32 tile of the lower triangle per CTA
// (the first nrows rows of W; nw is its row count per block; wdinv holds the
// reciprocal pivot of every W row)
__global__ void __launch_bounds__(256) k_contract_g_f64(const double* __restrict__ W,
                                                        const double* __restrict__ wdinv, int nw, int nrows,
                                                        int k, double* __restrict__ G) {
  const int b = blockIdx.y;
  // tile index -> (ti, tj) with ti >= tj
  int tile = blockIdx.x, ti = 0;
  while (tile > ti) {
    tile -= ti + 1;
    ti++;
  }
  const int tj = tile;
  const int t1_0 = ti * 32, t2_0 = tj * 32;
  __shared__ double Wa[32][33], Wb_[32][33];
  const double* Wblk = W + (int64_t)b * nw * k;
  const double* dinv_b = wdinv + (int64_t)b * nw;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  double acc[4] = {0, 0, 0, 0};
  for (int r0 = 0; r0 < nrows; r0 += 32) {
    for (int q = threadIdx.x; q < 32 * 32; q += 256) {
      const int rr = q >> 5, cc = q & 31;
      const int row = r0 + rr;
      double a = 0.0, bb = 0.0;
      if (row < nrows) {
        const double dinv = dinv_b[row];
        if (t1_0 + cc < k) a = Wblk[(int64_t)row * k + t1_0 + cc] * dinv;
        if (t2_0 + cc < k) bb = Wblk[(int64_t)row * k + t2_0 + cc];
      }
      Wa[rr][cc] = a;
      Wb_[rr][cc] = bb;
    }
    __syncthreads();
    for (int rr = 0; rr < 32; rr++) {
      const double bv = Wb_[rr][tx];
#pragma unroll
      for (int i = 0; i < 4; i++) acc[i] += Wa[rr][ty + 8 * i] * bv;
    }
    __syncthreads();
  }
  double* Gb = G + (int64_t)b * k * k;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int t1 = t1_0 + ty + 8 * i, t2 = t2_0 + tx;
    if (t1 < k && t2 < k) {
      Gb[(int64_t)t1 * k + t2] = acc[i];
      if (ti != tj) Gb[(int64_t)t2 * k + t1] = acc[i];
    }
  }
}

// G_b -= T_b[nT:, nT:]: after the nT pivots of the augmented tail its trailing
// k x k block holds -W_T^T D_T^{-1} W_T (lower triangle), the tail rows' share of G.
__global__ void k_add_tail_g(const double* __restrict__ Ta, int nT, int nTa, int k, double* __restrict__ G) {
  const int b = blockIdx.y;
  const double* Tb = Ta + (int64_t)b * nTa * nTa;
  double* Gb = G + (int64_t)b * k * k;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < k * k; q += gridDim.x * blockDim.x) {
    const int t1 = q / k, t2 = q - t1 * k;
    const int hi = max(t1, t2), lo = min(t1, t2);
    Gb[q] -= Tb[(int64_t)(nT + hi) + (int64_t)(nT + lo) * nTa];
  }
}

// reciprocal pivot of every W row of every block (used by the contraction and
// by the right-hand-side reduction of the solves)
__global__ void k_w_dinv(const double* __restrict__ Lx, int64_t pt, const int64_t* __restrict__ w_dpos, int nw,
                         int N, double* __restrict__ wdinv) {
  const int64_t total = (int64_t)nw * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = q / nw, row = q - b * nw;
    wdinv[q] = 1.0 / Lx[b * pt + w_dpos[row]];
  }
}

__global__ void k_init_s(double* __restrict__ S, int nC, int c_kind, const double* __restrict__ c_vals) {
  const int64_t n2 = (int64_t)nC * nC;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n2;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = q / nC, i = q - j * nC;  // column-major: row i, column j
    double v = 0.0;
    if (c_kind == 0) {
      if (i == j) v = c_vals[i];
    } else if (i >= j) {
      v = c_vals[i * nC + j];  // row-major input, lower triangle
    }
    S[q] = v;
  }
}

__global__ void k_assemble_s(const int64_t* __restrict__ s_key, const int64_t* __restrict__ s_ptr,
                             const int32_t* __restrict__ s_e1, const int32_t* __restrict__ s_e2,
                             const int32_t* __restrict__ e_t, const int32_t* __restrict__ e_block,
                             const double* __restrict__ b_vals, const double* __restrict__ G, int k,
                             int64_t nkeys, int nC, double* __restrict__ S) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nkeys;
       q += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t r = s_ptr[q]; r < s_ptr[q + 1]; r++) {
      const int e1 = s_e1[r], e2 = s_e2[r];
      const double* Gb = G + (int64_t)e_block[e1] * k * k;
      acc += b_vals[e1] * b_vals[e2] * Gb[(int64_t)e_t[e1] * k + e_t[e2]];
    }
    const int64_t key = s_key[q];
    const int64_t c1 = key / nC, c2 = key - c1 * nC;
    S[c1 + c2 * (int64_t)nC] -= acc;
  }
}

}  // namespace

namespace {

cudaError_t w_levels(Handle& h, const std::vector<int32_t>& lvl_ptr, const std::vector<int32_t>& lvl_chunks,
                     const int32_t* lvl_sn, cudaStream_t st) {
  const int k = h.cpl.k;
  for (int l = 0; l < h.sym.nlevels; l++) {
    const int s0 = lvl_ptr[l], s1 = lvl_ptr[l + 1];
    if (s1 == s0) continue;
    dim3 grid(s1 - s0, h.N, lvl_chunks[l]);
    k_w_solve<false><<<grid, 128, 0, st>>>(lvl_sn + s0, h.d, h.Lx, h.sym.panel_total, h.W, h.cpl.nw, k);
    h.launches++;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_w_solve(Handle& h, cudaStream_t st) {
  const int k = h.cpl.k;
  if (k == 0 || h.cpl.nw == 0 || h.tail_aug) return cudaSuccess;  // augmented: done before the tail
  return w_levels(h, h.reach_lvl_ptr, h.reach_lvl_chunks, h.d.reach_lvl_sn, st);
}

// Augmented tail: the W rows outside the tail, then the tail's rows Z (the
// right-hand side minus the updates from outside the tail), before the tail
// factor that completes them.
cudaError_t launch_w_solve_before_tail(Handle& h, cudaStream_t st) {
  const int k = h.cpl.k;
  cudaError_t e = w_levels(h, h.reach_lvl_ptr_nt, h.reach_lvl_chunks_nt, h.d.reach_lvl_sn_nt, st);
  if (e != cudaSuccess) return e;
  const int nts = h.tail_reach_sn;
  if (nts == 0) return cudaSuccess;
  dim3 grid(nts, h.N, 1);
  k_w_solve<true><<<grid, 128, 0, st>>>(h.d.tail_sn_list, h.d, h.Lx, h.sym.panel_total, h.W, h.cpl.nw, k);
  h.launches++;
  return cudaGetLastError();
}

cudaError_t launch_w_dinv(Handle& h, cudaStream_t st) {
  const int64_t total = (int64_t)h.cpl.nw * h.N;
  if (total == 0) return cudaSuccess;
  k_w_dinv<<<(int)std::min<int64_t>((total + 255) / 256, 152 * 8), 256, 0, st>>>(h.Lx, h.sym.panel_total, h.d.w_dpos,
                                                                              h.cpl.nw, h.N, h.wdinv);
  h.launches++;
  return cudaGetLastError();
}

cudaError_t launch_add_tail_g(Handle& h, cudaStream_t st) {
  if (!h.tail_aug) return cudaSuccess;
  const int k = h.cpl.k;
  dim3 grid((k * k + 255) / 256, h.N);
  k_add_tail_g<<<grid, 256, 0, st>>>(h.Tt, h.nT, h.nTa, k, h.G);
  h.launches++;
  return cudaGetLastError();
}

cudaError_t launch_contract_g(Handle& h, cudaStream_t st) {
  const int k = h.cpl.k;
  if (k == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(h.G, 0, sizeof(double) * (size_t)h.N * k * k, st);
  const int64_t nkeys = (int64_t)h.g_nkeys;
  if (e == cudaSuccess && nkeys > 0) {
    const int64_t total = nkeys * h.N;
    k_contract_g_sparse<<<(int)std::min<int64_t>((total + 255) / 256, 152 * 16), 256, 0, st>>>(
        h.d.g_key, h.d.g_ptr, h.d.g_row, nkeys, h.W, h.wdinv, h.cpl.nw, k, h.N, h.G);
    h.launches++;
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  return launch_add_tail_g(h, st);
}

cudaError_t launch_assemble_s(Handle& h, cudaStream_t st) {
  if (h.nC == 0) return cudaSuccess;
  const int64_t n2 = (int64_t)h.nC * h.nC;
  int grid = (int)std::min<int64_t>((n2 + 255) / 256, 152 * 32);
  {
    k_init_s<<<grid, 256, 0, st>>>(h.S, h.nC, h.c_kind, h.c_vals);
    h.launches++;
  }
  const int64_t nkeys = (int64_t)h.cpl.s_key.size();
  if (nkeys > 0) {
    int g2 = (int)std::min<int64_t>((nkeys + 255) / 256, 152 * 32);
    {
    k_assemble_s<<<g2, 256, 0, st>>>(h.d.s_key, h.d.s_ptr, h.d.s_e1, h.d.s_e2, h.d.e_t, h.d.e_block,
                                     h.b_vals, h.G, h.cpl.k, nkeys, h.nC, h.S);
    h.launches++;
  }
  }
  return cudaGetLastError();
}

}  // namespace kkt
