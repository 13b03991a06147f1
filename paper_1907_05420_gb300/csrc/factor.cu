// (a) Batched numeric LDL^T of the N blocks A_i = P L_i D_i L_i^T P^T
// (the block factorization of Algorithm 1), all blocks sharing one supernodal
// structure.
//
// Storage: block b's factor is one contiguous array of supernode panels;
// panel s is column-major m_s x w_s (its rows are sn_rows[s], the first w_s of
// them its own columns).  The diagonal of the w_s x w_s top block holds D,
// the rest of the panel holds L (unit diagonal implied).
//
// Schedule: supernodes are processed level by level of the supernodal
// elimination tree.  Per level two launches:
//   k_factor_update: left-looking updates of every supernode s of the level
//     from its descendants d,  P_s[rel(i), j - f_s] -= sum_k L_d[i,k] D_d[k] L_d[j,k],
//     one CTA per (32-row tile of s, block) so that the wide supernodes at the
//     top of the tree spread over many SMs;
//   k_panel_factor: dense LDL^T of the panel (1x1 pivots; a pivot below
//     pivot_eps*max|A_i| is replaced by the expected-sign value and counted).
// The top of the tree (the dense tail, a suffix of the supernodes) is left out
// of the level loop: once the rest is factored, its updates from outside the
// tail are applied (k_factor_update over the tail's lists) and the tail is factored as one
// dense triangle per block (tail.cu).
// Every entry is written by one thread in a fixed order: the result does not
// depend on scheduling.
#include "handle.h"
#include "pivot.cuh"

namespace kkt {

namespace {

__global__ void k_scatter_a(const double* __restrict__ a_vals, int64_t nnzA,
                            const int64_t* __restrict__ a_map, double* __restrict__ Lx,
                            int64_t pt, int N) {
  const int64_t total = nnzA * (int64_t)N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = q / nnzA, p = q - b * nnzA;
    Lx[b * pt + a_map[p]] = a_vals[q];
  }
}

// Inertia-correction shift of the copied values: +dw on the diagonal of the
// primal rows of every block, -dc on the dual rows, dcs on C's diagonal (+dw
// for primal coupling variables, -dc for multipliers).  One thread per
// (block, row) or C entry.
__global__ void k_shift_diag(double* __restrict__ a_vals, int64_t nnzA, const int32_t* __restrict__ diag_pos,
                             int nA, int nP, int N, double* __restrict__ c_vals, int nC, int c_kind, double dw,
                             double dc, double dcs) {
  const int64_t na = (int64_t)N * nA;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < na + nC;
       q += (int64_t)gridDim.x * blockDim.x) {
    if (q < na) {
      const int64_t b = q / nA;
      const int r = (int)(q - b * nA);
      a_vals[b * nnzA + diag_pos[r]] += r < nP ? dw : -dc;
    } else {
      const int64_t i = q - na;
      c_vals[c_kind == 0 ? i : i * nC + i] += dcs;
    }
  }
}

// max |a| of each block (threshold base of the pivot perturbation)
__global__ void k_block_absmax(const double* __restrict__ a_vals, int64_t nnzA,
                               double* __restrict__ anorm) {
  __shared__ double red[256];
  const double* a = a_vals + blockIdx.x * nnzA;
  double m = 0.0;
  for (int64_t p = threadIdx.x; p < nnzA; p += blockDim.x) m = fmax(m, fabs(a[p]));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) anorm[blockIdx.x] = red[0];
}

// One CTA per (32-row tile of supernode s, block; 128 threads).  The tile's update is
// accumulated in shared memory over the descendants d that meet the tile (in
// update order) and subtracted from the panel once.  For each update the rows
// of d that land in the tile ([ia, ib), listed per tile at analysis with only
// the updates that meet it) and the rows that land in s's columns ([r0, r1))
// are staged in shared memory, the latter pre-multiplied by D_d.  For the tail
// supernodes the lists hold only the updates from descendants outside the
// dense tail; their updates among themselves are the dense tail factor's.
constexpr int kTileRows = kFactorTileRows;
constexpr int kFactorThreads = 128;

__global__ void __launch_bounds__(kFactorThreads) k_factor_update(const int32_t* __restrict__ work,
                                                       const UpdPair* __restrict__ pairs, DevSym d,
                                                       double* __restrict__ Lx, int64_t pt,
                                                       const double* __restrict__ LDx, int64_t ldt) {
  __shared__ double acc[kTileRows][kMaxSnWidth + 1];
  __shared__ double Li[kTileRows][kMaxSnWidth + 1];
  __shared__ double Lj[kMaxSnWidth][kMaxSnWidth + 1];
  __shared__ int rs[kTileRows], tc[kMaxSnWidth];
  const int item = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
  const int s = work[4 * item], lo = work[4 * item + 1], hi = work[4 * item + 2];
  const int p0 = work[4 * item + 3], p1 = work[4 * item + 7];  // this item's updates, to the next item's
  const int ms = (int)(d.sn_rowptr[s + 1] - d.sn_rowptr[s]);
  const int f = d.sn_first[s], ws = d.sn_first[s + 1] - f;
  const int nrow = hi - lo;
  const double* Lb = Lx + b * pt;
  const double* LDb = LDx + b * ldt;
  double* P = Lx + b * pt + d.sn_valoff[s];
  for (int q = tid; q < kTileRows * (kMaxSnWidth + 1); q += blockDim.x) (&acc[0][0])[q] = 0.0;
  UpdPair Rn{};  // the next update's record, loaded during this one's products
  if (p0 < p1) Rn = pairs[p0];
  for (int p = p0; p < p1; p++) {
    const UpdPair R = Rn;
    const int ni = R.ib - R.ia, nj = R.r1 - R.r0, wd = R.wd, md = R.md;
    const double* Pd = Lb + R.val;
    const double* PDd = LDb + R.val;  // the same panel's L D (descendants lie outside the tail)
    const int32_t* Rd = d.sn_rows + R.rows;
    const int32_t* rel = d.upd_rel + R.rel;
    __syncthreads();  // the previous update's reads of Li/Lj are done
    for (int q = tid; q < ni * wd; q += blockDim.x) {
      const int i = q % ni, kk = q / ni;
      Li[i][kk] = Pd[(int64_t)kk * md + R.ia + i];
    }
    for (int q = tid; q < nj * wd; q += blockDim.x) {
      const int j = q % nj, kk = q / nj;
      Lj[j][kk] = PDd[(int64_t)kk * md + R.r0 + j];
    }
    for (int q = tid; q < ni; q += blockDim.x) rs[q] = rel[R.ia + q - R.r0] - lo;
    for (int q = tid; q < nj; q += blockDim.x) tc[q] = Rd[R.r0 + q] - f;
    __syncthreads();
    if (p + 1 < p1) Rn = pairs[p + 1];
    for (int q = tid; q < ni * nj; q += blockDim.x) {
      const int i = q % ni, j = q / ni;
      if (R.ia + i < R.r0 + j) continue;  // above the diagonal of the target
      double sum = 0.0;
      for (int kk = 0; kk < wd; kk++) sum += Li[i][kk] * Lj[j][kk];
      acc[rs[i]][tc[j]] += sum;
    }
  }
  __syncthreads();
  for (int q = tid; q < nrow * ws; q += blockDim.x) {
    const int r = q % nrow, c = q / nrow;
    P[(int64_t)c * ms + lo + r] -= acc[r][c];
  }
}

__global__ void __launch_bounds__(256) k_panel_factor(const int32_t* __restrict__ lvl_sn, DevSym d,
                                                      double* __restrict__ Lx, int64_t pt,
                                                      double* __restrict__ LDx, int64_t ldt,
                                                      const double* __restrict__ anorm,
                                                      double pivot_eps,
                                                      unsigned long long* __restrict__ counters) {
  const int s = lvl_sn[blockIdx.x], b = blockIdx.y;
  const int m = (int)(d.sn_rowptr[s + 1] - d.sn_rowptr[s]);
  const int f = d.sn_first[s], w = d.sn_first[s + 1] - f;
  double* P = Lx + b * pt + d.sn_valoff[s];
  const double thr = pivot_eps * anorm[b];
  __shared__ double dsh, dinv_sh;
  __shared__ int cnt[4];
  if (threadIdx.x < 4) cnt[threadIdx.x] = 0;
  for (int c = 0; c < w; c++) {
    if (threadIdx.x == 0) {
      double dv = P[(int64_t)c * m + c];
      const bool primal = d.col_primal[f + c] != 0;
      if (thr > 0.0 && fabs(dv) < thr) {
        dv = primal ? thr : -thr;
        cnt[3]++;
      }
      P[(int64_t)c * m + c] = dv;
      cnt[dv > 0.0 ? 0 : (dv < 0.0 ? 1 : 2)]++;
      dsh = dv;
      dinv_sh = pivot_recip(dv);
    }
    __syncthreads();
    const double dv = dsh, di = dinv_sh;
    double* colc = P + (int64_t)c * m;
    for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) colc[r] = colc[r] * di;
    __syncthreads();
    for (int c2 = c + 1; c2 < w; c2++) {
      const double l2 = colc[c2] * dv;
      double* col2 = P + (int64_t)c2 * m;
      for (int r = c2 + threadIdx.x; r < m; r += blockDim.x) col2[r] -= colc[r] * l2;
    }
    __syncthreads();
  }
  if (threadIdx.x < 4 && cnt[threadIdx.x]) atomicAdd(&counters[threadIdx.x], (unsigned long long)cnt[threadIdx.x]);
  // L D of the panel for the updates of its ancestors: column c's entries
  // times d_c, the product the updates would otherwise form per target tile
  double* PD = LDx + b * ldt + d.sn_valoff[s];
  for (int c = 0; c < w; c++) {
    const double dv = P[(int64_t)c * m + c];
    for (int r = threadIdx.x; r < m; r += blockDim.x) PD[(int64_t)c * m + r] = P[(int64_t)c * m + r] * dv;
  }
}

}  // namespace

cudaError_t launch_shift_diag(Handle& h, double dw, double dc, double dcs, cudaStream_t st) {
  const int64_t total = (int64_t)h.N * h.nA + h.nC;
  if (total == 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  k_shift_diag<<<grid, 256, 0, st>>>(h.a_vals, h.nnzA, h.d.diag_pos, h.nA, h.nP, h.N, h.c_vals, h.nC, h.c_kind,
                                     dw, dc, dcs);
  h.launches++;
  return cudaGetLastError();
}

cudaError_t launch_scatter_a(Handle& h, cudaStream_t st) {
  const int64_t pt = h.sym.panel_total;
  cudaError_t e = cudaMemsetAsync(h.Lx, 0, sizeof(double) * pt * h.N, st);
  if (e != cudaSuccess) return e;
  int64_t total = h.nnzA * h.N;
  int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  {
    k_scatter_a<<<grid, 256, 0, st>>>(h.a_vals, h.nnzA, h.d.a_map, h.Lx, pt, h.N);
    h.launches++;
  }
  {
    k_block_absmax<<<h.N, 256, 0, st>>>(h.a_vals, h.nnzA, h.anorm);
    h.launches++;
  }
  return cudaGetLastError();
}

cudaError_t launch_factor_levels(Handle& h, cudaStream_t st) {
  const int64_t pt = h.sym.panel_total;
  // supernodes outside the dense tail, level by level
  for (int l = 0; l < h.sym.nlevels; l++) {
    const int w0 = h.fwork_lvl_ptr[l], w1 = h.fwork_lvl_ptr[l + 1];
    if (l > 0 && w1 > w0) {
      dim3 grid(w1 - w0, h.N);
      const int kt = kt_begin(h, kFamFactorUpd, h.N * h.fupd_flops[l], st);
      k_factor_update<<<grid, kFactorThreads, 0, st>>>(h.d.fwork + 4 * w0, h.d.fpairs, h.d, h.Lx, pt, h.LDx,
                                                        h.ld_total);
      kt_end(h, kt, st);
      h.launches++;
    }
    const int s0 = h.flvl_ptr[l], s1 = h.flvl_ptr[l + 1];
    if (s1 > s0) {
      dim3 grid2(s1 - s0, h.N);
      k_panel_factor<<<grid2, 256, 0, st>>>(h.d.flvl_sn + s0, h.d, h.Lx, pt, h.LDx, h.ld_total, h.anorm,
                                            h.opt.pivot_eps,
                                            h.counters);
      h.launches++;
    }
  }
  if (h.nT > 0) {
    // updates of the tail from the rest of the tree (all factored by now), then
    // the dense factor of the tail; an augmented tail first takes the W rows
    // outside the tail and its own rows Z
    if (h.tail_aug) {
      cudaError_t e = launch_w_solve_before_tail(h, st);
      if (e != cudaSuccess) return e;
    }
    if (h.tail_items > 0) {
      dim3 grid(h.tail_items, h.N);
      const int kt = kt_begin(h, kFamFactorUpd, h.N * h.tupd_flops, st);
      k_factor_update<<<grid, kFactorThreads, 0, st>>>(h.d.twork, h.d.fpairs, h.d, h.Lx, pt, h.LDx, h.ld_total);
      kt_end(h, kt, st);
      h.launches++;
    }
    cudaError_t e = launch_dense_tail(h, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace kkt
