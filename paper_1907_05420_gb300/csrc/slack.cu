// Slack elimination around the solve (Sec. 2): the barrier method's Newton
// system (eq. SCOPFhessian) is reduced to the arrowhead K by eliminating the
// bound multipliers and the slacks of the inequality rows (eqs.
// SCOPFhessianSymmetric, SCOPFslackAtEnd, SCOPFhessianReduced), and the
// eliminated unknowns are recovered from the solution (eqs.
// SCOPFslackReduction, SCOPFhessianSymmetricRecovery):
//
//   A_i:  primal diagonals  += z / x              (H + X^-1 Z)
//         inequality rows:  diagonal = -(s / y)   (-L_s^-1, L_s = S^-1 Y)
//   C:    diagonal          += z_g / x_g
//   rhs:  primal rows       -(l_a + l_e / x)
//         equality rows     -l_c
//         inequality rows   -(l_d + (s / y) (l_b + l_f / s))
//   ds = (s / y) (dlI - l_b - l_f / s),  dz = -(l_e + z dx) / x,  dy = -(l_f + y ds) / s
//
// Every entry is computed by one thread with round-to-nearest intrinsics (no
// fused multiply-adds), in the order written above.
#include <vector>

#include "handle.h"

struct kkt_slack {
  kkt::Handle* h = nullptr;
  int32_t L = 0;              // inequality rows per block
  int32_t* ineq_of_row = nullptr;  // per row of A: its index among the inequality rows, -1 otherwise
  int32_t* ineq_rows = nullptr;    // the inequality rows
};

namespace kkt {
namespace {

// one thread per row of K: the diagonal entry of A_i or C and the right-hand side
__global__ void k_slack_reduce(const int32_t* __restrict__ diag_pos, const int32_t* __restrict__ ineq_of_row,
                               int nA, int nP, int N, int nC, int L, int64_t nnzA, int c_kind,
                               const double* __restrict__ x, const double* __restrict__ z,
                               const double* __restrict__ s, const double* __restrict__ y,
                               const double* __restrict__ la, const double* __restrict__ le,
                               const double* __restrict__ lcd, const double* __restrict__ lb,
                               const double* __restrict__ lf, const double* __restrict__ a_base,
                               const double* __restrict__ c_base, double* __restrict__ a_vals,
                               double* __restrict__ c_vals, double* __restrict__ rhs) {
  const int64_t nb = (int64_t)N * nA, total = nb + nC;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    if (q < nb) {
      const int64_t b = q / nA;
      const int r = (int)(q - b * nA);
      const int64_t pos = b * nnzA + diag_pos[r];
      if (r < nP) {
        const int64_t k = b * nP + r;
        a_vals[pos] = __dadd_rn(a_base[pos], __ddiv_rn(z[k], x[k]));
        rhs[q] = -__dadd_rn(la[k], __ddiv_rn(le[k], x[k]));
      } else {
        const int e = ineq_of_row[r];
        const double l = lcd[b * (nA - nP) + (r - nP)];
        if (e >= 0) {
          const int64_t j = b * L + e;
          const double sy = __ddiv_rn(s[j], y[j]);
          a_vals[pos] = -sy;
          rhs[q] = -__dadd_rn(l, __dmul_rn(sy, __dadd_rn(lb[j], __ddiv_rn(lf[j], s[j]))));
        } else {
          rhs[q] = -l;
        }
      }
    } else {
      const int c = (int)(q - nb);
      const int64_t k = (int64_t)N * nP + c;
      const int64_t cp = c_kind == 0 ? c : (int64_t)c * nC + c;
      c_vals[cp] = __dadd_rn(c_base[cp], __ddiv_rn(z[k], x[k]));
      rhs[q] = -__dadd_rn(la[k], __ddiv_rn(le[k], x[k]));
    }
  }
}

// one thread per primal variable (dz) and per inequality row (ds, dy)
__global__ void k_slack_recover(const int32_t* __restrict__ ineq_rows, int nA, int nP, int N, int nC, int L,
                                const double* __restrict__ x, const double* __restrict__ z,
                                const double* __restrict__ s, const double* __restrict__ y,
                                const double* __restrict__ le, const double* __restrict__ lb,
                                const double* __restrict__ lf, const double* __restrict__ dsol,
                                double* __restrict__ ds, double* __restrict__ dz, double* __restrict__ dy) {
  const int64_t nx = (int64_t)N * nP + nC, ni = (int64_t)N * L;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nx + ni;
       q += (int64_t)gridDim.x * blockDim.x) {
    if (q < nx) {
      double dx;
      if (q < (int64_t)N * nP) {
        const int64_t b = q / nP;
        dx = dsol[b * nA + (q - b * nP)];
      } else {
        dx = dsol[(int64_t)N * nA + (q - (int64_t)N * nP)];
      }
      dz[q] = __ddiv_rn(-__dadd_rn(le[q], __dmul_rn(z[q], dx)), x[q]);
    } else {
      const int64_t j = q - nx, b = j / L;
      const int e = (int)(j - b * L);
      const double dli = dsol[b * nA + ineq_rows[e]];
      const double sy = __ddiv_rn(s[j], y[j]);
      const double d = __dmul_rn(sy, __dsub_rn(__dsub_rn(dli, lb[j]), __ddiv_rn(lf[j], s[j])));
      ds[j] = d;
      dy[j] = __ddiv_rn(-__dadd_rn(lf[j], __dmul_rn(y[j], d)), s[j]);
    }
  }
}

inline int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

}  // namespace
}  // namespace kkt

using namespace kkt;

extern "C" {

kkt_status kkt_slack_create(kkt_handle* hh, int32_t n_ineq, const int32_t* ineq_rows, kkt_slack** out) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !out || n_ineq < 0 || (n_ineq > 0 && !ineq_rows)) {
    set_error("kkt_slack_create: invalid argument");
    return KKT_ERR_INVALID;
  }
  *out = nullptr;
  std::vector<int32_t> of_row(h->nA, -1);
  for (int32_t q = 0; q < n_ineq; q++) {
    const int32_t r = ineq_rows[q];
    if (r < h->nP || r >= h->nA || (q > 0 && r <= ineq_rows[q - 1])) {
      set_error("kkt_slack_create: inequality rows must be increasing multiplier rows of A (in [nP, nA))");
      return KKT_ERR_INVALID;
    }
    of_row[r] = q;
  }
  kkt_slack* sl = new (std::nothrow) kkt_slack();
  if (!sl) return KKT_ERR_OOM;
  sl->h = h;
  sl->L = n_ineq;
  cudaError_t e = cudaMalloc((void**)&sl->ineq_of_row, sizeof(int32_t) * (size_t)std::max(1, h->nA));
  if (e == cudaSuccess) e = cudaMalloc((void**)&sl->ineq_rows, sizeof(int32_t) * (size_t)std::max(1, n_ineq));
  if (e == cudaSuccess)
    e = cudaMemcpy(sl->ineq_of_row, of_row.data(), sizeof(int32_t) * (size_t)h->nA, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n_ineq > 0)
    e = cudaMemcpy(sl->ineq_rows, ineq_rows, sizeof(int32_t) * (size_t)n_ineq, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_error(std::string("kkt_slack_create: ") + cudaGetErrorString(e));
    kkt_slack_destroy(sl);
    return e == cudaErrorMemoryAllocation ? KKT_ERR_OOM : KKT_ERR_CUDA;
  }
  *out = sl;
  return KKT_OK;
}

kkt_status kkt_slack_reduce(kkt_slack* sl, const kkt_ipm_state* st, const double* a_base, const double* c_base,
                            double* a_vals, double* c_vals, double* rhs, void* stream) {
  if (!sl || !st || !a_base || !a_vals || !rhs || !st->x || !st->z || !st->la || !st->le || !st->lcd ||
      (sl->h->nC > 0 && (!c_base || !c_vals)) || (sl->L > 0 && (!st->s || !st->y || !st->lb || !st->lf))) {
    set_error("kkt_slack_reduce: null argument");
    return KKT_ERR_INVALID;
  }
  Handle& h = *sl->h;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  // the entries other than the diagonals keep their base values
  if (a_vals != a_base)
    KKT_CUDA(cudaMemcpyAsync(a_vals, a_base, sizeof(double) * (size_t)(h.nnzA * h.N), cudaMemcpyDeviceToDevice, s));
  const int64_t nc_vals = h.c_kind == 0 ? (int64_t)h.nC : (int64_t)h.nC * h.nC;
  if (c_vals != c_base && nc_vals > 0)
    KKT_CUDA(cudaMemcpyAsync(c_vals, c_base, sizeof(double) * (size_t)nc_vals, cudaMemcpyDeviceToDevice, s));
  const int64_t rows = (int64_t)h.N * h.nA + h.nC;
  k_slack_reduce<<<grid_of(rows), 256, 0, s>>>(h.d.diag_pos, sl->ineq_of_row, h.nA, h.nP, h.N, h.nC, sl->L,
                                              h.nnzA, h.c_kind, st->x, st->z, st->s, st->y, st->la, st->le,
                                              st->lcd, st->lb, st->lf, a_base, c_base, a_vals, c_vals, rhs);
  h.launches++;
  KKT_CUDA(cudaGetLastError());
  return KKT_OK;
}

kkt_status kkt_slack_recover(kkt_slack* sl, const kkt_ipm_state* st, const double* dsol, double* ds, double* dz,
                             double* dy, void* stream) {
  if (!sl || !st || !dsol || !dz || !st->x || !st->z || !st->le ||
      (sl->L > 0 && (!ds || !dy || !st->s || !st->y || !st->lb || !st->lf))) {
    set_error("kkt_slack_recover: null argument");
    return KKT_ERR_INVALID;
  }
  Handle& h = *sl->h;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  const int64_t n = (int64_t)h.N * h.nP + h.nC + (int64_t)h.N * sl->L;
  k_slack_recover<<<grid_of(n), 256, 0, s>>>(sl->ineq_rows, h.nA, h.nP, h.N, h.nC, sl->L, st->x, st->z, st->s,
                                             st->y, st->le, st->lb, st->lf, dsol, ds, dz, dy);
  h.launches++;
  KKT_CUDA(cudaGetLastError());
  return KKT_OK;
}

kkt_status kkt_slack_destroy(kkt_slack* sl) {
  if (!sl) return KKT_OK;
  if (sl->ineq_of_row) cudaFree(sl->ineq_of_row);
  if (sl->ineq_rows) cudaFree(sl->ineq_rows);
  delete sl;
  return KKT_OK;
}

}  // extern "C"
