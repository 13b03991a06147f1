// The steps of Algorithm 1 (Sec. 4.2) one at a time, for a solve whose
// blocks are spread over several processes (one GPU each):
//
//   kkt_factor_blocks   block factors and the local Schur complement
//                       C_p - sum_{i in p} B_i^T A_i^{-1} B_i of the handle's
//                       blocks (Algorithm 1: factorization, S_i, accumulation);
//   kkt_schur_matrix    the device buffer of that S, into which the root adds
//                       the other processes' parts (the reduce);
//   kkt_factor_schur    dense LDL^T of the reduced S (root only);
//   kkt_solve_front     t_p = r_g,p - sum_{i in p} B_i^T A_i^{-1} r_i (eq. SCsolve,
//                       the right-hand-side accumulation);
//   kkt_solve_coupling  x_g = S^{-1} t (root only);
//   kkt_solve_back      x_i = A_i^{-1} (r_i - B_i x_g) with the broadcast x_g
//                       (eq. SCsolve1, the local solves);
//   kkt_residual, kkt_abs_rowsums, kkt_norm_inf, kkt_accumulate: the pieces
//                       of FP64 refinement on the distributed K.
// The collectives themselves belong to the caller.  Every step is a kernel;
// the host only orders launches on the caller's stream.
#include <cmath>

#include "handle.h"

namespace kkt {

namespace {

__global__ void k_accumulate(double* __restrict__ dst, int64_t ld_dst, const double* __restrict__ src,
                             int64_t ld_src, int64_t rows, int64_t cols) {
  const int64_t total = rows * cols;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = q / rows, i = q - j * rows;
    dst[i + j * ld_dst] += src[i + j * ld_src];
  }
}

// out[b*nA + row] = sum_p |A_b[row, p]| over the full symmetric row
__global__ void k_rowsum_blocks(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ src,
                                const double* __restrict__ a_vals, int64_t nnzA, int nA, int N,
                                double* __restrict__ out) {
  const int64_t total = (int64_t)nA * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = q / nA;
    const int row = (int)(q - b * nA);
    const double* a = a_vals + b * nnzA;
    double acc = 0.0;
    for (int p = rowptr[row]; p < rowptr[row + 1]; p++) acc += fabs(a[src[p]]);
    out[q] = acc;
  }
}

// the rows of E also carry B's entries (each (block, E row) once)
__global__ void k_rowsum_b(const int32_t* __restrict__ bt_ptr, const double* __restrict__ b_vals,
                           const int32_t* __restrict__ E, int k, int nA, int N, double* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= k * N) return;
  const int b = q / k, t = q - b * k;
  const int32_t* bp = bt_ptr + (int64_t)b * (k + 1);
  double acc = 0.0;
  for (int e = bp[t]; e < bp[t + 1]; e++) acc += fabs(b_vals[e]);
  if (bp[t] < bp[t + 1]) out[(int64_t)b * nA + E[t]] += acc;
}

// coupling rows: sum |B column c| + sum |C row c|
__global__ void k_rowsum_g(const int32_t* __restrict__ t_ptr, const int32_t* __restrict__ t_e,
                           const double* __restrict__ b_vals, const double* __restrict__ c_vals, int c_kind,
                           int nC, double* __restrict__ out) {
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
  out[c] = acc;
}

// max |v| keeping NaN (see k_norms3)
__global__ void k_maxabs(const double* __restrict__ v, int64_t n, double* __restrict__ out) {
  __shared__ double sh[256];
  double m = 0.0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const double a = fabs(v[q]);
    m = (a > m || a != a) ? a : m;
  }
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double a = sh[threadIdx.x + s], b = sh[threadIdx.x];
      sh[threadIdx.x] = (a > b || a != a) ? a : b;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(sh[0]));
}

__global__ void k_f32_to_f64(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    b[q] = (double)a[q];
}

inline int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

kkt_status need(bool ok, const char* what) {
  if (ok) return KKT_OK;
  set_error(what);
  return KKT_ERR_STATE;
}

}  // namespace

cudaError_t launch_dense_factor_of(Handle& h, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(h.counters + kNumCounters, 0, sizeof(unsigned long long) * kNumCounters, st);
  if (e != cudaSuccess) return e;
  return h.opt.prec == KKT_FP64 ? launch_dense_ldlt(h, h.counters + kNumCounters, st)
                                : launch_dense_ldlt_tc(h, h.opt.prec, h.counters + kNumCounters, st);
}

}  // namespace kkt

using namespace kkt;

extern "C" {

kkt_status kkt_schur_matrix(kkt_handle* hh, double** S, int64_t* ld) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !S || !ld) {
    set_error("kkt_schur_matrix: null argument");
    return KKT_ERR_INVALID;
  }
  if (h->cum) {
    set_error("kkt_schur_matrix: the structured S (structured_s = 2) has no dense S");
    return KKT_ERR_INVALID;
  }
  *S = h->S;
  *ld = h->nC;
  return KKT_OK;
}

kkt_status kkt_factor_schur(kkt_handle* hh, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) {
    set_error("kkt_factor_schur: null handle");
    return KKT_ERR_INVALID;
  }
  if (h->cum) {
    set_error("kkt_factor_schur: the structured S (structured_s = 2) is factored by kkt_factor");
    return KKT_ERR_INVALID;
  }
  kkt_status s = need(h->blocks_factored, "kkt_factor_schur: no block factorization (kkt_factor_blocks first)");
  if (s != KKT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  h->stream = st;
  (void)cudaGetLastError();
  h->s_factor = (h->opt.prec == KKT_TF32 || h->opt.prec == KKT_BF16) ? 1 : 0;
  h->g_reduced = false;
  KKT_CUDA(launch_dense_factor_of(*h, st));
  KKT_CUDA(cudaEventRecord(h->ev_done, st));
  h->factored = true;
  h->schur_pending = false;
  return KKT_OK;
}

kkt_status kkt_schur_factor_copy(kkt_handle* hh, double* out, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || (!out && h->nC > 0)) {
    set_error("kkt_schur_factor_copy: null argument");
    return KKT_ERR_INVALID;
  }
  if (h->cum) {
    set_error("kkt_schur_factor_copy: the structured S (structured_s = 2) has no dense factor");
    return KKT_ERR_INVALID;
  }
  kkt_status s = need(h->factored, "kkt_schur_factor_copy: S is not factored");
  if (s != KKT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n2 = (int64_t)h->nC * h->nC;
  if (n2 == 0) return KKT_OK;
  if (h->s_factor == 1) {
    k_f32_to_f64<<<grid_of(n2), 256, 0, st>>>(h->S32, out, n2);
    h->launches++;
    KKT_CUDA(cudaGetLastError());
  } else {
    KKT_CUDA(cudaMemcpyAsync(out, h->S, sizeof(double) * (size_t)n2, cudaMemcpyDeviceToDevice, st));
  }
  return KKT_OK;
}

kkt_status kkt_accumulate(double* dst, int64_t ld_dst, const double* src, int64_t ld_src, int64_t rows,
                          int64_t cols, void* stream) {
  if (rows < 0 || cols < 0 || ((!dst || !src) && rows * cols > 0) || (cols > 1 && (ld_dst < rows || ld_src < rows))) {
    set_error("kkt_accumulate: invalid argument");
    return KKT_ERR_INVALID;
  }
  if (rows * cols == 0) return KKT_OK;
  k_accumulate<<<grid_of(rows * cols), 256, 0, (cudaStream_t)stream>>>(dst, ld_dst, src, ld_src, rows, cols);
  KKT_CUDA(cudaGetLastError());
  return KKT_OK;
}

kkt_status kkt_solve_front(kkt_handle* hh, const double* rhs, double* t, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !rhs || (!t && h->nC > 0)) {
    set_error("kkt_solve_front: null argument");
    return KKT_ERR_INVALID;
  }
  kkt_status s = need(h->blocks_factored, "kkt_solve_front: no block factorization");
  if (s != KKT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  h->stream = st;
  (void)cudaGetLastError();
  KKT_CUDA(launch_apply_front(*h, rhs, st));
  if (h->nC > 0) KKT_CUDA(cudaMemcpyAsync(t, h->tg, sizeof(double) * h->nC, cudaMemcpyDeviceToDevice, st));
  KKT_CUDA(cudaEventRecord(h->ev_done, st));
  h->front_done = true;
  return KKT_OK;
}

kkt_status kkt_solve_coupling(kkt_handle* hh, const double* t, double* xg, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || ((!t || !xg) && h->nC > 0) || (t == xg && h->nC > 0)) {
    set_error("kkt_solve_coupling: null or aliased argument");
    return KKT_ERR_INVALID;
  }
  kkt_status s = need(h->factored, "kkt_solve_coupling: S is not factored");
  if (s != KKT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  h->stream = st;
  (void)cudaGetLastError();
  if (h->nC > 0)
    KKT_CUDA(h->cum ? launch_cum_solve(*h, t, xg, st)
                    : h->s_factor == 1 ? launch_dense_solve_f32(*h, t, xg, st) : launch_dense_solve(*h, t, xg, st));
  KKT_CUDA(cudaEventRecord(h->ev_done, st));
  return KKT_OK;
}

kkt_status kkt_solve_back(kkt_handle* hh, const double* xg, double* x, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !x || (!xg && h->nC > 0)) {
    set_error("kkt_solve_back: null argument");
    return KKT_ERR_INVALID;
  }
  kkt_status s = need(h->front_done, "kkt_solve_back: no front half on this handle (kkt_solve_front first)");
  if (s != KKT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  h->stream = st;
  (void)cudaGetLastError();
  if (h->nC > 0) KKT_CUDA(cudaMemcpyAsync(h->xg, xg, sizeof(double) * h->nC, cudaMemcpyDeviceToDevice, st));
  KKT_CUDA(launch_apply_back(*h, x, st, false));
  KKT_CUDA(cudaEventRecord(h->ev_done, st));
  h->front_done = false;
  return KKT_OK;
}

kkt_status kkt_residual(kkt_handle* hh, const double* rhs, const double* x, double* rho, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !rhs || !x || !rho) {
    set_error("kkt_residual: null argument");
    return KKT_ERR_INVALID;
  }
  kkt_status s = need(h->blocks_factored, "kkt_residual: no values (kkt_factor or kkt_factor_blocks first)");
  if (s != KKT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  (void)cudaGetLastError();
  KKT_CUDA(launch_residual(*h, rhs, x, rho, st));
  return KKT_OK;
}

kkt_status kkt_abs_rowsums(kkt_handle* hh, double* out, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !out) {
    set_error("kkt_abs_rowsums: null argument");
    return KKT_ERR_INVALID;
  }
  kkt_status s = need(h->blocks_factored, "kkt_abs_rowsums: no values (kkt_factor or kkt_factor_blocks first)");
  if (s != KKT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  (void)cudaGetLastError();
  const int64_t nb = (int64_t)h->nA * h->N;
  k_rowsum_blocks<<<grid_of(nb), 256, 0, st>>>(h->d.full_rowptr, h->d.full_src, h->a_vals, h->nnzA, h->nA, h->N,
                                               out);
  h->launches++;
  const int k = h->cpl.k;
  if (k > 0) {
    k_rowsum_b<<<(k * h->N + 255) / 256, 256, 0, st>>>(h->d.bt_ptr, h->b_vals, h->d.E, k, h->nA, h->N, out);
    h->launches++;
  }
  if (h->nC > 0) {
    k_rowsum_g<<<(h->nC + 255) / 256, 256, 0, st>>>(h->d.t_ptr, h->d.t_e, h->b_vals, h->c_vals, h->c_kind, h->nC,
                                                    out + nb);
    h->launches++;
  }
  KKT_CUDA(cudaGetLastError());
  return KKT_OK;
}

kkt_status kkt_norm_inf(kkt_handle* hh, const double* v, int64_t n, double* out, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !out || n < 0 || (!v && n > 0)) {
    set_error("kkt_norm_inf: invalid argument");
    return KKT_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  (void)cudaGetLastError();
  KKT_CUDA(cudaMemsetAsync(h->red + 8, 0, sizeof(double), st));
  if (n > 0) {
    k_maxabs<<<grid_of(n), 256, 0, st>>>(v, n, h->red + 8);
    h->launches++;
  }
  KKT_CUDA(cudaMemcpyAsync(h->host_red + 5, h->red + 8, sizeof(double), cudaMemcpyDeviceToHost, st));
  KKT_CUDA(cudaStreamSynchronize(st));
  *out = h->host_red[5];
  return KKT_OK;
}

}  // extern "C"
