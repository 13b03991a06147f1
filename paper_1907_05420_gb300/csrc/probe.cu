// FP64 FMA throughput of the current device: the denominator of the roofline
// of the FP64-bound phases (block factor, FP64 Schur contraction, FP64 dense
// factor).  Each thread runs 8 independent FMA chains, so the FP64 pipe, not
// latency, limits the rate.  Also the pivot reciprocal of the factor kernels
// beside CUDA's own FP64 division, for the tests.
#include <cuda_runtime.h>

#include <algorithm>

#include "handle.h"
#include "pivot.cuh"

namespace kkt {
namespace {

__global__ void __launch_bounds__(256) k_fp64_fma(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; i++) x[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; i++) s += x[i];
  if (s == 12345.678) out[0] = s;  // keeps the chains alive
}

__global__ void k_recip_pair(const double* __restrict__ d, int64_t n, double* __restrict__ recip,
                             double* __restrict__ quot) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    recip[q] = pivot_recip(d[q]);
    quot[q] = 1.0 / d[q];
  }
}

}  // namespace
}  // namespace kkt

extern "C" kkt_status kkt_probe_pivot_reciprocal(const double* d, int64_t n, double* recip, double* quotient,
                                                 void* stream) {
  using namespace kkt;
  if (n < 0 || (n > 0 && (!d || !recip || !quotient))) {
    set_error("kkt_probe_pivot_reciprocal: invalid argument");
    return KKT_ERR_INVALID;
  }
  if (n == 0) return KKT_OK;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  k_recip_pair<<<grid, 256, 0, (cudaStream_t)stream>>>(d, n, recip, quotient);
  KKT_CUDA(cudaGetLastError());
  return KKT_OK;
}

extern "C" kkt_status kkt_measure_fp64_peak(double* gflops) {
  using namespace kkt;
  if (!gflops) return KKT_ERR_INVALID;
  int dev = 0, sms = 0;
  KKT_CUDA(cudaGetDevice(&dev));
  KKT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double* out = nullptr;
  KKT_CUDA(cudaMalloc(&out, sizeof(double)));
  cudaEvent_t e0, e1;
  KKT_CUDA(cudaEventCreate(&e0));
  KKT_CUDA(cudaEventCreate(&e1));
  const int blocks = sms * 8, threads = 256, iters = 4096;
  k_fp64_fma<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 5; rep++) {
    cudaEventRecord(e0);
    k_fp64_fma<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) {
    set_error(std::string("kkt_measure_fp64_peak: ") + cudaGetErrorString(err));
    return KKT_ERR_CUDA;
  }
  const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
  *gflops = flops / (best * 1e-3) / 1e9;
  return KKT_OK;
}
