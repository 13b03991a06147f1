// (b) Schur contraction G_i = W_i^T D_i^{-1} W_i on the tensor cores (tcgen05)
// for the TF32 / BF16 modes.
//
// The blocks are quasidefinite, so the sign of every pivot is known from the
// pattern (primal +, multiplier -).  With w_rho the rows of W_i scaled by
// |d_rho|^{-1/2}, G_i = sum_{d>0} w w^T - sum_{d<0} w w^T: one operand tile
// serves as both MMA operands, and the two sums go to two tensor-memory
// accumulators.  The reach rows are visited primal first, each group padded to
// 64-row chunks, so every chunk feeds one accumulator.
//
// One CTA per block: the 128 threads stream the chunks of W (converted to TF32
// or BF16 into the K-major core-matrix layout of shared memory, two buffers),
// one thread issues the MMAs (M = N = 128 covering k <= 128 columns of W), and
// four warps drain tensor memory into G_i in FP64.
#include <cuda_bf16.h>

#include "handle.h"

namespace kkt {

namespace {

constexpr int GK = 64;          // rows of W per chunk (reduction length of one stage)
constexpr int GM = 128;         // columns of W covered (M = N of the MMA)
constexpr long long kWait = 4000000000LL;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(bar), "r"(parity)
                 : "memory");
    if (done) return true;
    if (clock64() - t0 > kWait) return false;
  }
}

template <int BF16>
__global__ void __launch_bounds__(128, 1) k_contract_g_tc(const double* __restrict__ W,
                                                          const double* __restrict__ Lx, int64_t pt,
                                                          const int64_t* __restrict__ w_dpos,
                                                          const int32_t* __restrict__ g_rows, int nchunks,
                                                          int nchunks_pos, int nw, int k,
                                                          double* __restrict__ G, int* err) {
  constexpr int ESZ = BF16 ? 2 : 4;
  constexpr int KPC = 16 / ESZ;             // K elements per 16-byte core row
  constexpr int KG = GK / KPC;              // cores along K
  constexpr int BUF = GM / 8 * KG * 128;    // bytes of one chunk image
  constexpr int KSTEPS = GK * ESZ / 32;     // MMAs per chunk (32 bytes of K each)
  extern __shared__ __align__(128) uint8_t gbuf[];  // two chunk images of BUF bytes
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  const int b = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double* Wb = W + (int64_t)b * nw * k;
  const double* Pb = Lx + b * pt;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(su32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | ((uint32_t)(BF16 ? 1 : 2) << 7) | ((uint32_t)(BF16 ? 1 : 2) << 10) |
                         ((uint32_t)(GM >> 3) << 17) | ((uint32_t)(GM >> 4) << 24);
  bool ok = true;
  uint32_t phase[2] = {0u, 0u};
  bool first_pos = true, first_neg = true;
  for (int c = 0; c < nchunks; c++) {
    const int sb = c & 1;
    if (c >= 2) {
      // the MMAs of chunk c-2 read this buffer: wait for their commit
      if (!wait_parity(su32(&bar[sb]), phase[sb])) {
        atomicExch(err, 4);
        ok = false;
      }
      phase[sb] ^= 1u;
    }
    // thread t converts column t of the 64 rows of this chunk
    uint8_t* dst = gbuf + sb * BUF;
    const int t = tid;
    for (int j = 0; j < GK; j++) {
      const int rho = g_rows[c * GK + j];
      float v = 0.f;
      if (rho >= 0 && t < k) v = (float)(Wb[(int64_t)rho * k + t] * rsqrt(fabs(Pb[w_dpos[rho]])));
      uint8_t* p = dst + ((t / 8) * KG + j / KPC) * 128 + (t % 8) * 16 + (j % KPC) * ESZ;
      if (BF16) *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v);
      else *reinterpret_cast<float*>(p) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const bool pos = c < nchunks_pos;
      const uint32_t dtm = tmem + (pos ? 0u : (uint32_t)GM);
      for (int ks = 0; ks < KSTEPS; ks++) {
        const uint64_t dsc = desc(su32(dst + ks * 256), 128, KG * 128);
        const uint32_t acc = (pos ? first_pos : first_neg) ? 0u : 1u;
        if (pos) first_pos = false;
        else first_neg = false;
        if (BF16)
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtm),
                       "l"(dsc), "l"(dsc), "r"(idesc), "r"(acc));
        else
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtm),
                       "l"(dsc), "l"(dsc), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&bar[sb]))
                   : "memory");
    }
    // broadcast the first-use flags are only tracked by thread 0
  }
  // drain: wait for the last (up to two) commits
  for (int c = (nchunks >= 2 ? nchunks - 2 : 0); c < nchunks; c++) {
    const int sb = c & 1;
    if (!wait_parity(su32(&bar[sb]), phase[sb])) {
      atomicExch(err, 4);
      ok = false;
      wait_parity(su32(&bar[sb]), phase[sb]);  // second bounded window before tensor memory is freed
    }
    phase[sb] ^= 1u;
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int t1 = warp * 32 + lane;
    double* Gb = G + (int64_t)b * k * k;
    const bool has_pos = nchunks_pos > 0, has_neg = nchunks > nchunks_pos;
    for (int c0 = 0; c0 < GM; c0 += 32) {
      uint32_t rp[32], rn[32];
#pragma unroll
      for (int j = 0; j < 32; j++) rp[j] = rn[j] = 0u;
      if (has_pos) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(rp[0]), "=r"(rp[1]), "=r"(rp[2]), "=r"(rp[3]), "=r"(rp[4]), "=r"(rp[5]), "=r"(rp[6]), "=r"(rp[7]),
              "=r"(rp[8]), "=r"(rp[9]), "=r"(rp[10]), "=r"(rp[11]), "=r"(rp[12]), "=r"(rp[13]), "=r"(rp[14]), "=r"(rp[15]),
              "=r"(rp[16]), "=r"(rp[17]), "=r"(rp[18]), "=r"(rp[19]), "=r"(rp[20]), "=r"(rp[21]), "=r"(rp[22]), "=r"(rp[23]),
              "=r"(rp[24]), "=r"(rp[25]), "=r"(rp[26]), "=r"(rp[27]), "=r"(rp[28]), "=r"(rp[29]), "=r"(rp[30]), "=r"(rp[31])
            : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
      }
      if (has_neg) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(rn[0]), "=r"(rn[1]), "=r"(rn[2]), "=r"(rn[3]), "=r"(rn[4]), "=r"(rn[5]), "=r"(rn[6]), "=r"(rn[7]),
              "=r"(rn[8]), "=r"(rn[9]), "=r"(rn[10]), "=r"(rn[11]), "=r"(rn[12]), "=r"(rn[13]), "=r"(rn[14]), "=r"(rn[15]),
              "=r"(rn[16]), "=r"(rn[17]), "=r"(rn[18]), "=r"(rn[19]), "=r"(rn[20]), "=r"(rn[21]), "=r"(rn[22]), "=r"(rn[23]),
              "=r"(rn[24]), "=r"(rn[25]), "=r"(rn[26]), "=r"(rn[27]), "=r"(rn[28]), "=r"(rn[29]), "=r"(rn[30]), "=r"(rn[31])
            : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(GM + c0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
      }
      if (t1 < k) {
#pragma unroll
        for (int j = 0; j < 32; j++) {
          const int t2 = c0 + j;
          if (t2 < k) Gb[(int64_t)t1 * k + t2] = (double)__uint_as_float(rp[j]) - (double)__uint_as_float(rn[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

}  // namespace

// Kernel attributes set once (before any launch, outside stream capture).
cudaError_t schur_tc_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_contract_g_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       2 * (GM / 8) * (GK / 8) * 128);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_contract_g_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * (GM / 8) * (GK / 4) * 128);
  return e;
}

bool contract_g_tc_supported(const Handle& h) { return h.cpl.k > 0 && h.cpl.k <= GM && h.cpl.nw > 0; }

cudaError_t launch_contract_g_tc(Handle& h, int bf16, cudaStream_t st) {
  const int nchunks = h.g_nchunks, npos = h.g_nchunks_pos;
  const int smem = 2 * (GM / 8) * (GK / (16 / (bf16 ? 2 : 4))) * 128;
  cudaError_t e;
  if (bf16)
    k_contract_g_tc<1><<<h.N, 128, smem, st>>>(h.W, h.Lx, h.sym.panel_total, h.d.w_dpos, h.d.g_rows, nchunks, npos,
                                           h.cpl.nw, h.cpl.k, h.G, h.dev_err);
  else
    k_contract_g_tc<0><<<h.N, 128, smem, st>>>(h.W, h.Lx, h.sym.panel_total, h.d.w_dpos, h.d.g_rows, nchunks, npos,
                                           h.cpl.nw, h.cpl.k, h.G, h.dev_err);
  h.launches++;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_add_tail_g(h, st);
}

}  // namespace kkt
