// (c) Dense LDL^T of S with the trailing update on the tensor cores
// (tcgen05 MMA into tensor memory), in three arithmetics:
//
//   TF32 / BF16:  S held in FP32; the update S22 -= Y L21^T takes Y = L21 D and
//                 L21 rounded to TF32 or BF16 and accumulates in FP32.
//   F64 (emulated): S held in FP64.  Each row of Y and of L21 is scaled by a
//                 power of two 2^e and cut into 7 signed 8-bit digits,
//                 v = 2^e sum_s d_s 2^{-8(s+1)}, |d_s| <= 255, so every digit is
//                 an exact BF16 integer and every digit product is exact in
//                 FP32.  The 28 digit pairs with s + t <= 6 are accumulated per
//                 level d = s + t in 7 FP32 tensor-memory accumulators (levels
//                 0-3 stay below 2^24 and are exact for a 64-wide panel; the
//                 rounding of levels >= 4 is below 2^-56 of the product), and
//                 the levels are recombined in FP64:
//                   (Y L^T)_ij = 2^{e_i+f_j} sum_d 2^{-8(d+2)} acc_d[i][j].
//                 This is the FP64 product to within ~2^-50 relative.
//
// The blocked right-looking factorization (panel width 64) is that of
// dense.cu; only the trailing update and its operand preparation live here:
//   k_tc_slice:  writes the tile images of the update operands (the exact
//                shared-memory layout of one 128-row A block or 64-row B block,
//                all digit slices contiguous) and the row scales;
//   k_tc_update: (TF32, BF16) one CTA per 128 x 64 lower tile of the trailing
//                matrix; the images arrive by bulk copy, one thread issues the
//                MMAs, four warps drain tensor memory and update S;
//   k_tc_update_emu: (emulated FP64) one CTA per run of up to 8 tiles of a tile
//                row, with loads, products and the read-modify-write of S
//                overlapped across the run (below).
//
// Shared-memory operand layout (K-major, no swizzle): an 8-row x 16-byte core
// matrix is 128 contiguous bytes; cores are ordered K-fastest, so the
// descriptor's leading byte offset (along K) is 128 and its stride byte offset
// (along M/N) is 128 * (cores per row group).
#include <cuda_bf16.h>

#include "dense_kernels.cuh"
#include "emu_arith.cuh"

namespace kkt {

namespace {

constexpr int TM = 128;       // rows of an A block (MMA M)
constexpr int TN = 64;        // rows of a B block (MMA N)
constexpr int TK = kDenseNB;  // panel width = reduction length
constexpr int kEmuLevels = 7;
static_assert(kEmuLevels == kEmuSlices, "level d holds the digit pairs sa + sb = d, 0 <= sa, sb <= d");
constexpr long long kWaitBudget = 4000000000LL;  // cycles (~2 s)

struct ModeCfg {
  int kind;     // 0 bf16 operands, 1 tf32 operands
  int slices;   // digit slices per operand
  int levels;   // accumulators in tensor memory
  int esz;      // bytes per operand element
};

__host__ __device__ constexpr ModeCfg mode_cfg(int mode) {
  // mode: 0 = TF32, 1 = BF16, 2 = FP64 emulated on BF16 digit slices
  return mode == 0 ? ModeCfg{1, 1, 1, 4} : (mode == 1 ? ModeCfg{0, 1, 1, 2} : ModeCfg{0, kEmuSlices, kEmuLevels, 2});
}

__host__ __device__ constexpr int kgroups_of(int mode) { return TK * mode_cfg(mode).esz / 16; }
__host__ __device__ constexpr int slice_bytes(int mode, int rows) { return rows / 8 * kgroups_of(mode) * 128; }
__host__ __device__ constexpr int image_bytes(int mode, int rows) {
  return mode_cfg(mode).slices * slice_bytes(mode, rows);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the fifth-generation tensor core
  return d;                // base offset 0, no swizzle
}

// The descriptor of the operand at byte offset off from the one desc
// describes: shared-memory addresses stay below 256 KB, so the 14-bit address
// field (address / 16) takes off / 16 without a carry into the other fields.
__device__ __forceinline__ uint64_t umma_desc_at(uint64_t desc, uint32_t off) { return desc + (uint64_t)(off >> 4); }

__device__ __forceinline__ void mma_bf16(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitBudget) return false;
  }
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%"
      "19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}



// Images of the operands of one panel step.  Rows rho in [0, m) are trailing
// rows base + rho.  A = Y (rows of L21 D, from Y with leading dimension n),
// B = L21 (columns k0..k0+63 of S).  Rows >= m are written as zeros.
// Batched over blockIdx.y (the dense tails of the block factors): matrix b
// is S + b * ts.s, its Y, images and scales are offset by the other strides.
struct TcStrides {
  int64_t s = 0, y = 0, img_a = 0, img_b = 0, scale = 0;
};

// One 16-byte core-matrix row of each of the 7 digit slices: the BF16 digits
// (unsigned base-256 digits of |v| 2^-e, with the sign of v) of 8 consecutive
// K entries, stored at dst + s * slice_stride for slice s.  table holds the
// BF16 bit patterns of the 256 byte values (no conversion instructions).
__device__ __forceinline__ void emu_store_core_row(const double (&v)[8], int e_exp, const uint32_t* table,
                                                   uint8_t* dst, int slice_stride) {
  uint32_t packed[kEmuSlices][4];
#pragma unroll
  for (int e = 0; e < 8; e++) {
    long long vb;
    const unsigned long long a = digits7(v[e], e_exp, vb);
    const uint32_t sgn = vb < 0 ? 0x8000u : 0u;
#pragma unroll
    for (int s = 0; s < kEmuSlices; s++) {
      const uint32_t h = table[(a >> (8 * (kEmuSlices - 1 - s))) & 0xFFull] | sgn;
      packed[s][e >> 1] = (e & 1) ? (packed[s][e >> 1] | (h << 16)) : h;
    }
  }
#pragma unroll
  for (int s = 0; s < kEmuSlices; s++)
    *reinterpret_cast<uint4*>(dst + (int64_t)s * slice_stride) =
        make_uint4(packed[s][0], packed[s][1], packed[s][2], packed[s][3]);
}

template <int MODE, class T>
__global__ void __launch_bounds__(256) k_tc_slice(const T* __restrict__ S0, const T* __restrict__ Y0,
                                                  int n, int k0, int kb, int m, uint8_t* __restrict__ imgA0,
                                                  uint8_t* __restrict__ imgB0, double* __restrict__ scaleA0,
                                                  double* __restrict__ scaleB0, int mpadA, int mpadB,
                                                  TcStrides ts) {
  const int64_t bb = blockIdx.y;
  const T* S = S0 + bb * ts.s;
  const T* Y = Y0 + bb * ts.y;
  uint8_t* imgA = imgA0 + bb * ts.img_a;
  uint8_t* imgB = imgB0 + bb * ts.img_b;
  double* scaleA = scaleA0 + bb * ts.scale;
  double* scaleB = scaleB0 + bb * ts.scale;
  constexpr ModeCfg cfg = mode_cfg(MODE);
  constexpr int KG = kgroups_of(MODE);
  constexpr int kpc = 16 / cfg.esz;  // elements per 16-byte core row
  __shared__ uint32_t bf16_of_byte[256];
  if (MODE == 2) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
      bf16_of_byte[i] = bf16_bits_of_byte((uint32_t)i);
    __syncthreads();
  }
  const int base = k0 + kb;
  const int total = mpadA + mpadB;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const bool isA = q < mpadA;
    const int rho = isA ? q : q - mpadA;
    const int rows_blk = isA ? TM : TN;
    uint8_t* img = isA ? imgA : imgB;
    const T* src = isA ? Y : S;
    const int64_t col0 = isA ? 0 : k0;  // Y columns are 0..63, L21 columns k0..k0+63
    const int blk = rho / rows_blk, rr = rho % rows_blk, g = rr / 8, r8 = rr % 8;
    uint8_t* blk_img = img + (int64_t)blk * image_bytes(MODE, rows_blk);
    const bool live = rho < m;
    double e_scale = 1.0;
    int e_exp = 0;
    if (MODE == 2) {
      // e = ilogb(max |v|) + 1 from the largest exponent field; rows whose
      // largest entry is subnormal (or zero) take the FP64 route
      int emax = 0;
      if (live)
        for (int c = 0; c < kb; c++) emax = max(emax, exp_field((double)src[(int64_t)(base + rho) + (col0 + c) * n]));
      if (emax > 0) {
        e_exp = emax - 1023 + 1;  // |v| < 2^e
      } else {
        double amax = 0.0;
        if (live)
          for (int c = 0; c < kb; c++) amax = fmax(amax, fabs((double)src[(int64_t)(base + rho) + (col0 + c) * n]));
        e_exp = amax > 0.0 ? ilogb(amax) + 1 : 0;
      }
      e_scale = ldexp(1.0, e_exp);
      if (isA) scaleA[rho] = e_scale;
      else scaleB[rho] = e_scale;
    }
    for (int kq = 0; kq < KG; kq++) {
      // one 16-byte core row: elements kq*kpc .. kq*kpc+kpc-1
      if (MODE == 2) {
        // BF16 bit patterns of the signed digits, from the table of the 256
        // byte values (no conversion instructions)
        double v[8] = {};
#pragma unroll
        for (int e = 0; e < kpc; e++) {
          const int c = kq * kpc + e;  // columns >= kb (a ragged panel) are zero
          v[e] = (live && c < kb) ? (double)src[(int64_t)(base + rho) + (col0 + c) * n] : 0.0;
        }
        emu_store_core_row(v, e_exp, bf16_of_byte, blk_img + (g * KG + kq) * 128 + r8 * 16,
                           slice_bytes(MODE, rows_blk));
      } else if (MODE == 1) {
        __align__(16) __nv_bfloat16 h[8];
#pragma unroll
        for (int e = 0; e < 8; e++)
          h[e] = __float2bfloat16_rn((live && kq * kpc + e < kb)
                                         ? (float)src[(int64_t)(base + rho) + (col0 + kq * kpc + e) * n]
                                         : 0.f);
        *reinterpret_cast<uint4*>(blk_img + (g * KG + kq) * 128 + r8 * 16) = *reinterpret_cast<const uint4*>(h);
      } else {
        __align__(16) float f[4];
#pragma unroll
        for (int e = 0; e < 4; e++)
          f[e] = (live && kq * kpc + e < kb) ? (float)src[(int64_t)(base + rho) + (col0 + kq * kpc + e) * n] : 0.f;
        *reinterpret_cast<uint4*>(blk_img + (g * KG + kq) * 128 + r8 * 16) = *reinterpret_cast<const uint4*>(f);
      }
    }
  }
}

// tile list: (I, J) with J <= 2I + 1 (tiles that hold part of the lower
// triangle).  jmode 0: all of them; 1: the first tile column (J = 0, the next
// panel's columns); 2: the others (J >= 1).
__device__ __forceinline__ void tile_of(int t, int TJ, int jmode, int& I, int& J) {
  if (jmode == 1) {
    I = t;
    J = 0;
    return;
  }
  // row I of the list has min(2I+2, TJ) tiles, one fewer without J = 0
  const int skip = jmode == 2 ? 1 : 0;
  int i = 0;
  for (;;) {
    const int cnt = min(2 * i + 2, TJ) - skip;
    if (t < cnt) break;
    t -= cnt;
    i++;
  }
  I = i;
  J = t + skip;
}

template <int MODE, class T>
__global__ void __launch_bounds__(128, 1) k_tc_update(T* __restrict__ S0, int n, int k0, int kb, int m, int TJ, int jmode,
                                                      const uint8_t* __restrict__ imgA0,
                                                      const uint8_t* __restrict__ imgB0,
                                                      const double* __restrict__ scaleA0,
                                                      const double* __restrict__ scaleB0, int* err,
                                                      TcStrides ts) {
  const int64_t bb = blockIdx.y;
  T* S = S0 + bb * ts.s;
  const uint8_t* imgA = imgA0 + bb * ts.img_a;
  const uint8_t* imgB = imgB0 + bb * ts.img_b;
  static_assert(MODE != 2, "the emulated-FP64 update is k_tc_update_emu");
  (void)scaleA0;
  (void)scaleB0;
  constexpr ModeCfg cfg = mode_cfg(MODE);
  constexpr int KG = kgroups_of(MODE);
  constexpr int A_BYTES = image_bytes(MODE, TM), B_BYTES = image_bytes(MODE, TN);
  constexpr int A_SLICE = slice_bytes(MODE, TM), B_SLICE = slice_bytes(MODE, TN);
  constexpr uint32_t TMEM_COLS = cfg.levels * TN <= 32 ? 32 : (cfg.levels * TN <= 64 ? 64 : (cfg.levels * TN <= 128 ? 128 : (cfg.levels * TN <= 256 ? 256 : 512)));
  constexpr int MMA_K_BYTES = 32;  // one MMA consumes 32 bytes of K (16 bf16 or 8 tf32)
  constexpr int KSTEPS = TK * cfg.esz / MMA_K_BYTES;
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + A_BYTES;
  __shared__ __align__(8) uint64_t bar_load, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int I, J;
  tile_of(blockIdx.x, TJ, jmode, I, J);
  const int base = k0 + kb;

  if (tid == 0) {
    s_ok = 1;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_load)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_mma)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  if (tid == 0) {
    // bulk copies of the two images (16 KB pieces), completion on bar_load
    const uint32_t bl = smem_u32(&bar_load);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bl), "r"((uint32_t)(A_BYTES + B_BYTES))
                 : "memory");
    const uint8_t* srcA = imgA + (int64_t)I * A_BYTES;
    const uint8_t* srcB = imgB + (int64_t)J * B_BYTES;
    for (int off = 0; off < A_BYTES; off += 16384) {
      const uint32_t sz = (uint32_t)min(16384, A_BYTES - off);
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(sA + off)),
                   "l"(srcA + off), "r"(sz), "r"(bl)
                   : "memory");
    }
    for (int off = 0; off < B_BYTES; off += 16384) {
      const uint32_t sz = (uint32_t)min(16384, B_BYTES - off);
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(sB + off)),
                   "l"(srcB + off), "r"(sz), "r"(bl)
                   : "memory");
    }
    if (!mbar_wait(bl, 0)) {
      atomicExch(err, 2);
      s_ok = 0;
      mbar_wait(bl, 0);  // give copies still in flight a second bounded window before exit
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t idesc = (1u << 4) | ((uint32_t)(cfg.kind == 0 ? 1 : 2) << 7) |
                             ((uint32_t)(cfg.kind == 0 ? 1 : 2) << 10) | ((uint32_t)(TN >> 3) << 17) |
                             ((uint32_t)(TM >> 4) << 24);
      for (int d = 0; d < cfg.levels; d++) {
        const uint32_t dtm = tmem + (uint32_t)(d * TN);
        bool first = true;
        for (int sa = 0; sa < cfg.slices; sa++) {
          const int sb = d - sa;
          if (cfg.slices > 1 && (sb < 0 || sb >= cfg.slices)) continue;
          const int sbb = cfg.slices > 1 ? sb : 0;
          for (int ks = 0; ks < KSTEPS; ks++) {
            const uint64_t ad = umma_desc(smem_u32(sA + sa * A_SLICE + ks * MMA_K_BYTES * 8), 128, KG * 128);
            const uint64_t bd = umma_desc(smem_u32(sB + sbb * B_SLICE + ks * MMA_K_BYTES * 8), 128, KG * 128);
            const uint32_t acc = first ? 0u : 1u;
            first = false;
            if (cfg.kind == 0)
              asm volatile(
                  "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                      dtm),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            else
              asm volatile(
                  "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
                      dtm),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bar_mma))
                   : "memory");
    }
  }
  __syncthreads();
  bool ok = s_ok != 0;
  if (ok) {
    if (!mbar_wait(smem_u32(&bar_mma), 0)) {
      atomicExch(err, 3);
      ok = false;
      mbar_wait(smem_u32(&bar_mma), 0);  // second bounded window before tensor memory is freed
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int rho = I * TM + warp * 32 + lane;  // this thread's tile row
    const int row = base + rho;
    for (int cc = 0; cc < TN / 32; cc++) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), r);
      if (rho < m) {
        // all loads of the 32 columns first, then the stores: 32 loads in flight
        T cur[32];
#pragma unroll
        for (int j = 0; j < 32; j++) {
          const int cj = J * TN + cc * 32 + j;
          const int col = base + cj;
          cur[j] = (cj < m && row >= col) ? S[(int64_t)row + (int64_t)col * n] : T(0);
        }
#pragma unroll
        for (int j = 0; j < 32; j++) {
          const int cj = J * TN + cc * 32 + j;
          const int col = base + cj;
          if (cj < m && row >= col) S[(int64_t)row + (int64_t)col * n] = cur[j] - (T)__uint_as_float(r[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// ---- Emulated-FP64 update, pipelined over a run of tiles ----
//
// One CTA per task: up to kEmuRun consecutive tiles (I, J) of one tile row I.
// The A image of the row (7 digit slices of 128 rows, 112 KB) is loaded once;
// the B images (56 KB) go through two shared-memory buffers; the 28 digit
// products of each tile accumulate in tensor memory (7 levels x 64 columns).
// Warps with fixed roles:
//   warp 0 (one lane): bulk copies of A and of the B images, ahead by one;
//   warp 1 (one lane): tensor-memory allocation and the MMAs of each tile,
//                      started once the epilogue has drained the previous one;
//   warps 2-9:         the epilogue, one tile row and 32 columns per thread
//                      (warp w reads tensor-memory lanes 32 (w mod 4) ...):
//                      the 7 levels are read and folded into one integer W
//                      per entry first, tensor memory is handed back, and only
//                      then are the FP64 bit patterns built and S read,
//                      updated and written, so that the next tile's products
//                      run during this tile's bit building and global
//                      read-modify-write.
// The scaled product W 2^{e_i+f_j-56} is built as an FP64 bit pattern with
// integer operations (W rounded once, exponents added), and the levels are
// read out of FP32 without conversion instructions, which on this GPU share
// the narrow FP64 pipe; one FP64 addition per entry is left.
// Every wait is bounded: a timeout sets *err, makes the other roles stop, lets
// the copies and products in flight finish (bounded again) and frees tensor
// memory before the CTA exits.
// Epilogue warps: 8 (two per tensor-memory lane quadrant, 32 columns per
// thread).  With 10 warps a thread has 168 registers; 4 epilogue warps of 64
// columns (255 registers) left one warp per scheduler and ran 1.7x slower.
constexpr int kEpiWarps = 8;
constexpr int kEpiCols = TN * 4 / kEpiWarps;     // tile columns per epilogue thread
constexpr int kEmuThreads = 64 + 32 * kEpiWarps;  // producer, MMA issuer, epilogue
// A image and two B buffers (229,376 bytes)
__host__ __device__ constexpr int emu_smem_bytes() { return image_bytes(2, TM) + 2 * image_bytes(2, TN); }

__device__ __forceinline__ bool mbar_wait_ab(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitBudget) return false;
  }
}

__device__ __forceinline__ void bulk_load(uint8_t* dst, const uint8_t* src, int bytes, uint32_t bar) {
  for (int off = 0; off < bytes; off += 16384) {
    const uint32_t sz = (uint32_t)min(16384, bytes - off);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst + off)),
                 "l"(src + off), "r"(sz), "r"(bar)
                 : "memory");
  }
}

// The S entries an epilogue thread will read and write for one tile (its row,
// columns base + cj0 .. base + cj0 + COLS - 1 below mcol and on or below the
// diagonal) prefetched into L2 while the tile's products run: for the 32 rows
// of a warp one prefetch per column covers whole cache lines, and the
// read-modify-write after the products then waits on L2 instead of DRAM.
template <class T, int COLS>
__device__ __forceinline__ void prefetch_tile_row(const T* S, int n, int row, bool live_row, int base, int cj0,
                                                  int mcol) {
  if (!live_row) return;
#pragma unroll 8
  for (int j = 0; j < COLS; j++) {
    const int cj = cj0 + j, col = base + cj;
    if (cj < mcol && row >= col)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(S + (int64_t)row + (int64_t)col * n));
  }
}

// The epilogue's read-out of tensor memory: the 7 levels of this thread's
// kEpiCols columns (16-column loads) folded into W = V 2^16 + round(256 c),
// V the exact integer of levels 0-3 and c the FP32 sum of levels 4-6.  Only
// this part holds tensor memory; the FP64 bit patterns are built after it is
// handed back.
__device__ __forceinline__ void emu_fold(uint32_t taddr, long long (&W)[kEpiCols]) {
#pragma unroll
  for (int hh = 0; hh < kEpiCols / 16; hh++) {
    long long V[16];
    float cf[16];
#pragma unroll
    for (int j = 0; j < 16; j++) {
      V[j] = 0;
      cf[j] = 0.f;
    }
#pragma unroll
    for (int d = 0; d < kEmuLevels; d++) {
      uint32_t r[16];
      tmem_ld16(taddr + (uint32_t)(d * TN + hh * 16), r);
#pragma unroll
      for (int j = 0; j < 16; j++) {
        const float fv = __uint_as_float(r[j]);
        if (d < 4) V[j] = V[j] * 256 + exact_f2i(fv);  // levels 0-3: exact integers below 2^24
        else cf[j] += fv * (d == 4 ? 1.f : (d == 5 ? 0.00390625f : 0.0000152587890625f));
      }
    }
#pragma unroll
    for (int j = 0; j < 16; j++) W[hh * 16 + j] = V[j] * 65536 + round_f2ll(cf[j] * 256.f);  // 256 c can pass 2^31
  }
}

// S[row, col] += -W 2^{e_i + f_j - 56} for the thread's columns col = base +
// cj, cj = cj0 .. cj0 + kEpiCols - 1, that lie below mcol and on or below the
// diagonal; 16 loads of S in flight per thread.  Lane l's ebl is the exponent
// f_j of column cj0 + l; every lane of the warp takes part (the exponents go
// through shuffles).
__device__ __forceinline__ void emu_apply(double* __restrict__ S, int n, int row, bool live_row, int base, int cj0,
                                          int mcol, int ea, int ebl, const long long (&W)[kEpiCols]) {
#pragma unroll
  for (int hh = 0; hh < kEpiCols / 16; hh++) {
    double cur[16];
#pragma unroll
    for (int j = 0; j < 16; j++) {
      const int cj = cj0 + hh * 16 + j, col = base + cj;
      cur[j] = (live_row && cj < mcol && row >= col) ? S[(int64_t)row + (int64_t)col * n] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 16; j++) {
      const int c = hh * 16 + j, cj = cj0 + c, col = base + cj;
      const int eb = __shfl_sync(0xffffffffu, ebl, c);
      const double nd = neg_scaled(W[c], ea + eb);
      if (live_row && cj < mcol && row >= col) S[(int64_t)row + (int64_t)col * n] = cur[j] + nd;
    }
  }
}

__global__ void __launch_bounds__(kEmuThreads, 1)
    k_tc_update_emu(double* __restrict__ S0, int n, int k0, int kb, int m, int mcol, int TI, int TJ, int jmode,
                    const uint8_t* __restrict__ imgA0, const uint8_t* __restrict__ imgB0,
                    const double* __restrict__ scaleA0, const double* __restrict__ scaleB0, int* err,
                    TcStrides ts) {
  constexpr ModeCfg cfg = mode_cfg(2);
  constexpr int KG = kgroups_of(2);
  constexpr int A_BYTES = image_bytes(2, TM), B_BYTES = image_bytes(2, TN);
  constexpr int A_SLICE = slice_bytes(2, TM), B_SLICE = slice_bytes(2, TN);
  constexpr uint32_t TMEM_COLS = 512;  // 7 levels x 64 columns
  constexpr int MMA_K_BYTES = 32;
  constexpr int KSTEPS = TK * cfg.esz / MMA_K_BYTES;
  static_assert(cfg.levels * TN <= (int)TMEM_COLS, "levels must fit tensor memory");
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + A_BYTES;  // two buffers of B_BYTES
  __shared__ __align__(8) uint64_t bar_a, bar_bfull[2], bar_bempty[2], bar_tfull, bar_tempty;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;

  const int64_t bb = blockIdx.y;
  double* S = S0 + bb * ts.s;
  const uint8_t* imgA = imgA0 + bb * ts.img_a;
  const uint8_t* imgB = imgB0 + bb * ts.img_b;
  const double* scaleA = scaleA0 + bb * ts.scale;
  const double* scaleB = scaleB0 + bb * ts.scale;
  // task -> tile row I and its run of tiles [j0, j1)
  int I, j0, j1;
  emu_task(blockIdx.x, TI, TJ, jmode, I, j0, j1);
  const int ntile = max(0, j1 - j0);
  const int base = k0 + kb;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_a)));
    for (int s = 0; s < 2; s++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_bfull[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_bempty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_tfull)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_tempty)), "r"(kEpiWarps));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0 && ntile > 0) {
      // producer
      const uint32_t ba = smem_u32(&bar_a);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ba), "r"((uint32_t)A_BYTES)
                   : "memory");
      bulk_load(sA, imgA + (int64_t)I * A_BYTES, A_BYTES, ba);
      int armed[2] = {0, 0};  // loads issued per B buffer
      for (int u = 0; u < ntile; u++) {
        const int s = u & 1;
        if (u >= 2 && !mbar_wait_ab(smem_u32(&bar_bempty[s]), (uint32_t)(((u >> 1) - 1) & 1), &s_abort)) {
          if (!s_abort) atomicExch(err, 4);
          s_abort = 1;
          break;
        }
        const uint32_t bf = smem_u32(&bar_bfull[s]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bf), "r"((uint32_t)B_BYTES)
                     : "memory");
        bulk_load(sB + s * B_BYTES, imgB + (int64_t)(j0 + u) * B_BYTES, B_BYTES, bf);
        armed[s]++;
      }
      // the copies issued must land before the CTA's shared memory goes away
      volatile int never = 0;
      mbar_wait_ab(ba, 0u, &never);
      for (int s = 0; s < 2; s++)
        if (armed[s] > 0) mbar_wait_ab(smem_u32(&bar_bfull[s]), (uint32_t)((armed[s] - 1) & 1), &never);
    }
  } else if (warp == 1) {
    if (lane == 0 && ntile > 0) {
      // MMA issuer
      int issued = 0;
      if (!mbar_wait_ab(smem_u32(&bar_a), 0u, &s_abort)) {
        if (!s_abort) atomicExch(err, 5);
        s_abort = 1;
      } else {
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                               ((uint32_t)(TM >> 4) << 24);
        for (int u = 0; u < ntile; u++) {
          const int s = u & 1;
          if (!mbar_wait_ab(smem_u32(&bar_bfull[s]), (uint32_t)((u >> 1) & 1), &s_abort) ||
              (u >= 1 && !mbar_wait_ab(smem_u32(&bar_tempty), (uint32_t)((u - 1) & 1), &s_abort))) {
            if (!s_abort) atomicExch(err, 6);
            s_abort = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint64_t a0 = umma_desc(smem_u32(sA), 128, KG * 128);
          const uint64_t b0 = umma_desc(smem_u32(sB + s * B_BYTES), 128, KG * 128);
          // level d takes the digit pairs sa + sb = d
#pragma unroll
          for (int d = 0; d < kEmuLevels; d++) {
            const uint32_t dtm = tmem + (uint32_t)(d * TN);
#pragma unroll
            for (int sa = 0; sa <= d; sa++)
#pragma unroll
              for (int ks = 0; ks < KSTEPS; ks++)
                mma_bf16(dtm, umma_desc_at(a0, sa * A_SLICE + ks * MMA_K_BYTES * 8),
                         umma_desc_at(b0, (d - sa) * B_SLICE + ks * MMA_K_BYTES * 8), idesc,
                         (sa == 0 && ks == 0) ? 0u : 1u);
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&bar_bempty[s]))
                       : "memory");
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&bar_tfull))
                       : "memory");
          issued++;
        }
      }
      // products in flight must finish before tensor memory is freed
      volatile int never = 0;
      if (issued > 0) mbar_wait_ab(smem_u32(&bar_tfull), (uint32_t)((issued - 1) & 1), &never);
    }
  } else {
    // epilogue: tile row rho = I*128 + 32 (warp mod 4) + lane, columns
    // cbase .. cbase + kEpiCols - 1 of each tile
    const int q = warp & 3, cbase = ((warp - 2) >> 2) * kEpiCols;
    const int rho = I * TM + q * 32 + lane;
    const int row = base + rho;
    const bool live_row = rho < m;
    const int ea = pow2_exponent(live_row ? scaleA[rho] : 1.0) - 56;
    for (int u = 0; u < ntile; u++) {
      const int J = j0 + u;
      const int cj0 = J * TN + cbase;
      // exponents of this lane's column scales, shared across the warp below
      int ebl[kEpiCols / 32];
#pragma unroll
      for (int g = 0; g < kEpiCols / 32; g++)
        ebl[g] = pow2_exponent(cj0 + g * 32 + lane < m ? scaleB[cj0 + g * 32 + lane] : 1.0);
      prefetch_tile_row<double, kEpiCols>(S, n, row, live_row, base, cj0, mcol);
      bool ok = true;
      if (lane == 0) ok = mbar_wait_ab(smem_u32(&bar_tfull), (uint32_t)(u & 1), &s_abort);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) {
        if (lane == 0) {
          if (!s_abort) atomicExch(err, 7);
          s_abort = 1;
        }
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      long long W[kEpiCols];
      emu_fold(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)cbase, W);
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar_tempty)) : "memory");
      emu_apply(S, n, row, live_row, base, cj0, mcol, ea, ebl[0], W);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// ---- Emulated-FP64 panel of a 64-column step ----
//
// The panel of a step, Y = A21 L11^{-T} and L21 = Y D1^{-1} (the rows below
// the diagonal block), as a product on the tensor cores instead of one
// substitution per row on the FP64 pipe: W = L11^{-1} is formed per matrix
// in FP64 (k_panel_inverse_slice, 64 x 64: column j of W by the substitution
// that k_dense_panel_t runs for a row, applied to the unit vector e_j; the
// same launch slices the rows of A21 into digits), and
// Y = A21 W^T is one 64-column product with K = 64 in the format of the
// 64-wide emulated update (7 BF16 digit slices, 7 exact tensor-memory levels,
// the same fold), written instead of accumulated (k_tc_panel_emu).  The
// rounding differs from the substitution's: the product is within the
// rounding of an FP64 dot product with W's rows, W within that of the
// substitution, so the panel's residual A21 - Y L11^T grows with the
// condition of the unit lower triangle L11, which the diagonal blocks of
// these quasidefinite matrices keep small.

// The two operands of k_tc_panel_emu for matrix blockIdx.y, in one launch.
// CTA 0: W = L11^{-1} (the kb x kb unit lower triangle at (k0, k0) after
// k_dense_diag_t) and the digit image of its rows, the B operand: row i of B
// is row i of W (K index = column), rows and columns >= kb zero, the row
// scales in scaleB[0..63].  CTAs 1..: the digit image of the rows of A21
// (columns k0 .. k0 + kb of the rows below the diagonal block, rows >= m
// zero), the A operand, with the row scales and layout of k_tc_slice.
__global__ void __launch_bounds__(256) k_panel_inverse_slice(const double* __restrict__ S0, int n, int k0, int kb,
                                                             int m, int mpadA, uint8_t* __restrict__ imgA0,
                                                             uint8_t* __restrict__ imgB0,
                                                             double* __restrict__ scaleA0,
                                                             double* __restrict__ scaleB0, TcStrides ts) {
  constexpr int KG = kgroups_of(2);
  __shared__ double M[TK][TK + 1];  // L11 by rows, then W by rows
  __shared__ uint32_t bf16_of_byte[256];
  const int64_t bb = blockIdx.y;
  const double* S = S0 + bb * ts.s;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) bf16_of_byte[i] = bf16_bits_of_byte((uint32_t)i);
  __syncthreads();
  if (blockIdx.x > 0) {
    uint8_t* imgA = imgA0 + bb * ts.img_a;
    double* scaleA = scaleA0 + bb * ts.scale;
    for (int rho = (blockIdx.x - 1) * blockDim.x + threadIdx.x; rho < mpadA;
         rho += (gridDim.x - 1) * blockDim.x) {
      const bool live = rho < m;
      const double* src = S + (int64_t)(k0 + kb + rho) + (int64_t)k0 * n;  // column c at src[c n]
      // e = ilogb(max |v|) + 1 from the largest exponent field; rows whose
      // largest entry is subnormal (or zero) take the FP64 route
      int emax = 0;
      if (live)
        for (int c = 0; c < kb; c++) emax = max(emax, exp_field(src[(int64_t)c * n]));
      int e_exp;
      if (emax > 0) {
        e_exp = emax - 1023 + 1;  // |v| < 2^e
      } else {
        double amax = 0.0;
        if (live)
          for (int c = 0; c < kb; c++) amax = fmax(amax, fabs(src[(int64_t)c * n]));
        e_exp = amax > 0.0 ? ilogb(amax) + 1 : 0;
      }
      scaleA[rho] = ldexp(1.0, e_exp);
      const int rr = rho % TM;
      uint8_t* blk_img = imgA + (int64_t)(rho / TM) * image_bytes(2, TM) + (rr / 8) * KG * 128 + (rr % 8) * 16;
      for (int kq = 0; kq < KG; kq++) {
        double v[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
          const int c = kq * 8 + e;
          v[e] = (live && c < kb) ? src[(int64_t)c * n] : 0.0;
        }
        emu_store_core_row(v, e_exp, bf16_of_byte, blk_img + kq * 128, slice_bytes(2, TM));
      }
    }
    return;
  }
  uint8_t* imgB = imgB0 + bb * ts.img_b;
  double* scaleB = scaleB0 + bb * ts.scale;
  for (int q = threadIdx.x; q < TK * TK; q += blockDim.x) {
    const int c = q / TK, j = q - c * TK;
    M[j][c] = (j > c && j < kb) ? S[(int64_t)(k0 + j) + (int64_t)(k0 + c) * n] : 0.0;
  }
  __syncthreads();
  // column jc of W: w L11^T = e_jc solved as a row, subtracted in increasing c
  const int jc = threadIdx.x;
  double w[TK];
  if (jc < TK) {
#pragma unroll
    for (int c = 0; c < TK; c++) w[c] = (c == jc && c < kb) ? 1.0 : 0.0;
#pragma unroll
    for (int j = 1; j < TK; j++) {
      double acc = w[j];
#pragma unroll
      for (int c = 0; c < j; c++) acc -= w[c] * M[j][c];
      w[j] = acc;
    }
  }
  __syncthreads();  // every read of L11 is done
  if (jc < TK) {
#pragma unroll
    for (int i = 0; i < TK; i++) M[i][jc] = w[i];
  }
  __syncthreads();
  // the digit image: 64 rows x 8 core rows of K, two per thread
  for (int q = threadIdx.x; q < TK * KG; q += blockDim.x) {
    const int i = q / KG, kq = q - i * KG;
    int emax = 0;
    double amax = 0.0;
    for (int c = 0; c < TK; c++) {
      emax = max(emax, exp_field(M[i][c]));
      amax = fmax(amax, fabs(M[i][c]));
    }
    // |w| < 2^e; rows whose largest entry is subnormal (or zero) take ilogb
    const int e_exp = emax > 0 ? emax - 1023 + 1 : (amax > 0.0 ? ilogb(amax) + 1 : 0);
    if (kq == 0) scaleB[i] = ldexp(1.0, e_exp);
    double v[8];
#pragma unroll
    for (int e = 0; e < 8; e++) v[e] = M[i][kq * 8 + e];
    emu_store_core_row(v, e_exp, bf16_of_byte, imgB + ((i / 8) * KG + kq) * 128 + (i % 8) * 16,
                       slice_bytes(2, TN));
  }
}

// Y = A21 W^T for the 128-row tile blockIdx.x of matrix blockIdx.y: the A
// image of the tile and the B image of W (k_panel_inverse_slice) are copied once,
// thread 0 issues the 112 MMAs (28 digit pairs x 4 K steps of 16) into the 7
// levels, and 8 warps (two per tensor-memory lane quadrant, 32 columns each)
// fold the levels and write Y (leading dimension n) and L21 = Y D1^{-1} into
// the panel's columns of S.  Both waits are bounded (a timeout sets *err).
__host__ __device__ constexpr int panel_emu_smem_bytes() { return image_bytes(2, TM) + image_bytes(2, TN); }

__global__ void __launch_bounds__(256, 1) k_tc_panel_emu(double* __restrict__ S0, double* __restrict__ Y0, int n,
                                                         int k0, int kb, int m, const uint8_t* __restrict__ imgA0,
                                                         const uint8_t* __restrict__ imgB0,
                                                         const double* __restrict__ scaleA0,
                                                         const double* __restrict__ scaleB0, int* err,
                                                         TcStrides ts) {
  constexpr int KG = kgroups_of(2);
  constexpr int A_BYTES = image_bytes(2, TM), B_BYTES = image_bytes(2, TN);
  constexpr int A_SLICE = slice_bytes(2, TM), B_SLICE = slice_bytes(2, TN);
  constexpr uint32_t TMEM_COLS = 512;  // 7 levels x 64 columns
  constexpr int KSTEPS = TK * 2 / 32;  // MMAs of K = 16 per level and digit pair
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + A_BYTES;
  __shared__ __align__(8) uint64_t bar_load, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int s_ok;
  __shared__ double dinv[TK];
  const int64_t bb = blockIdx.y;
  const int I = blockIdx.x;
  double* S = S0 + bb * ts.s;
  double* Y = Y0 + bb * ts.y;
  const uint8_t* imgA = imgA0 + bb * ts.img_a + (int64_t)I * A_BYTES;
  const uint8_t* imgB = imgB0 + bb * ts.img_b;
  const double* scaleA = scaleA0 + bb * ts.scale;
  const double* scaleB = scaleB0 + bb * ts.scale;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int base = k0 + kb;

  if (tid == 0) {
    s_ok = 1;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_load)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_mma)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (tid < TK) dinv[tid] = tid < kb ? 1.0 / S[(int64_t)(k0 + tid) + (int64_t)(k0 + tid) * n] : 0.0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  if (tid == 0) {
    const uint32_t bl = smem_u32(&bar_load);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bl), "r"((uint32_t)(A_BYTES + B_BYTES))
                 : "memory");
    bulk_load(sA, imgA, A_BYTES, bl);
    bulk_load(sB, imgB, B_BYTES, bl);
    if (!mbar_wait(bl, 0)) {
      atomicExch(err, 17);
      s_ok = 0;
      mbar_wait(bl, 0);  // give copies still in flight a second bounded window before exit
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                             ((uint32_t)(TM >> 4) << 24);
      const uint64_t a0 = umma_desc(smem_u32(sA), 128, KG * 128);
      const uint64_t b0 = umma_desc(smem_u32(sB), 128, KG * 128);
#pragma unroll
      for (int d = 0; d < kEmuLevels; d++) {
#pragma unroll
        for (int sa = 0; sa <= d; sa++)
#pragma unroll
          for (int ks = 0; ks < KSTEPS; ks++)
            mma_bf16(tmem + (uint32_t)(d * TN), umma_desc_at(a0, sa * A_SLICE + ks * 256),
                     umma_desc_at(b0, (d - sa) * B_SLICE + ks * 256), idesc, (sa == 0 && ks == 0) ? 0u : 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bar_mma))
                   : "memory");
    }
  }
  __syncthreads();
  bool ok = s_ok != 0;
  if (ok && !mbar_wait(smem_u32(&bar_mma), 0)) {
    if (tid == 0) atomicExch(err, 18);
    ok = false;
    mbar_wait(smem_u32(&bar_mma), 0);  // second bounded window before tensor memory is freed
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int q = warp & 3, cbase = (warp >> 2) * kEpiCols;
    const int rho = I * TM + q * 32 + lane;
    const int row = base + rho;
    const bool live_row = rho < m;
    const int ea = pow2_exponent(live_row ? scaleA[rho] : 1.0) - 56;
    const int ebl = pow2_exponent(cbase + lane < kb ? scaleB[cbase + lane] : 1.0);
    long long W[kEpiCols];
    emu_fold(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)cbase, W);
#pragma unroll
    for (int c = 0; c < kEpiCols; c++) {
      const int j = cbase + c;
      const int eb = __shfl_sync(0xffffffffu, ebl, c);
      const double y = -neg_scaled(W[c], ea + eb);
      if (live_row && j < kb) {
        Y[(int64_t)row + (int64_t)j * n] = y;
        S[(int64_t)row + (int64_t)(k0 + j) * n] = y * dinv[j];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// ---- Emulated-FP64 update of a 256-wide outer panel ----
//
// The emulated factors (dense tails of the block factors, S in the emulated
// mode and the FP64 fallback) also run in outer panels of 256 columns: the
// 64-wide steps update only the outer panel's own columns, and the rest of the
// trailing matrix takes one update with K = 256, so that each trailing entry
// pays one epilogue (levels folded, FP64 bits built, read-modify-write) per
// 256 columns of K instead of per 64.
//
// One 256-wide operand image per outer panel (k_slice_wide): every row of Y
// (= L D) and of L over the panel's columns is scaled by a power of two 2^e
// common to the 256 columns, |v| < 2^(e-1), and cut into 7 balanced base-256
// digits in [-128, 128] (balanced7).  A digit product is then at most 2^14, so
// the FP32 tensor-memory levels 0..3 of a K = 256 accumulation stay below 2^24
// and exact, as the 64-wide update's unsigned digits do for K = 64, and the
// fold and FP64 recombination of the epilogue are the same.  Levels 4..6 round
// only where their partial sums pass 2^24, which keeps the error of the
// product within the worst-case rounding of an FP64 dot product of 256 terms.
//
// Image layout (per matrix and operand): 64-row blocks; in a block, for each
// 32-column K chunk (8 of them) and each digit slice (7), the 8 row groups x 4
// core matrices along K x 128 bytes (4 KB).  One shared-memory stage holds one
// K chunk of a 128 x 64 tile: A 7 x 8 KB, B 7 x 4 KB.
constexpr int kEwW = 256;                          // outer panel width
constexpr int kEwChunk = 32;                       // K per stage
constexpr int kEwChunks = kEwW / kEwChunk;         // 8
constexpr int kEwPiece = 4096;                     // one (block, chunk, slice): 8 row groups x 4 x 128 B
constexpr int kEwBlockBytes = kEwChunks * kEmuSlices * kEwPiece;  // 64 rows: 229,376 bytes
constexpr int kEwStageA = kEmuSlices * 2 * kEwPiece;  // 128 rows, 57,344 bytes
constexpr int kEwStageB = kEmuSlices * kEwPiece;      // 64 rows, 28,672 bytes
constexpr int kEwStages = 2;
__host__ __device__ constexpr int ew_smem_bytes() { return kEwStages * (kEwStageA + kEwStageB); }  // 168 KB

// rows rho in [0, mpad) of the outer trailing matrix of matrix blockIdx.y:
// operand A = rows of Y (columns 0..kw-1 of Yw, leading dimension n), operand
// B = rows of L (columns K0..K0+kw-1 of S); rows >= m and columns >= kw are zero.
__global__ void __launch_bounds__(128) k_slice_wide(const double* __restrict__ S0, const double* __restrict__ Yw0,
                                                    int n, int K0, int kw, int base, int m, int mpad,
                                                    uint8_t* __restrict__ imgA0, uint8_t* __restrict__ imgB0,
                                                    double* __restrict__ scaleA0, double* __restrict__ scaleB0,
                                                    int64_t s_stride, int64_t y_stride, int64_t img_stride,
                                                    int64_t scale_stride) {
  const int64_t bb = blockIdx.y;
  __shared__ uint32_t bf16_of_byte[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) bf16_of_byte[i] = bf16_bits_of_byte((uint32_t)i);
  __syncthreads();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 2 * mpad) return;
  const bool isA = q < mpad;
  const int rho = isA ? q : q - mpad;
  const bool live = rho < m;
  const double* src = isA ? Yw0 + bb * y_stride : S0 + bb * s_stride + (int64_t)K0 * n;  // column 0 of the operand
  const int64_t row = (int64_t)base + rho;
  uint8_t* img = (isA ? imgA0 : imgB0) + bb * img_stride;
  // e = ilogb(max |v|) + 2, so that |v| < 2^(e-1); rows whose largest entry is
  // subnormal or zero take the FP64 route
  int emax = 0;
  if (live)
    for (int c = 0; c < kw; c++) emax = max(emax, exp_field(src[row + (int64_t)c * n]));
  int e_exp;
  if (emax > 0) {
    e_exp = emax - 1023 + 2;
  } else {
    double amax = 0.0;
    if (live)
      for (int c = 0; c < kw; c++) amax = fmax(amax, fabs(src[row + (int64_t)c * n]));
    e_exp = amax > 0.0 ? ilogb(amax) + 2 : 0;
  }
  (isA ? scaleA0 : scaleB0)[bb * scale_stride + rho] = ldexp(1.0, e_exp);
  const int blk = rho >> 6, rr = rho & 63, g = rr >> 3, r8 = rr & 7;
  uint8_t* bimg = img + (int64_t)blk * kEwBlockBytes + (g * 4) * 128 + r8 * 16;
  for (int k = 0; k < kEwChunks; k++) {
#pragma unroll
    for (int kq = 0; kq < 4; kq++) {
      uint32_t packed[kEmuSlices][4];
#pragma unroll
      for (int e = 0; e < 8; e++) {
        const int c = k * kEwChunk + kq * 8 + e;
        const double v = (live && c < kw) ? src[row + (int64_t)c * n] : 0.0;
        long long vb;
        const unsigned long long a = digits7(v, e_exp, vb);
        int d[kEmuSlices];
        balanced7(a, d);
        const uint32_t neg = vb < 0 ? 0x8000u : 0u;
#pragma unroll
        for (int sl = 0; sl < kEmuSlices; sl++) {
          const int t = d[sl];
          const uint32_t hbits = t == 0 ? 0u : (bf16_of_byte[t < 0 ? -t : t] | ((t < 0 ? 0x8000u : 0u) ^ neg));
          packed[sl][e >> 1] = (e & 1) ? (packed[sl][e >> 1] | (hbits << 16)) : hbits;
        }
      }
#pragma unroll
      for (int sl = 0; sl < kEmuSlices; sl++)
        *reinterpret_cast<uint4*>(bimg + ((int64_t)(k * kEmuSlices + sl)) * kEwPiece + kq * 128) =
            make_uint4(packed[sl][0], packed[sl][1], packed[sl][2], packed[sl][3]);
    }
  }
}

// The K = 256 emulated update: one CTA per run of up to kEmuRun tiles (I, J)
// of one tile row I (128 x 64 tiles of the lower triangle, J <= 2I + 1);
// jmode 1 takes J < 4 (the next outer panel's 256 columns), 2 the rest.
// Warp roles as in k_tc_update_emu: warp 0 copies the K chunks of A and B of
// every tile through two shared-memory stages, warp 1 issues the 56 MMAs of
// each chunk (28 digit pairs x 2 K steps of 16) into 7 tensor-memory levels,
// warps 2..9 fold the levels of a finished tile, hand tensor memory back and
// read-modify-write S.  Every wait is bounded, as there.
__global__ void __launch_bounds__(kEmuThreads, 1)
    k_tc_update_emu_wide(double* __restrict__ S0, int n, int base, int m, int TI, int TJ, int jmode, int nchunk,
                         const uint8_t* __restrict__ imgA0, const uint8_t* __restrict__ imgB0,
                         const double* __restrict__ scaleA0, const double* __restrict__ scaleB0,
                         int64_t s_stride, int64_t img_stride, int64_t scale_stride, int* err) {
  constexpr uint32_t TMEM_COLS = 512;  // 7 levels x 64 columns
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar_full[kEwStages], bar_empty[kEwStages], bar_tfull, bar_tempty;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;
  const int64_t bb = blockIdx.y;
  double* S = S0 + bb * s_stride;
  const uint8_t* imgA = imgA0 + bb * img_stride;
  const uint8_t* imgB = imgB0 + bb * img_stride;
  const double* scaleA = scaleA0 + bb * scale_stride;
  const double* scaleB = scaleB0 + bb * scale_stride;
  int I, j0, j1;
  emu_task(blockIdx.x, TI, TJ, jmode, I, j0, j1, 4);
  const int ntile = max(0, j1 - j0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    s_abort = 0;
    for (int st = 0; st < kEwStages; st++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_full[st])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_empty[st])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_tfull)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_tempty)), "r"(kEpiWarps));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const int nsteps = ntile * nchunk;

  if (warp == 0) {
    if (lane == 0 && ntile > 0) {
      // producer: chunk g = u * nchunk + k of tile u into stage g & 1
      int armed[kEwStages] = {0, 0};
      for (int g = 0; g < nsteps; g++) {
        const int st = g & 1, u = g / nchunk, k = g - u * nchunk, J = j0 + u;
        if (g >= kEwStages && !mbar_wait_ab(smem_u32(&bar_empty[st]), (uint32_t)(((g >> 1) - 1) & 1), &s_abort)) {
          if (!s_abort) atomicExch(err, 13);
          s_abort = 1;
          break;
        }
        const uint32_t bf = smem_u32(&bar_full[st]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bf),
                     "r"((uint32_t)(kEwStageA + kEwStageB))
                     : "memory");
        uint8_t* sA = smem + st * (kEwStageA + kEwStageB);
        uint8_t* sB = sA + kEwStageA;
        for (int sl = 0; sl < kEmuSlices; sl++) {
          const int64_t piece = ((int64_t)k * kEmuSlices + sl) * kEwPiece;
          bulk_load(sA + sl * 2 * kEwPiece, imgA + (int64_t)(2 * I) * kEwBlockBytes + piece, kEwPiece, bf);
          bulk_load(sA + sl * 2 * kEwPiece + kEwPiece, imgA + (int64_t)(2 * I + 1) * kEwBlockBytes + piece, kEwPiece,
                    bf);
          bulk_load(sB + sl * kEwPiece, imgB + (int64_t)J * kEwBlockBytes + piece, kEwPiece, bf);
        }
        armed[st]++;
      }
      volatile int never = 0;
      for (int st = 0; st < kEwStages; st++)
        if (armed[st] > 0) mbar_wait_ab(smem_u32(&bar_full[st]), (uint32_t)((armed[st] - 1) & 1), &never);
    }
  } else if (warp == 1) {
    if (lane == 0 && ntile > 0) {
      // MMA issuer
      uint32_t last_bar = 0, last_par = 0;
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                             ((uint32_t)(TM >> 4) << 24);
      bool stop = false;
      for (int u = 0; u < ntile && !stop; u++) {
        if (u >= 1 && !mbar_wait_ab(smem_u32(&bar_tempty), (uint32_t)((u - 1) & 1), &s_abort)) {
          if (!s_abort) atomicExch(err, 14);
          s_abort = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int k = 0; k < nchunk; k++) {
          const int g = u * nchunk + k, st = g & 1;
          if (!mbar_wait_ab(smem_u32(&bar_full[st]), (uint32_t)((g >> 1) & 1), &s_abort)) {
            if (!s_abort) atomicExch(err, 15);
            s_abort = 1;
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint8_t* sA = smem + st * (kEwStageA + kEwStageB);
          const uint64_t a0 = umma_desc(smem_u32(sA), 128, 512);
          const uint64_t b0 = umma_desc(smem_u32(sA + kEwStageA), 128, 512);
          // level d takes the digit pairs sa + sb = d
#pragma unroll
          for (int d = 0; d < kEmuLevels; d++) {
            const uint32_t dtm = tmem + (uint32_t)(d * TN);
#pragma unroll
            for (int sa = 0; sa <= d; sa++)
#pragma unroll
              for (int ks = 0; ks < kEwChunk / 16; ks++)
                mma_bf16(dtm, umma_desc_at(a0, sa * 2 * kEwPiece + ks * 256),
                         umma_desc_at(b0, (d - sa) * kEwPiece + ks * 256), idesc,
                         (k == 0 && sa == 0 && ks == 0) ? 0u : 1u);
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&bar_empty[st]))
                       : "memory");
          last_bar = smem_u32(&bar_empty[st]);
          last_par = (uint32_t)((g >> 1) & 1);
        }
        if (stop) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bar_tfull))
                     : "memory");
        last_bar = smem_u32(&bar_tfull);
        last_par = (uint32_t)(u & 1);
      }
      volatile int never = 0;
      if (last_bar) mbar_wait_ab(last_bar, last_par, &never);
    }
  } else {
    // epilogue (as in k_tc_update_emu)
    const int q = warp & 3, cbase = ((warp - 2) >> 2) * kEpiCols;
    const int rho = I * TM + q * 32 + lane;
    const int row = base + rho;
    const bool live_row = rho < m;
    const int ea = pow2_exponent(live_row ? scaleA[rho] : 1.0) - 56;
    for (int u = 0; u < ntile; u++) {
      const int J = j0 + u;
      const int cj0 = J * TN + cbase;
      int ebl[kEpiCols / 32];
#pragma unroll
      for (int g2 = 0; g2 < kEpiCols / 32; g2++)
        ebl[g2] = pow2_exponent(cj0 + g2 * 32 + lane < m ? scaleB[cj0 + g2 * 32 + lane] : 1.0);
      prefetch_tile_row<double, kEpiCols>(S, n, row, live_row, base, cj0, m);
      bool ok = true;
      if (lane == 0) ok = mbar_wait_ab(smem_u32(&bar_tfull), (uint32_t)(u & 1), &s_abort);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) {
        if (lane == 0) {
          if (!s_abort) atomicExch(err, 16);
          s_abort = 1;
        }
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      long long W[kEpiCols];
      emu_fold(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)cbase, W);
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar_tempty)) : "memory");
      emu_apply(S, n, row, live_row, base, cj0, m, ea, ebl[0], W);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// ---- TF32 trailing update of a 256-wide outer panel (two-level blocking) ----
//
// The TF32 factor of S runs the 64-wide panel steps above inside outer panels
// of kWideW = 256 columns: the inner steps update only the outer panel's own
// columns, and the rest of the trailing matrix takes one update with K = 256
// per outer panel, S22 -= [Y_0 .. Y_3] [L_0 .. L_3]^T, which reads and writes
// S a quarter as often as four 64-wide updates.  The operands are the images
// the inner panel kernels wrote (one set per inner step: Y and L21 of the rows
// below that step, 8-row x 16-byte core matrices, 16 cores along K), read at
// the row offset of the outer trailing matrix in each set.
//
// One CTA per run of up to kWideRun tiles (I, J), J <= I, of one tile row I
// (tiles of 128 x 128):
//   warp 0 (one lane): bulk copies: the row's A operand (4 chunks of 128 rows
//                      x 64 columns, 128 KB, once), then the B chunks of every
//                      tile through kWideStages shared-memory stages;
//   warp 1 (one lane): tensor-memory allocation and the MMAs (M = N = 128,
//                      K = 8 per instruction, 32 per tile) into one of two
//                      tensor-memory accumulators, so that the products of
//                      the next tile run during this tile's epilogue;
//   warps 2-9:         the epilogue, two warps per tensor-memory lane quadrant
//                      (64 columns per thread): read the accumulator, hand it
//                      back, read-modify-write the lower-triangle entries of S.
// Every wait is bounded: a timeout sets *err, makes the other roles stop, lets
// the copies and products in flight finish (bounded again) and frees tensor
// memory before the CTA exits.
constexpr int kWideW = 256;                        // outer panel width (K of the update)
constexpr int kWideChunks = kWideW / TK;           // 64-column chunks (image sets)
constexpr int kWideTile = 128;                     // output tile: 128 x 128
constexpr int kWideChunkBytes = kWideTile / 8 * 16 * 128;  // one chunk of 128 rows (TF32), 32 KB
constexpr int kWideStages = 3;                     // B chunk stages
constexpr int kWideRun = 8;                        // tiles per CTA
constexpr int kWideEpiWarps = 8;
constexpr int kWideThreads = 64 + 32 * kWideEpiWarps;
__host__ __device__ constexpr int wide_smem_bytes() {
  return kWideChunks * kWideChunkBytes + kWideStages * kWideChunkBytes;  // 224 KB
}
static_assert(wide_smem_bytes() <= 227 * 1024 - 256, "wide update exceeds shared memory");

// tile columns [jlo, jhi) of tile row I for jmode (0 all J <= I, 1 J < 2, 2 J >= 2)
__host__ __device__ inline void wide_row_range(int I, int jmode, int& jlo, int& jhi) {
  jlo = jmode == 2 ? 2 : 0;
  jhi = jmode == 1 ? (I + 1 < 2 ? I + 1 : 2) : I + 1;
}

__host__ __device__ inline int wide_row_tasks(int I, int jmode) {
  int jlo, jhi;
  wide_row_range(I, jmode, jlo, jhi);
  return jhi > jlo ? (jhi - jlo + kWideRun - 1) / kWideRun : 0;
}

__host__ inline int wide_tasks(int TI, int jmode) {
  int t = 0;
  for (int I = 0; I < TI; I++) t += wide_row_tasks(I, jmode);
  return t;
}

__global__ void __launch_bounds__(kWideThreads, 1)
    k_tc_update_wide(float* __restrict__ S, int n, int base, int m, int TI, int jmode,
                     const uint8_t* __restrict__ imgA, const uint8_t* __restrict__ imgB, int64_t set_bytes,
                     int* err) {
  constexpr int KG = kgroups_of(0);                 // 16 core matrices along a 64-column chunk
  constexpr int KSTEPS = TK * 4 / 32;               // 8 MMAs of K = 8 per chunk
  constexpr uint32_t TMEM_COLS = 2 * kWideTile;     // two 128-column accumulators
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* sA = smem;                               // kWideChunks chunks of 128 rows
  uint8_t* sB = smem + kWideChunks * kWideChunkBytes;  // kWideStages stages
  __shared__ __align__(8) uint64_t bar_a, bar_full[kWideStages], bar_empty[kWideStages], bar_accf[2], bar_acce[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;

  // task -> tile row I and its run [j0, j1)
  int I = 0, t = blockIdx.x;
  for (;;) {
    const int c = wide_row_tasks(I, jmode);
    if (t < c || I + 1 >= TI) break;
    t -= c;
    I++;
  }
  int jlo, jhi;
  wide_row_range(I, jmode, jlo, jhi);
  const int j0 = jlo + t * kWideRun, j1 = min(j0 + kWideRun, jhi);
  const int ntile = max(0, j1 - j0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_a)));
    for (int q = 0; q < kWideStages; q++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_empty[q])));
    }
    for (int q = 0; q < 2; q++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_accf[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_acce[q])), "r"(kWideEpiWarps));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  // image set c holds the rows below inner step c; the outer trailing matrix
  // starts (kWideChunks - 1 - c) * 64 rows into it
  auto chunk_src = [&](const uint8_t* img, int c, int row0) -> const uint8_t* {
    const int64_t rho = (int64_t)(kWideChunks - 1 - c) * TK + row0;
    return img + (int64_t)c * set_bytes + rho * (KG * 16);
  };

  if (warp == 0) {
    if (lane == 0 && ntile > 0) {
      // producer
      const uint32_t ba = smem_u32(&bar_a);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ba),
                   "r"((uint32_t)(kWideChunks * kWideChunkBytes))
                   : "memory");
      for (int c = 0; c < kWideChunks; c++)
        bulk_load(sA + c * kWideChunkBytes, chunk_src(imgA, c, I * kWideTile), kWideChunkBytes, ba);
      int armed[kWideStages] = {};
      const int nchunk = ntile * kWideChunks;
      for (int g = 0; g < nchunk; g++) {
        const int q = g % kWideStages;
        if (g >= kWideStages &&
            !mbar_wait_ab(smem_u32(&bar_empty[q]), (uint32_t)((g / kWideStages - 1) & 1), &s_abort)) {
          if (!s_abort) atomicExch(err, 8);
          s_abort = 1;
          break;
        }
        const uint32_t bf = smem_u32(&bar_full[q]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bf), "r"((uint32_t)kWideChunkBytes)
                     : "memory");
        const int J = j0 + g / kWideChunks, c = g % kWideChunks;
        bulk_load(sB + q * kWideChunkBytes, chunk_src(imgB, c, J * kWideTile), kWideChunkBytes, bf);
        armed[q]++;
      }
      // the copies issued must land before the CTA's shared memory goes away
      volatile int never = 0;
      mbar_wait_ab(ba, 0u, &never);
      for (int q = 0; q < kWideStages; q++)
        if (armed[q] > 0) mbar_wait_ab(smem_u32(&bar_full[q]), (uint32_t)((armed[q] - 1) & 1), &never);
    }
  } else if (warp == 1) {
    if (lane == 0 && ntile > 0) {
      // MMA issuer
      uint32_t last_bar = 0, last_par = 0;  // the barrier of the last commit and its phase parity
      if (!mbar_wait_ab(smem_u32(&bar_a), 0u, &s_abort)) {
        if (!s_abort) atomicExch(err, 9);
        s_abort = 1;
      } else {
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kWideTile >> 3) << 17) |
                               ((uint32_t)(kWideTile >> 4) << 24);
        bool stop = false;
        for (int u = 0; u < ntile && !stop; u++) {
          const int b = u & 1;
          if (u >= 2 && !mbar_wait_ab(smem_u32(&bar_acce[b]), (uint32_t)(((u >> 1) - 1) & 1), &s_abort)) {
            if (!s_abort) atomicExch(err, 10);
            s_abort = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t dtm = tmem + (uint32_t)(b * kWideTile);
          for (int c = 0; c < kWideChunks; c++) {
            const int g = u * kWideChunks + c, q = g % kWideStages;
            if (!mbar_wait_ab(smem_u32(&bar_full[q]), (uint32_t)((g / kWideStages) & 1), &s_abort)) {
              if (!s_abort) atomicExch(err, 11);
              s_abort = 1;
              stop = true;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int ks = 0; ks < KSTEPS; ks++) {
              const uint64_t ad = umma_desc(smem_u32(sA + c * kWideChunkBytes + ks * 256), 128, KG * 128);
              const uint64_t bd = umma_desc(smem_u32(sB + q * kWideChunkBytes + ks * 256), 128, KG * 128);
              const uint32_t acc = (c == 0 && ks == 0) ? 0u : 1u;
              asm volatile(
                  "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, "
                  "p;\n}" ::"r"(dtm),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar_empty[q]))
                         : "memory");
            last_bar = smem_u32(&bar_empty[q]);
            last_par = (uint32_t)((g / kWideStages) & 1);
          }
          if (stop) break;
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&bar_accf[b]))
                       : "memory");
          last_bar = smem_u32(&bar_accf[b]);
          last_par = (uint32_t)((u >> 1) & 1);
        }
        // products in flight must finish before tensor memory is freed: the
        // last commit covers every MMA issued before it
        volatile int never = 0;
        if (last_bar) mbar_wait_ab(last_bar, last_par, &never);
      }
    }
  } else {
    // epilogue: tile row rho = I*128 + 32 (warp mod 4) + lane, columns
    // h*64 .. h*64 + 63 of each tile
    const int qd = warp & 3, h = (warp - 2) >> 2;
    const int rho = I * kWideTile + qd * 32 + lane;
    const int row = base + rho;
    const bool live_row = rho < m;
    for (int u = 0; u < ntile; u++) {
      const int b = u & 1, J = j0 + u;
      prefetch_tile_row<float, 64>(S, n, row, live_row, base, J * kWideTile + h * 64, m);
      bool ok = true;
      if (lane == 0) ok = mbar_wait_ab(smem_u32(&bar_accf[b]), (uint32_t)((u >> 1) & 1), &s_abort);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) {
        if (lane == 0) {
          if (!s_abort) atomicExch(err, 12);
          s_abort = 1;
        }
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      uint32_t r0[32], r1[32];
      const uint32_t ta = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * kWideTile + h * 64);
      tmem_ld32(ta, r0);
      tmem_ld32(ta + 32, r1);
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar_acce[b])) : "memory");
      if (live_row) {
        const int cj0 = J * kWideTile + h * 64;
        float cur[32];
#pragma unroll
        for (int j = 0; j < 32; j++) {
          const int cj = cj0 + j, col = base + cj;
          cur[j] = (cj < m && row >= col) ? S[(int64_t)row + (int64_t)col * n] : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 32; j++) {
          const int cj = cj0 + j, col = base + cj;
          if (cj < m && row >= col) S[(int64_t)row + (int64_t)col * n] = cur[j] - __uint_as_float(r0[j]);
        }
#pragma unroll
        for (int j = 0; j < 32; j++) {
          const int cj = cj0 + 32 + j, col = base + cj;
          cur[j] = (cj < m && row >= col) ? S[(int64_t)row + (int64_t)col * n] : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 32; j++) {
          const int cj = cj0 + 32 + j, col = base + cj;
          if (cj < m && row >= col) S[(int64_t)row + (int64_t)col * n] = cur[j] - __uint_as_float(r1[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// ---- FP32 panel kernels for the TF32 / BF16 modes (same steps as the FP64 ones in dense.cu) ----

__global__ void k_to_f32(const double* __restrict__ S, float* __restrict__ S32, int64_t n2) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n2; q += (int64_t)gridDim.x * blockDim.x)
    S32[q] = (float)S[q];
}

// One blocked LDL^T of nb matrices of order n (matrix b at S + b * ts.s):
// diagonal block and panel on the CUDA cores, trailing update on the tensor
// cores.  rend: per 64-wide panel, one past its last nonzero row (or null).
//
// Lookahead: the update of step k is split into its first tile column (the
// next panel's 64 columns) and the rest, so that the next diagonal block and
// panel run while the rest of the update does.  The critical chain (diagonal
// block, panel, slicing, first tile column) runs on the handle's high-priority
// stream, whose blocks the scheduler dispatches ahead of the rest's waiting
// blocks on the side stream.  The next step's slicing waits for the rest (it
// overwrites the operand images the rest reads); the caller's stream joins
// both at the end.
template <int MODE, class T>
cudaError_t factor_tc(Handle& h, T* S, T* Y, int n, int npiv, int nb, const TcStrides& ts, const PivotRule& rule,
                      const int32_t* rend_of_panel, unsigned long long* counters, uint8_t* imgA,
                      uint8_t* imgB, double* scaleA, double* scaleB, cudaStream_t caller) {
  constexpr int A_BYTES = image_bytes(MODE, TM), B_BYTES = image_bytes(MODE, TN);
  const int smem = A_BYTES + B_BYTES;
  cudaStream_t side = h.side_stream;
  cudaStream_t st = caller;
  const int prio = side ? h.prio_hi : 0;  // the critical chain's launches outrank the rest of the update
  bool side_busy = false;
  cudaError_t e = cudaSuccess;
  if (side && h.hi_stream) {  // fork the critical chain onto the high-priority stream
    e = cudaEventRecord(h.ev_main, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h.hi_stream, h.ev_main, 0);
    if (e != cudaSuccess) return e;
    st = h.hi_stream;
  }
  for (int k0 = 0; k0 < npiv && e == cudaSuccess; k0 += TK) {
    const int kb = std::min(TK, npiv - k0);
    const int kd = kt_begin(h, kFamDiag, nb * (2.0 / 3.0) * kb * kb * kb, st);
    launch_prio(k_dense_diag_t<T>, dim3(nb), dim3(256), 0, st, prio, S, n, k0, kb, ts.s, rule, counters);
    kt_end(h, kd, st);
    h.launches++;
    // rows below the envelope of the panel's columns stay zero (no pivoting)
    const int rend = rend_of_panel ? rend_of_panel[k0 / TK] : n;
    const int m = rend - k0 - kb;
    if (m <= 0) continue;
    // TF32 (one matrix): the panel kernel writes the update's operand images
    // itself, so it waits for the previous update's rest, which reads them
    constexpr bool fused = MODE == 0;
    const bool fuse = fused && nb == 1;
    if (side_busy && fuse) {
      e = cudaStreamWaitEvent(st, h.ev_side, 0);
      side_busy = false;
      if (e != cudaSuccess) break;
    }
    Tf32Images img;
    if (fuse) {
      img.A = imgA;
      img.B = imgB;
    }
    launch_dense_panel<T>(S, Y, n, k0, kb, rend, nb, ts.s, ts.y, st, prio, img);
    h.launches++;
    if (side_busy) {
      e = cudaStreamWaitEvent(st, h.ev_side, 0);
      side_busy = false;
      if (e != cudaSuccess) break;
    }
    const int TI = (m + TM - 1) / TM, TJ = (m + TN - 1) / TN;
    const int mpadA = TI * TM, mpadB = TJ * TN;
    if (!fuse) {
      const int sgrid = std::max(1, std::min((mpadA + mpadB + 255) / 256, 152 * 8 / nb));
      launch_prio(k_tc_slice<MODE, T>, dim3(sgrid, nb), dim3(256), 0, st, prio, S, Y, n, k0, kb, m, imgA, imgB,
                  scaleA, scaleB, mpadA, mpadB, ts);
      h.launches++;
    }
    int tiles = 0;
    for (int I = 0; I < TI; I++) tiles += std::min(2 * I + 2, TJ);
    // one launch of the update over the tiles of jmode (0 all, 1 J = 0, 2 J >= 1)
    auto update = [&](int jmode, cudaStream_t us, int uprio) -> cudaError_t {
      h.launches++;
      const int c0 = jmode == 2 ? TN : 0, c1 = jmode == 1 ? TN : m;
      const int kt = kt_begin(h, MODE == 2 ? kFamEmu : kFamTc, nb * update_flops(m, c0, c1, kb), us);
      cudaError_t le;
      if constexpr (MODE == 2) {
        int tasks = 0;
        for (int I = 0; I < TI; I++) tasks += emu_row_tasks(I, TJ, jmode);
        le = launch_prio(k_tc_update_emu, dim3(tasks, nb), dim3(kEmuThreads), emu_smem_bytes(), us, uprio,
                         (double*)S, n, k0, kb, m, m, TI, TJ, jmode, (const uint8_t*)imgA, (const uint8_t*)imgB,
                         (const double*)scaleA, (const double*)scaleB, h.dev_err, ts);
      } else {
        const int cnt = jmode == 0 ? tiles : (jmode == 1 ? TI : tiles - TI);
        le = launch_prio(k_tc_update<MODE, T>, dim3(cnt, nb), dim3(128), smem, us, uprio, S, n, k0, kb, m, TJ,
                         jmode, (const uint8_t*)imgA, (const uint8_t*)imgB, (const double*)scaleA,
                         (const double*)scaleB, h.dev_err, ts);
      }
      kt_end(h, kt, us);
      return le;
    };
    if (!side || TJ < 2) {
      e = update(0, st, 0);
      continue;
    }
    e = cudaEventRecord(h.ev_main, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, h.ev_main, 0);
    if (e != cudaSuccess) break;
    e = update(2, side, 0);
    if (e == cudaSuccess) e = cudaEventRecord(h.ev_side, side);
    side_busy = true;
    if (e == cudaSuccess) e = update(1, st, prio);
  }
  if (side_busy && e == cudaSuccess) e = cudaStreamWaitEvent(caller, h.ev_side, 0);
  if (st != caller && e == cudaSuccess) {  // join the high-priority chain
    e = cudaEventRecord(h.ev_main, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, h.ev_main, 0);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

// The emulated-FP64 factor with 256-wide outer panels (k_slice_wide and
// k_tc_update_emu_wide above), for nb matrices of order n with npiv pivots.
// Per outer panel K0: its 64-wide steps (diagonal block, panel writing Y into
// the panel's columns of Yw, per-step images, k_tc_update_emu over the outer
// panel's own remaining columns); then the 256-wide images and the outer
// update of the rest: its first four tile columns (the next outer panel's
// columns) on the high-priority chain, the others on the side stream,
// overlapping the next outer panel's steps.  The next panel's slicing waits
// for the side stream (it overwrites the images the rest reads).
struct EwBuffers {
  double* Yw = nullptr;   // per matrix: n x 256, leading dimension n
  int64_t y_stride = 0;
  uint8_t* A = nullptr;   // per matrix: the 256-wide images of Y and of L
  uint8_t* B = nullptr;
  int64_t img_stride = 0;
  double* sA = nullptr;   // per matrix: row scales
  double* sB = nullptr;
  int64_t scale_stride = 0;
};

cudaError_t factor_emu_wide(Handle& h, double* S, int n, int npiv, int nb, const TcStrides& ts, const PivotRule& rule,
                            unsigned long long* counters, uint8_t* imgA, uint8_t* imgB, double* scaleA,
                            double* scaleB, const EwBuffers& ew, cudaStream_t caller) {
  cudaStream_t side = h.side_stream;
  cudaStream_t st = caller;
  const int prio = side ? h.prio_hi : 0;
  bool side_busy = false;
  cudaError_t e = cudaSuccess;
  if (side && h.hi_stream) {
    e = cudaEventRecord(h.ev_main, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h.hi_stream, h.ev_main, 0);
    if (e != cudaSuccess) return e;
    st = h.hi_stream;
  }
  TcStrides ti = ts;  // the per-step images, with Y taken from Yw
  ti.y = ew.y_stride;
  for (int K0 = 0; K0 < npiv && e == cudaSuccess; K0 += kEwW) {
    const int Wb = std::min(kEwW, npiv - K0);
    for (int c = 0; c * TK < Wb && e == cudaSuccess; c++) {
      const int k0 = K0 + c * TK, kb = std::min(TK, npiv - k0);
      const int kd = kt_begin(h, kFamDiag, nb * (2.0 / 3.0) * kb * kb * kb, st);
      launch_prio(k_dense_diag_t<double>, dim3(nb), dim3(256), 0, st, prio, S, n, k0, kb, ts.s, rule, counters);
      kt_end(h, kd, st);
      h.launches++;
      const int m = n - k0 - kb;
      if (m <= 0) continue;
      double* Yc = ew.Yw + (int64_t)c * TK * n;
      {
        // the panel as a product: W = L11^{-1}, the digit image of A21 (rows
        // below the diagonal block, columns k0 .. k0 + kb of S), Y = A21 W^T
        const int TIp = (m + TM - 1) / TM;
        const int kp = kt_begin(h, kFamPanelEmu, nb * (double)m * kb * (kb - 1), st);
        const int pgrid = std::max(1, std::min((TIp * TM + 255) / 256, 152 * 8 / nb));
        launch_prio(k_panel_inverse_slice, dim3(1 + pgrid, nb), dim3(256), 0, st, prio, (const double*)S, n, k0, kb,
                    m, TIp * TM, imgA, imgB, scaleA, scaleB, ti);
        e = launch_prio(k_tc_panel_emu, dim3(TIp, nb), dim3(256), panel_emu_smem_bytes(), st, prio, S, Yc, n, k0, kb,
                        m, (const uint8_t*)imgA, (const uint8_t*)imgB, (const double*)scaleA, (const double*)scaleB,
                        h.dev_err, ti);
        kt_end(h, kp, st);
        h.launches += 2;
        if (e != cudaSuccess) break;
      }
      // the outer panel's own remaining columns
      const int TJl = (K0 + Wb - (k0 + kb) + TN - 1) / TN;
      if (TJl <= 0) continue;
      const int TI = (m + TM - 1) / TM, mpadA = TI * TM, mpadB = TJl * TN;
      const int sgrid = std::max(1, std::min((mpadA + mpadB + 255) / 256, 152 * 8 / nb));
      launch_prio(k_tc_slice<2, double>, dim3(sgrid, nb), dim3(256), 0, st, prio, (const double*)S,
                  (const double*)Yc, n, k0, kb, m, imgA, imgB, scaleA, scaleB, mpadA, mpadB, ti);
      h.launches++;
      int tasks = 0;
      for (int I = 0; I < TI; I++) tasks += emu_row_tasks(I, TJl, 0);
      const int kt = kt_begin(h, kFamEmu, nb * update_flops(m, 0, K0 + Wb - (k0 + kb), kb), st);
      // columns past the outer panel (the augmented rows of a tail) belong to the outer update
      e = launch_prio(k_tc_update_emu, dim3(tasks, nb), dim3(kEmuThreads), emu_smem_bytes(), st, prio, S, n, k0, kb,
                      m, K0 + Wb - (k0 + kb), TI, TJl, 0, (const uint8_t*)imgA, (const uint8_t*)imgB, (const double*)scaleA,
                      (const double*)scaleB, h.dev_err, ti);
      kt_end(h, kt, st);
      h.launches++;
    }
    const int base = K0 + Wb, m = n - base;
    if (m <= 0 || e != cudaSuccess) break;
    if (side_busy) {  // the rest of the previous outer update still reads the images
      e = cudaStreamWaitEvent(st, h.ev_side, 0);
      side_busy = false;
      if (e != cudaSuccess) break;
    }
    const int TI = (m + TM - 1) / TM, TJ = (m + TN - 1) / TN, mpad = TI * TM;
    launch_prio(k_slice_wide, dim3((2 * mpad + 127) / 128, nb), dim3(128), 0, st, prio, (const double*)S,
                (const double*)ew.Yw, n, K0, Wb, base, m, mpad, ew.A, ew.B, ew.sA, ew.sB, ts.s, ew.y_stride,
                ew.img_stride, ew.scale_stride);
    h.launches++;
    const int nchunk = (Wb + kEwChunk - 1) / kEwChunk;
    auto wide = [&](int jmode, cudaStream_t us, int uprio) -> cudaError_t {
      int tasks = 0;
      for (int I = 0; I < TI; I++) tasks += emu_row_tasks(I, TJ, jmode, 4);
      if (tasks == 0) return cudaSuccess;
      h.launches++;
      const int c0 = jmode == 2 ? 4 * TN : 0, c1 = jmode == 1 ? 4 * TN : m;
      const int kt = kt_begin(h, kFamEmuWide, nb * update_flops(m, c0, c1, Wb), us);
      const cudaError_t le = launch_prio(k_tc_update_emu_wide, dim3(tasks, nb), dim3(kEmuThreads), ew_smem_bytes(),
                                         us, uprio, S, n, base, m, TI, TJ, jmode, nchunk, (const uint8_t*)ew.A,
                                         (const uint8_t*)ew.B, (const double*)ew.sA, (const double*)ew.sB, ts.s,
                                         ew.img_stride, ew.scale_stride, h.dev_err);
      kt_end(h, kt, us);
      return le;
    };
    if (!side || TJ <= 4) {
      e = wide(0, st, prio);
      continue;
    }
    e = wide(1, st, prio);
    if (e == cudaSuccess) e = cudaEventRecord(h.ev_main, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, h.ev_main, 0);
    if (e == cudaSuccess) e = wide(2, side, 0);
    if (e == cudaSuccess) e = cudaEventRecord(h.ev_side, side);
    side_busy = e == cudaSuccess;
  }
  if (side_busy && e == cudaSuccess) e = cudaStreamWaitEvent(caller, h.ev_side, 0);
  if (st != caller && e == cudaSuccess) {
    e = cudaEventRecord(h.ev_main, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, h.ev_main, 0);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

// The TF32 factor of S with 256-wide outer panels (k_tc_update_wide above).
// Per outer panel K0: its four 64-wide steps (diagonal block, panel with the
// operand images in set c of the panel's parity, update of the panel's own
// remaining columns), then the outer update of the rest, split as in
// factor_tc: its first two tile columns (the next outer panel's 256 columns)
// on the high-priority chain, the rest on the side stream, overlapping the
// next outer panel's steps.  The image sets alternate between two parities, so
// that the next panel does not overwrite the images the rest still reads.
cudaError_t factor_tf32_wide(Handle& h, float* S, float* Y, int n, unsigned long long* counters, cudaStream_t caller) {
  constexpr int B_BYTES = image_bytes(0, TN), A_BYTES = image_bytes(0, TM);
  cudaStream_t side = h.side_stream;
  cudaStream_t st = caller;
  const int prio = side ? h.prio_hi : 0;
  bool side_busy = false;
  cudaError_t e = cudaSuccess;
  if (side && h.hi_stream) {
    e = cudaEventRecord(h.ev_main, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h.hi_stream, h.ev_main, 0);
    if (e != cudaSuccess) return e;
    st = h.hi_stream;
  }
  const int64_t sb = h.tw_set_bytes;
  for (int K0 = 0, j = 0; K0 < n && e == cudaSuccess; K0 += kWideW, j++) {
    const int Wb = std::min(kWideW, n - K0);
    uint8_t* setA = h.tw_img + (int64_t)(j & 1) * 2 * kWideChunks * sb;  // [parity][A sets | B sets]
    uint8_t* setB = setA + kWideChunks * sb;
    for (int c = 0; c * TK < Wb && e == cudaSuccess; c++) {
      const int k0 = K0 + c * TK, kb = std::min(TK, n - k0);
      const int kd = kt_begin(h, kFamDiag, (2.0 / 3.0) * kb * kb * kb, st);
      launch_prio(k_dense_diag_t<float>, dim3(1), dim3(256), 0, st, prio, S, n, k0, kb, (int64_t)0, PivotRule{},
                  counters);
      kt_end(h, kd, st);
      h.launches++;
      const int m = n - k0 - kb;
      if (m <= 0) continue;
      Tf32Images img;
      img.A = setA + c * sb;
      img.B = setB + c * sb;
      launch_dense_panel<float>(S, Y, n, k0, kb, n, 1, 0, 0, st, prio, img);
      h.launches++;
      // the rest of this outer panel's columns
      const int TJl = (K0 + Wb - (k0 + kb) + TN - 1) / TN;
      if (TJl <= 0) continue;
      const int TI = (m + TM - 1) / TM;
      int tiles = 0;
      for (int I = 0; I < TI; I++) tiles += std::min(2 * I + 2, TJl);
      const int kt = kt_begin(h, kFamTc, update_flops(m, 0, K0 + Wb - (k0 + kb), kb), st);
      e = launch_prio(k_tc_update<0, float>, dim3(tiles), dim3(128), A_BYTES + B_BYTES, st, prio, S, n, k0, kb, m,
                      TJl, 0, (const uint8_t*)img.A, (const uint8_t*)img.B, (const double*)nullptr,
                      (const double*)nullptr, h.dev_err, TcStrides{});
      kt_end(h, kt, st);
      h.launches++;
    }
    const int base = K0 + Wb, m = n - base;
    if (m <= 0 || e != cudaSuccess) break;
    // the rest of the previous outer update must be done before this one
    if (side_busy) {
      e = cudaStreamWaitEvent(st, h.ev_side, 0);
      side_busy = false;
      if (e != cudaSuccess) break;
    }
    const int TI = (m + kWideTile - 1) / kWideTile;
    auto wide = [&](int jmode, cudaStream_t us, int uprio) -> cudaError_t {
      const int tasks = wide_tasks(TI, jmode);
      if (tasks == 0) return cudaSuccess;
      h.launches++;
      const int c0 = jmode == 2 ? 2 * kWideTile : 0, c1 = jmode == 1 ? 2 * kWideTile : m;
      const int kt = kt_begin(h, kFamWide, update_flops(m, c0, c1, kWideW), us);
      const cudaError_t le = launch_prio(k_tc_update_wide, dim3(tasks), dim3(kWideThreads), wide_smem_bytes(), us,
                                         uprio, S, n, base, m, TI, jmode, (const uint8_t*)setA, (const uint8_t*)setB,
                                         sb, h.dev_err);
      kt_end(h, kt, us);
      return le;
    };
    if (!side || TI <= 2) {
      e = wide(0, st, prio);
      continue;
    }
    e = wide(1, st, prio);
    if (e == cudaSuccess) e = cudaEventRecord(h.ev_main, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, h.ev_main, 0);
    if (e == cudaSuccess) e = wide(2, side, 0);
    if (e == cudaSuccess) e = cudaEventRecord(h.ev_side, side);
    side_busy = e == cudaSuccess;
  }
  (void)B_BYTES;
  if (side_busy && e == cudaSuccess) e = cudaStreamWaitEvent(caller, h.ev_side, 0);
  if (st != caller && e == cudaSuccess) {
    e = cudaEventRecord(h.ev_main, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, h.ev_main, 0);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

// Kernel attributes set once (before any launch, outside stream capture).
cudaError_t dense_tc_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_update<0, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       image_bytes(0, TM) + image_bytes(0, TN));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_update<1, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             image_bytes(1, TM) + image_bytes(1, TN));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_update_emu, cudaFuncAttributeMaxDynamicSharedMemorySize, emu_smem_bytes());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_update_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, wide_smem_bytes());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_update_emu_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, ew_smem_bytes());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_panel_emu, cudaFuncAttributeMaxDynamicSharedMemorySize, panel_emu_smem_bytes());
  return e;
}

int64_t emu_wide_image_bytes(int n) {
  // 64-row blocks of the largest outer trailing matrix, in whole 128-row tiles
  const int64_t rows = ((int64_t)n + TM - 1) / TM * TM + TM;
  return rows / 64 * kEwBlockBytes;
}

bool emu_wide_applies(int npiv) { return npiv >= 2 * kEwW; }

int64_t tf32_wide_set_bytes(int n) {
  // rows of one image set: the rows below an inner step, read in whole
  // 128-row tiles from up to 192 rows into the set
  const int64_t rows = ((int64_t)n + kWideTile - 1) / kWideTile * kWideTile + 2 * kWideW;
  return rows * (kgroups_of(0) * 16);
}

bool tf32_wide_applies(int n, bool structured) { return !structured && n >= 2 * kWideW; }

int64_t tc_image_bytes(int n, int mode) {
  const int TI = (n + TM - 1) / TM + 1, TJ = (n + TN - 1) / TN + 1;
  const int m = mode == KKT_TF32 ? 0 : (mode == KKT_BF16 ? 1 : 2);
  const int ia = m == 0 ? image_bytes(0, TM) : (m == 1 ? image_bytes(1, TM) : image_bytes(2, TM));
  const int ib = m == 0 ? image_bytes(0, TN) : (m == 1 ? image_bytes(1, TN) : image_bytes(2, TN));
  return (int64_t)TI * ia + (int64_t)TJ * ib;
}

int64_t tc_image_bytes_a(int n, int mode) {
  const int TI = (n + TM - 1) / TM + 1;
  const int ia = mode == KKT_TF32 ? image_bytes(0, TM) : (mode == KKT_BF16 ? image_bytes(1, TM) : image_bytes(2, TM));
  return (int64_t)TI * ia;
}

// The dense factor of S in precision `mode`.  TF32/BF16 factor the FP32 copy
// S32 (S itself is kept for the FP64 fallback); the emulated FP64 mode
// factors S in place.  `counters` receives the pivot signs.
cudaError_t launch_dense_ldlt_tc(Handle& h, int mode, unsigned long long* counters, cudaStream_t st) {
  const int n = h.nC;
  if (n == 0) return cudaSuccess;
  const int32_t* rend = h.panel_rend.empty() ? nullptr : h.panel_rend.data();
  const TcStrides one{};
  cudaError_t e;
  if (mode == KKT_F64_EMULATED) {
    if (h.ew_s_A && !rend) {
      EwBuffers ew;
      ew.Yw = h.ew_s_Y;
      ew.y_stride = (int64_t)n * kEwW;
      ew.A = h.ew_s_A;
      ew.B = h.ew_s_B;
      ew.sA = h.ew_s_scale;
      ew.sB = h.ew_s_scale + (n + 2 * TM);
      e = factor_emu_wide(h, h.S, n, n, 1, one, PivotRule{}, counters, h.tc_imgA, h.tc_imgB, h.tc_scaleA, h.tc_scaleB,
                          ew, st);
    } else {
      e = factor_tc<2, double>(h, h.S, h.Ypanel, n, n, 1, one, PivotRule{}, rend, counters, h.tc_imgA, h.tc_imgB,
                               h.tc_scaleA, h.tc_scaleB, st);
    }
    return e != cudaSuccess ? e : launch_diag_inverse(h, false, st);
  }
  const int64_t n2 = (int64_t)n * n;
  k_to_f32<<<(int)std::min<int64_t>((n2 + 255) / 256, 152 * 32), 256, 0, st>>>(h.S, h.S32, n2);
  h.launches++;
  if (mode == KKT_TF32 && h.tw_img && !rend)
    e = factor_tf32_wide(h, h.S32, h.Y32, n, counters, st);
  else if (mode == KKT_TF32)
    e = factor_tc<0, float>(h, h.S32, h.Y32, n, n, 1, one, PivotRule{}, rend, counters, h.tc_imgA, h.tc_imgB,
                            h.tc_scaleA, h.tc_scaleB, st);
  else
    e = factor_tc<1, float>(h, h.S32, h.Y32, n, n, 1, one, PivotRule{}, rend, counters, h.tc_imgA, h.tc_imgB,
                            h.tc_scaleA, h.tc_scaleB, st);
  return e != cudaSuccess ? e : launch_diag_inverse(h, true, st);
}

// The dense tails of the N block factors in emulated FP64: the batched
// blocked LDL^T above with the static-pivot rule of the block factors.
cudaError_t launch_tail_factor_emulated(Handle& h, cudaStream_t st) {
  const int nTa = h.nTa;
  TcStrides ts;
  ts.s = (int64_t)nTa * nTa;
  ts.y = (int64_t)nTa * TK;
  ts.img_a = tc_image_bytes_a(nTa, KKT_F64_EMULATED);
  ts.img_b = tc_image_bytes(nTa, KKT_F64_EMULATED) - ts.img_a;
  ts.scale = (int64_t)nTa + 256;
  const PivotRule rule{h.anorm, h.opt.pivot_eps, h.d.col_primal + h.sym.tail_col};
  if (h.ew_t_A) {
    EwBuffers ew;
    ew.Yw = h.ew_t_Y;
    ew.y_stride = (int64_t)nTa * kEwW;
    ew.A = h.ew_t_A;
    ew.B = h.ew_t_B;
    ew.img_stride = emu_wide_image_bytes(nTa);
    ew.sA = h.ew_t_scale;
    ew.sB = h.ew_t_scale + (nTa + 2 * TM);
    ew.scale_stride = 2 * ((int64_t)nTa + 2 * TM);
    return factor_emu_wide(h, h.Tt, nTa, h.nT, h.N, ts, rule, h.counters, h.t_imgA, h.t_imgB, h.t_scaleA,
                           h.t_scaleB, ew, st);
  }
  return factor_tc<2, double>(h, h.Tt, h.TY, nTa, h.nT, h.N, ts, rule, nullptr, h.counters, h.t_imgA,
                              h.t_imgB, h.t_scaleA, h.t_scaleB, st);
}

// Diagonal block and panel of one 64-wide step of the FP64 factor (shared by
// the FP64 path, whose trailing update runs on the CUDA cores).
cudaError_t launch_dense_diag_panel_f64(Handle& h, int k0, int kb, int rend, unsigned long long* counters,
                                        cudaStream_t st) {
  const int n = h.nC;
  const int kd = kt_begin(h, kFamDiag, (2.0 / 3.0) * kb * kb * kb, st);
  k_dense_diag_t<double><<<1, 256, 0, st>>>(h.S, n, k0, kb, 0, PivotRule{}, counters);
  kt_end(h, kd, st);
  h.launches++;
  if (rend - k0 - kb > 0) {
    launch_dense_panel<double>(h.S, h.Ypanel, n, k0, kb, rend, 1, 0, 0, st);
    h.launches++;
  }
  return cudaGetLastError();
}

}  // namespace kkt
