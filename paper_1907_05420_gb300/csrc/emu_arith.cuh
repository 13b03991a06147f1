// Exact integer and FP32 arithmetic of the emulated-FP64 tensor-core update
// (dense_tc.cu): digit slicing of the FP64 operands, read-out of the FP32
// digit-product levels, and the FP64 bit pattern of the scaled product.
//
// The GPU has few FP64 instructions, and its conversion instructions share the
// same narrow pipe, so everything here is integer or FP32 work.  The functions
// compile for the device and for the host (g++ or nvcc), so that the CPU tests
// can check them against exact rational arithmetic.
#pragma once
#include <cstdint>
#include <cstring>
#include <cmath>

#ifdef __CUDACC__
#define KKT_HD __host__ __device__ __forceinline__
#else
#define KKT_HD inline
#endif

namespace kkt {

constexpr int kEmuSlices = 7;  // base-256 digits per FP64 operand

KKT_HD long long bits_of(double v) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(v);
#else
  long long b;
  std::memcpy(&b, &v, sizeof b);
  return b;
#endif
}

KKT_HD double double_of(long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(b);
#else
  double v;
  std::memcpy(&v, &b, sizeof v);
  return v;
#endif
}

KKT_HD int bits_of(float v) {
#ifdef __CUDA_ARCH__
  return __float_as_int(v);
#else
  int b;
  std::memcpy(&b, &v, sizeof b);
  return b;
#endif
}

// leading zeros of a nonzero 64-bit / 32-bit value
KKT_HD int clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return __builtin_clzll(x);
#endif
}

KKT_HD int clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __clz((int)x);
#else
  return __builtin_clz(x);
#endif
}

KKT_HD int imin(int a, int b) {
#ifdef __CUDA_ARCH__
  return min(a, b);
#else
  return a < b ? a : b;
#endif
}

KKT_HD float fma32(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return fmaf(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}

// The 7 base-256 digits of u = v / 2^e in (-1, 1), truncated toward zero:
// q = trunc(|u| 2^56), and digit s is byte 6 - s of q with the sign of v.
// Computed on the raw bits: |v| = m 2^(E - 1075) with m the 53-bit significand
// and E the biased exponent (a subnormal has E = 0, no implicit bit and
// exponent -1074), so q is m shifted by E - 1075 + 56 - e; |v| < 2^e bounds q
// below 2^56.  Returns q; the sign of v is the sign bit of b.
KKT_HD unsigned long long digits7(double v, int e, long long& b) {
  b = bits_of(v);
  const int E = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = (unsigned long long)(b & 0xFFFFFFFFFFFFFll) | (E ? (1ull << 52) : 0ull);
  const int sh = (E ? E : 1) - 1075 + 56 - e;
  return sh >= 0 ? (sh < 64 ? m << sh : 0ull) : (sh > -64 ? m >> (-sh) : 0ull);
}

// The 7 base-256 digits of q < 2^55 rebalanced into [-128, 128]: q =
// sum_s d_s 256^(6 - s) with d_s in [-128, 127] for s >= 1 and d_0 in
// [0, 128] (a digit of 128 or more borrows 256 from itself and carries one
// into the next more significant digit; q < 2^55 keeps the top digit at most
// 127 + 1).  Every digit product is then at most 2^14 in magnitude.
KKT_HD void balanced7(unsigned long long q, int (&d)[kEmuSlices]) {
  int carry = 0;
  for (int s = kEmuSlices - 1; s >= 0; s--) {
    int t = (int)((q >> (8 * (kEmuSlices - 1 - s))) & 0xFFull) + carry;
    carry = 0;
    if (s > 0 && t >= 128) {
      t -= 256;
      carry = 1;
    }
    d[s] = t;
  }
}

// Biased exponent field of a double (0 for zero and subnormals).
KKT_HD int exp_field(double v) { return (int)((bits_of(v) >> 52) & 0x7FF); }

// BF16 bit pattern of an integer 0 <= v < 256 (exact: 8 significant bits).
KKT_HD uint32_t bf16_bits_of_byte(uint32_t v) {
  if (v == 0) return 0u;
  const int e = 31 - clz32(v);  // 0..7
  return ((uint32_t)(127 + e) << 7) | ((v << (7 - e)) & 0x7Fu);
}

// FP32 additions of M = 1.5 * 2^23 put a rounded integer |k| < 2^22 into the
// low significand bits of M + k, read back with an integer subtraction.
constexpr float kMagic = 12582912.0f;   // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;  // bit pattern of kMagic

// x an integer-valued FP32 number, |x| < 2^30: x exactly as int32
// (x = 256 hi + lo with hi = rn(x / 256) and |lo| <= 128, both exact).
KKT_HD int exact_f2i(float x) {
  const float r = fma32(x, 0.00390625f, kMagic);
  const float hi = r - kMagic;
  const float lo = fma32(-256.0f, hi, x);
  return (bits_of(r) - kMagicBits) * 256 + (bits_of(lo + kMagic) - kMagicBits);
}

// round-to-nearest-even of an FP32 x, |x| < 2^37, as int64
// (x = 65536 hi + lo with hi = rn(x / 65536), lo exact, |lo| <= 2^15).
KKT_HD long long round_f2ll(float x) {
  const float r = fma32(x, 0x1p-16f, kMagic);
  const float hi = r - kMagic;
  const float lo = fma32(-65536.0f, hi, x);
  return (long long)(bits_of(r) - kMagicBits) * 65536 + (bits_of(lo + kMagic) - kMagicBits);
}

// Exponent e of a positive power of two 2^e (normal or subnormal).
KKT_HD int pow2_exponent(double s) {
  const long long b = bits_of(s);
  const int E = (int)((b >> 52) & 0x7FF);
  return E ? E - 1023 : (63 - clz64((unsigned long long)b)) - 1074;
}

// -RN(W 2^eoff) as an FP64 bit pattern, built with integer operations for
// every W (|W| < 2^63) and eoff: a normal result keeps the top 53 bits of |W|
// (round to nearest even, the carry may bump the exponent), a subnormal one the
// bits down to 2^-1074, and a result beyond the largest finite value is an
// infinity.  One rounding of the exact value, as fma(-W, 2^eoff, 0) would do.
KKT_HD double neg_scaled(long long W, int eoff) {
  const unsigned long long sgn = W < 0 ? 0ull : (1ull << 63);  // sign of -W
  const unsigned long long a = W < 0 ? (unsigned long long)(-W) : (unsigned long long)W;
  const int lz = clz64(a | 1ull);  // a = 0 handled below
  const unsigned long long x = a << lz;  // leading one at bit 63
  const int be = (63 - lz) + eoff + 1023;  // biased exponent of a normal result
  const int drop = be >= 1 ? 11 : imin(64, 12 - be);  // low bits of x rounded off
  unsigned long long mant = drop < 64 ? x >> drop : 0ull;
  const unsigned long long rem = drop < 64 ? x & ((1ull << drop) - 1ull) : x;
  const unsigned long long half = 1ull << (drop - 1);
  if (rem > half || (rem == half && (mant & 1ull))) mant++;
  unsigned long long bits = be >= 1 ? ((unsigned long long)(be - 1) << 52) + mant : mant;
  if (12 - be > 64) bits = 0ull;  // below half the smallest subnormal
  if (be >= 2047) bits = 0x7FF0000000000000ull;
  return double_of((long long)(a == 0 ? 0ull : (sgn | bits)));
}

// ---- tiles of the trailing update (128-row by 64-column tiles) ----
// Tile (I, J) holds part of the lower triangle when J <= 2I + 1.  A task is a
// run of at most kEmuRun consecutive tiles of one tile row; jmode 0 takes all
// tiles, 1 the first jsplit tile columns (J < jsplit: the next panel's
// columns), 2 the others.
constexpr int kEmuRun = 8;

// tile columns [jlo, jhi) of tile row I for jmode
KKT_HD void emu_row_range(int I, int TJ, int jmode, int& jlo, int& jhi, int jsplit = 1) {
  const int cnt = imin(2 * I + 2, TJ);
  jlo = jmode == 2 ? jsplit : 0;
  jhi = jmode == 1 ? imin(jsplit, cnt) : cnt;
}

KKT_HD int emu_row_tasks(int I, int TJ, int jmode, int jsplit = 1) {
  int jlo, jhi;
  emu_row_range(I, TJ, jmode, jlo, jhi, jsplit);
  return jhi > jlo ? (jhi - jlo + kEmuRun - 1) / kEmuRun : 0;
}

// task t (of the sum of emu_row_tasks over the TI rows) -> row I, tiles [j0, j1)
KKT_HD void emu_task(int t, int TI, int TJ, int jmode, int& I, int& j0, int& j1, int jsplit = 1) {
  I = 0;
  for (;;) {
    const int c = emu_row_tasks(I, TJ, jmode, jsplit);
    if (t < c || I + 1 >= TI) break;
    t -= c;
    I++;
  }
  int jlo, jhi;
  emu_row_range(I, TJ, jmode, jlo, jhi, jsplit);
  j0 = jlo + t * kEmuRun;
  j1 = imin(j0 + kEmuRun, jhi);
}

}  // namespace kkt
