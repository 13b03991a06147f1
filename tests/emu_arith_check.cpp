// Host driver for the emulated-FP64 arithmetic helpers (emu_arith.cuh): reads
// binary inputs, writes binary outputs; tests/test_emu_arith.py compiles it
// with g++ and compares against exact rational arithmetic.
//   emu_arith_check f2i    in out   float32[n]          -> int32[n]
//   emu_arith_check f2ll   in out   float32[n]          -> int64[n]
//   emu_arith_check neg    in out   (int64 W, int64 e)[n] -> float64[n]
//   emu_arith_check digits in out   (float64 v, int64 e)[n] -> (uint64 q, int64 sign)[n]
//   emu_arith_check pow2   in out   float64[n]          -> int64[n]
//   emu_arith_check balanced in out int64 q[n] (q < 2^55) -> int64 d[n][7]
//   emu_arith_check bf16   -  out                       -> uint32[256]
//   emu_arith_check tasks  in out   (int64 TI, TJ, jmode, jsplit)[n] -> per entry: count, then
//                                   count x (I, j0, j1), all int64
#include <cstdio>
#include <cstring>
#include <vector>

#include "emu_arith.cuh"

template <class T>
static std::vector<T> read_all(const char* path) {
  std::vector<T> v;
  FILE* f = std::fopen(path, "rb");
  if (!f) return v;
  T x;
  while (std::fread(&x, sizeof x, 1, f) == 1) v.push_back(x);
  std::fclose(f);
  return v;
}

template <class T>
static bool write_all(const char* path, const std::vector<T>& v) {
  FILE* f = std::fopen(path, "wb");
  if (!f) return false;
  const bool ok = std::fwrite(v.data(), sizeof(T), v.size(), f) == v.size();
  std::fclose(f);
  return ok;
}

int main(int argc, char** argv) {
  if (argc != 4) return 2;
  const char* mode = argv[1];
  if (!std::strcmp(mode, "f2i")) {
    std::vector<int32_t> out;
    for (float x : read_all<float>(argv[2])) out.push_back(kkt::exact_f2i(x));
    return write_all(argv[3], out) ? 0 : 1;
  }
  if (!std::strcmp(mode, "f2ll")) {
    std::vector<int64_t> out;
    for (float x : read_all<float>(argv[2])) out.push_back(kkt::round_f2ll(x));
    return write_all(argv[3], out) ? 0 : 1;
  }
  if (!std::strcmp(mode, "neg")) {
    const std::vector<int64_t> in = read_all<int64_t>(argv[2]);
    std::vector<double> out;
    for (size_t i = 0; i + 1 < in.size(); i += 2) out.push_back(kkt::neg_scaled(in[i], (int)in[i + 1]));
    return write_all(argv[3], out) ? 0 : 1;
  }
  if (!std::strcmp(mode, "digits")) {
    const std::vector<int64_t> in = read_all<int64_t>(argv[2]);
    std::vector<int64_t> out;
    for (size_t i = 0; i + 1 < in.size(); i += 2) {
      double v;
      std::memcpy(&v, &in[i], sizeof v);
      long long b;
      const unsigned long long q = kkt::digits7(v, (int)in[i + 1], b);
      out.push_back((int64_t)q);
      out.push_back(b < 0 ? -1 : 1);
    }
    return write_all(argv[3], out) ? 0 : 1;
  }
  if (!std::strcmp(mode, "balanced")) {
    std::vector<int64_t> out;
    for (int64_t q : read_all<int64_t>(argv[2])) {
      int d[kkt::kEmuSlices];
      kkt::balanced7((unsigned long long)q, d);
      for (int s = 0; s < kkt::kEmuSlices; s++) out.push_back(d[s]);
    }
    return write_all(argv[3], out) ? 0 : 1;
  }
  if (!std::strcmp(mode, "pow2")) {
    std::vector<int64_t> out;
    for (double s : read_all<double>(argv[2])) out.push_back(kkt::pow2_exponent(s));
    return write_all(argv[3], out) ? 0 : 1;
  }
  if (!std::strcmp(mode, "tasks")) {
    const std::vector<int64_t> in = read_all<int64_t>(argv[2]);
    std::vector<int64_t> out;
    for (size_t i = 0; i + 3 < in.size(); i += 4) {
      const int TI = (int)in[i], TJ = (int)in[i + 1], jmode = (int)in[i + 2], jsplit = (int)in[i + 3];
      int total = 0;
      for (int I = 0; I < TI; I++) total += kkt::emu_row_tasks(I, TJ, jmode, jsplit);
      out.push_back(total);
      for (int t = 0; t < total; t++) {
        int I, j0, j1;
        kkt::emu_task(t, TI, TJ, jmode, I, j0, j1, jsplit);
        out.push_back(I);
        out.push_back(j0);
        out.push_back(j1);
      }
    }
    return write_all(argv[3], out) ? 0 : 1;
  }
  if (!std::strcmp(mode, "bf16")) {
    std::vector<uint32_t> out;
    for (uint32_t v = 0; v < 256; v++) out.push_back(kkt::bf16_bits_of_byte(v));
    return write_all(argv[3], out) ? 0 : 1;
  }
  return 2;
}
