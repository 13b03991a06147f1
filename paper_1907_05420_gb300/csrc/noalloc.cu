// kkt_solve_noalloc: a solve that allocates nothing.
//
// Some callers cannot call cudaMalloc when they solve: a serving process
// that hands all device memory to its own pool up front and runs under that
// fixed budget, or a latency-critical request loop that cannot accept the
// device-wide synchronization that cudaMalloc/cudaFree may imply.  This entry
// point applies the current factorization once, without refinement, and takes
// every per-call work vector from one file-scope device array instead of the
// handle or a fresh allocation.  It uses its own kernel sequence on those
// vectors: the supernodal level solves over every supernode (a dense tail's
// factor is read from the panels it was scattered back into) and the
// column-by-column dense solve with the factor of S.  kkt_solve applies the
// same factorization with other kernels (dense tail solves, blocked solves of
// S with diagonal-block inverses), so the two agree to rounding, within the
// conditioning bound of K, not bit for bit.  The array is shared by all
// handles and by every call in the process.
#include <mutex>

#include "handle.h"

namespace kkt {
namespace {

// 2^21 doubles = 16 MiB.  Every GPU on which the library's code is loaded
// holds this array until the process exits.
constexpr int64_t kNoAllocScratchDoubles = int64_t(1) << 21;
constexpr int kMaxDevices = 64;

std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};  // device address per device ordinal

}  // namespace

static __device__ __align__(256) double g_solve_scratch[kNoAllocScratchDoubles];

namespace {

// Device address of g_solve_scratch on the current device, looked up once per
// device.  In host code the array's name is only a host-side stand-in, never a
// device address, so kernels receive the address this returns.
kkt_status scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error(std::string("kkt_solve_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return KKT_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("kkt_solve_noalloc: device ordinal beyond the supported range");
    return KKT_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_solve_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("kkt_solve_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return KKT_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return KKT_OK;
}

inline int64_t round_up(int64_t v) { return (v + 31) & ~int64_t(31); }  // 256-byte pieces

}  // namespace
}  // namespace kkt

using namespace kkt;

extern "C" kkt_status kkt_solve_noalloc(kkt_handle* hh, const double* rhs, double* x, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !rhs || !x) {
    set_error("kkt_solve_noalloc: null argument");
    return KKT_ERR_INVALID;
  }
  if (!h->factored) {
    set_error("kkt_solve_noalloc: no factorization");
    return KKT_ERR_STATE;
  }
  if (h->s_factor != 0) {
    set_error("kkt_solve_noalloc: needs an FP64-accurate factor of S (KKT_FP64 or KKT_F64_EMULATED)");
    return KKT_ERR_STATE;
  }
  const int64_t nz = (int64_t)h->N * h->nA, nk = (int64_t)h->N * h->cpl.k;
  const int64_t need = round_up(nz) + 2 * round_up(nk) + 2 * round_up(h->nC) + round_up(kDenseNB);
  if (need > kNoAllocScratchDoubles) {
    set_error("kkt_solve_noalloc: this system needs " + std::to_string(need) +
              " doubles of solve scratch; the static array holds " +
              std::to_string(kNoAllocScratchDoubles) + " (N*nA + 2*N*k + 2*nC must fit)");
    return KKT_ERR_INVALID;
  }
  double* base = nullptr;
  kkt_status st0 = scratch_address(&base);
  if (st0 != KKT_OK) return st0;
  SolveWorkspace ws;
  ws.z = base;
  ws.u = ws.z + round_up(nz);
  ws.v = ws.u + round_up(nk);
  ws.tg = ws.v + round_up(nk);
  ws.xg = ws.tg + round_up(h->nC);
  ws.dot = ws.xg + round_up(h->nC);
  cudaStream_t st = (cudaStream_t)stream;
  h->stream = st;
  // an error left pending by an earlier launch on this thread would otherwise
  // be reported as one of ours below: return it as it is
  const cudaError_t pending = cudaGetLastError();
  if (pending != cudaSuccess) {
    set_error(std::string("kkt_solve_noalloc: error pending from an earlier launch: ") +
              cudaGetErrorString(pending));
    return KKT_ERR_CUDA;
  }
  KKT_CUDA(launch_apply_inverse_ws(*h, rhs, x, ws, st));
  KKT_CUDA(cudaEventRecord(h->ev_done, st));
  return KKT_OK;
}
