// Internal state of a kkt_handle: symbolic structures (host and device),
// numeric buffers, and the kernel entry points shared by the .cu files.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/kkt_schur.h"
#include "symbolic.h"

namespace kkt {

// Records a CUDA error and returns from the enclosing kkt_status function.
void set_error(const std::string& msg);
#define KKT_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      ::kkt::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));         \
      return KKT_ERR_CUDA;                                                          \
    }                                                                               \
  } while (0)

// One update of a factor work item (a 32-row tile of supernode s) by a
// descendant d that meets the tile, with everything the update kernel reads
// about d, so that one load gives it.
struct UpdPair {
  int64_t rel;   // offset of the update's relative row map in upd_rel
  int64_t val;   // offset of d's panel in a block's factor
  int64_t rows;  // offset of d's row list in sn_rows
  int32_t ia, ib;  // d's rows [ia, ib) land in the tile
  int32_t r0, r1;  // d's rows [r0, r1) are columns of s
  int32_t md, wd;  // rows and columns of d's panel
};
static_assert(sizeof(UpdPair) == 48, "UpdPair layout");

// Device copies of the symbolic structures.
struct DevSym {
  int32_t* sn_first = nullptr;
  int64_t* sn_rowptr = nullptr;
  int32_t* sn_rows = nullptr;
  int64_t* sn_valoff = nullptr;
  int64_t* upd_ptr = nullptr;
  int32_t* upd_src = nullptr;
  int32_t* upd_r0 = nullptr;
  int32_t* upd_r1 = nullptr;
  int64_t* upd_reloff = nullptr;
  int32_t* upd_rel = nullptr;
  int32_t* lvl_sn = nullptr;
  int32_t* perm = nullptr;
  int64_t* a_map = nullptr;
  int32_t* col_primal = nullptr;   // per column (elimination order): 1 if primal
  int64_t* col_dpos = nullptr;     // per column: panel position of its pivot
  int32_t* diag_pos = nullptr;     // per row of A (pattern order): position of its diagonal entry
  // factor update work items: (supernode, first panel row, last panel row)
  int32_t* fwork = nullptr;        // 4 ints per item: s, lo, hi, its first update in fpairs (a closing item ends the list)
  UpdPair* fpairs = nullptr;       // per item, the updates of s that meet the tile
  // symmetric full CSR of A for the residual: entry p reads a_vals[full_src[p]]
  int32_t* full_rowptr = nullptr;
  int32_t* full_col = nullptr;
  int32_t* full_src = nullptr;
  // coupling
  int32_t* b_row = nullptr;
  int32_t* b_col = nullptr;
  int32_t* b_blockptr = nullptr;
  int32_t* e_t = nullptr;
  int32_t* e_block = nullptr;
  int32_t* wpos = nullptr;
  int32_t* sn_wrow = nullptr;
  int64_t* w_dpos = nullptr;       // per W row: panel position of its pivot
  int32_t* w_col = nullptr;        // per W row: its column (elimination order)
  int32_t* reach_lvl_sn = nullptr;
  int64_t* s_key = nullptr;
  int64_t* s_ptr = nullptr;
  int32_t* s_e1 = nullptr;
  int32_t* s_e2 = nullptr;
  int32_t* t_ptr = nullptr;
  int32_t* t_e = nullptr;
  int32_t* bt_ptr = nullptr;
  int32_t* E = nullptr;            // the k rows of A carrying B's nonzeros
  int32_t* g_rows = nullptr;       // W rows in contraction order: primal chunks, then multiplier chunks
  int32_t* trsv_jlo = nullptr;     // envelope of S (structured mode): first column block of each row block
  int32_t* trsv_jhi = nullptr;     // one past the last row block of each column block
  int32_t* flvl_sn = nullptr;      // supernodes outside the dense tail, by level (block factor)
  int32_t* twork = nullptr;        // factor work items of the dense-tail supernodes
  int32_t* upd_ntail = nullptr;    // per supernode: leading updates from outside the tail
  int32_t* reach_lvl_sn_nt = nullptr;  // reach supernodes outside the tail, by level
  int32_t* tail_sn_list = nullptr;     // the tail supernodes in the reach of E
  int32_t* tail_wrow = nullptr;        // per tail column: its W row (-1 outside the reach)
  int32_t* wt_ptr = nullptr;           // per supernode: the columns of W on it (wt_idx)
  int32_t* wt_idx = nullptr;
  int32_t* g_key = nullptr;            // sparse contraction: entries t1 * k + t2 of G
  int64_t* g_ptr = nullptr;            // their rows g_row[g_ptr[e] .. g_ptr[e+1])
  int32_t* g_row = nullptr;
  // structured S of the cumulative coupling: per block and storage unit the
  // (index into E, B entry) lists of its own period's columns (y) and of the
  // later periods' (z); pairs of B entries that must hold equal values
  int32_t* cum_y_ptr = nullptr;
  int32_t* cum_y_t = nullptr;
  int32_t* cum_y_e = nullptr;
  int32_t* cum_z_ptr = nullptr;
  int32_t* cum_z_t = nullptr;
  int32_t* cum_z_e = nullptr;
  int32_t* cum_check = nullptr;
};

// Counters written by the kernels (device, int64).
enum Counter { kPos = 0, kNeg, kZero, kPerturbed, kNumCounters };
// counters[0..3]: block pivots; counters[4..7]: pivots of the current factor of S

struct Handle {
  // sizes
  int32_t N = 0, nA = 0, nP = 0, nC = 0, c_kind = 0;
  int64_t nnzA = 0, nnzB = 0, nnzFull = 0;
  kkt_options opt{};
  Symbolic sym;
  Coupling cpl;
  DevSym d;
  std::vector<int32_t> fwork_lvl_ptr;  // factor work items per level
  std::vector<int32_t> lvl_ptr;        // supernodes per level (host copy)
  std::vector<int32_t> reach_lvl_ptr;
  std::vector<int32_t> panel_rend;     // structured mode: per 64-wide panel, one past its last nonzero row
  std::vector<int32_t> flvl_ptr;       // supernodes outside the dense tail per level (factor)
  int32_t nT = 0;                      // columns of the dense tail (0 = none)
  double tail_ratio = 0.0;             // cost ratio the tail was chosen with
  double last_delta_w = 0.0;           // inertia correction: the last successful shift > 0 (0: none yet)
  int32_t nTa = 0;                     // order of the tail matrices: nT, plus k augmented rows
  bool tail_aug = false;               // tail augmented by the k coupling rows (Sec. 4.2)
  int32_t nw_nt = 0;                   // W rows outside the tail (the first ones)
  int32_t tail_reach_sn = 0;           // tail supernodes in the reach of E
  std::vector<int32_t> reach_lvl_ptr_nt;  // reach supernodes outside the tail per level
  std::vector<int32_t> reach_lvl_chunks, reach_lvl_chunks_nt;  // W solve: 32-column chunks per level
  int64_t g_nkeys = 0;                 // nonzero entries of the sparse contraction
  int32_t tail_items = 0;              // factor work items of the tail supernodes
  std::vector<double> fupd_flops;      // algorithmic flops of one block's supernodal updates, per level
  double tupd_flops = 0.0;             // and of the tail's updates from outside it

  // numeric buffers
  double* Lx = nullptr;       // N * panel_total
  double* LDx = nullptr;      // N * ld_total: L D of the panels outside the dense tail
  int64_t ld_total = 0;       // entries of those panels per block (sn_valoff[tail_sn])
  double* a_vals = nullptr;   // N * nnzA (FP64 copy for the residual)
  double* b_vals = nullptr;   // nnzB
  double* c_vals = nullptr;   // nC or nC*nC
  double* anorm = nullptr;    // N: max |a| per block
  double* W = nullptr;        // N * nw * k, row-major per block
  double* G = nullptr;        // N * k * k
  double* wdinv = nullptr;    // N * nw: reciprocal pivot of each W row
  double* S = nullptr;        // nC * nC column-major (lower triangle used)
  double* Ypanel = nullptr;   // nC * kDenseNB scratch of the dense factor
  double* Xinv = nullptr;     // ceil(nC/64) * 64 * 64: inverses of the diagonal blocks of the factor of S
  double* Sdinv = nullptr;    // nC: reciprocal pivots of the factor of S
  double* Tt = nullptr;       // N * nT * nT: dense tails of the block factors (column-major)
  double* TY = nullptr;       // N * nT * kDenseNB: panel scratch of the tail factor
  double* Xtail = nullptr;    // N * ceil(nT/64) * 64 * 64: inverses of the tails' diagonal blocks
  int tail_mode = 0;          // 0 none, 1 FP64 on the CUDA cores, 2 emulated FP64 on the tensor cores
  uint8_t* t_imgA = nullptr;  // per block: tensor-core operand images of one tail panel step
  uint8_t* t_imgB = nullptr;
  double* t_scaleA = nullptr; // per block: row scales of the emulated update (nT + 256)
  double* t_scaleB = nullptr;
  float* S32 = nullptr;       // nC * nC FP32 copy factored in the TF32/BF16 modes
  float* Y32 = nullptr;       // nC * kDenseNB FP32 panel scratch
  uint8_t* tw_img = nullptr;  // TF32 factor of S with 256-wide outer panels: 2 parities x (4 Y + 4 L21) image sets
  // emulated-FP64 factors with 256-wide outer panels: Y of the outer panel,
  // its 256-wide operand images and row scales (for S, and per block for the tails)
  double* ew_s_Y = nullptr;
  uint8_t *ew_s_A = nullptr, *ew_s_B = nullptr;
  double* ew_s_scale = nullptr;
  double* ew_t_Y = nullptr;
  uint8_t *ew_t_A = nullptr, *ew_t_B = nullptr;
  double* ew_t_scale = nullptr;
  int64_t tw_set_bytes = 0;   // bytes of one image set
  uint8_t* tc_imgA = nullptr; // tensor-core operand images of one panel step
  uint8_t* tc_imgB = nullptr;
  double* tc_scaleA = nullptr;  // row scales of the emulated FP64 update
  double* tc_scaleB = nullptr;
  int s_factor = 0;           // current factor of S: 0 FP64-accurate in S, 1 FP32 in S32
  bool g_reduced = false;     // S assembled from a TF32/BF16 contraction
  int g_nchunks = 0, g_nchunks_pos = 0;  // 64-row chunks of g_rows (positive-pivot chunks first)
  double* knorm = nullptr;    // ||K||_inf
  unsigned long long* counters = nullptr;  // kNumCounters
  // solve work vectors
  double* r = nullptr;        // nK: right-hand side being solved
  double* z = nullptr;        // N * nA
  double* u = nullptr;        // N * k
  double* v = nullptr;        // N * k
  double* tg = nullptr;       // nC
  double* xg = nullptr;       // nC
  double* x = nullptr;        // nK iterate
  double* dx = nullptr;       // nK correction
  double* rho = nullptr;      // nK residual
  double* rhs = nullptr;      // nK original right-hand side
  double* red = nullptr;      // reduction scratch (norms; [16, 528) the dot products' partial sums)
  double* gm_V = nullptr;     // GMRES refinement: gmres_restart + 1 Krylov vectors of nK
  double* gm_Z = nullptr;     // and their preconditioned images (gmres_restart vectors)
  double* host_red = nullptr; // pinned
  int* trsv_flags = nullptr;  // 2 * ceil(nC/64): block-ready epochs of the dense triangular solves
  unsigned* trsv_ticket = nullptr;  // 2 tickets (forward, backward)
  int* dev_err = nullptr;     // set when a bounded device wait runs out
  // device-side refinement (opt.device_refine): the solve graph and its loop state
  // (eta, eta_prev, steps, outcome: 0 converged, 1 stopped above the tolerance, 2 not finite)
  // one graph per kind of factor of S (s_factor: the FP32 one of the TF32/BF16
  // modes, or the FP64-accurate one, also after a fallback), built at first use
  cudaGraphExec_t solve_exec[2] = {nullptr, nullptr};
  bool solve_graph_failed[2] = {false, false};
  bool solve_capturing = false;  // the dense triangular solves clear their flags instead of advancing an epoch
  double* rstate = nullptr;
  // structured S of the cumulative coupling (structured_s = 2, cumulative.cu):
  // ns x ns blocks, column-major, N of each unless noted
  bool cum = false;
  int32_t cum_ns = 0;          // coupling variables per period
  int64_t cum_npairs = 0;      // B entries whose values must repeat
  int* cum_err = nullptr;      // set by the factor when they do not
  double* cum_H = nullptr;     // 3 per block: Y^T G Y, Z^T G Y, Z^T G Z
  double* cum_Sd = nullptr;    // S_d (eq. GlobalSchur)
  double* cum_So = nullptr;    // S_o (the last unused)
  double* cum_Q = nullptr;     // N x (2ns)^2: the augmented matrix of each period, factored in place
  double* cum_QY = nullptr;    // 2ns x 64: panel scratch of its factor
  double* cum_Linv = nullptr;  // L_j^{-1}
  double* cum_M = nullptr;     // M_j = L21_j L_j^{-1} (the last zero)
  double* cum_Mt = nullptr;    // M_j^T
  double* cum_D = nullptr;     // N x ns: the pivots
  // FP32 copies of the period factors in the TF32/BF16 modes (the FP64 ones are the fallback)
  float *cum_Q32 = nullptr, *cum_QY32 = nullptr, *cum_Linv32 = nullptr, *cum_M32 = nullptr, *cum_Mt32 = nullptr;
  float* cum_D32 = nullptr;
  int trsv_epoch = 1;          // the last epoch of a direct triangular solve of S (graph solves use 1)
  int64_t device_bytes = 0;

  bool factored = false;
  bool blocks_factored = false;  // block factors and the assembled S are current (kkt_factor_blocks)
  bool front_done = false;       // z holds a front half (kkt_solve_front) that kkt_solve_back may finish
  bool timed_factor = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_f0 = nullptr, ev_f1 = nullptr;
  cudaEvent_t ev_fa = nullptr, ev_fb = nullptr;  // phase boundaries inside kkt_factor
  cudaEvent_t ev_s0 = nullptr, ev_s1 = nullptr;  // around kkt_solve
  cudaEvent_t ev_done = nullptr;  // end of the handle's last factor/solve (outlives the caller's stream)
  // CUDA graph of the factor's launch sequence (captured at the first kkt_factor)
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side_stream = nullptr;  // second stream of the dense factors' lookahead
  cudaStream_t hi_stream = nullptr;    // high-priority stream of the lookahead's critical chain
  cudaStream_t early_stream = nullptr; // kkt_solve's front half, overlapping the factor of S
  cudaEvent_t ev_early = nullptr;
  bool schur_pending = false;          // ev_fb marks the Schur assembly of a factor not yet solved with
  int prio_hi = 0;                     // its priority (also set on the chain's launches)
  cudaEvent_t ev_main = nullptr, ev_side = nullptr;
  cudaGraphExec_t factor_exec = nullptr;
  bool graph_failed = false;
  bool capturing = false;
  int64_t graph_launches = 0;
  int64_t launches = 0;                          // kernels launched since analyze
  kkt_info info{};
  // per-launch timing of the dominant kernels (opt.time_kernels): event pairs,
  // the family and algorithmic flops of each timed launch; kt_used counts the
  // launches of the current factor (fixed by the graph capture when graphs are on)
  std::vector<cudaEvent_t> kt_ev;
  std::vector<int> kt_fam;
  std::vector<double> kt_flops;
  int kt_used = 0;
  int kt_graph_used = 0;  // timed launches inside the factor's graph
};

enum KernelFamily {
  kFamEmu = 0, kFamWide, kFamTc, kFamDenseF64, kFamFactorUpd, kFamDiag, kFamEmuWide, kFamPanelEmu, kNumFamilies
};
// An event before a timed launch on `st` (returns its slot, -1 when not timing
// or the pool is full) and one after it.
int kt_begin(Handle& h, int fam, double flops, cudaStream_t st);
void kt_end(Handle& h, int slot, cudaStream_t st);
// algorithmic flops of a trailing update with inner dimension kb over the
// entries of the lower triangle of an m x m trailing matrix in columns [c0, c1)
inline double update_flops(int64_t m, int64_t c0, int64_t c1, int64_t kb) {
  if (c1 > m) c1 = m;
  if (c0 >= c1) return 0.0;
  // entries (i, j) with c0 <= j < c1 and j <= i < m
  const double e = (double)(c1 - c0) * (double)m - 0.5 * ((double)c1 * (c1 - 1) - (double)c0 * (c0 - 1));
  return 2.0 * (double)kb * e;
}

constexpr int kDenseNB = 64;
constexpr int kFactorTileRows = 32;  // rows of a work item of the supernodal update (factor.cu)

// ---- kernel attributes, set once per device before any launch ----
cudaError_t dense_prepare();
cudaError_t dense_tc_prepare();
cudaError_t schur_tc_prepare();
// ---- kernel launchers (factor.cu) ----
// a_vals[i][diag(r)] += dw for primal rows r, -= dc for dual rows; C's diagonal += dcs
cudaError_t launch_shift_diag(Handle& h, double dw, double dc, double dcs, cudaStream_t st);
cudaError_t launch_scatter_a(Handle& h, cudaStream_t st);
cudaError_t launch_factor_levels(Handle& h, cudaStream_t st);
// ---- (tail.cu) ----
cudaError_t launch_dense_tail(Handle& h, cudaStream_t st);
cudaError_t launch_tail_factor_emulated(Handle& h, cudaStream_t st);  // (dense_tc.cu)
// ---- (schur.cu) ----
cudaError_t launch_w_solve(Handle& h, cudaStream_t st);
cudaError_t launch_w_solve_before_tail(Handle& h, cudaStream_t st);
cudaError_t launch_add_tail_g(Handle& h, cudaStream_t st);
cudaError_t launch_w_dinv(Handle& h, cudaStream_t st);
cudaError_t launch_contract_g(Handle& h, cudaStream_t st);
cudaError_t launch_assemble_s(Handle& h, cudaStream_t st);
// ---- (schur_tc.cu) ----
bool contract_g_tc_supported(const Handle& h);
cudaError_t launch_contract_g_tc(Handle& h, int bf16, cudaStream_t st);
// ---- (dense.cu) ----
cudaError_t launch_dense_ldlt(Handle& h, unsigned long long* counters, cudaStream_t st);
cudaError_t launch_dense_solve(Handle& h, const double* t, double* x, cudaStream_t st);
cudaError_t launch_dense_solve_f32(Handle& h, const double* t, double* x, cudaStream_t st);
cudaError_t launch_diag_inverse(Handle& h, bool f32, cudaStream_t st);
cudaError_t launch_tail_inverse(Handle& h, cudaStream_t st);
cudaError_t launch_tail_fsolve(Handle& h, double* z, cudaStream_t st);  // (tail.cu)
cudaError_t launch_tail_bsolve(Handle& h, double* z, cudaStream_t st);
// ---- (dense_tc.cu) ----
cudaError_t launch_dense_ldlt_tc(Handle& h, int mode, unsigned long long* counters, cudaStream_t st);
int64_t tc_image_bytes_a(int n, int mode);
cudaError_t launch_dense_diag_panel_f64(Handle& h, int k0, int kb, int rend, unsigned long long* counters,
                                        cudaStream_t st);
int64_t tc_image_bytes(int n, int mode);
int64_t tf32_wide_set_bytes(int n);                 // one image set of the 256-wide TF32 factor of S
int64_t emu_wide_image_bytes(int n);                // one operand image of the 256-wide emulated update, order n
bool emu_wide_applies(int npiv);                    // whether the emulated factors take 256-wide outer panels
bool tf32_wide_applies(int n, bool structured);     // whether that factor is used for S of order n
// ---- (solve.cu) ----
cudaError_t launch_apply_inverse(Handle& h, const double* rhs, double* out, cudaStream_t st);
cudaError_t launch_apply_front(Handle& h, const double* rhs, cudaStream_t st);
cudaError_t launch_apply_back(Handle& h, double* out, cudaStream_t st, bool solve_s = true);
cudaError_t launch_dense_factor_of(Handle& h, cudaStream_t st);  // (shard.cu) factor of S in the handle's mode
cudaError_t launch_residual(Handle& h, const double* rhs, const double* x, double* rho,
                            cudaStream_t st);
cudaError_t launch_knorm(Handle& h, cudaStream_t st);
cudaError_t launch_axpy(Handle& h, double* y, const double* x, int64_t n, cudaStream_t st);
cudaError_t launch_norms(Handle& h, const double* rho, const double* x, const double* rhs,
                         cudaStream_t st);
// GMRES refinement: deterministic dot product into device *out (scratch red[16..16+512)), y += a x, y = a x
cudaError_t launch_dot(Handle& h, const double* a, const double* b, int64_t n, double* out, cudaStream_t st);
cudaError_t launch_axpby(Handle& h, double* y, double a, const double* x, int64_t n, cudaStream_t st);
cudaError_t launch_scale_into(Handle& h, double* y, double a, const double* x, int64_t n, cudaStream_t st);

// ---- (cumulative.cu) structured S of the cumulative coupling ----
constexpr int kCumMaxStor = 4096;            // coupling variables per period at most
constexpr int kCumInverseSmem = 200 * 1024;  // dynamic shared memory of its inverse kernel
struct CumPattern {
  int32_t ns = 0;
  std::vector<int32_t> y_ptr, y_t, y_e;  // per block: ns + 1 offsets; (E index, B entry) per entry
  std::vector<int32_t> z_ptr, z_t, z_e;
  std::vector<int32_t> check;            // pairs (entry, entry it must equal)
};
// Checks that B has the cumulative structure and builds the lists ("" on success).
std::string analyze_cumulative(const kkt_pattern* pat, const Coupling& C, CumPattern& out);
cudaError_t cum_prepare();
cudaError_t launch_cum_assemble(Handle& h, cudaStream_t st);   // S_d, S_o from G and B
// the period steps in FP32 (f32: the TF32/BF16 modes) or FP64
cudaError_t launch_cum_factor(Handle& h, unsigned long long* counters, cudaStream_t st, bool f32);
cudaError_t launch_cum_solve(Handle& h, const double* t, double* x, cudaStream_t st);

// Solve work vectors supplied by the caller instead of the handle.
struct SolveWorkspace {
  double* z;    // N * nA
  double* u;    // N * k
  double* v;    // N * k
  double* tg;   // nC
  double* xg;   // nC
  double* dot;  // kDenseNB
};
cudaError_t launch_apply_inverse_ws(Handle& h, const double* rhs, double* out,
                                    const SolveWorkspace& ws, cudaStream_t st);
cudaError_t launch_dense_solve_ws(Handle& h, const double* t, double* x, double* dot,
                                  cudaStream_t st);

}  // namespace kkt
