// C ABI: kkt_analyze / kkt_factor / kkt_solve / kkt_get_info / kkt_destroy.
//
// Host orchestration only: every arithmetic step of the factor and of the
// solve runs in the kernels of factor.cu, schur.cu, dense.cu and solve.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>

#include "handle.h"

namespace kkt {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

int kt_begin(Handle& h, int fam, double flops, cudaStream_t st) {
  if (!h.opt.time_kernels || 2 * (size_t)(h.kt_used + 1) > h.kt_ev.size()) return -1;
  const int slot = h.kt_used++;
  h.kt_fam[slot] = fam;
  h.kt_flops[slot] = flops;
  cudaEventRecordWithFlags(h.kt_ev[2 * slot], st, h.capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
  return slot;
}

void kt_end(Handle& h, int slot, cudaStream_t st) {
  if (slot < 0) return;
  cudaEventRecordWithFlags(h.kt_ev[2 * slot + 1], st, h.capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
}

namespace {

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& v, int64_t& bytes) {
  size_t n = v.empty() ? 1 : v.size();
  cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * n);
  if (e != cudaSuccess) return e;
  bytes += (int64_t)(sizeof(T) * n);
  if (!v.empty()) e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
  return e;
}

template <class T>
cudaError_t dalloc(T** dst, int64_t count, int64_t& bytes) {
  size_t n = count > 0 ? (size_t)count : 1;
  cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * n);
  if (e == cudaSuccess) bytes += (int64_t)(sizeof(T) * n);
  return e;
}

kkt_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return KKT_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? KKT_ERR_OOM : KKT_ERR_CUDA;
}

void free_all(Handle* h) {
  void* ptrs[] = {h->d.sn_first, h->d.sn_rowptr, h->d.sn_rows, h->d.sn_valoff, h->d.upd_ptr,
                  h->d.upd_src, h->d.upd_r0, h->d.upd_r1, h->d.upd_reloff, h->d.upd_rel,
                  h->d.lvl_sn, h->d.perm, h->d.a_map, h->d.col_primal, h->d.col_dpos, h->d.diag_pos, h->d.fwork, h->d.fpairs,
                  h->d.full_rowptr, h->d.full_col, h->d.full_src, h->d.b_row, h->d.b_col,
                  h->d.b_blockptr, h->d.e_t, h->d.e_block, h->d.wpos, h->d.sn_wrow, h->d.w_dpos,
                  h->d.w_col, h->d.reach_lvl_sn, h->d.s_key, h->d.s_ptr, h->d.s_e1, h->d.s_e2,
                  h->d.t_ptr, h->d.t_e, h->d.bt_ptr, h->d.E, h->d.g_rows, h->d.trsv_jlo, h->d.trsv_jhi,
                  h->d.flvl_sn, h->d.twork, h->d.upd_ntail, h->d.reach_lvl_sn_nt, h->d.tail_sn_list, h->d.tail_wrow, h->d.wt_ptr, h->d.wt_idx,
                  h->d.g_key, h->d.g_ptr, h->d.g_row, h->Xinv, h->Sdinv, h->wdinv, h->Xtail, h->Tt, h->TY, h->t_imgA, h->t_imgB,
                  h->t_scaleA, h->t_scaleB, h->Lx, h->LDx, h->a_vals, h->b_vals,
                  h->c_vals, h->anorm, h->W, h->G, h->S, h->Ypanel, h->knorm, h->counters, h->r,
                  h->z, h->u, h->v, h->tg, h->xg, h->x, h->dx, h->rho, h->rhs, h->red,
                  h->trsv_flags, h->trsv_ticket, h->dev_err, h->S32, h->Y32, h->tw_img, h->ew_s_Y, h->ew_s_A,
                  h->ew_s_B, h->ew_s_scale, h->ew_t_Y, h->ew_t_A, h->ew_t_B, h->ew_t_scale, h->tc_imgA,
                  h->tc_imgB, h->tc_scaleA, h->tc_scaleB, h->gm_V, h->gm_Z, h->d.cum_y_ptr, h->d.cum_y_t,
                  h->d.cum_y_e, h->d.cum_z_ptr, h->d.cum_z_t, h->d.cum_z_e, h->d.cum_check, h->cum_err,
                  h->rstate, h->cum_Q32, h->cum_QY32, h->cum_Linv32, h->cum_M32, h->cum_Mt32, h->cum_D32, h->cum_H, h->cum_Sd, h->cum_So, h->cum_Q, h->cum_QY, h->cum_Linv, h->cum_M, h->cum_Mt,
                  h->cum_D};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->host_red) cudaFreeHost(h->host_red);
  cudaEvent_t evs[] = {h->ev_f0, h->ev_f1, h->ev_fa, h->ev_fb, h->ev_s0, h->ev_s1, h->ev_done};
  for (cudaEvent_t ev : evs)
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : h->kt_ev)
    if (ev) cudaEventDestroy(ev);
  if (h->factor_exec) cudaGraphExecDestroy(h->factor_exec);
  for (cudaGraphExec_t ex : h->solve_exec)
    if (ex) cudaGraphExecDestroy(ex);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side_stream) cudaStreamDestroy(h->side_stream);
  if (h->early_stream) cudaStreamDestroy(h->early_stream);
  if (h->ev_early) cudaEventDestroy(h->ev_early);
  if (h->hi_stream) cudaStreamDestroy(h->hi_stream);
  if (h->ev_main) cudaEventDestroy(h->ev_main);
  if (h->ev_side) cudaEventDestroy(h->ev_side);
}

// An event record that becomes a node of the graph while the factor is captured.
cudaError_t record(Handle& h, cudaEvent_t ev, cudaStream_t st) {
  return cudaEventRecordWithFlags(ev, st, h.capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// The device work of kkt_factor after the input copies: every launch depends
// only on the handle's buffers and options, so the sequence is captured once
// as a CUDA graph and replayed.
cudaError_t enqueue_factor(Handle& h, cudaStream_t st, bool with_s = true) {
  h.kt_used = 0;
  cudaError_t e = cudaMemsetAsync(h.counters, 0, sizeof(unsigned long long) * 2 * kNumCounters, st);
#define STEP(x) \
  if (e == cudaSuccess) e = (x)
  STEP(launch_scatter_a(h, st));
  STEP(launch_factor_levels(h, st));
  STEP(record(h, h.ev_fa, st));
  STEP(launch_w_dinv(h, st));
  STEP(launch_w_solve(h, st));
  if (h.g_reduced) {
    STEP(launch_contract_g_tc(h, h.opt.prec == KKT_BF16 ? 1 : 0, st));
  } else {
    STEP(launch_contract_g(h, st));
  }
  if (h.cum) {
    STEP(launch_cum_assemble(h, st));
  } else {
    STEP(launch_assemble_s(h, st));
  }
  STEP(record(h, h.ev_fb, st));
  if (!with_s) {
    // the factor of S is left to kkt_factor_schur (a sharded solve reduces S first)
  } else if (h.cum) {
    STEP(launch_cum_factor(h, h.counters + kNumCounters, st, h.opt.prec == KKT_TF32 || h.opt.prec == KKT_BF16));
  } else if (h.opt.prec == KKT_FP64) {
    STEP(launch_dense_ldlt(h, h.counters + kNumCounters, st));
  } else {
    STEP(launch_dense_ldlt_tc(h, h.opt.prec, h.counters + kNumCounters, st));
  }
  STEP(launch_knorm(h, st));
#undef STEP
  return e;
}

// The convergence test of the refinement on the device (device_refine): the
// same test as kkt_solve's loop, from the norms of this step's residual, and
// the decision whether the loop's body runs again (the body applies the
// factorization to the residual, adds the correction and recomputes the
// residual and its norms).  st: eta, eta_prev, steps, outcome (0 converged or
// still running, 1 stopped above the tolerance, 2 a non-finite iterate, 3 a
// non-finite K or right-hand side).
__global__ void k_refine_decide(const double* __restrict__ red, const double* __restrict__ knorm, double tol,
                                int max_steps, double* __restrict__ st, cudaGraphConditionalHandle loop,
                                int first) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (first) {
    st[1] = INFINITY;
    st[2] = 0.0;
  }
  const double r0 = red[0], r1 = red[1], r2 = red[2], kn = knorm[0];
  unsigned int again = 0;
  double eta, outcome;
  if (!isfinite(r2) || !isfinite(kn)) {
    eta = NAN;
    outcome = 3.0;  // a NaN or Inf in K or the right-hand side: no iterate can meet the test
  } else {
    const bool finite_x = isfinite(r0) && isfinite(r1);
    eta = finite_x ? r0 / (kn * r1 + r2) : NAN;
    if (finite_x && r0 == 0.0) eta = 0.0;
    const double steps = st[2];
    if (eta <= tol) {
      outcome = 0.0;
    } else {
      const bool stalled = !(eta < 0.5 * st[1]) || !isfinite(eta);
      if (steps >= (double)max_steps || (steps > 0.0 && stalled) || !finite_x) {
        outcome = finite_x ? 1.0 : 2.0;
      } else {
        outcome = 0.0;
        again = 1;
        st[1] = eta;
        st[2] = steps + 1.0;
      }
    }
  }
  st[0] = eta;
  st[3] = outcome;
  cudaGraphSetConditional(loop, again);
}

// Captures enqueue_factor into h.factor_exec; on any failure the handle keeps
// launching directly.
void capture_factor(Handle& h) {
  const int64_t l0 = h.launches;
  cudaGraph_t g = nullptr;
  h.capturing = true;
  cudaError_t e = cudaStreamBeginCapture(h.cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = enqueue_factor(h, h.cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(h.cap_stream, &g);
    e = e1 != cudaSuccess ? e1 : e2;
  }
  h.capturing = false;
  if (e == cudaSuccess && g) e = cudaGraphInstantiate(&h.factor_exec, g, cudaGraphInstantiateFlagUseNodePriority);
  if (g) cudaGraphDestroy(g);
  h.graph_launches = h.launches - l0;
  h.launches = l0;
  if (e != cudaSuccess || !h.factor_exec) {
    h.graph_failed = true;
    h.factor_exec = nullptr;
    (void)cudaGetLastError();
  }
}

}  // namespace
}  // namespace kkt

using namespace kkt;

extern "C" {

void kkt_default_options(kkt_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->prec = KKT_FP64;
  opt->refine_tol = 1e-10;
  opt->max_refine = 10;
  opt->pivot_eps = 1e-20;
  opt->use_graphs = 1;
  opt->fp64_fallback = 1;
  opt->dense_tail = -1;
  opt->gmres_restart = 8;
  opt->device_refine = 0;
}

const char* kkt_status_string(kkt_status s) {
  switch (s) {
    case KKT_OK: return "ok";
    case KKT_ERR_INVALID: return "invalid argument";
    case KKT_ERR_OOM: return "out of memory";
    case KKT_ERR_CUDA: return "CUDA error";
    case KKT_ERR_ZERO_PIVOT: return "zero pivot";
    case KKT_ERR_INERTIA: return "wrong inertia";
    case KKT_ERR_NOT_CONVERGED: return "refinement did not converge";
    case KKT_ERR_TIMEOUT: return "device wait timed out";
    case KKT_ERR_STATE: return "call out of order";
    case KKT_ERR_NONFINITE: return "NaN or Inf in the system or the solution";
  }
  return "unknown status";
}

const char* kkt_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace {

// One analysis with the dense tail chosen at cost ratio `tail_ratio`.  With
// `sym0` and `cpl0`, the ordering, supernodes and coupling reach are copied
// from an earlier analysis of the same pattern instead of being recomputed
// (they do not depend on the tail).
kkt_status analyze_one(const kkt_pattern* pat, const kkt_options* opt, double tail_ratio, const Symbolic* sym0,
                       const Coupling* cpl0, kkt_handle** out) {
  *out = nullptr;
  if (!pat->a_rowptr || !pat->a_col || !pat->b_blockptr || (pat->c_kind != 0 && pat->c_kind != 1) ||
      pat->N <= 0 || pat->nA <= 0 || pat->nC < 0) {
    set_error("kkt_analyze: malformed pattern descriptor");
    return KKT_ERR_INVALID;
  }
  const int64_t nnzB = pat->b_blockptr[pat->N];
  if (nnzB > 0 && (!pat->b_row || !pat->b_col)) {
    set_error("kkt_analyze: B has entries but no row/col arrays");
    return KKT_ERR_INVALID;
  }
  auto t0 = std::chrono::steady_clock::now();
  Handle* h = new (std::nothrow) Handle();
  if (!h) return KKT_ERR_OOM;
  kkt_default_options(&h->opt);
  if (opt) h->opt = *opt;
  if (h->opt.prec < KKT_FP64 || h->opt.prec > KKT_F64_EMULATED) {
    set_error("kkt_analyze: unknown precision mode");
    delete h;
    return KKT_ERR_INVALID;
  }
  if (h->opt.structured_s < 0 || h->opt.structured_s > 2) {
    set_error("kkt_analyze: structured_s must be 0, 1 or 2");
    delete h;
    return KKT_ERR_INVALID;
  }
  if (h->opt.device_refine != 0 && (h->opt.device_refine != 1 || h->opt.refine_mode != 0)) {
    set_error("kkt_analyze: device_refine must be 0, or 1 with refine_mode 0");
    delete h;
    return KKT_ERR_INVALID;
  }
  if ((h->opt.refine_mode != 0 && h->opt.refine_mode != 1) || h->opt.gmres_restart < 1 || h->opt.gmres_restart > 64) {
    set_error("kkt_analyze: refine_mode must be 0 or 1 and gmres_restart in [1, 64]");
    delete h;
    return KKT_ERR_INVALID;
  }
  h->N = pat->N;
  h->nA = pat->nA;
  h->nP = pat->nP;
  h->nC = pat->nC;
  h->c_kind = pat->c_kind;

  std::string err;
  if (sym0 && cpl0) {
    h->sym = *sym0;
    h->cpl = *cpl0;
  } else {
    err = analyze_pattern(pat->nA, pat->nP, pat->a_rowptr, pat->a_col, pat->a_vals_hint,
                          pat->a_vals_hint ? 1 : 0, h->sym);
    if (err.empty())
      err = analyze_coupling(h->sym, pat->N, pat->nC, pat->b_blockptr, pat->b_row, pat->b_col, h->cpl,
                             h->opt.structured_s != 2);
  }
  CumPattern cum;
  if (err.empty() && h->opt.structured_s == 2 && pat->nC > 0) {
    err = analyze_cumulative(pat, h->cpl, cum);
    h->cum = err.empty();
    h->cum_ns = cum.ns;
    h->cum_npairs = (int64_t)cum.check.size() / 2;
  }
  if (!err.empty()) {
    set_error("kkt_analyze: " + err);
    delete h;
    return KKT_ERR_INVALID;
  }
  // dense tail: -1 (default) picks the emulated tail in the reduced-precision
  // modes and none in the plain FP64 mode
  h->tail_mode = h->opt.dense_tail < 0 ? (h->opt.prec == KKT_FP64 ? 1 : 2) : h->opt.dense_tail;
  if (h->tail_mode < 0 || h->tail_mode > 2) {
    set_error("kkt_analyze: dense_tail must be -1, 0, 1 or 2");
    delete h;
    return KKT_ERR_INVALID;
  }
  h->tail_ratio = tail_ratio;
  if (h->tail_mode)
    choose_tail(h->sym, h->N, h->tail_mode == 2 ? kTailMaxBytesTC : kTailMaxBytes, kTailMinCols, tail_ratio);
  else choose_tail(h->sym, h->N, 0, 0);  // no tail fits in 0 bytes
  const Symbolic& S = h->sym;
  const Coupling& C = h->cpl;
  const int32_t n = S.n;
  h->nT = n - S.tail_col;
  if (h->nT == 0) h->tail_mode = 0;
  // Augmented tail: the k coupling rows are appended to each tail triangle, and
  // its factorization also yields W's tail rows and the tail's share of G
  // (Sec. 4.2, the incomplete factorization of the augmented matrix); the tail's
  // W rows (those of its supernodes in the reach of E) come after all others.
  std::vector<int32_t> tail_wrow;
  h->nw_nt = tail_w_rows(S, C, tail_wrow);
  h->tail_aug = h->tail_mode != 0 && h->nT > 0 && C.k > 0;
  if (!h->tail_aug) h->nw_nt = C.nw;
  h->nTa = h->nT + (h->tail_aug ? C.k : 0);
  h->nnzA = pat->a_rowptr[n];
  h->nnzB = nnzB;
  // position of every row's diagonal entry (the inertia-correction shift)
  std::vector<int32_t> diag_pos(n, -1);
  for (int32_t r = 0; r < n; r++)
    for (int32_t p = pat->a_rowptr[r]; p < pat->a_rowptr[r + 1]; p++)
      if (pat->a_col[p] == r) diag_pos[r] = p;
  if (std::find(diag_pos.begin(), diag_pos.end(), -1) != diag_pos.end()) {
    set_error("kkt_analyze: a row of A has no diagonal entry");
    delete h;
    return KKT_ERR_INVALID;
  }
  h->lvl_ptr = S.lvl_ptr;
  h->reach_lvl_ptr = C.reach_lvl_ptr;
  // reach supernodes outside the tail, by level (the W solve before the tail)
  std::vector<int32_t> reach_lvl_sn_nt, tail_sn_list;
  h->reach_lvl_ptr_nt.assign(S.nlevels + 1, 0);
  for (int l = 0; l < S.nlevels; l++) {
    for (int q = C.reach_lvl_ptr[l]; q < C.reach_lvl_ptr[l + 1]; q++)
      if (C.reach_lvl_sn[q] < S.tail_sn) reach_lvl_sn_nt.push_back(C.reach_lvl_sn[q]);
    h->reach_lvl_ptr_nt[l + 1] = (int32_t)reach_lvl_sn_nt.size();
  }
  for (int s = S.tail_sn; s < S.nsuper; s++)
    if (C.sn_wrow[s] >= 0) tail_sn_list.push_back(s);  // tail supernodes in the reach of E
  h->tail_reach_sn = (int32_t)tail_sn_list.size();
  // W solve: per level, the most 32-column chunks of any of its supernodes
  auto chunks_of = [&](const std::vector<int32_t>& ptr, const std::vector<int32_t>& sn, std::vector<int32_t>& out) {
    out.assign(S.nlevels, 1);
    for (int l = 0; l < S.nlevels; l++)
      for (int q = ptr[l]; q < ptr[l + 1]; q++) {
        const int s = sn[q], nts = C.wt_ptr[s + 1] - C.wt_ptr[s];
        out[l] = std::max(out[l], (nts + 31) / 32);
      }
  };
  chunks_of(h->reach_lvl_ptr, C.reach_lvl_sn, h->reach_lvl_chunks);
  chunks_of(h->reach_lvl_ptr_nt, reach_lvl_sn_nt, h->reach_lvl_chunks_nt);
  // sparse contraction over the W rows outside the (augmented) tail
  std::vector<int32_t> g_key, g_row;
  std::vector<int64_t> g_ptr;
  g_gather(S, C, h->tail_aug ? S.tail_sn : S.nsuper, g_key, g_ptr, g_row);
  h->g_nkeys = (int64_t)g_key.size();

  // factor work items: 32-row tiles of every supernode outside the dense tail,
  // grouped by level, then those of the tail supernodes; per item the updates
  // that meet the tile, as (update index within s's list, rows [ia, ib) of the
  // descendant that land in the tile), from the item's offset to the next item's
  std::vector<int32_t> fwork, twork, flvl_sn;
  std::vector<UpdPair> fpairs;
  // algorithmic flops of the updates of each work item: descendant d adds w_d
  // multiply-adds to every target entry (row i, column j) of the tile with
  // i >= j, i one of d's rows in the tile ([ia, ib)), j one in s's columns ([r0, r1))
  double item_flops = 0.0;
  auto pair_flops = [&](int64_t ia, int64_t ib, int64_t r0, int64_t r1, int64_t wd) {
    double cnt = 0.0;
    const int64_t a = std::max(ia, r0), z = std::min(ib, r1);  // i in [r0, r1): i - r0 + 1 targets
    if (z > a) cnt += 0.5 * (double)(z - a) * (double)((a - r0 + 1) + (z - r0));
    const int64_t a2 = std::max(ia, r1);  // i >= r1: all r1 - r0 targets
    if (ib > a2) cnt += (double)(ib - a2) * (double)(r1 - r0);
    return 2.0 * (double)wd * cnt;
  };
  auto add_items = [&](int s, std::vector<int32_t>& items) {
    int m = (int)(S.sn_rowptr[s + 1] - S.sn_rowptr[s]);
    for (int lo = 0; lo < m; lo += kFactorTileRows) {
      const int hi = std::min(m, lo + kFactorTileRows);
      items.push_back(s);
      items.push_back(lo);
      items.push_back(hi);
      items.push_back((int32_t)fpairs.size());
      for (int64_t u = S.upd_ptr[s]; u < S.upd_ptr[s + 1]; u++) {
        const int32_t* rel = S.upd_rel.data() + S.upd_reloff[u];
        const int64_t nrel = S.upd_reloff[u + 1] - S.upd_reloff[u];
        const int32_t ia = S.upd_r0[u] + (int32_t)(std::lower_bound(rel, rel + nrel, lo) - rel);
        const int32_t ib = S.upd_r0[u] + (int32_t)(std::lower_bound(rel, rel + nrel, hi) - rel);
        const int dd = S.upd_src[u];
        // the tail's own updates among its supernodes run in the dense tail factor
        const bool counted = !(s >= S.tail_sn && u - S.upd_ptr[s] >= S.upd_ntail[s]);
        if (counted && ia < ib) {
          UpdPair pr;
          pr.rel = S.upd_reloff[u];
          pr.val = S.sn_valoff[dd];
          pr.rows = S.sn_rowptr[dd];
          pr.ia = ia;
          pr.ib = ib;
          pr.r0 = S.upd_r0[u];
          pr.r1 = S.upd_r1[u];
          pr.md = (int32_t)(S.sn_rowptr[dd + 1] - S.sn_rowptr[dd]);
          pr.wd = S.sn_first[dd + 1] - S.sn_first[dd];
          fpairs.push_back(pr);
          item_flops += pair_flops(ia, ib, S.upd_r0[u], S.upd_r1[u], S.sn_first[dd + 1] - S.sn_first[dd]);
        }
      }
    }
  };
  h->fwork_lvl_ptr.assign(S.nlevels + 1, 0);
  h->flvl_ptr.assign(S.nlevels + 1, 0);
  h->fupd_flops.assign(S.nlevels, 0.0);
  for (int l = 0; l < S.nlevels; l++) {
    item_flops = 0.0;
    for (int q = S.lvl_ptr[l]; q < S.lvl_ptr[l + 1]; q++) {
      const int s = S.lvl_sn[q];
      if (s >= S.tail_sn) continue;
      flvl_sn.push_back(s);
      add_items(s, fwork);
    }
    h->fupd_flops[l] = item_flops;
    h->fwork_lvl_ptr[l + 1] = (int32_t)(fwork.size() / 4);
    h->flvl_ptr[l + 1] = (int32_t)flvl_sn.size();
  }
  // a closing item after each list gives its last item the end of its updates
  const auto close_items = [&](std::vector<int32_t>& items) {
    items.insert(items.end(), {0, 0, 0, (int32_t)fpairs.size()});
  };
  close_items(fwork);
  item_flops = 0.0;
  for (int s = S.tail_sn; s < S.nsuper; s++) add_items(s, twork);
  h->tupd_flops = item_flops;
  h->tail_items = (int32_t)(twork.size() / 4);
  close_items(twork);
  // per-column pivot position and primal flag
  std::vector<int64_t> col_dpos(n);
  std::vector<int32_t> col_primal(n);
  for (int s = 0; s < S.nsuper; s++) {
    int f = S.sn_first[s], w = S.sn_first[s + 1] - f;
    int64_t m = S.sn_rowptr[s + 1] - S.sn_rowptr[s];
    for (int c = 0; c < w; c++) col_dpos[f + c] = S.sn_valoff[s] + (int64_t)c * m + c;
  }
  for (int j = 0; j < n; j++) col_primal[j] = S.perm[j] < S.nP ? 1 : 0;
  // W rows
  std::vector<int64_t> w_dpos(C.nw);
  std::vector<int32_t> w_col(C.nw);
  for (int s = 0; s < S.nsuper; s++) {
    if (C.sn_wrow[s] < 0) continue;
    int f = S.sn_first[s], w = S.sn_first[s + 1] - f;
    for (int c = 0; c < w; c++) {
      w_col[C.sn_wrow[s] + c] = f + c;
      w_dpos[C.sn_wrow[s] + c] = col_dpos[f + c];
    }
  }
  // W rows in contraction order: primal (positive pivot) rows, then multiplier
  // rows, each group padded with -1 to whole 64-row chunks
  std::vector<int32_t> g_rows;
  {
    std::vector<int32_t> pos_rows, neg_rows;
    // with the augmented tail, the tail rows' share of G comes from the tail factor
    const int nw_contract = h->nw_nt;
    for (int r = 0; r < nw_contract; r++) (col_primal[w_col[r]] ? pos_rows : neg_rows).push_back(r);
    auto pad = [](std::vector<int32_t>& v) {
      while (v.size() % 64) v.push_back(-1);
    };
    pad(pos_rows);
    pad(neg_rows);
    h->g_nchunks_pos = (int)(pos_rows.size() / 64);
    h->g_nchunks = h->g_nchunks_pos + (int)(neg_rows.size() / 64);
    g_rows = pos_rows;
    g_rows.insert(g_rows.end(), neg_rows.begin(), neg_rows.end());
  }
  // row envelope of S for the structured mode
  std::vector<int32_t> trsv_jlo, trsv_jhi;
  if (h->opt.structured_s == 1 && h->nC > 0) s_envelope(C, h->c_kind, kDenseNB, h->panel_rend, trsv_jlo, trsv_jhi);
  // symmetric full CSR of A with source positions
  std::vector<int32_t> full_rowptr(n + 1, 0), full_col, full_src;
  for (int r = 0; r < n; r++)
    for (int p = pat->a_rowptr[r]; p < pat->a_rowptr[r + 1]; p++) {
      full_rowptr[r + 1]++;
      if (pat->a_col[p] != r) full_rowptr[pat->a_col[p] + 1]++;
    }
  for (int r = 0; r < n; r++) full_rowptr[r + 1] += full_rowptr[r];
  full_col.resize(full_rowptr[n]);
  full_src.resize(full_rowptr[n]);
  {
    std::vector<int32_t> fill(full_rowptr.begin(), full_rowptr.end() - 1);
    for (int r = 0; r < n; r++)
      for (int p = pat->a_rowptr[r]; p < pat->a_rowptr[r + 1]; p++) {
        int c = pat->a_col[p];
        full_col[fill[r]] = c;
        full_src[fill[r]++] = p;
        if (c != r) {
          full_col[fill[c]] = r;
          full_src[fill[c]++] = p;
        }
      }
  }
  h->nnzFull = full_rowptr[n];
  std::vector<int32_t> b_row(pat->b_row ? pat->b_row : nullptr, pat->b_row ? pat->b_row + nnzB : nullptr);
  std::vector<int32_t> b_col(pat->b_col ? pat->b_col : nullptr, pat->b_col ? pat->b_col + nnzB : nullptr);
  std::vector<int32_t> b_blockptr(pat->b_blockptr, pat->b_blockptr + pat->N + 1);

  int64_t& by = h->device_bytes;
  cudaError_t e = cudaSuccess;
#define UP(dst, vec) \
  if (e == cudaSuccess) e = upload(&h->d.dst, vec, by)
  UP(sn_first, S.sn_first);
  UP(sn_rowptr, S.sn_rowptr);
  UP(sn_rows, S.sn_rows);
  UP(sn_valoff, S.sn_valoff);
  UP(upd_ptr, S.upd_ptr);
  UP(upd_src, S.upd_src);
  UP(upd_r0, S.upd_r0);
  UP(upd_r1, S.upd_r1);
  UP(upd_reloff, S.upd_reloff);
  UP(upd_rel, S.upd_rel);
  UP(lvl_sn, S.lvl_sn);
  UP(perm, S.perm);
  UP(a_map, S.a_map);
  UP(col_primal, col_primal);
  UP(col_dpos, col_dpos);
  UP(diag_pos, diag_pos);
  UP(fwork, fwork);
  UP(fpairs, fpairs);
  UP(flvl_sn, flvl_sn);
  UP(twork, twork);
  UP(upd_ntail, S.upd_ntail);
  UP(full_rowptr, full_rowptr);
  UP(full_col, full_col);
  UP(full_src, full_src);
  UP(b_row, b_row);
  UP(b_col, b_col);
  UP(b_blockptr, b_blockptr);
  UP(e_t, C.e_t);
  UP(e_block, C.e_block);
  UP(wpos, C.wpos);
  UP(sn_wrow, C.sn_wrow);
  UP(w_dpos, w_dpos);
  UP(w_col, w_col);
  UP(reach_lvl_sn, C.reach_lvl_sn);
  UP(reach_lvl_sn_nt, reach_lvl_sn_nt);
  UP(tail_sn_list, tail_sn_list);
  UP(tail_wrow, tail_wrow);
  UP(wt_ptr, C.wt_ptr);
  UP(wt_idx, C.wt_idx);
  UP(g_key, g_key);
  UP(g_ptr, g_ptr);
  UP(g_row, g_row);
  UP(s_key, C.s_key);
  UP(s_ptr, C.s_ptr);
  UP(s_e1, C.s_e1);
  UP(s_e2, C.s_e2);
  UP(t_ptr, C.t_ptr);
  UP(t_e, C.t_e);
  UP(bt_ptr, C.bt_ptr);
  UP(E, C.E);
  UP(g_rows, g_rows);
  if (!trsv_jlo.empty()) {
    UP(trsv_jlo, trsv_jlo);
    UP(trsv_jhi, trsv_jhi);
  }
  if (h->cum) {
    UP(cum_y_ptr, cum.y_ptr);
    UP(cum_y_t, cum.y_t);
    UP(cum_y_e, cum.y_e);
    UP(cum_z_ptr, cum.z_ptr);
    UP(cum_z_t, cum.z_t);
    UP(cum_z_e, cum.z_e);
    UP(cum_check, cum.check);
  }
#undef UP
  const int64_t nK = (int64_t)h->N * n + h->nC;
  const int64_t k = C.k;
#define AL(dst, T, cnt) \
  if (e == cudaSuccess) e = dalloc<T>(&h->dst, cnt, by)
  AL(Lx, double, S.panel_total * h->N);
  h->ld_total = std::max<int64_t>(1, S.sn_valoff[S.tail_sn]);
  AL(LDx, double, h->ld_total * h->N);
  AL(a_vals, double, h->nnzA * h->N);
  AL(b_vals, double, nnzB);
  AL(c_vals, double, h->c_kind == 0 ? (int64_t)h->nC : (int64_t)h->nC * h->nC);
  AL(anorm, double, h->N);
  AL(W, double, (int64_t)C.nw * k * h->N);
  AL(G, double, k * k * h->N);
  AL(wdinv, double, (int64_t)C.nw * h->N);
  // the dense S and its factor's buffers (none with the structured S)
  const int64_t nCd = h->cum ? 0 : h->nC;
  AL(S, double, nCd * nCd);
  AL(Ypanel, double, nCd * kDenseNB);
  AL(Xinv, double, (int64_t)((nCd + kDenseNB - 1) / kDenseNB) * kDenseNB * kDenseNB);
  if (h->cum) {
    const int64_t ns = h->cum_ns, nn = ns * ns;
    AL(cum_err, int, 1);
    AL(cum_H, double, 3 * nn * h->N);
    AL(cum_Sd, double, nn * h->N);
    AL(cum_So, double, nn * h->N);
    AL(cum_Q, double, 4 * nn * h->N);
    AL(cum_QY, double, 2 * ns * kDenseNB);
    AL(cum_Linv, double, nn * h->N);
    AL(cum_M, double, nn * h->N);
    AL(cum_Mt, double, nn * h->N);
    AL(cum_D, double, ns * h->N);
    // the last period has no M_j: it stays zero; the flag starts clear
    if (e == cudaSuccess) e = cudaMemset(h->cum_M, 0, sizeof(double) * (size_t)(nn * h->N));
    if (e == cudaSuccess) e = cudaMemset(h->cum_Mt, 0, sizeof(double) * (size_t)(nn * h->N));
    if (e == cudaSuccess) e = cudaMemset(h->cum_err, 0, sizeof(int));
    if (h->opt.prec == KKT_TF32 || h->opt.prec == KKT_BF16) {
      AL(cum_Q32, float, 4 * nn * h->N);
      AL(cum_QY32, float, 2 * ns * kDenseNB);
      AL(cum_Linv32, float, nn * h->N);
      AL(cum_M32, float, nn * h->N);
      AL(cum_Mt32, float, nn * h->N);
      AL(cum_D32, float, ns * h->N);
      if (e == cudaSuccess) e = cudaMemset(h->cum_M32, 0, sizeof(float) * (size_t)(nn * h->N));
      if (e == cudaSuccess) e = cudaMemset(h->cum_Mt32, 0, sizeof(float) * (size_t)(nn * h->N));
    }
  }
  AL(Sdinv, double, h->nC);
  if (h->nT > 0) {
    AL(Xtail, double, (int64_t)((h->nT + kDenseNB - 1) / kDenseNB) * kDenseNB * kDenseNB * h->N);
    AL(Tt, double, (int64_t)h->nTa * h->nTa * h->N);
    AL(TY, double, (int64_t)h->nTa * kDenseNB * h->N);
  }
  if (h->tail_mode == 2) {
    const int64_t ia = tc_image_bytes_a(h->nTa, KKT_F64_EMULATED);
    const int64_t ib = tc_image_bytes(h->nTa, KKT_F64_EMULATED) - ia;
    AL(t_imgA, uint8_t, ia * h->N);
    AL(t_imgB, uint8_t, ib * h->N);
    AL(t_scaleA, double, ((int64_t)h->nTa + 256) * h->N);
    AL(t_scaleB, double, ((int64_t)h->nTa + 256) * h->N);
    if (emu_wide_applies(h->nT)) {  // 256-wide outer panels of the tails
      AL(ew_t_Y, double, (int64_t)h->nTa * 256 * h->N);
      AL(ew_t_A, uint8_t, emu_wide_image_bytes(h->nTa) * h->N);
      AL(ew_t_B, uint8_t, emu_wide_image_bytes(h->nTa) * h->N);
      AL(ew_t_scale, double, 2 * ((int64_t)h->nTa + 256) * h->N);
    }
  }
  AL(knorm, double, 1);
  AL(counters, unsigned long long, 2 * kNumCounters);  // second half: discarded counts
  AL(z, double, (int64_t)h->N * n);
  AL(u, double, k * h->N);
  AL(v, double, k * h->N);
  AL(tg, double, h->nC);
  AL(xg, double, h->nC);
  AL(x, double, nK);
  AL(dx, double, nK);
  AL(rho, double, nK);
  AL(rhs, double, nK);
  AL(red, double, 1024);
  AL(rstate, double, 4);
  if (h->opt.refine_mode == 1) {
    const int m = std::max(1, h->opt.gmres_restart);
    AL(gm_V, double, (int64_t)(m + 1) * nK);
    AL(gm_Z, double, (int64_t)m * nK);
  }
  AL(trsv_flags, int, 2 * ((h->nC + kDenseNB - 1) / kDenseNB));
  if ((h->opt.prec == KKT_TF32 || h->opt.prec == KKT_BF16) && !h->cum) {
    AL(S32, float, (int64_t)h->nC * h->nC);
    AL(Y32, float, (int64_t)h->nC * kDenseNB);
  }
  if (h->opt.prec == KKT_TF32 && !h->cum && tf32_wide_applies(h->nC, h->opt.structured_s != 0)) {
    h->tw_set_bytes = tf32_wide_set_bytes(h->nC);
    AL(tw_img, uint8_t, 16 * h->tw_set_bytes);
    // rows past the trailing matrix are read (and masked) in whole tiles: keep them finite
    if (e == cudaSuccess) e = cudaMemset(h->tw_img, 0, (size_t)(16 * h->tw_set_bytes));
  }
  if (h->opt.prec != KKT_FP64 && h->nC > 0 && !h->cum) {
    // operand images sized for the largest panel step; the FP64 fallback of the
    // reduced modes uses the emulated path, so size for the larger of the two
    const int mode_img = KKT_F64_EMULATED;
    const int64_t ia = tc_image_bytes_a(h->nC, mode_img);
    const int64_t itot = tc_image_bytes(h->nC, mode_img);
    AL(tc_imgA, uint8_t, ia);
    AL(tc_imgB, uint8_t, itot - ia);
    AL(tc_scaleA, double, (int64_t)h->nC + 256);
    AL(tc_scaleB, double, (int64_t)h->nC + 256);
    if (emu_wide_applies(h->nC) && !h->opt.structured_s) {  // the emulated factor of S (mode or fallback)
      AL(ew_s_Y, double, (int64_t)h->nC * 256);
      AL(ew_s_A, uint8_t, emu_wide_image_bytes(h->nC));
      AL(ew_s_B, uint8_t, emu_wide_image_bytes(h->nC));
      AL(ew_s_scale, double, 2 * ((int64_t)h->nC + 256));
    }
  }
  AL(trsv_ticket, unsigned, 2);
  AL(dev_err, int, 1);
#undef AL
  if (e == cudaSuccess)
    e = cudaMemset(h->trsv_flags, 0, sizeof(int) * (size_t)std::max(1, 2 * ((h->nC + kDenseNB - 1) / kDenseNB)));
  if (e == cudaSuccess) e = cudaMemset(h->dev_err, 0, sizeof(int));
  // W's structurally zero entries are never written: clear it once
  if (e == cudaSuccess) e = cudaMemset(h->W, 0, sizeof(double) * (size_t)std::max<int64_t>(1, (int64_t)C.nw * C.k * h->N));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h->host_red, sizeof(double) * 8);
  for (cudaEvent_t* ev : {&h->ev_f0, &h->ev_f1, &h->ev_fa, &h->ev_fb, &h->ev_s0, &h->ev_s1, &h->ev_done})
    if (e == cudaSuccess) e = cudaEventCreate(ev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->early_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_early, cudaEventDisableTiming);
  if (e == cudaSuccess) {
    int lo = 0, hi = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->hi_stream, cudaStreamNonBlocking, hi);
    h->prio_hi = hi;
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_main, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_side, cudaEventDisableTiming);
  if (e == cudaSuccess && h->opt.time_kernels) {
    // an upper bound on the timed launches of one factor and its fallback
    const int64_t slots = 8 * ((int64_t)(h->nTa + 63) / 64 + (h->nC + 63) / 64) + 2 * S.nlevels + 64;
    h->kt_ev.assign(2 * slots, nullptr);
    h->kt_fam.assign(slots, 0);
    h->kt_flops.assign(slots, 0.0);
    for (auto& ev : h->kt_ev)
      if (e == cudaSuccess) e = cudaEventCreate(&ev);
  }
  if (e == cudaSuccess) e = dense_prepare();
  if (e == cudaSuccess) e = dense_tc_prepare();
  if (e == cudaSuccess) e = schur_tc_prepare();
  if (e == cudaSuccess && h->cum) e = cum_prepare();
  if (e != cudaSuccess) {
    kkt_status st = cuda_status(e, "kkt_analyze");
    free_all(h);
    delete h;
    return st;
  }
  h->info.nnz_l = S.nnzL;
  h->info.panel_doubles = S.panel_total;
  h->info.n_supernodes = S.nsuper;
  h->info.n_levels = S.nlevels;
  h->info.k_coupling_rows = C.k;
  h->info.w_rows = C.nw;
  h->info.factor_flops = S.flops;
  h->info.schur_block = h->cum ? h->cum_ns : 0;
  h->info.ms_analyze =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = reinterpret_cast<kkt_handle*>(h);
  return KKT_OK;
}

// Device time of one kkt_factor (the second of two, after the graph capture
// of the first) on representative values: every block takes the values hint,
// B is zero, C the identity.
double time_factor(kkt_handle* hh, const kkt_pattern* pat) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  const int64_t nA_vals = h->nnzA * h->N, nb = std::max<int64_t>(1, h->nnzB);
  const int64_t nc = h->c_kind == 0 ? h->nC : (int64_t)h->nC * h->nC;
  std::vector<double> a((size_t)nA_vals), b((size_t)nb, 0.0), c((size_t)std::max<int64_t>(1, nc), 0.0);
  for (int i = 0; i < h->N; i++) std::copy(pat->a_vals_hint, pat->a_vals_hint + h->nnzA, a.begin() + i * h->nnzA);
  for (int64_t q = 0; q < h->nC; q++) c[h->c_kind == 0 ? q : q * h->nC + q] = 1.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double ms = -1.0;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
      kkt_factor(hh, a.data(), b.data(), c.data(), 0, nullptr) == KKT_OK && cudaDeviceSynchronize() == cudaSuccess &&
      cudaEventRecord(e0, nullptr) == cudaSuccess && kkt_factor(hh, a.data(), b.data(), c.data(), 0, nullptr) == KKT_OK &&
      cudaEventRecord(e1, nullptr) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) {
    float f = 0.f;
    if (cudaEventElapsedTime(&f, e0, e1) == cudaSuccess) ms = f;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  (void)cudaGetLastError();
  return ms;
}

// The factor of the input values with the inertia-correction shift (dw, dc;
// dcs on C's diagonal) applied to the device copy (none when dw and dc are 0).
kkt_status factor_values(Handle* h, const double* a_vals, const double* b_vals, const double* c_vals,
                         int32_t on_device, cudaStream_t st, double dw, double dc, double dcs, bool with_s = true) {
  h->stream = st;
  (void)cudaGetLastError();  // drop a stale non-sticky error left by an unrelated call
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const int64_t nc_vals = h->c_kind == 0 ? (int64_t)h->nC : (int64_t)h->nC * h->nC;
  KKT_CUDA(cudaEventRecord(h->ev_f0, st));
  KKT_CUDA(cudaMemcpyAsync(h->a_vals, a_vals, sizeof(double) * h->nnzA * h->N, kind, st));
  if (h->nnzB > 0) KKT_CUDA(cudaMemcpyAsync(h->b_vals, b_vals, sizeof(double) * h->nnzB, kind, st));
  if (nc_vals > 0) KKT_CUDA(cudaMemcpyAsync(h->c_vals, c_vals, sizeof(double) * nc_vals, kind, st));
  if (dw != 0.0 || dc != 0.0) KKT_CUDA(launch_shift_diag(*h, dw, dc, dcs, st));
  // the split factor (kkt_factor_blocks) keeps the FP64 contraction: its S may
  // take other processes' parts, which a fallback could not rebuild
  h->g_reduced = with_s && (h->opt.prec == KKT_TF32 || h->opt.prec == KKT_BF16) && h->opt.reduced_contraction &&
                 contract_g_tc_supported(*h);
  h->s_factor = (h->opt.prec == KKT_TF32 || h->opt.prec == KKT_BF16) ? 1 : 0;
  if (with_s && h->opt.use_graphs && !h->graph_failed && !h->factor_exec) {
    capture_factor(*h);
    h->kt_graph_used = h->kt_used;
  }
  if (with_s && h->factor_exec) {
    KKT_CUDA(cudaGraphLaunch(h->factor_exec, st));
    h->launches += h->graph_launches;
    h->kt_used = h->kt_graph_used;  // the graph re-records the events of its timed launches
  } else {
    KKT_CUDA(enqueue_factor(*h, st, with_s));
  }
  h->info.fell_back_fp64 = 0;
  h->schur_pending = with_s;
  KKT_CUDA(cudaEventRecord(h->ev_f1, st));
  KKT_CUDA(cudaEventRecord(h->ev_done, st));
  h->blocks_factored = true;
  h->front_done = false;
  h->factored = with_s;
  h->timed_factor = with_s;
  return KKT_OK;
}

// The factor of S redone FP64-accurately (emulated FP64 on the tensor cores)
// after a reduced-precision one, from an FP64 contraction if G was reduced.
kkt_status refactor_s_fp64(Handle* h, cudaStream_t st) {
  KKT_CUDA(cudaMemsetAsync(h->counters + kNumCounters, 0, sizeof(unsigned long long) * kNumCounters, st));
  if (h->g_reduced) {
    // S was assembled from a reduced-precision contraction: rebuild it in FP64
    KKT_CUDA(launch_contract_g(*h, st));
    KKT_CUDA(h->cum ? launch_cum_assemble(*h, st) : launch_assemble_s(*h, st));
    h->g_reduced = false;
  }
  if (h->cum) {
    KKT_CUDA(launch_cum_factor(*h, h->counters + kNumCounters, st, false));  // the FP64 period steps
  } else {
    KKT_CUDA(launch_dense_ldlt_tc(*h, KKT_F64_EMULATED, h->counters + kNumCounters, st));
  }
  h->s_factor = 0;
  h->info.fell_back_fp64 = 1;
  return KKT_OK;
}

// The solve graph of device_refine: apply the factorization to h->rhs into
// h->x, residual, norms and the test; then a WHILE node whose body is one
// refinement step (apply to the residual, x += dx, residual, norms, test).
// The application depends on the kind of factor of S the handle holds
// (h.s_factor), so there is one graph per kind.  On any failure the handle
// keeps the host loop for that kind.
void build_solve_graph(Handle& h) {
  const int sf = h.s_factor;
  const int64_t nK = (int64_t)h.N * h.nA + h.nC;
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle loop{};
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&loop, g, 0, cudaGraphCondAssignDefault);
  const int64_t l0 = h.launches;
  h.solve_capturing = true;
  auto capture_into = [&](cudaGraph_t target, bool prologue) -> cudaError_t {
    cudaError_t c = cudaStreamBeginCaptureToGraph(h.cap_stream, target, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
    if (c != cudaSuccess) return c;
    cudaError_t w;
    if (prologue) {
      w = launch_apply_inverse(h, h.rhs, h.x, h.cap_stream);
    } else {
      w = launch_apply_inverse(h, h.rho, h.dx, h.cap_stream);
      if (w == cudaSuccess) w = launch_axpy(h, h.x, h.dx, nK, h.cap_stream);
    }
    if (w == cudaSuccess) w = launch_residual(h, h.rhs, h.x, h.rho, h.cap_stream);
    if (w == cudaSuccess) w = launch_norms(h, h.rho, h.x, h.rhs, h.cap_stream);
    if (w == cudaSuccess) {
      k_refine_decide<<<1, 32, 0, h.cap_stream>>>(h.red, h.knorm, h.opt.refine_tol, h.opt.max_refine, h.rstate,
                                                   loop, prologue ? 1 : 0);
      w = cudaGetLastError();
    }
    cudaGraph_t out = nullptr;
    c = cudaStreamEndCapture(h.cap_stream, &out);
    return w != cudaSuccess ? w : c;
  };
  if (e == cudaSuccess) e = capture_into(g, true);
  // the loop node after every leaf of the prologue
  std::vector<cudaGraphNode_t> leaves;
  if (e == cudaSuccess) {
    size_t nn = 0;
    e = cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess && nn) e = cudaGraphGetNodes(g, nodes.data(), &nn);
    for (size_t i = 0; e == cudaSuccess && i < nn; i++) {
      size_t nd = 0;
      e = cudaGraphNodeGetDependentNodes(nodes[i], nullptr, nullptr, &nd);
      if (e == cudaSuccess && nd == 0) leaves.push_back(nodes[i]);
    }
  }
  if (e == cudaSuccess) {
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = loop;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t wnode = nullptr;
    e = cudaGraphAddNode(&wnode, g, leaves.data(), nullptr, leaves.size(), &np);
    if (e == cudaSuccess) e = capture_into(np.conditional.phGraph_out[0], false);
  }
  h.solve_capturing = false;
  h.launches = l0;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h.solve_exec[sf], g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess || !h.solve_exec[sf]) {
    h.solve_graph_failed[sf] = true;
    h.solve_exec[sf] = nullptr;
    (void)cudaGetLastError();
  }
}

// One cycle of GMRES refinement (right preconditioning by the factorization
// K~): from the residual rho = r - K x in h->rho, up to `budget` Krylov steps
// z_j = K~^{-1} v_j, w = K z_j, modified Gram-Schmidt against v_0..v_j, Givens
// rotations on the Hessenberg column; stops once the residual estimate |g_{j+1}|
// (a 2-norm, so a bound on the infinity norm) is below `target`.  Then x +=
// sum_j y_j z_j with H y = g solved on the host.  `its` receives the steps taken.
kkt_status gmres_cycle(Handle* h, cudaStream_t st, double target, int budget, int& its) {
  const int64_t nK = (int64_t)h->N * h->nA + h->nC;
  const int m = std::min(budget, std::max(1, h->opt.gmres_restart));
  double* V = h->gm_V;
  double* Z = h->gm_Z;
  its = 0;
  auto dot = [&](const double* a, const double* b, double& out) -> kkt_status {
    KKT_CUDA(launch_dot(*h, a, b, nK, h->red + 8, st));
    KKT_CUDA(cudaMemcpyAsync(h->host_red + 6, h->red + 8, sizeof(double), cudaMemcpyDeviceToHost, st));
    KKT_CUDA(cudaStreamSynchronize(st));
    out = h->host_red[6];
    return KKT_OK;
  };
  double beta2 = 0.0;
  kkt_status ks = dot(h->rho, h->rho, beta2);
  if (ks != KKT_OK) return ks;
  const double beta = std::sqrt(beta2);
  if (!(beta > 0.0) || !std::isfinite(beta)) return KKT_OK;
  KKT_CUDA(launch_scale_into(*h, V, 1.0 / beta, h->rho, nK, st));
  KKT_CUDA(cudaMemsetAsync(h->dx, 0, sizeof(double) * (size_t)nK, st));  // zero right-hand side for K z
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), g(m + 1, 0.0);
  auto Hc = [&](int i, int j) -> double& { return H[(size_t)j * (m + 1) + i]; };
  g[0] = beta;
  int k = 0;
  for (int j = 0; j < m; j++) {
    double* vj = V + (size_t)j * nK;
    double* zj = Z + (size_t)j * nK;
    double* u = V + (size_t)(j + 1) * nK;
    KKT_CUDA(launch_apply_inverse(*h, vj, zj, st));
    KKT_CUDA(launch_residual(*h, h->dx, zj, u, st));  // u = -K z_j
    for (int i = 0; i <= j; i++) {
      double d = 0.0;
      ks = dot(u, V + (size_t)i * nK, d);
      if (ks != KKT_OK) return ks;
      Hc(i, j) = -d;  // (K z_j, v_i)
      KKT_CUDA(launch_axpby(*h, u, -d, V + (size_t)i * nK, nK, st));  // u = -(w - sum h_ij v_i)
    }
    double hn2 = 0.0;
    ks = dot(u, u, hn2);
    if (ks != KKT_OK) return ks;
    const double hn = std::sqrt(hn2);
    Hc(j + 1, j) = hn;
    k = j + 1;
    its = k;
    if (!std::isfinite(hn)) break;
    if (hn > 0.0) KKT_CUDA(launch_scale_into(*h, u, -1.0 / hn, u, nK, st));
    for (int i = 0; i < j; i++) {  // earlier rotations on the new column
      const double t = cs[i] * Hc(i, j) + sn[i] * Hc(i + 1, j);
      Hc(i + 1, j) = -sn[i] * Hc(i, j) + cs[i] * Hc(i + 1, j);
      Hc(i, j) = t;
    }
    const double r = std::hypot(Hc(j, j), Hc(j + 1, j));
    cs[j] = r > 0.0 ? Hc(j, j) / r : 1.0;
    sn[j] = r > 0.0 ? Hc(j + 1, j) / r : 0.0;
    Hc(j, j) = r;
    Hc(j + 1, j) = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    if (std::fabs(g[j + 1]) <= target || hn == 0.0) break;
  }
  // back substitution R y = g, then x += Z y
  std::vector<double> y(k, 0.0);
  for (int i = k - 1; i >= 0; i--) {
    double t = g[i];
    for (int l = i + 1; l < k; l++) t -= Hc(i, l) * y[l];
    y[i] = Hc(i, i) != 0.0 ? t / Hc(i, i) : 0.0;
  }
  for (int i = 0; i < k; i++)
    if (y[i] != 0.0 && std::isfinite(y[i])) KKT_CUDA(launch_axpby(*h, h->x, y[i], Z + (size_t)i * nK, nK, st));
  return KKT_OK;
}

}  // namespace

extern "C" {

kkt_status kkt_analyze(const kkt_pattern* pat, const kkt_options* opt, kkt_handle** out) {
  if (!pat || !out) {
    set_error("kkt_analyze: null argument");
    return KKT_ERR_INVALID;
  }
  *out = nullptr;
  kkt_options o;
  kkt_default_options(&o);
  if (opt) o = *opt;
  auto t0 = std::chrono::steady_clock::now();
  if (!(o.tail_ratio >= 0.0)) {
    set_error("kkt_analyze: tail_ratio must be >= 0");
    return KKT_ERR_INVALID;
  }
  kkt_handle* best = nullptr;
  kkt_status st = analyze_one(pat, &o, o.tail_ratio > 0.0 ? o.tail_ratio : kTailRatio, nullptr, nullptr, &best);
  if (st != KKT_OK) return st;
  // Autotuning of the dense tail: the candidate cost ratios give tails of
  // different sizes; each distinct one is set up (on a copy of the first
  // analysis) and timed once on the values hint, and the fastest factor is kept.
  if (o.autotune && o.tail_ratio == 0.0 && pat->a_vals_hint && reinterpret_cast<Handle*>(best)->nT > 0) {
    double best_ms = time_factor(best, pat);
    std::vector<int32_t> tried = {reinterpret_cast<Handle*>(best)->nT};
    // the first analysis, kept while `best` may be replaced
    const Symbolic sym0 = reinterpret_cast<Handle*>(best)->sym;
    const Coupling cpl0 = reinterpret_cast<Handle*>(best)->cpl;
    for (double r : {1.0, 1.25, 2.0, 3.0}) {
      kkt_handle* cand = nullptr;
      if (analyze_one(pat, &o, r, &sym0, &cpl0, &cand) != KKT_OK) continue;
      const int32_t nT = reinterpret_cast<Handle*>(cand)->nT;
      if (std::find(tried.begin(), tried.end(), nT) != tried.end()) {
        kkt_destroy(cand);
        continue;
      }
      tried.push_back(nT);
      const double ms = time_factor(cand, pat);
      if (ms > 0.0 && (best_ms <= 0.0 || ms < best_ms)) {
        kkt_destroy(best);
        best = cand;
        best_ms = ms;
      } else {
        kkt_destroy(cand);
      }
    }
    Handle* h = reinterpret_cast<Handle*>(best);
    h->info.autotune_candidates = (int32_t)tried.size();
    h->info.ms_analyze = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  *out = best;
  return KKT_OK;
}

kkt_status kkt_factor(kkt_handle* hh, const double* a_vals, const double* b_vals,
                      const double* c_vals, int32_t on_device, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !a_vals || (h->nnzB > 0 && !b_vals) || (h->nC > 0 && !c_vals)) {
    set_error("kkt_factor: null argument");
    return KKT_ERR_INVALID;
  }
  return factor_values(h, a_vals, b_vals, c_vals, on_device, (cudaStream_t)stream, 0.0, 0.0, 0.0);
}

kkt_status kkt_factor_blocks(kkt_handle* hh, const double* a_vals, const double* b_vals, const double* c_vals,
                             int32_t on_device, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !a_vals || (h->nnzB > 0 && !b_vals) || (h->nC > 0 && !c_vals)) {
    set_error("kkt_factor_blocks: null argument");
    return KKT_ERR_INVALID;
  }
  if (h->cum) {
    set_error("kkt_factor_blocks: the structured S (structured_s = 2) has no dense S to reduce");
    return KKT_ERR_INVALID;
  }
  return factor_values(h, a_vals, b_vals, c_vals, on_device, (cudaStream_t)stream, 0.0, 0.0, 0.0, false);
}

void kkt_default_inertia_options(kkt_inertia_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->delta_w_init = 1e-4;
  opt->delta_w_min = 1e-20;
  opt->delta_w_max = 1e40;
  opt->grow_first = 100.0;
  opt->grow = 8.0;
  opt->shrink = 1.0 / 3.0;
  opt->delta_c = 1e-8;
  opt->max_trials = 40;
}

kkt_status kkt_factor_inertia(kkt_handle* hh, const double* a_vals, const double* b_vals, const double* c_vals,
                              int32_t on_device, void* stream, const kkt_inertia_options* opt,
                              kkt_inertia_result* result) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !a_vals || (h->nnzB > 0 && !b_vals) || (h->nC > 0 && !c_vals)) {
    set_error("kkt_factor_inertia: null argument");
    return KKT_ERR_INVALID;
  }
  kkt_inertia_options o;
  kkt_default_inertia_options(&o);
  if (opt) o = *opt;
  if (!(o.delta_w_init > 0.0) || !(o.delta_w_min > 0.0) || !(o.delta_w_max >= o.delta_w_init) ||
      !(o.grow_first > 1.0) || !(o.grow > 1.0) || !(o.shrink > 0.0 && o.shrink < 1.0) || !(o.delta_c >= 0.0) ||
      o.max_trials < 1 || (o.coupling_dual != 0 && o.coupling_dual != 1)) {
    set_error("kkt_factor_inertia: invalid options");
    return KKT_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // expected pivot signs: blocks (N*nP, N*nD, 0); S (nC, 0, 0), or (0, nC, 0)
  // when the coupling variables are multipliers
  const uint64_t pos_blk = (uint64_t)h->N * h->nP, neg_blk = (uint64_t)h->N * (h->nA - h->nP);
  const uint64_t pos_s = o.coupling_dual ? 0 : (uint64_t)h->nC, neg_s = o.coupling_dual ? (uint64_t)h->nC : 0;
  unsigned long long c[2 * kNumCounters];
  int dev_err = 0, cum_err = 0;
  auto read_counts = [&]() -> kkt_status {
    KKT_CUDA(cudaMemcpyAsync(c, h->counters, sizeof(c), cudaMemcpyDeviceToHost, st));
    KKT_CUDA(cudaMemcpyAsync(&dev_err, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (h->cum) KKT_CUDA(cudaMemcpyAsync(&cum_err, h->cum_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    KKT_CUDA(cudaStreamSynchronize(st));
    if (dev_err != 0) {
      set_error("kkt_factor_inertia: a bounded device wait ran out");
      return KKT_ERR_TIMEOUT;
    }
    if (cum_err != 0) {
      set_error("kkt_factor_inertia: B's values do not repeat over the later periods (structured_s = 2)");
      return KKT_ERR_INVALID;
    }
    return KKT_OK;
  };
  double dw = 0.0, dc = 0.0;          // the next trial's shifts
  double used_dw = 0.0, used_dc = 0.0;  // those of the factor the handle holds
  int32_t trials = 0;
  kkt_status status = KKT_ERR_INERTIA;
  for (;;) {
    kkt_status fs = factor_values(h, a_vals, b_vals, c_vals, on_device, st, dw, dc, o.coupling_dual ? -dc : dw);
    used_dw = dw;
    used_dc = dc;
    if (fs == KKT_OK) fs = read_counts();
    if (fs != KKT_OK) return fs;
    trials++;
    const bool blocks_ok =
        c[kPos] == pos_blk && c[kNeg] == neg_blk && c[kZero] == 0 && c[kPerturbed] == 0;
    auto s_right = [&]() {
      return c[kNumCounters + kPos] == pos_s && c[kNumCounters + kNeg] == neg_s && c[kNumCounters + kZero] == 0;
    };
    bool s_ok = s_right();
    if (blocks_ok && !s_ok && h->s_factor == 1) {
      // reduced-precision pivot signs of S are not reliable: recount them on
      // an FP64-accurate factor before shifting
      fs = refactor_s_fp64(h, st);
      if (fs == KKT_OK) fs = read_counts();
      if (fs != KKT_OK) return fs;
      s_ok = s_right();
    }
    if (blocks_ok && s_ok) {
      status = KKT_OK;
      break;
    }
    if (trials >= o.max_trials) break;
    if (c[kZero] > 0 || c[kPerturbed] > 0 || c[kNumCounters + kZero] > 0) dc = o.delta_c;  // singular
    double next;
    if (dw == 0.0) next = h->last_delta_w > 0.0 ? std::max(o.delta_w_min, o.shrink * h->last_delta_w) : o.delta_w_init;
    else next = dw * (h->last_delta_w > 0.0 ? o.grow : o.grow_first);
    if (next > o.delta_w_max) break;
    dw = next;
  }
  if (status == KKT_OK && used_dw > 0.0) h->last_delta_w = used_dw;
  if (result) {
    result->delta_w = used_dw;
    result->delta_c = used_dc;
    result->trials = trials;
    result->reserved = 0;
  }
  if (status != KKT_OK) set_error("kkt_factor_inertia: no shift within the limits gave the expected inertia");
  return status;
}


kkt_status kkt_solve(kkt_handle* hh, const double* rhs, double* x, int32_t nrhs, int32_t on_device,
                     void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !rhs || !x || nrhs < 1) {
    set_error("kkt_solve: invalid argument");
    return KKT_ERR_INVALID;
  }
  if (!h->factored) {
    set_error("kkt_solve: no factorization");
    return KKT_ERR_STATE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  h->stream = st;
  (void)cudaGetLastError();
  auto t0 = std::chrono::steady_clock::now();
  const int64_t nK = (int64_t)h->N * h->nA + h->nC;
  kkt_status result = KKT_OK;
  KKT_CUDA(cudaEventRecord(h->ev_s0, st));
  for (int32_t q = 0; q < nrhs; q++) {
    const double* rq = rhs + q * nK;
    double* xq = x + q * nK;
    const bool early = q == 0 && h->opt.early_solve && h->schur_pending;
    const int sf = h->s_factor;
    if (h->opt.device_refine && !early && !h->solve_exec[sf] && !h->solve_graph_failed[sf]) build_solve_graph(*h);
    const bool on_graph = h->opt.device_refine && !early && h->solve_exec[sf];
    int steps = 0, before_fallback = 0;  // steps of this refinement, of the one before the FP64 fallback
    bool nonfinite = false, host_loop = true;
    double eta = INFINITY, eta_prev = INFINITY;
    if (on_graph) {
      // the application and the refinement loop on the device; one read of the outcome
      KKT_CUDA(cudaMemcpyAsync(h->rhs, rq, sizeof(double) * nK,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
      KKT_CUDA(cudaGraphLaunch(h->solve_exec[sf], st));
      KKT_CUDA(cudaMemcpyAsync(h->host_red, h->rstate, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
      KKT_CUDA(cudaMemcpyAsync(h->host_red + 4, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
      if (h->cum) KKT_CUDA(cudaMemcpyAsync(h->host_red + 5, h->cum_err, sizeof(int), cudaMemcpyDeviceToHost, st));
      KKT_CUDA(cudaStreamSynchronize(st));
      if (*reinterpret_cast<int*>(h->host_red + 4) != 0) {
        set_error("kkt_solve: a bounded device wait ran out");
        return KKT_ERR_TIMEOUT;
      }
      if (h->cum && *reinterpret_cast<int*>(h->host_red + 5) != 0) {
        set_error("kkt_solve: B's values do not repeat over the later periods (structured_s = 2)");
        return KKT_ERR_INVALID;
      }
      eta = h->host_red[0];
      steps = (int)h->host_red[2];
      const int outcome = (int)h->host_red[3];
      host_loop = false;
      if (outcome == 3) {
        nonfinite = true;  // a NaN or Inf among the values of K or the right-hand side
      } else if (outcome != 0 && h->s_factor == 1 && h->opt.fp64_fallback) {
        // stopped above the tolerance with the FP32 factor of S: the fallback
        // and its refinement run on the host, as without device_refine
        const kkt_status rs = refactor_s_fp64(h, st);
        if (rs != KKT_OK) return rs;
        KKT_CUDA(launch_apply_inverse(*h, h->rhs, h->x, st));
        before_fallback = steps + 1;
        steps = 0;
        host_loop = true;
      } else if (outcome == 2) {
        nonfinite = true;
      }
    } else if (early) {
      // the front half needs only the block factors and W: it starts when the
      // preceding factor's Schur assembly ends, beside the dense factor of S
      KKT_CUDA(cudaStreamWaitEvent(h->early_stream, h->ev_fb, 0));
      KKT_CUDA(cudaMemcpyAsync(h->rhs, rq, sizeof(double) * nK,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->early_stream));
      KKT_CUDA(launch_apply_front(*h, h->rhs, h->early_stream));
      KKT_CUDA(cudaEventRecord(h->ev_early, h->early_stream));
      KKT_CUDA(cudaStreamWaitEvent(st, h->ev_early, 0));
      KKT_CUDA(launch_apply_back(*h, h->x, st));
    } else {
      KKT_CUDA(cudaMemcpyAsync(h->rhs, rq, sizeof(double) * nK,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
      KKT_CUDA(launch_apply_inverse(*h, h->rhs, h->x, st));
    }
    h->schur_pending = false;
    while (host_loop) {
      KKT_CUDA(launch_residual(*h, h->rhs, h->x, h->rho, st));
      KKT_CUDA(launch_norms(*h, h->rho, h->x, h->rhs, st));
      KKT_CUDA(cudaMemcpyAsync(h->host_red, h->red, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
      KKT_CUDA(cudaMemcpyAsync(h->host_red + 3, h->knorm, sizeof(double), cudaMemcpyDeviceToHost, st));
      KKT_CUDA(cudaMemcpyAsync(h->host_red + 4, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
      if (h->cum) KKT_CUDA(cudaMemcpyAsync(h->host_red + 5, h->cum_err, sizeof(int), cudaMemcpyDeviceToHost, st));
      KKT_CUDA(cudaStreamSynchronize(st));
      if (*reinterpret_cast<int*>(h->host_red + 4) != 0) {
        set_error("kkt_solve: a bounded device wait ran out");
        return KKT_ERR_TIMEOUT;
      }
      if (h->cum && *reinterpret_cast<int*>(h->host_red + 5) != 0) {
        set_error("kkt_solve: B's values do not repeat over the later periods (structured_s = 2)");
        return KKT_ERR_INVALID;
      }
      const double* hr = h->host_red;
      // hr: ||rho||, ||x||, ||r|| (inf-norms that keep NaN) and ||K||_inf
      if (!std::isfinite(hr[2]) || !std::isfinite(hr[3])) {
        // a NaN or Inf among the values of K or the right-hand side: no
        // iterate can meet the test, and eta would be meaningless
        eta = NAN;
        nonfinite = true;
        break;
      }
      const bool iterate_finite = std::isfinite(hr[0]) && std::isfinite(hr[1]);
      eta = iterate_finite ? hr[0] / (hr[3] * hr[1] + hr[2]) : NAN;
      if (iterate_finite && hr[0] == 0.0) eta = 0.0;  // exact: K x = r in FP64
      if (eta <= h->opt.refine_tol) break;
      const bool stalled = !(eta < 0.5 * eta_prev) || !std::isfinite(eta);
      if (steps >= h->opt.max_refine || (steps > 0 && stalled) || !iterate_finite) {
        if (h->s_factor == 1 && h->opt.fp64_fallback) {
          // refinement with the FP32 factor of S stalls: refactor S (still the
          // assembled FP64 matrix) FP64-accurately and restart from its solve
          const kkt_status rs = refactor_s_fp64(h, st);
          if (rs != KKT_OK) return rs;
          KKT_CUDA(launch_apply_inverse(*h, h->rhs, h->x, st));
          eta_prev = INFINITY;
          // the refinement starts over on the FP64-accurate factor, with its own budget
          before_fallback += steps + 1;
          steps = 0;
          continue;
        }
        if (!iterate_finite) nonfinite = true;
        break;
      }
      eta_prev = eta;
      if (h->opt.refine_mode == 1) {
        // a cycle aims at the residual whose eta is the target (its 2-norm
        // estimate bounds the infinity norm the test uses)
        int its = 0;
        const kkt_status gs =
            gmres_cycle(h, st, h->opt.refine_tol * (hr[3] * hr[1] + hr[2]), h->opt.max_refine - steps, its);
        if (gs != KKT_OK) return gs;
        if (its == 0) break;
        steps += its;
        continue;
      }
      KKT_CUDA(launch_apply_inverse(*h, h->rho, h->dx, st));
      KKT_CUDA(launch_axpy(*h, h->x, h->dx, nK, st));
      steps++;
    }
    KKT_CUDA(cudaMemcpyAsync(xq, h->x, sizeof(double) * nK,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    h->info.refine_steps = before_fallback + steps;
    h->info.rel_residual = eta;
    if (nonfinite) result = KKT_ERR_NONFINITE;
    else if (!(eta <= h->opt.refine_tol) && result == KKT_OK) result = KKT_ERR_NOT_CONVERGED;
  }
  KKT_CUDA(cudaEventRecord(h->ev_s1, st));
  KKT_CUDA(cudaEventRecord(h->ev_done, st));
  KKT_CUDA(cudaStreamSynchronize(st));
  {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_s0, h->ev_s1) == cudaSuccess) h->info.ms_solve_device = ms;
  }
  h->info.ms_solve =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (result == KKT_ERR_NONFINITE)
    set_error("kkt_solve: NaN or Inf in the values of K, the right-hand side or the solution");
  else if (result != KKT_OK)
    set_error("kkt_solve: refinement stopped above refine_tol");
  return result;
}

kkt_status kkt_get_info(kkt_handle* hh, kkt_info* info) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !info) {
    set_error("kkt_get_info: null argument");
    return KKT_ERR_INVALID;
  }
  KKT_CUDA(cudaEventSynchronize(h->ev_done));
  if (h->factored) {
    unsigned long long c[2 * kNumCounters];
    KKT_CUDA(cudaMemcpy(c, h->counters, sizeof(c), cudaMemcpyDeviceToHost));
    h->info.n_pos = (int64_t)(c[kPos] + c[kNumCounters + kPos]);
    h->info.n_neg = (int64_t)(c[kNeg] + c[kNumCounters + kNeg]);
    h->info.n_zero = (int64_t)(c[kZero] + c[kNumCounters + kZero]);
    h->info.n_perturbed = (int64_t)c[kPerturbed];
    if (h->timed_factor) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, h->ev_f0, h->ev_f1) == cudaSuccess) h->info.ms_factor = ms;
      if (cudaEventElapsedTime(&ms, h->ev_f0, h->ev_fa) == cudaSuccess) h->info.ms_block_factor = ms;
      if (cudaEventElapsedTime(&ms, h->ev_fa, h->ev_fb) == cudaSuccess) h->info.ms_schur_assembly = ms;
      if (cudaEventElapsedTime(&ms, h->ev_fb, h->ev_f1) == cudaSuccess) h->info.ms_dense_factor = ms;
      h->timed_factor = false;
    }
  }
  h->info.device_bytes = h->device_bytes;
  h->info.n_launches = h->launches;
  h->info.dense_tail_cols = h->nT;
  h->info.tail_ratio = h->nT > 0 ? h->tail_ratio : 0.0;
  h->info.tail_augmented = h->tail_aug ? 1 : 0;
  *info = h->info;
  return KKT_OK;
}

kkt_status kkt_kernel_stats(kkt_handle* hh, int32_t family, kkt_kernel_stat* out) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !out || family < 0 || family >= kNumFamilies) {
    set_error("kkt_kernel_stats: invalid argument");
    return KKT_ERR_INVALID;
  }
  std::memset(out, 0, sizeof(*out));
  KKT_CUDA(cudaEventSynchronize(h->ev_done));
  for (int q = 0; q < h->kt_used; q++) {
    if (h->kt_fam[q] != family) continue;
    float ms = 0.f;
    KKT_CUDA(cudaEventElapsedTime(&ms, h->kt_ev[2 * q], h->kt_ev[2 * q + 1]));
    out->launches++;
    out->ms_total += ms;
    out->ms_max = std::max(out->ms_max, (double)ms);
    out->flops += h->kt_flops[q];
  }
  return KKT_OK;
}

kkt_status kkt_destroy(kkt_handle* hh) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return KKT_OK;
  cudaEventSynchronize(h->ev_done);
  free_all(h);
  delete h;
  return KKT_OK;
}

}  // extern "C"
