// Host-only inspection of the symbolic analysis (no CUDA): the structures that
// kkt_analyze uploads, exposed as int64 arrays for tests and tools.
#include <cstring>
#include <string>

#include "../../include/kkt_symbolic.h"
#include "symbolic.h"

namespace {
thread_local std::string g_err;

struct Inspect {
  int32_t N = 0;
  kkt::Symbolic S;
  kkt::Coupling C;
  std::vector<int32_t> panel_rend, jlo, jhi;
};

template <class T>
int64_t copy_out(const std::vector<T>& v, int64_t* out) {
  if (out)
    for (size_t i = 0; i < v.size(); i++) out[i] = (int64_t)v[i];
  return (int64_t)v.size();
}
}  // namespace

extern "C" {

kkt_symbolic* kkt_symbolic_create(int32_t nA, int32_t nP, const int32_t* a_rowptr, const int32_t* a_col,
                                  const double* a_vals_hint, int32_t N, int32_t nC,
                                  const int32_t* b_blockptr, const int32_t* b_row, const int32_t* b_col,
                                  int32_t c_kind) {
  Inspect* in = new Inspect();
  in->N = N;
  std::string e = kkt::analyze_pattern(nA, nP, a_rowptr, a_col, a_vals_hint, a_vals_hint ? 1 : 0, in->S);
  if (e.empty()) e = kkt::analyze_coupling(in->S, N, nC, b_blockptr, b_row, b_col, in->C);
  if (!e.empty()) {
    g_err = e;
    delete in;
    return nullptr;
  }
  kkt::s_envelope(in->C, c_kind, 64, in->panel_rend, in->jlo, in->jhi);
  kkt::choose_tail(in->S, N, kkt::kTailMaxBytes, kkt::kTailMinCols);
  return reinterpret_cast<kkt_symbolic*>(in);
}

int64_t kkt_symbolic_get(const kkt_symbolic* sym, const char* name, int64_t* out) {
  const Inspect* in = reinterpret_cast<const Inspect*>(sym);
  if (!in || !name) return -1;
  const kkt::Symbolic& S = in->S;
  const kkt::Coupling& C = in->C;
  const std::string n(name);
  if (n == "perm") return copy_out(S.perm, out);
  if (n == "partner") return copy_out(S.partner, out);
  if (n == "sn_first") return copy_out(S.sn_first, out);
  if (n == "sn_rowptr") return copy_out(S.sn_rowptr, out);
  if (n == "sn_rows") return copy_out(S.sn_rows, out);
  if (n == "sn_valoff") return copy_out(S.sn_valoff, out);
  if (n == "sn_parent") return copy_out(S.sn_parent, out);
  if (n == "sn_level") return copy_out(S.sn_level, out);
  if (n == "a_map") return copy_out(S.a_map, out);
  if (n == "upd_ptr") return copy_out(S.upd_ptr, out);
  if (n == "upd_src") return copy_out(S.upd_src, out);
  if (n == "upd_r0") return copy_out(S.upd_r0, out);
  if (n == "upd_r1") return copy_out(S.upd_r1, out);
  if (n == "upd_reloff") return copy_out(S.upd_reloff, out);
  if (n == "upd_rel") return copy_out(S.upd_rel, out);
  if (n == "E") return copy_out(C.E, out);
  if (n == "e_t") return copy_out(C.e_t, out);
  if (n == "wpos") return copy_out(C.wpos, out);
  if (n == "sn_wrow") return copy_out(C.sn_wrow, out);
  if (n == "s_key") return copy_out(C.s_key, out);
  if (n == "panel_rend") return copy_out(in->panel_rend, out);
  if (n == "jlo") return copy_out(in->jlo, out);
  if (n == "jhi") return copy_out(in->jhi, out);
  if (n == "colcount") return copy_out(S.colcount, out);
  if (n == "wt_ptr") return copy_out(C.wt_ptr, out);
  if (n == "wt_idx") return copy_out(C.wt_idx, out);
  if (n == "upd_ntail") return copy_out(S.upd_ntail, out);
  if (n == "tail_wrow") {
    std::vector<int32_t> tw;
    kkt::tail_w_rows(S, C, tw);
    return copy_out(tw, out);
  }
  if (n == "stats") {
    std::vector<int32_t> tw;
    const int32_t nw_before = kkt::tail_w_rows(S, C, tw);
    std::vector<int64_t> st = {S.n, S.nsuper, S.nlevels, S.panel_total, S.nnzL,
                               C.k, C.nw,     S.tail_sn, S.tail_col,    nw_before};
    return copy_out(st, out);
  }
  return -1;
}

int32_t kkt_symbolic_choose_tail(kkt_symbolic* sym, double ratio, int64_t max_bytes) {
  Inspect* in = reinterpret_cast<Inspect*>(sym);
  if (!in || !(ratio > 0.0)) return -1;
  kkt::choose_tail(in->S, in->N, max_bytes, kkt::kTailMinCols, ratio);
  return in->S.n - in->S.tail_col;
}

void kkt_symbolic_destroy(kkt_symbolic* sym) { delete reinterpret_cast<Inspect*>(sym); }

const char* kkt_symbolic_error(void) { return g_err.c_str(); }

}  // extern "C"
