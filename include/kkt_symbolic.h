/*
 * kkt_symbolic.h -- host-only inspection of the symbolic analysis that
 * kkt_analyze performs (no CUDA needed): ordering, elimination tree,
 * supernodes, update maps, reach of B's rows and envelope of S.  Used by the
 * CPU tests of the host logic; the solver itself does not need it.
 */
#ifndef KKT_SYMBOLIC_H
#define KKT_SYMBOLIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kkt_symbolic kkt_symbolic;

/* Runs the analysis of kkt_analyze on a pattern (arguments as in kkt_pattern;
 * host arrays, read during the call).  NULL on a malformed pattern, with the
 * reason in kkt_symbolic_error(). */
kkt_symbolic* kkt_symbolic_create(int32_t nA, int32_t nP, const int32_t* a_rowptr, const int32_t* a_col,
                                  const double* a_vals_hint, int32_t N, int32_t nC,
                                  const int32_t* b_blockptr, const int32_t* b_row, const int32_t* b_col,
                                  int32_t c_kind);

/* Copies the named array as int64 into out (may be NULL to query the length)
 * and returns its length, or -1 for an unknown name.  Names: perm, partner,
 * sn_first, sn_rowptr, sn_rows, sn_valoff, sn_parent, sn_level, a_map, upd_ptr,
 * upd_src, upd_r0, upd_r1, upd_reloff, upd_rel, E, e_t, wpos, sn_wrow, s_key,
 * panel_rend, jlo, jhi, colcount, upd_ntail, stats (n, nsuper, nlevels,
 * panel_total, nnzL, k, nw, tail_sn, tail_col, nw_before_tail), tail_wrow
 * (per tail column its W row, -1 outside the reach), wt_ptr / wt_idx (per
 * supernode the columns of W that are nonzero on it).  The dense tail is
 * chosen as kkt_analyze chooses it with the dense_tail option on. */
int64_t kkt_symbolic_get(const kkt_symbolic* sym, const char* name, int64_t* out);

/* Re-chooses the dense tail with cost ratio `ratio` and the byte cap
 * `max_bytes` for the N triangles (kkt_analyze uses 24 GiB for the FP64
 * CUDA-core tail and 96 GiB for the tensor-core tail; the default ratio is
 * 1.5), as kkt_analyze's option tail_ratio does; later kkt_symbolic_get calls
 * see the new tail.  Returns its number of columns, or -1 for a NULL handle or
 * a ratio <= 0. */
int32_t kkt_symbolic_choose_tail(kkt_symbolic* sym, double ratio, int64_t max_bytes);

void kkt_symbolic_destroy(kkt_symbolic* sym);

const char* kkt_symbolic_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KKT_SYMBOLIC_H */
