// Host-side symbolic analysis of the shared block pattern (internal header).
//
// The N diagonal blocks A_i of the arrowhead system share one sparsity
// pattern (Sec. 4.1, eq. hessianPerm: every period has the same network), so
// the ordering, elimination tree, supernode partition and every index map
// below are computed once and reused by all N numeric factorizations.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace kkt {

// Supernodes never exceed this many columns, so a whole panel column block
// fits the shared-memory tiles of the factor kernels.
constexpr int kMaxSnWidth = 32;

// Dense tail limits: at least this many columns, and at most this many bytes
// for the N dense triangles held at once.  A tail whose updates run in FP64 on
// the CUDA cores gains nothing from growing past the supernodal work it
// replaces (both run at the FP64 rate), so its cap is smaller; a tail updated
// on the tensor cores may take the whole dense top of a large grid's tree.
constexpr int32_t kTailMinCols = 16;
constexpr int64_t kTailMaxBytes = int64_t(24) << 30;    // FP64 CUDA-core tail
constexpr int64_t kTailMaxBytesTC = int64_t(96) << 30;  // emulated-FP64 tensor-core tail

struct Symbolic {
  int32_t n = 0;   // block size nA
  int32_t nP = 0;  // primal rows come first
  std::vector<int32_t> perm;   // perm[k] = original row eliminated k-th
  std::vector<int32_t> iperm;  // inverse
  std::vector<int32_t> partner;  // per original multiplier row: its pivot partner (or -1)

  // supernodes (columns in elimination order)
  int32_t nsuper = 0;
  std::vector<int32_t> sn_first;    // nsuper+1; columns [sn_first[s], sn_first[s+1])
  std::vector<int64_t> sn_rowptr;   // nsuper+1; rows of s in sn_rows[...]
  std::vector<int32_t> sn_rows;     // sorted; the first w_s rows are s's own columns
  std::vector<int64_t> sn_valoff;   // nsuper+1; panel offsets (column-major m_s x w_s)
  std::vector<int32_t> sn_parent;   // supernodal elimination tree (-1 = root)
  std::vector<int32_t> sn_level;    // height above the leaves
  std::vector<int32_t> col_sn;      // column -> supernode
  int64_t panel_total = 0;          // doubles per block
  int32_t nlevels = 0;

  // numeric assembly: each entry of the caller's lower CSR -> panel position
  std::vector<int64_t> a_map;       // nnzA

  // left-looking update lists: for supernode s, updates from descendants d
  // upd_ptr[s]..upd_ptr[s+1] index upd_*; each record names d and the
  // first row position (within d's row list) that falls into s's columns.
  std::vector<int64_t> upd_ptr;
  std::vector<int32_t> upd_src;     // d
  std::vector<int32_t> upd_r0;      // first row index (position in d's rows) >= sn_first[s]
  std::vector<int32_t> upd_r1;      // one past the last row position inside s's columns
  // for update u: rows r0..m_d-1 of d map to positions upd_rel[upd_reloff[u] + (i - r0)] in s
  std::vector<int64_t> upd_reloff;
  std::vector<int32_t> upd_rel;
  // supernodes grouped by level (level 0 = leaves)
  std::vector<int32_t> lvl_ptr;
  std::vector<int32_t> lvl_sn;

  // statistics
  int64_t nnzL = 0;       // strictly lower nonzeros of L (exact, no padding)
  double flops = 0;       // factorization flops per block
  std::vector<int32_t> colcount;  // per column: strictly lower nonzeros of L

  // dense tail: columns [tail_col, n), the supernodes tail_sn .. nsuper-1.  A
  // suffix of the postorder is closed under the elimination-tree parent, so
  // every row of a tail supernode is a tail column and the tail is one dense
  // lower triangle per block.  tail_sn == nsuper when there is none.
  int32_t tail_sn = 0, tail_col = 0;
  std::vector<int32_t> upd_ntail;  // per supernode: its leading updates from non-tail descendants
};

// Picks the dense tail: the longest suffix of supernodes whose dense factor
// costs at most `ratio` times the exact sparse flops of its columns, has at
// least min_cols columns, and whose N dense triangles (nT^2 doubles each) fit
// max_bytes.  Fills tail_sn, tail_col and upd_ntail.
constexpr double kTailRatio = 1.5;
void choose_tail(Symbolic& S, int32_t N, int64_t max_bytes, int32_t min_cols, double ratio = kTailRatio);

// Coupling analysis: B_i (COO per block) against the block factor.
// With E the sorted union of the rows that carry a nonzero of some B_i
// (k = |E| rows), B_i = E M_i and
//   B_i^T A_i^{-1} B_i = M_i^T (E^T A_i^{-1} E) M_i = M_i^T G_i M_i,
//   G_i = W_i^T D_i^{-1} W_i,   W_i = L_i^{-1} P^T E.
// W_i is nonzero only on the elimination-tree reach of E, so it is stored
// for the reach supernodes only (nw rows x k columns).
struct Coupling {
  int32_t N = 0, nC = 0, k = 0;
  int64_t nnzB = 0;
  std::vector<int32_t> E;            // k original row indices
  std::vector<int32_t> e_t;          // per B entry: its index t in E
  std::vector<int32_t> e_block;      // per B entry: its block
  std::vector<int32_t> wpos;         // per t: W row holding the unit right-hand side
  std::vector<int32_t> sn_wrow;      // per supernode: first W row (-1 = outside the reach)
  int32_t nw = 0;                    // W rows
  std::vector<int32_t> reach_lvl_ptr;  // reach supernodes grouped by level
  std::vector<int32_t> reach_lvl_sn;
  // lower triangle of sum_i M_i^T G_i M_i, gathered per output entry
  std::vector<int64_t> s_key;        // c1 * nC + c2 (c1 >= c2), sorted
  std::vector<int64_t> s_ptr;        // records of entry q: s_ptr[q]..s_ptr[q+1]
  std::vector<int32_t> s_e1, s_e2;   // B entry pair of each record (same block)
  // t = r_g - sum_i M_i^T u_i, gathered per coupling column
  std::vector<int32_t> t_ptr;        // nC + 1
  std::vector<int32_t> t_e;          // B entries of that column, block order
  // v_i = M_i x_g: B entries of block i with index t lie in bt_ptr[i*(k+1)+t] ..
  std::vector<int32_t> bt_ptr;       // N * (k + 1)
  // Column t of W is L^{-1} P^T e_{E_t}: nonzero only on the supernodes of
  // the elimination-tree path from E_t's supernode to the root.  Per supernode
  // the columns whose path it is on, sorted (empty outside the reach).
  std::vector<int32_t> wt_ptr;       // nsuper + 1
  std::vector<int32_t> wt_idx;
};

// Gather lists of the contraction G = W^T D^{-1} W over the W rows of the
// supernodes before `tail_sn`, by structure: entry (t1 >= t2) collects the
// rows whose supernode has both t1 and t2 among its columns.  Keys t1 * k + t2
// sorted; rows ascending per key.
void g_gather(const Symbolic& S, const Coupling& C, int32_t tail_sn, std::vector<int32_t>& g_key,
              std::vector<int64_t>& g_ptr, std::vector<int32_t>& g_row);

// s_records = false leaves the gather records of S empty (the structured S of
// the cumulative coupling does without them).
std::string analyze_coupling(const Symbolic& S, int32_t N, int32_t nC, const int32_t* b_blockptr,
                             const int32_t* b_row, const int32_t* b_col, Coupling& out,
                             bool s_records = true);

// Row envelope of S = C - sum_i M_i^T G_i M_i (the structured factor): for each
// 64-wide panel p, one past the last row that can be nonzero in its columns
// (panel_rend), and per 64-row block the first / one-past-last block of the
// triangular solves (jlo, jhi).  LDL^T without pivoting keeps the envelope.
void s_envelope(const Coupling& C, int32_t c_kind, int32_t block, std::vector<int32_t>& panel_rend,
                std::vector<int32_t>& jlo, std::vector<int32_t>& jhi);

// W rows of the tail: per tail column, its W row (-1 outside the reach of E).
// W rows are numbered in supernode order, so the tail's come after all others;
// returns the number of W rows outside the tail.
int32_t tail_w_rows(const Symbolic& S, const Coupling& C, std::vector<int32_t>& wrow_of_tail_col);

// Returns an empty string on success, else a description of the problem.
std::string analyze_pattern(int32_t n, int32_t nP, const int32_t* rowptr, const int32_t* col,
                            const double* vals_hint, int32_t hint_blocks, Symbolic& out);

}  // namespace kkt
