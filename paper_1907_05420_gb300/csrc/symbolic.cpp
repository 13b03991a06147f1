// Symbolic analysis of the shared pattern of the blocks A_i.
//
// Every IPM iteration factors A_i = L_i D_i L_i^T (Algorithm 1) on
// one unchanging pattern, so the ordering, elimination tree, supernodes and
// every index map are built here once per pattern.
//
// Ordering.  A_i = [H_i J_i^T; J_i -delta I] is quasidefinite, so any
// symmetric order admits 1x1 pivots in exact arithmetic.  In FP64 a
// multiplier row used as a pivot before its dominant primal neighbour has
// been eliminated contributes a pivot of size ~delta and growth ~1/delta.
// Each multiplier is therefore paired with its partner: the primal neighbour
// with the largest |coupling| in the value hint.  Partner and multipliers are
// contracted into one node, the contracted graph is ordered by weighted
// minimum degree, and the expansion puts the partner right before its
// multipliers.  The multiplier pivot is then -delta - a_p^2/h_p - ..., and an
// update through it is bounded by h_p (a_max / a_p)^2 <= ||A||.
#include "symbolic.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <queue>
#include <utility>

namespace kkt {
namespace {

struct Graph {
  int32_t n = 0;
  std::vector<std::vector<int32_t>> adj;  // sorted, no self loops
  std::vector<int64_t> weight;
};

// Weighted minimum degree on an explicit elimination graph.  The degree of a
// node is the total weight (number of variables) of its current neighbours.
// Lazy heap: stale entries are skipped when popped.
//
// A node's neighbours are a sorted list while few and a bitset once the list
// would take more bits than the bitset (dense rows near the top of the tree):
// merging the eliminated node's neighbours into a bitset is a pass over the
// words they span, and its degree is updated by the weights of the
// neighbours it gains.  Both forms give the same sets and degrees, so the
// order is that of plain sorted-list merges.
//
// Once the node taken is adjacent to every remaining node, its elimination
// leaves a clique.  In a clique of total weight W a node's degree is W - w(v),
// and each later elimination lowers all of them by the same amount, so the
// heap would take the rest by decreasing weight, ties by node number; that
// order is appended directly instead of eliminating the clique node by node
// (whose merges cost the cube of its size).
std::vector<int32_t> weighted_min_degree(Graph& g) {
  const int32_t n = g.n;
  const int32_t words = (n + 63) / 64;
  const size_t dense_at = std::max<size_t>(64, (size_t)n / 32);
  std::vector<std::vector<uint64_t>> bits(n);  // empty: the sorted list g.adj[v] holds v's neighbours
  std::vector<int64_t> deg(n, 0);
  for (int32_t v = 0; v < n; v++)
    for (int32_t u : g.adj[v]) deg[v] += g.weight[u];
  using Key = std::pair<std::pair<int64_t, int64_t>, int32_t>;  // (deg, weight), node
  std::priority_queue<Key, std::vector<Key>, std::greater<Key>> heap;
  for (int32_t v = 0; v < n; v++) heap.push({{deg[v], g.weight[v]}, v});
  std::vector<char> gone(n, 0);
  std::vector<int32_t> order;
  order.reserve(n);
  std::vector<int32_t> merged, np;
  std::vector<uint64_t> npbits(words, 0);
  int32_t remaining = n;
  while (!heap.empty()) {
    Key top = heap.top();
    heap.pop();
    int32_t p = top.second;
    if (gone[p] || top.first.first != deg[p]) continue;
    gone[p] = 1;
    order.push_back(p);
    remaining--;
    // p's neighbours, ascending
    np.clear();
    if (bits[p].empty()) {
      np.swap(g.adj[p]);
    } else {
      for (int32_t w = 0; w < words; w++)
        for (uint64_t m = bits[p][w]; m; m &= m - 1) np.push_back(w * 64 + __builtin_ctzll(m));
      std::vector<uint64_t>().swap(bits[p]);
    }
    if ((int32_t)np.size() == remaining) {
      // p is adjacent to all remaining nodes: they form a clique after it
      std::sort(np.begin(), np.end(), [&](int32_t a, int32_t b) {
        return g.weight[a] != g.weight[b] ? g.weight[a] > g.weight[b] : a < b;
      });
      order.insert(order.end(), np.begin(), np.end());
      break;
    }
    if (np.empty()) continue;
    for (int32_t x : np) npbits[x >> 6] |= 1ull << (x & 63);
    const int32_t w0 = np.front() >> 6, w1 = np.back() >> 6;
    for (int32_t u : np) {
      // neighbours of u <- (neighbours of u U np) \ {u, p}, and their weight
      int64_t d;
      if (bits[u].empty()) {
        std::vector<int32_t>& au = g.adj[u];
        merged.clear();
        merged.reserve(au.size() + np.size());
        d = 0;
        size_t a = 0, b = 0;
        while (a < au.size() || b < np.size()) {
          int32_t x;
          if (b >= np.size() || (a < au.size() && au[a] < np[b])) x = au[a++];
          else if (a >= au.size() || np[b] < au[a]) x = np[b++];
          else { x = au[a++]; b++; }
          if (x == u || x == p) continue;
          merged.push_back(x);
          d += g.weight[x];
        }
        au.swap(merged);
        if (au.size() > dense_at) {  // switch u to a bitset
          bits[u].assign(words, 0);
          for (int32_t x : au) bits[u][x >> 6] |= 1ull << (x & 63);
          std::vector<int32_t>().swap(au);
        }
      } else {
        uint64_t* bu = bits[u].data();
        d = deg[u] - g.weight[p];  // p was a neighbour of u
        bu[p >> 6] &= ~(1ull << (p & 63));
        for (int32_t w = w0; w <= w1; w++) {
          uint64_t add = npbits[w] & ~bu[w];
          if (w == (u >> 6)) add &= ~(1ull << (u & 63));
          if (!add) continue;
          bu[w] |= add;
          for (uint64_t m = add; m; m &= m - 1) d += g.weight[w * 64 + __builtin_ctzll(m)];
        }
      }
      deg[u] = d;
      heap.push({{d, g.weight[u]}, u});
    }
    for (int32_t x : np) npbits[x >> 6] = 0;
  }
  return order;
}

// Upper pattern of P A P^T by columns: for column k, rows i < k.
void permuted_upper(int32_t n, const int32_t* rowptr, const int32_t* col,
                    const std::vector<int32_t>& iperm, std::vector<int64_t>& ptr,
                    std::vector<int32_t>& rows) {
  ptr.assign(n + 1, 0);
  for (int32_t r = 0; r < n; r++)
    for (int32_t p = rowptr[r]; p < rowptr[r + 1]; p++) {
      int32_t a = iperm[r], b = iperm[col[p]];
      if (a != b) ptr[std::max(a, b) + 1]++;
    }
  for (int32_t k = 0; k < n; k++) ptr[k + 1] += ptr[k];
  rows.assign(ptr[n], 0);
  std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
  for (int32_t r = 0; r < n; r++)
    for (int32_t p = rowptr[r]; p < rowptr[r + 1]; p++) {
      int32_t a = iperm[r], b = iperm[col[p]];
      if (a != b) rows[fill[std::max(a, b)]++] = std::min(a, b);
    }
}

// Elimination tree by path compression over virtual ancestors.
std::vector<int32_t> etree(int32_t n, const std::vector<int64_t>& ptr,
                           const std::vector<int32_t>& rows) {
  std::vector<int32_t> parent(n, -1), anc(n, -1);
  for (int32_t k = 0; k < n; k++) {
    for (int64_t p = ptr[k]; p < ptr[k + 1]; p++) {
      int32_t i = rows[p];
      while (i != -1 && i < k) {
        int32_t next = anc[i];
        anc[i] = k;
        if (next == -1) {
          parent[i] = k;
          break;
        }
        i = next;
      }
    }
  }
  return parent;
}

std::vector<int32_t> postorder(int32_t n, const std::vector<int32_t>& parent) {
  std::vector<int32_t> head(n, -1), next(n, -1), post;
  post.reserve(n);
  for (int32_t j = n - 1; j >= 0; j--) {
    if (parent[j] >= 0) {
      next[j] = head[parent[j]];
      head[parent[j]] = j;
    }
  }
  std::vector<int32_t> stack;
  for (int32_t r = 0; r < n; r++) {
    if (parent[r] != -1) continue;
    stack.push_back(r);
    while (!stack.empty()) {
      int32_t v = stack.back();
      int32_t c = head[v];
      if (c == -1) {
        stack.pop_back();
        post.push_back(v);
      } else {
        head[v] = next[c];
        stack.push_back(c);
      }
    }
  }
  return post;
}

}  // namespace

std::string analyze_pattern(int32_t n, int32_t nP, const int32_t* rowptr, const int32_t* col,
                            const double* vals_hint, int32_t hint_blocks, Symbolic& S) {
  S = Symbolic();
  S.n = n;
  S.nP = nP;
  if (n <= 0) return "nA must be positive";
  if (nP < 0 || nP > n) return "nP must lie in [0, nA]";
  if (rowptr[0] != 0) return "a_rowptr[0] must be 0";
  for (int32_t r = 0; r < n; r++) {
    if (rowptr[r + 1] <= rowptr[r]) return "every row of A needs its diagonal entry";
    for (int32_t p = rowptr[r]; p < rowptr[r + 1]; p++) {
      if (col[p] < 0 || col[p] > r) return "a_col must hold lower-triangle columns in [0,row]";
      if (p > rowptr[r] && col[p] <= col[p - 1]) return "a_col must be strictly increasing per row";
    }
    if (col[rowptr[r + 1] - 1] != r) return "every row of A needs its diagonal entry";
  }
  const int64_t nnz = rowptr[n];

  // --- partners: each multiplier row pairs with its dominant primal neighbour
  std::vector<int32_t> deg(n, 0);
  for (int32_t r = 0; r < n; r++)
    for (int32_t p = rowptr[r]; p < rowptr[r + 1]; p++)
      if (col[p] != r) {
        deg[r]++;
        deg[col[p]]++;
      }
  S.partner.assign(n, -1);
  for (int32_t r = nP; r < n; r++) {
    double best = -1.0;
    int32_t bc = -1;
    for (int32_t p = rowptr[r]; p < rowptr[r + 1]; p++) {
      int32_t c = col[p];
      if (c >= nP) continue;
      double w;
      if (vals_hint) {
        w = 0.0;
        for (int32_t b = 0; b < hint_blocks; b++) w = std::max(w, std::fabs(vals_hint[(int64_t)b * nnz + p]));
      } else {
        w = (double)deg[c];  // structural fallback: best-connected primal neighbour
      }
      if (w > best) {
        best = w;
        bc = c;
      }
    }
    S.partner[r] = bc;
  }

  // --- contracted graph
  std::vector<int32_t> gid(n, -1);
  int32_t ng = 0;
  for (int32_t v = 0; v < nP; v++) gid[v] = ng++;
  for (int32_t r = nP; r < n; r++) gid[r] = S.partner[r] >= 0 ? gid[S.partner[r]] : ng++;
  Graph g;
  g.n = ng;
  g.adj.assign(ng, {});
  g.weight.assign(ng, 0);
  for (int32_t v = 0; v < n; v++) g.weight[gid[v]]++;
  for (int32_t r = 0; r < n; r++)
    for (int32_t p = rowptr[r]; p < rowptr[r + 1]; p++) {
      int32_t a = gid[r], b = gid[col[p]];
      if (a == b) continue;
      g.adj[a].push_back(b);
      g.adj[b].push_back(a);
    }
  for (auto& a : g.adj) {
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
  }
  std::vector<int32_t> gorder = weighted_min_degree(g);
  std::vector<std::vector<int32_t>> members(ng);
  for (int32_t v = 0; v < n; v++) members[gid[v]].push_back(v);  // primal (partner) first
  std::vector<int32_t> perm0;
  perm0.reserve(n);
  for (int32_t gg : gorder)
    for (int32_t v : members[gg]) perm0.push_back(v);

  // --- elimination tree, postorder, final permutation
  std::vector<int32_t> iperm0(n);
  for (int32_t k = 0; k < n; k++) iperm0[perm0[k]] = k;
  std::vector<int64_t> uptr;
  std::vector<int32_t> urows;
  permuted_upper(n, rowptr, col, iperm0, uptr, urows);
  std::vector<int32_t> par0 = etree(n, uptr, urows);
  std::vector<int32_t> post = postorder(n, par0);
  S.perm.resize(n);
  S.iperm.resize(n);
  for (int32_t k = 0; k < n; k++) S.perm[k] = perm0[post[k]];
  for (int32_t k = 0; k < n; k++) S.iperm[S.perm[k]] = k;
  permuted_upper(n, rowptr, col, S.iperm, uptr, urows);
  std::vector<int32_t> parent = etree(n, uptr, urows);

  // --- column counts (strictly lower) by row-subtree traversal
  std::vector<int32_t> cnt(n, 0), mark(n, -1), nchild(n, 0);
  for (int32_t k = 0; k < n; k++) {
    mark[k] = k;
    for (int64_t p = uptr[k]; p < uptr[k + 1]; p++) {
      for (int32_t i = urows[p]; mark[i] != k; i = parent[i]) {
        mark[i] = k;
        cnt[i]++;
      }
    }
  }
  for (int32_t j = 0; j < n; j++)
    if (parent[j] >= 0) nchild[parent[j]]++;
  S.nnzL = 0;
  S.flops = 0;
  S.colcount.assign(cnt.begin(), cnt.begin() + n);
  for (int32_t j = 0; j < n; j++) {
    S.nnzL += cnt[j];
    S.flops += (double)cnt[j] * (cnt[j] + 3);  // scale column, rank-1 update of the rest
  }

  // --- fundamental supernodes, then relaxed amalgamation, then width cap
  std::vector<int32_t> first;
  for (int32_t j = 0; j < n; j++) {
    bool join = j > 0 && parent[j - 1] == j && cnt[j - 1] == cnt[j] + 1 && nchild[j] == 1;
    if (!join) first.push_back(j);
  }
  first.push_back(n);
  // merge a supernode into its parent when contiguous and cheap in zeros
  {
    int32_t ns = (int32_t)first.size() - 1;
    std::vector<int32_t> sf(first.begin(), first.end() - 1), sl(first.begin() + 1, first.end());
    std::vector<int64_t> m(ns);   // rows of the supernode (incl. own columns)
    std::vector<int64_t> zeros(ns, 0);
    std::vector<int32_t> cs(n);
    for (int32_t s = 0; s < ns; s++) {
      m[s] = (int64_t)(sl[s] - sf[s]) + cnt[sl[s] - 1];
      for (int32_t j = sf[s]; j < sl[s]; j++) cs[j] = s;
    }
    std::vector<int32_t> alive(ns, 1);
    // walk from the top: merging child c (ends right before s) into s
    for (int32_t s = ns - 1; s >= 0; s--) {
      if (!alive[s]) continue;
      while (sf[s] > 0) {
        int32_t c = cs[sf[s] - 1];
        if (!alive[c]) break;
        int32_t lastc = sl[c] - 1;
        if (parent[lastc] != sf[s]) break;  // c is not a child of s
        int64_t wc = sl[c] - sf[c], ws = sl[s] - sf[s];
        if (wc + ws > kMaxSnWidth) break;
        // merged panel: (wc + m_s) rows x (wc + ws) columns, lower part only
        auto tri = [](int64_t w, int64_t mm) { return w * mm - w * (w - 1) / 2; };
        int64_t before = tri(wc, m[c]) + tri(ws, m[s]);
        int64_t after = tri(wc + ws, wc + m[s]);
        int64_t z = zeros[c] + zeros[s] + (after - before);
        bool ok = (wc + ws <= 4) || z <= (int64_t)(0.15 * (double)after);
        if (!ok) break;
        zeros[s] = z;
        m[s] = wc + m[s];
        sf[s] = sf[c];
        for (int32_t j = sf[c]; j < sl[c]; j++) cs[j] = s;
        alive[c] = 0;
      }
    }
    first.clear();
    for (int32_t s = 0; s < ns; s++)
      if (alive[s]) {
        int32_t w = sl[s] - sf[s];
        for (int32_t j = sf[s]; j < sl[s]; j += kMaxSnWidth) first.push_back(j);
        (void)w;
      }
    first.push_back(n);
  }
  S.nsuper = (int32_t)first.size() - 1;
  S.sn_first = first;
  S.col_sn.assign(n, 0);
  for (int32_t s = 0; s < S.nsuper; s++)
    for (int32_t j = first[s]; j < first[s + 1]; j++) S.col_sn[j] = s;

  // --- supernode parents and row structures (bottom-up unions)
  S.sn_parent.assign(S.nsuper, -1);
  for (int32_t s = 0; s < S.nsuper; s++) {
    int32_t last = first[s + 1] - 1;
    S.sn_parent[s] = parent[last] >= 0 ? S.col_sn[parent[last]] : -1;
  }
  std::vector<std::vector<int32_t>> rows(S.nsuper);
  std::vector<std::vector<int32_t>> kids(S.nsuper);
  for (int32_t s = 0; s < S.nsuper; s++)
    if (S.sn_parent[s] >= 0) kids[S.sn_parent[s]].push_back(s);
  // lower pattern by columns of P A P^T: for column j, rows i > j
  std::vector<std::vector<int32_t>> lcols(n);
  for (int32_t k = 0; k < n; k++)
    for (int64_t p = uptr[k]; p < uptr[k + 1]; p++) lcols[urows[p]].push_back(k);
  std::vector<int32_t> stamp(n, -1);
  for (int32_t s = 0; s < S.nsuper; s++) {  // children precede parents (postorder)
    int32_t f = first[s], l = first[s + 1];
    std::vector<int32_t>& R = rows[s];
    for (int32_t j = f; j < l; j++) {
      R.push_back(j);
      stamp[j] = s;
    }
    for (int32_t j = f; j < l; j++)
      for (int32_t i : lcols[j])
        if (i >= l && stamp[i] != s) {
          stamp[i] = s;
          R.push_back(i);
        }
    for (int32_t c : kids[s])
      for (int32_t i : rows[c])
        if (i >= l && stamp[i] != s) {
          stamp[i] = s;
          R.push_back(i);
        }
    std::sort(R.begin() + (l - f), R.end());
  }
  S.sn_rowptr.assign(S.nsuper + 1, 0);
  S.sn_valoff.assign(S.nsuper + 1, 0);
  for (int32_t s = 0; s < S.nsuper; s++) {
    int64_t m = (int64_t)rows[s].size(), w = first[s + 1] - first[s];
    S.sn_rowptr[s + 1] = S.sn_rowptr[s] + m;
    S.sn_valoff[s + 1] = S.sn_valoff[s] + m * w;
  }
  S.panel_total = S.sn_valoff[S.nsuper];
  S.sn_rows.resize(S.sn_rowptr[S.nsuper]);
  for (int32_t s = 0; s < S.nsuper; s++)
    std::copy(rows[s].begin(), rows[s].end(), S.sn_rows.begin() + S.sn_rowptr[s]);

  // --- levels
  S.sn_level.assign(S.nsuper, 0);
  S.nlevels = 0;
  for (int32_t s = 0; s < S.nsuper; s++) {
    if (S.sn_parent[s] >= 0)
      S.sn_level[S.sn_parent[s]] = std::max(S.sn_level[S.sn_parent[s]], S.sn_level[s] + 1);
    S.nlevels = std::max(S.nlevels, S.sn_level[s] + 1);
  }

  // --- map of the caller's lower CSR into the panels
  S.a_map.assign(nnz, -1);
  for (int32_t r = 0; r < n; r++)
    for (int32_t p = rowptr[r]; p < rowptr[r + 1]; p++) {
      int32_t a = S.iperm[r], b = S.iperm[col[p]];
      int32_t j = std::min(a, b), i = std::max(a, b);
      int32_t s = S.col_sn[j];
      const int32_t* R = S.sn_rows.data() + S.sn_rowptr[s];
      int64_t m = S.sn_rowptr[s + 1] - S.sn_rowptr[s];
      const int32_t* it = std::lower_bound(R, R + m, i);
      if (it == R + m || *it != i) return "internal: entry missing from supernode structure";
      S.a_map[p] = S.sn_valoff[s] + (int64_t)(j - first[s]) * m + (it - R);
    }

  // --- left-looking update lists
  std::vector<std::vector<int32_t>> ud(S.nsuper), u0(S.nsuper), u1(S.nsuper);
  for (int32_t d = 0; d < S.nsuper; d++) {
    int64_t m = S.sn_rowptr[d + 1] - S.sn_rowptr[d];
    const int32_t* R = S.sn_rows.data() + S.sn_rowptr[d];
    int32_t w = first[d + 1] - first[d];
    int64_t q = w;
    while (q < m) {
      int32_t s = S.col_sn[R[q]];
      int64_t q1 = q;
      while (q1 < m && R[q1] < first[s + 1]) q1++;
      ud[s].push_back(d);
      u0[s].push_back((int32_t)q);
      u1[s].push_back((int32_t)q1);
      q = q1;
    }
  }
  S.upd_ptr.assign(S.nsuper + 1, 0);
  for (int32_t s = 0; s < S.nsuper; s++) S.upd_ptr[s + 1] = S.upd_ptr[s] + (int64_t)ud[s].size();
  S.upd_src.reserve(S.upd_ptr[S.nsuper]);
  for (int32_t s = 0; s < S.nsuper; s++) {
    S.upd_src.insert(S.upd_src.end(), ud[s].begin(), ud[s].end());
    S.upd_r0.insert(S.upd_r0.end(), u0[s].begin(), u0[s].end());
    S.upd_r1.insert(S.upd_r1.end(), u1[s].begin(), u1[s].end());
  }
  // relative row positions of each update inside its target
  const int64_t nupd = S.upd_ptr[S.nsuper];
  S.upd_reloff.assign(nupd + 1, 0);
  for (int32_t s = 0; s < S.nsuper; s++)
    for (int64_t u = S.upd_ptr[s]; u < S.upd_ptr[s + 1]; u++) {
      int32_t d = S.upd_src[u];
      int64_t md = S.sn_rowptr[d + 1] - S.sn_rowptr[d];
      S.upd_reloff[u + 1] = S.upd_reloff[u] + (md - S.upd_r0[u]);
    }
  S.upd_rel.resize(S.upd_reloff[nupd]);
  for (int32_t s = 0; s < S.nsuper; s++) {
    const int32_t* Rs = S.sn_rows.data() + S.sn_rowptr[s];
    int64_t ms = S.sn_rowptr[s + 1] - S.sn_rowptr[s];
    for (int64_t u = S.upd_ptr[s]; u < S.upd_ptr[s + 1]; u++) {
      int32_t d = S.upd_src[u];
      const int32_t* Rd = S.sn_rows.data() + S.sn_rowptr[d];
      int64_t md = S.sn_rowptr[d + 1] - S.sn_rowptr[d];
      int64_t pos = 0;
      for (int64_t i = S.upd_r0[u]; i < md; i++) {
        while (pos < ms && Rs[pos] < Rd[i]) pos++;
        if (pos >= ms || Rs[pos] != Rd[i]) return "internal: update row missing from target structure";
        S.upd_rel[S.upd_reloff[u] + (i - S.upd_r0[u])] = (int32_t)pos;
      }
    }
  }
  // level lists
  S.lvl_ptr.assign(S.nlevels + 1, 0);
  for (int32_t s = 0; s < S.nsuper; s++) S.lvl_ptr[S.sn_level[s] + 1]++;
  for (int32_t l = 0; l < S.nlevels; l++) S.lvl_ptr[l + 1] += S.lvl_ptr[l];
  S.lvl_sn.resize(S.nsuper);
  {
    std::vector<int32_t> fill(S.lvl_ptr.begin(), S.lvl_ptr.end() - 1);
    for (int32_t s = 0; s < S.nsuper; s++) S.lvl_sn[fill[S.sn_level[s]]++] = s;
  }
  return std::string();
}

std::string analyze_coupling(const Symbolic& S, int32_t N, int32_t nC, const int32_t* b_blockptr,
                             const int32_t* b_row, const int32_t* b_col, Coupling& C, bool s_records) {
  C = Coupling();
  C.N = N;
  C.nC = nC;
  if (N <= 0) return "N must be positive";
  if (nC < 0) return "nC must be non-negative";
  if (b_blockptr[0] != 0) return "b_blockptr[0] must be 0";
  for (int32_t i = 0; i < N; i++)
    if (b_blockptr[i + 1] < b_blockptr[i]) return "b_blockptr must be non-decreasing";
  C.nnzB = b_blockptr[N];
  const int32_t n = S.n;
  std::vector<int32_t> tpos(n, -1);
  for (int64_t e = 0; e < C.nnzB; e++) {
    if (b_row[e] < 0 || b_row[e] >= n) return "b_row out of range";
    if (b_col[e] < 0 || b_col[e] >= nC) return "b_col out of range";
    tpos[b_row[e]] = 0;
  }
  for (int32_t i = 0; i < N; i++)
    for (int32_t e = b_blockptr[i] + 1; e < b_blockptr[i + 1]; e++)
      if (b_row[e] < b_row[e - 1] || (b_row[e] == b_row[e - 1] && b_col[e] <= b_col[e - 1]))
        return "B entries must be sorted by (row, col) within a block, without duplicates";
  for (int32_t r = 0; r < n; r++)
    if (tpos[r] == 0) {
      tpos[r] = (int32_t)C.E.size();
      C.E.push_back(r);
    }
  C.k = (int32_t)C.E.size();
  C.e_t.resize(C.nnzB);
  C.e_block.resize(C.nnzB);
  for (int32_t i = 0; i < N; i++)
    for (int32_t e = b_blockptr[i]; e < b_blockptr[i + 1]; e++) {
      C.e_t[e] = tpos[b_row[e]];
      C.e_block[e] = i;
    }
  // reach of E in the supernodal tree
  std::vector<char> in(S.nsuper, 0);
  for (int32_t r : C.E)
    for (int32_t s = S.col_sn[S.iperm[r]]; s >= 0 && !in[s]; s = S.sn_parent[s]) in[s] = 1;
  C.sn_wrow.assign(S.nsuper, -1);
  C.nw = 0;
  for (int32_t s = 0; s < S.nsuper; s++)
    if (in[s]) {
      C.sn_wrow[s] = C.nw;
      C.nw += S.sn_first[s + 1] - S.sn_first[s];
    }
  C.wpos.resize(C.k);
  for (int32_t t = 0; t < C.k; t++) {
    int32_t j = S.iperm[C.E[t]], s = S.col_sn[j];
    C.wpos[t] = C.sn_wrow[s] + (j - S.sn_first[s]);
  }
  // columns of W per supernode: walk each column's path to the root
  {
    std::vector<std::vector<int32_t>> cols(S.nsuper);
    for (int32_t t = 0; t < C.k; t++)
      for (int32_t s = S.col_sn[S.iperm[C.E[t]]]; s >= 0; s = S.sn_parent[s]) cols[s].push_back(t);
    C.wt_ptr.assign(S.nsuper + 1, 0);
    for (int32_t s = 0; s < S.nsuper; s++) C.wt_ptr[s + 1] = C.wt_ptr[s] + (int32_t)cols[s].size();
    C.wt_idx.reserve(C.wt_ptr[S.nsuper]);
    for (int32_t s = 0; s < S.nsuper; s++) C.wt_idx.insert(C.wt_idx.end(), cols[s].begin(), cols[s].end());
  }
  C.reach_lvl_ptr.assign(S.nlevels + 1, 0);
  for (int32_t s = 0; s < S.nsuper; s++)
    if (in[s]) C.reach_lvl_ptr[S.sn_level[s] + 1]++;
  for (int32_t l = 0; l < S.nlevels; l++) C.reach_lvl_ptr[l + 1] += C.reach_lvl_ptr[l];
  C.reach_lvl_sn.resize(C.reach_lvl_ptr[S.nlevels]);
  {
    std::vector<int32_t> fill(C.reach_lvl_ptr.begin(), C.reach_lvl_ptr.end() - 1);
    for (int32_t s = 0; s < S.nsuper; s++)
      if (in[s]) C.reach_lvl_sn[fill[S.sn_level[s]]++] = s;
  }
  // S gather records: pairs of entries of one block, lower triangle
  struct Rec {
    int64_t key;
    int32_t e1, e2;
  };
  std::vector<Rec> recs;
  for (int32_t i = 0; s_records && i < N; i++)
    for (int32_t e1 = b_blockptr[i]; e1 < b_blockptr[i + 1]; e1++)
      for (int32_t e2 = b_blockptr[i]; e2 < b_blockptr[i + 1]; e2++)
        if (b_col[e1] >= b_col[e2]) recs.push_back({(int64_t)b_col[e1] * nC + b_col[e2], e1, e2});
  std::stable_sort(recs.begin(), recs.end(), [](const Rec& a, const Rec& b) { return a.key < b.key; });
  C.s_ptr.push_back(0);
  for (size_t q = 0; q < recs.size(); q++) {
    if (q == 0 || recs[q].key != recs[q - 1].key) {
      if (q) C.s_ptr.push_back((int64_t)q);
      C.s_key.push_back(recs[q].key);
    }
    C.s_e1.push_back(recs[q].e1);
    C.s_e2.push_back(recs[q].e2);
  }
  C.s_ptr.push_back((int64_t)recs.size());
  if (recs.empty()) C.s_ptr.assign(1, 0);
  // t gather: entries per coupling column, block order
  C.t_ptr.assign(nC + 1, 0);
  for (int64_t e = 0; e < C.nnzB; e++) C.t_ptr[b_col[e] + 1]++;
  for (int32_t c = 0; c < nC; c++) C.t_ptr[c + 1] += C.t_ptr[c];
  C.t_e.resize(C.nnzB);
  {
    std::vector<int32_t> fill(C.t_ptr.begin(), C.t_ptr.end() - 1);
    for (int64_t e = 0; e < C.nnzB; e++) C.t_e[fill[b_col[e]]++] = (int32_t)e;
  }
  // entries of block i with index t
  C.bt_ptr.assign((size_t)N * (C.k + 1), 0);
  for (int32_t i = 0; i < N; i++) {
    int32_t* bp = C.bt_ptr.data() + (size_t)i * (C.k + 1);
    int32_t e = b_blockptr[i];
    for (int32_t t = 0; t <= C.k; t++) {
      while (e < b_blockptr[i + 1] && C.e_t[e] < t) e++;
      bp[t] = e;
    }
  }
  return std::string();
}

void s_envelope(const Coupling& C, int32_t c_kind, int32_t block, std::vector<int32_t>& panel_rend,
                std::vector<int32_t>& jlo, std::vector<int32_t>& jhi) {
  const int32_t nC = C.nC, nbk = (nC + block - 1) / block;
  panel_rend.assign(nbk, 0);
  jlo.assign(nbk, 0);
  jhi.assign(nbk, 0);
  if (nC == 0) return;
  std::vector<int32_t> first(nC);
  for (int32_t r = 0; r < nC; r++) first[r] = c_kind == 0 ? r : 0;
  for (int64_t key : C.s_key) {
    const int32_t c1 = (int32_t)(key / nC), c2 = (int32_t)(key % nC);
    first[c1] = std::min(first[c1], c2);
  }
  // last_row[c] = max{r : first[r] <= c}
  std::vector<int32_t> maxrow(nC, -1), last_row(nC, -1);
  for (int32_t r = 0; r < nC; r++) maxrow[first[r]] = std::max(maxrow[first[r]], r);
  int32_t run = -1;
  for (int32_t c = 0; c < nC; c++) {
    run = std::max(run, maxrow[c]);
    last_row[c] = run;
  }
  for (int32_t p = 0; p < nbk; p++) {
    const int32_t cend = std::min(nC, (p + 1) * block);
    panel_rend[p] = std::max(cend, last_row[cend - 1] + 1);
    jhi[p] = (panel_rend[p] + block - 1) / block;
    int32_t fmin = nC;
    for (int32_t r = p * block; r < cend; r++) fmin = std::min(fmin, first[r]);
    jlo[p] = fmin / block;
  }
}

void choose_tail(Symbolic& S, int32_t N, int64_t max_bytes, int32_t min_cols, double ratio) {
  const int32_t n = S.n;
  S.tail_sn = S.nsuper;
  S.tail_col = n;
  double suffix = 0.0;  // exact sparse flops of columns >= sn_first[t]
  for (int32_t t = S.nsuper - 1; t >= 0; t--) {
    for (int32_t j = S.sn_first[t]; j < S.sn_first[t + 1]; j++)
      suffix += (double)S.colcount[j] * (S.colcount[j] + 3);
    const double nT = (double)(n - S.sn_first[t]);
    if (nT < min_cols) continue;
    if ((double)N * nT * nT * 8.0 > (double)max_bytes) break;
    if (nT * nT * nT / 3.0 <= ratio * suffix) {
      S.tail_sn = t;
      S.tail_col = S.sn_first[t];
    }
  }
  S.upd_ntail.assign(S.nsuper, 0);
  for (int32_t s = 0; s < S.nsuper; s++) {
    int32_t c = 0;
    for (int64_t u = S.upd_ptr[s]; u < S.upd_ptr[s + 1]; u++)
      if (S.upd_src[u] < S.tail_sn) c++;  // update lists are in increasing descendant order
    S.upd_ntail[s] = c;
  }
}

int32_t tail_w_rows(const Symbolic& S, const Coupling& C, std::vector<int32_t>& wrow_of_tail_col) {
  const int32_t nT = S.n - S.tail_col;
  wrow_of_tail_col.assign(nT, -1);
  int32_t before = C.nw;
  for (int32_t s = S.tail_sn; s < S.nsuper; s++) {
    if (C.sn_wrow[s] < 0) continue;
    before = std::min(before, C.sn_wrow[s]);
    for (int32_t j = S.sn_first[s]; j < S.sn_first[s + 1]; j++)
      wrow_of_tail_col[j - S.tail_col] = C.sn_wrow[s] + (j - S.sn_first[s]);
  }
  return before;
}

void g_gather(const Symbolic& S, const Coupling& C, int32_t tail_sn, std::vector<int32_t>& g_key,
              std::vector<int64_t>& g_ptr, std::vector<int32_t>& g_row) {
  std::vector<std::pair<int32_t, int32_t>> recs;  // (key, W row)
  for (int32_t s = 0; s < tail_sn; s++) {
    if (C.sn_wrow[s] < 0) continue;
    const int32_t* T = C.wt_idx.data() + C.wt_ptr[s];
    const int32_t nt = C.wt_ptr[s + 1] - C.wt_ptr[s];
    for (int32_t c = 0; c < S.sn_first[s + 1] - S.sn_first[s]; c++)
      for (int32_t a = 0; a < nt; a++)
        for (int32_t b = 0; b <= a; b++) {
          const int32_t t1 = std::max(T[a], T[b]), t2 = std::min(T[a], T[b]);
          recs.push_back({t1 * C.k + t2, C.sn_wrow[s] + c});
        }
  }
  std::sort(recs.begin(), recs.end());
  g_key.clear();
  g_ptr.assign(1, 0);
  g_row.clear();
  for (size_t i = 0; i < recs.size(); i++) {
    if (i == 0 || recs[i].first != recs[i - 1].first) {
      if (i > 0) g_ptr.push_back((int64_t)g_row.size());
      g_key.push_back(recs[i].first);
    }
    g_row.push_back(recs[i].second);
  }
  if (!recs.empty()) g_ptr.push_back((int64_t)g_row.size());
}

}  // namespace kkt
