/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU reference for the Schur-complement solve of the
 * block-arrowhead KKT system K = [blockdiag(A_0..A_{N-1}) B; B^T C]
 * (Sec. 4.2, eqs. hessianPerm, SCform, SCsolve, SCsolve1; Algorithm 1).
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * load this file.  It shares no code with the CUDA path.
 *
 * Steps, each in the order the method states them:
 *   1. minimum-degree ordering of the shared pattern of A_i (explicit
 *      elimination graph, smallest current degree first, ties to the
 *      smallest index);
 *   2. A_i = L_i D_i L_i^T by the up-looking sparse algorithm with 1x1
 *      pivots in that order (the block factorization of Algorithm 1);
 *   3. S = C - sum_i B_i^T A_i^{-1} B_i, one full solve per nonzero column
 *      of B_i ("backsolve" assembly, Sec. 4.2) and
 *      t = r_g - sum_i B_i^T A_i^{-1} r_i (eq. SCsolve);
 *   4. dense S = L_s D_s L_s^T (Crout form, no pivoting) and S x_g = t
 *      (the dense factor and solve of Algorithm 1, eq. SCsolve);
 *   5. x_i = A_i^{-1} (r_i - B_i x_g) (eq. SCsolve1);
 *   6. inertia = sign counts of all D_i and D_s (Haynsworth additivity;
 *      the inertia test of Sec. 2.3).
 *
 * Notation follows K = [A B; B^T C] (B_i is nA x nC, right column), i.e. the
 * transpose of the paper's B_i.  Pivots are never perturbed here: an exactly
 * zero pivot is reported as an error.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_NOMEM (-2)
#define ORC_ERR_ZERO_PIVOT (-3)

/* ------------------------------------------------------------------ */
/* 1. minimum-degree ordering on the explicit elimination graph        */
/* ------------------------------------------------------------------ */

typedef struct {
  int32_t *v;
  int32_t len, cap;
} ivec;

static int ivec_reserve(ivec *a, int32_t cap) {
  if (a->cap >= cap) return 0;
  int32_t nc = a->cap ? a->cap : 4;
  while (nc < cap) nc *= 2;
  int32_t *p = (int32_t *)realloc(a->v, sizeof(int32_t) * (size_t)nc);
  if (!p) return -1;
  a->v = p;
  a->cap = nc;
  return 0;
}

/* perm[k] = original index of the k-th eliminated node.
   n_primal < n: nodes >= n_primal (multipliers) become eligible only once
   all their original neighbours below n_primal are eliminated (mode 1). */
int orc_min_degree_ex(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t n_primal,
                      int32_t *perm);
int orc_min_degree(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t *perm) {
  return orc_min_degree_ex(n, rowptr, col, n, perm);
}
int orc_min_degree_ex(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t n_primal,
                      int32_t *perm) {
  if (n < 0) return ORC_ERR_INVALID;
  int32_t *wait = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  if (!wait) return ORC_ERR_NOMEM;
  ivec *adj = (ivec *)calloc((size_t)(n > 0 ? n : 1), sizeof(ivec));
  char *done = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
  int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  ivec tmp = {0, 0, 0};
  if (!adj || !done || !mark) return ORC_ERR_NOMEM;
  for (int32_t i = 0; i < n; i++) mark[i] = -1;
  /* symmetric adjacency (no self loops) */
  for (int32_t r = 0; r < n; r++)
    for (int32_t p = rowptr[r]; p < rowptr[r + 1]; p++) {
      int32_t c = col[p];
      if (c < 0 || c >= n) return ORC_ERR_INVALID;
      if (c == r) continue;
      if (ivec_reserve(&adj[r], adj[r].len + 1) || ivec_reserve(&adj[c], adj[c].len + 1))
        return ORC_ERR_NOMEM;
      adj[r].v[adj[r].len++] = c;
      adj[c].v[adj[c].len++] = r;
    }
  /* remove duplicate neighbours */
  for (int32_t r = 0; r < n; r++) {
    int32_t w = 0;
    for (int32_t q = 0; q < adj[r].len; q++) {
      int32_t u = adj[r].v[q];
      if (mark[u] == r) continue;
      mark[u] = r;
      adj[r].v[w++] = u;
    }
    adj[r].len = w;
  }
  for (int32_t i = 0; i < n; i++) mark[i] = -1;
  /* multipliers wait for their primal neighbours: oadj lists, for each
     primal node, its multiplier neighbours in the original graph */
  int32_t *optr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  int32_t *oadj = NULL;
  if (!optr) return ORC_ERR_NOMEM;
  for (int32_t r = n_primal; r < n; r++)
    for (int32_t q = 0; q < adj[r].len; q++)
      if (adj[r].v[q] < n_primal) {
        wait[r]++;
        optr[adj[r].v[q] + 1]++;
      }
  for (int32_t i = 0; i < n; i++) optr[i + 1] += optr[i];
  oadj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(optr[n] > 0 ? optr[n] : 1));
  if (!oadj) return ORC_ERR_NOMEM;
  {
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!fill) return ORC_ERR_NOMEM;
    for (int32_t i = 0; i < n; i++) fill[i] = optr[i];
    for (int32_t r = n_primal; r < n; r++)
      for (int32_t q = 0; q < adj[r].len; q++)
        if (adj[r].v[q] < n_primal) oadj[fill[adj[r].v[q]]++] = r;
    free(fill);
  }

  for (int32_t k = 0; k < n; k++) {
    int32_t best = -1;
    for (int32_t i = 0; i < n; i++)
      if (!done[i] && wait[i] == 0 && (best < 0 || adj[i].len < adj[best].len)) best = i;
    if (best < 0) return ORC_ERR_INVALID;
    perm[k] = best;
    done[best] = 1;
    if (best < n_primal)
      for (int32_t q = optr[best]; q < optr[best + 1]; q++) wait[oadj[q]]--;
    ivec *nb = &adj[best];
    /* eliminating `best` joins its neighbours into a clique */
    for (int32_t q = 0; q < nb->len; q++) {
      int32_t u = nb->v[q];
      ivec *au = &adj[u];
      tmp.len = 0;
      /* mark current neighbours of u */
      for (int32_t t = 0; t < au->len; t++) mark[au->v[t]] = u;
      if (ivec_reserve(&tmp, au->len + nb->len)) return ORC_ERR_NOMEM;
      for (int32_t t = 0; t < au->len; t++)
        if (au->v[t] != best) tmp.v[tmp.len++] = au->v[t];
      for (int32_t t = 0; t < nb->len; t++) {
        int32_t w = nb->v[t];
        if (w != u && mark[w] != u) {
          tmp.v[tmp.len++] = w;
          mark[w] = u;
        }
      }
      /* reset marks for the next neighbour */
      for (int32_t t = 0; t < tmp.len; t++) mark[tmp.v[t]] = -1;
      mark[best] = -1;
      if (ivec_reserve(au, tmp.len)) return ORC_ERR_NOMEM;
      memcpy(au->v, tmp.v, sizeof(int32_t) * (size_t)tmp.len);
      au->len = tmp.len;
    }
    free(nb->v);
    nb->v = NULL;
    nb->len = nb->cap = 0;
  }
  for (int32_t i = 0; i < n; i++) free(adj[i].v);
  free(adj);
  free(done);
  free(mark);
  free(tmp.v);
  free(wait);
  free(optr);
  free(oadj);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* 2. sparse LDL^T: symbolic (elimination tree, column counts), numeric */
/* ------------------------------------------------------------------ */

typedef struct {
  int32_t n;
  int32_t *perm, *iperm;   /* perm[new] = old */
  int32_t *up_ptr, *up_row; /* permuted matrix, column k holds rows <= k */
  int64_t *up_src;         /* position of each entry in the caller's values */
  int32_t *parent;         /* elimination tree */
  int64_t *Lp;             /* column starts of strictly-lower L */
  int64_t nnzL;
} orc_symbolic;

static void sym_free(orc_symbolic *s) {
  free(s->perm);
  free(s->iperm);
  free(s->up_ptr);
  free(s->up_row);
  free(s->up_src);
  free(s->parent);
  free(s->Lp);
  memset(s, 0, sizeof(*s));
}

static int sym_analyze(int32_t n, const int32_t *rowptr, const int32_t *col, const int32_t *perm,
                       orc_symbolic *s) {
  memset(s, 0, sizeof(*s));
  s->n = n;
  size_t nn = (size_t)(n > 0 ? n : 1);
  int64_t nnz = rowptr[n];
  s->perm = (int32_t *)malloc(sizeof(int32_t) * nn);
  s->iperm = (int32_t *)malloc(sizeof(int32_t) * nn);
  s->up_ptr = (int32_t *)calloc(nn + 1, sizeof(int32_t));
  s->up_row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  s->up_src = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
  s->parent = (int32_t *)malloc(sizeof(int32_t) * nn);
  s->Lp = (int64_t *)calloc(nn + 1, sizeof(int64_t));
  int32_t *flag = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *cnt = (int32_t *)calloc(nn, sizeof(int32_t));
  if (!s->perm || !s->iperm || !s->up_ptr || !s->up_row || !s->up_src || !s->parent || !s->Lp ||
      !flag || !cnt)
    return ORC_ERR_NOMEM;
  for (int32_t k = 0; k < n; k++) {
    s->perm[k] = perm[k];
    s->iperm[k] = -1;
  }
  for (int32_t k = 0; k < n; k++) {
    if (perm[k] < 0 || perm[k] >= n || s->iperm[perm[k]] >= 0) return ORC_ERR_INVALID;
    s->iperm[perm[k]] = k;
  }
  /* permuted entries, placed in column max(pr,pc) with row min(pr,pc) */
  for (int32_t r = 0; r < n; r++)
    for (int32_t p = rowptr[r]; p < rowptr[r + 1]; p++) {
      int32_t a = s->iperm[r], b = s->iperm[col[p]];
      int32_t c = a > b ? a : b;
      s->up_ptr[c + 1]++;
    }
  for (int32_t k = 0; k < n; k++) s->up_ptr[k + 1] += s->up_ptr[k];
  for (int32_t k = 0; k < n; k++) cnt[k] = s->up_ptr[k];
  for (int32_t r = 0; r < n; r++)
    for (int32_t p = rowptr[r]; p < rowptr[r + 1]; p++) {
      int32_t a = s->iperm[r], b = s->iperm[col[p]];
      int32_t c = a > b ? a : b, rr = a > b ? b : a;
      int32_t q = cnt[c]++;
      s->up_row[q] = rr;
      s->up_src[q] = p;
    }
  /* elimination tree: parent[i] = min{k > i : L[k,i] != 0} */
  for (int32_t k = 0; k < n; k++) {
    s->parent[k] = -1;
    flag[k] = k;
    for (int32_t p = s->up_ptr[k]; p < s->up_ptr[k + 1]; p++) {
      int32_t i = s->up_row[p];
      /* climb from i to the root of its current subtree, stopping at nodes
         already visited for row k */
      while (i != k && flag[i] != k) {
        if (s->parent[i] == -1) s->parent[i] = k;
        flag[i] = k;
        i = s->parent[i];
      }
    }
  }
  /* column counts: row k of L is the set of nodes reached from A[0:k,k]
     by climbing the tree, stopping at k or at an already visited node */
  for (int32_t k = 0; k < n; k++) cnt[k] = 0;
  for (int32_t k = 0; k < n; k++) {
    flag[k] = k;
    for (int32_t p = s->up_ptr[k]; p < s->up_ptr[k + 1]; p++) {
      int32_t i = s->up_row[p];
      while (flag[i] != k) {
        cnt[i]++;
        flag[i] = k;
        i = s->parent[i];
      }
    }
  }
  s->Lp[0] = 0;
  for (int32_t k = 0; k < n; k++) s->Lp[k + 1] = s->Lp[k] + cnt[k];
  s->nnzL = s->Lp[n];
  free(flag);
  free(cnt);
  return ORC_OK;
}

typedef struct {
  int32_t *Li; /* row indices of L, per column in increasing order */
  double *Lx;
  double *D;
  double *y;
  int32_t *pattern, *stack, *flag, *Lnz;
} orc_numeric;

static int num_alloc(const orc_symbolic *s, orc_numeric *f) {
  size_t nn = (size_t)(s->n > 0 ? s->n : 1);
  size_t nl = (size_t)(s->nnzL > 0 ? s->nnzL : 1);
  f->Li = (int32_t *)malloc(sizeof(int32_t) * nl);
  f->Lx = (double *)malloc(sizeof(double) * nl);
  f->D = (double *)malloc(sizeof(double) * nn);
  f->y = (double *)calloc(nn, sizeof(double));
  f->pattern = (int32_t *)malloc(sizeof(int32_t) * nn);
  f->stack = (int32_t *)malloc(sizeof(int32_t) * nn);
  f->flag = (int32_t *)malloc(sizeof(int32_t) * nn);
  f->Lnz = (int32_t *)malloc(sizeof(int32_t) * nn);
  if (!f->Li || !f->Lx || !f->D || !f->y || !f->pattern || !f->stack || !f->flag || !f->Lnz)
    return ORC_ERR_NOMEM;
  return ORC_OK;
}

static void num_free(orc_numeric *f) {
  free(f->Li);
  free(f->Lx);
  free(f->D);
  free(f->y);
  free(f->pattern);
  free(f->stack);
  free(f->flag);
  free(f->Lnz);
  memset(f, 0, sizeof(*f));
}

/* Up-looking LDL^T: row k of L solves L[0:k,0:k] (D l_k) = A[0:k,k]; the
   nonzero rows of that triangular solve are the tree reach of A[0:k,k]. */
static int num_factor(const orc_symbolic *s, const double *vals, orc_numeric *f) {
  int32_t n = s->n;
  for (int32_t k = 0; k < n; k++) {
    f->Lnz[k] = 0;
    f->flag[k] = -1;
  }
  for (int32_t k = 0; k < n; k++) {
    int32_t top = n;
    f->flag[k] = k;
    f->y[k] = 0.0;
    for (int32_t p = s->up_ptr[k]; p < s->up_ptr[k + 1]; p++) {
      int32_t i = s->up_row[p];
      f->y[i] += vals[s->up_src[p]];
      int32_t len = 0;
      while (f->flag[i] != k) {
        f->stack[len++] = i;
        f->flag[i] = k;
        i = s->parent[i];
      }
      while (len > 0) f->pattern[--top] = f->stack[--len];
    }
    double dk = f->y[k];
    f->y[k] = 0.0;
    for (; top < n; top++) {
      int32_t j = f->pattern[top];
      double yj = f->y[j];
      f->y[j] = 0.0;
      int64_t p0 = s->Lp[j], p1 = s->Lp[j] + f->Lnz[j];
      for (int64_t p = p0; p < p1; p++) f->y[f->Li[p]] -= f->Lx[p] * yj;
      double lkj = yj / f->D[j];
      dk -= lkj * yj;
      f->Li[p1] = k;
      f->Lx[p1] = lkj;
      f->Lnz[j]++;
    }
    if (dk == 0.0) return ORC_ERR_ZERO_PIVOT;
    f->D[k] = dk;
  }
  return ORC_OK;
}

/* x = A^{-1} b with A = P L D L^T P^T; work has n entries */
static void num_solve(const orc_symbolic *s, const orc_numeric *f, const double *b, double *x,
                      double *work) {
  int32_t n = s->n;
  for (int32_t k = 0; k < n; k++) work[k] = b[s->perm[k]];
  for (int32_t j = 0; j < n; j++) {
    double wj = work[j];
    for (int64_t p = s->Lp[j]; p < s->Lp[j + 1]; p++) work[f->Li[p]] -= f->Lx[p] * wj;
  }
  for (int32_t j = 0; j < n; j++) work[j] /= f->D[j];
  for (int32_t j = n - 1; j >= 0; j--) {
    double wj = work[j];
    for (int64_t p = s->Lp[j]; p < s->Lp[j + 1]; p++) wj -= f->Lx[p] * work[f->Li[p]];
    work[j] = wj;
  }
  for (int32_t k = 0; k < n; k++) x[s->perm[k]] = work[k];
}

int64_t orc_nnz_l(int32_t n, const int32_t *rowptr, const int32_t *col, const int32_t *perm) {
  orc_symbolic s;
  int rc = sym_analyze(n, rowptr, col, perm, &s);
  int64_t r = rc == ORC_OK ? s.nnzL : rc;
  sym_free(&s);
  return r;
}

/* Factor one sparse symmetric matrix and return dense L (unit lower, in the
   permuted order, row-major n x n) and D.  For small matrices in tests. */
int orc_ldlt_dense(int32_t n, const int32_t *rowptr, const int32_t *col, const double *vals,
                   const int32_t *perm, double *Ldense, double *D) {
  orc_symbolic s;
  orc_numeric f;
  int rc = sym_analyze(n, rowptr, col, perm, &s);
  if (rc) return rc;
  rc = num_alloc(&s, &f);
  if (!rc) rc = num_factor(&s, vals, &f);
  if (!rc) {
    memset(Ldense, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int32_t j = 0; j < n; j++) {
      Ldense[(size_t)j * n + j] = 1.0;
      D[j] = f.D[j];
      for (int64_t p = s.Lp[j]; p < s.Lp[j + 1]; p++) Ldense[(size_t)f.Li[p] * n + j] = f.Lx[p];
    }
  }
  num_free(&f);
  sym_free(&s);
  return rc;
}

/* x = A^{-1} b for one sparse symmetric matrix in the given ordering */
int orc_sparse_solve(int32_t n, const int32_t *rowptr, const int32_t *col, const double *vals,
                     const int32_t *perm, const double *b, double *x) {
  orc_symbolic s;
  orc_numeric f;
  int rc = sym_analyze(n, rowptr, col, perm, &s);
  if (rc) return rc;
  rc = num_alloc(&s, &f);
  if (!rc) rc = num_factor(&s, vals, &f);
  if (!rc) {
    double *w = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!w) rc = ORC_ERR_NOMEM;
    else {
      num_solve(&s, &f, b, x, w);
      free(w);
    }
  }
  num_free(&f);
  sym_free(&s);
  return rc;
}

/* X = A^{-1} B for nrhs right-hand sides (column j of B and X at j * n): one
   factorization, then the solve of algorithm 1's local systems per column. */
int orc_sparse_solve_multi(int32_t n, const int32_t *rowptr, const int32_t *col, const double *vals,
                           const int32_t *perm, int32_t nrhs, const double *B, double *X) {
  orc_symbolic s;
  orc_numeric f;
  if (nrhs < 0) return ORC_ERR_INVALID;
  int rc = sym_analyze(n, rowptr, col, perm, &s);
  if (rc) return rc;
  rc = num_alloc(&s, &f);
  if (!rc) rc = num_factor(&s, vals, &f);
  if (!rc) {
    double *w = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!w) rc = ORC_ERR_NOMEM;
    else {
      for (int32_t j = 0; j < nrhs; j++) num_solve(&s, &f, B + (size_t)j * n, X + (size_t)j * n, w);
      free(w);
    }
  }
  num_free(&f);
  sym_free(&s);
  return rc;
}

/* ------------------------------------------------------------------ */
/* 4. dense LDL^T of S (Crout form), in place, row-major full storage   */
/* ------------------------------------------------------------------ */

/* On return the strict lower triangle of S holds L_s and the diagonal D_s.
   l_ij = (s_ij - sum_{k<j} l_ik d_k l_jk) / d_j,  d_j = s_jj - sum_k l_jk^2 d_k.
   w holds n entries of scratch. */
static int dense_ldlt(int64_t n, double *S, double *w) {
  for (int64_t j = 0; j < n; j++) {
    double *rj = S + j * n;
    for (int64_t k = 0; k < j; k++) w[k] = rj[k] * S[k * n + k]; /* l_jk d_k */
    double dj = rj[j];
    for (int64_t k = 0; k < j; k++) dj -= rj[k] * w[k];
    if (dj == 0.0) return ORC_ERR_ZERO_PIVOT;
    rj[j] = dj;
#pragma omp parallel for schedule(static)
    for (int64_t i = j + 1; i < n; i++) {
      double *ri = S + i * n;
      double sij = ri[j];
      for (int64_t k = 0; k < j; k++) sij -= ri[k] * w[k];
      ri[j] = sij / dj;
    }
  }
  return ORC_OK;
}

static void dense_ldlt_solve(int64_t n, const double *F, double *x) {
  for (int64_t i = 0; i < n; i++) {
    double v = x[i];
    for (int64_t k = 0; k < i; k++) v -= F[i * n + k] * x[k];
    x[i] = v;
  }
  for (int64_t i = 0; i < n; i++) x[i] /= F[i * n + i];
  for (int64_t i = n - 1; i >= 0; i--) {
    double v = x[i];
    for (int64_t k = i + 1; k < n; k++) v -= F[k * n + i] * x[k];
    x[i] = v;
  }
}

int orc_dense_ldlt(int64_t n, double *S, int64_t *inertia) {
  double *w = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!w) return ORC_ERR_NOMEM;
  int rc = dense_ldlt(n, S, w);
  free(w);
  if (rc == ORC_OK && inertia) {
    inertia[0] = inertia[1] = inertia[2] = 0;
    for (int64_t j = 0; j < n; j++) {
      double d = S[j * n + j];
      inertia[d > 0 ? 0 : (d < 0 ? 1 : 2)]++;
    }
  }
  return rc;
}

int orc_dense_ldlt_solve(int64_t n, const double *F, double *x) {
  dense_ldlt_solve(n, F, x);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* arrowhead K: products and norms (plain definitions)                 */
/* ------------------------------------------------------------------ */

/* y = K x.  C is diagonal (c_kind 0, nC values) or full symmetric
   (c_kind 1, nC*nC values, row-major). */
int orc_kkt_matvec(int32_t N, int32_t nA, int32_t nC, const int32_t *a_rowptr,
                   const int32_t *a_col, const double *a_vals, const int32_t *b_blockptr,
                   const int32_t *b_row, const int32_t *b_col, const double *b_vals,
                   int32_t c_kind, const double *c_vals, const double *x, double *y) {
  int64_t nnzA = a_rowptr[nA];
  int64_t nK = (int64_t)N * nA + nC;
  const double *xg = x + (int64_t)N * nA;
  double *yg = y + (int64_t)N * nA;
  for (int64_t k = 0; k < nK; k++) y[k] = 0.0;
  for (int32_t i = 0; i < N; i++) {
    const double *v = a_vals + (int64_t)i * nnzA;
    const double *xi = x + (int64_t)i * nA;
    double *yi = y + (int64_t)i * nA;
    for (int32_t r = 0; r < nA; r++)
      for (int32_t p = a_rowptr[r]; p < a_rowptr[r + 1]; p++) {
        int32_t c = a_col[p];
        yi[r] += v[p] * xi[c];
        if (c != r) yi[c] += v[p] * xi[r];
      }
    for (int32_t p = b_blockptr[i]; p < b_blockptr[i + 1]; p++) {
      yi[b_row[p]] += b_vals[p] * xg[b_col[p]];
      yg[b_col[p]] += b_vals[p] * xi[b_row[p]];
    }
  }
  if (c_kind == 0) {
    for (int32_t c = 0; c < nC; c++) yg[c] += c_vals[c] * xg[c];
  } else {
    for (int32_t r = 0; r < nC; r++)
      for (int32_t c = 0; c < nC; c++) yg[r] += c_vals[(int64_t)r * nC + c] * xg[c];
  }
  return ORC_OK;
}

/* ||K||_inf = max row sum of |K| */
double orc_kkt_norm_inf(int32_t N, int32_t nA, int32_t nC, const int32_t *a_rowptr,
                        const int32_t *a_col, const double *a_vals, const int32_t *b_blockptr,
                        const int32_t *b_row, const int32_t *b_col, const double *b_vals,
                        int32_t c_kind, const double *c_vals) {
  int64_t nnzA = a_rowptr[nA];
  int64_t nK = (int64_t)N * nA + nC;
  double *rs = (double *)calloc((size_t)(nK > 0 ? nK : 1), sizeof(double));
  if (!rs) return -1.0;
  double *rg = rs + (int64_t)N * nA;
  for (int32_t i = 0; i < N; i++) {
    const double *v = a_vals + (int64_t)i * nnzA;
    double *ri = rs + (int64_t)i * nA;
    for (int32_t r = 0; r < nA; r++)
      for (int32_t p = a_rowptr[r]; p < a_rowptr[r + 1]; p++) {
        ri[r] += fabs(v[p]);
        if (a_col[p] != r) ri[a_col[p]] += fabs(v[p]);
      }
    for (int32_t p = b_blockptr[i]; p < b_blockptr[i + 1]; p++) {
      ri[b_row[p]] += fabs(b_vals[p]);
      rg[b_col[p]] += fabs(b_vals[p]);
    }
  }
  if (c_kind == 0) {
    for (int32_t c = 0; c < nC; c++) rg[c] += fabs(c_vals[c]);
  } else {
    for (int32_t r = 0; r < nC; r++)
      for (int32_t c = 0; c < nC; c++) rg[r] += fabs(c_vals[(int64_t)r * nC + c]);
  }
  double m = 0.0;
  for (int64_t k = 0; k < nK; k++) m = rs[k] > m ? rs[k] : m;
  free(rs);
  return m;
}

/* ------------------------------------------------------------------ */
/* 3-6. the Schur-complement solve                                     */
/* ------------------------------------------------------------------ */

/* distinct nonzero columns of block i's B, in increasing order */
static int32_t block_cols(const int32_t *b_col, int32_t p0, int32_t p1, int32_t *out,
                          int32_t *mark, int32_t stamp) {
  int32_t k = 0;
  for (int32_t p = p0; p < p1; p++)
    if (mark[b_col[p]] != stamp) {
      mark[b_col[p]] = stamp;
      out[k++] = b_col[p];
    }
  /* insertion sort: k is small */
  for (int32_t a = 1; a < k; a++) {
    int32_t v = out[a], b = a - 1;
    while (b >= 0 && out[b] > v) {
      out[b + 1] = out[b];
      b--;
    }
    out[b + 1] = v;
  }
  return k;
}

/*
 * Solve K x = rhs.  Host arrays only.
 *   perm:       ordering of A's pattern (from orc_min_degree), nA entries
 *   S_out:      optional, nC*nC row-major: the assembled S = C - sum B^T A^-1 B
 *   t_out:      optional, nC: t = r_g - sum B^T A^-1 r_i
 *   inertia:    [n_pos, n_neg, n_zero] of K from the signs of all pivots
 *   nthreads:   OpenMP threads (0 = runtime default)
 */
int orc_kkt_solve(int32_t N, int32_t nA, int32_t nC, const int32_t *a_rowptr,
                  const int32_t *a_col, const double *a_vals, const int32_t *b_blockptr,
                  const int32_t *b_row, const int32_t *b_col, const double *b_vals,
                  int32_t c_kind, const double *c_vals, const double *rhs, const int32_t *perm,
                  double *x, double *S_out, double *t_out, int64_t *inertia, int32_t nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  if (N < 0 || nA < 0 || nC < 0) return ORC_ERR_INVALID;
  int64_t nnzA = a_rowptr[nA];
  orc_symbolic s;
  int rc = sym_analyze(nA, a_rowptr, a_col, perm, &s);
  if (rc) return rc;

  /* per-block workspace */
  orc_numeric *F = (orc_numeric *)calloc((size_t)(N > 0 ? N : 1), sizeof(orc_numeric));
  int32_t *kcols = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N + 1));
  double *S = (double *)calloc((size_t)nC * (size_t)nC + 1, sizeof(double));
  double *t = (double *)calloc((size_t)nC + 1, sizeof(double));
  double **Sloc = (double **)calloc((size_t)(N > 0 ? N : 1), sizeof(double *));
  double **tloc = (double **)calloc((size_t)(N > 0 ? N : 1), sizeof(double *));
  int32_t **cols = (int32_t **)calloc((size_t)(N > 0 ? N : 1), sizeof(int32_t *));
  int *brc = (int *)calloc((size_t)(N > 0 ? N : 1), sizeof(int));
  if (!F || !kcols || !S || !t || !Sloc || !tloc || !cols || !brc) return ORC_ERR_NOMEM;

  /* parts 2 and 3 above: per block factor, local Schur contribution, local RHS term */
#pragma omp parallel
  {
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nC > 0 ? nC : 1));
    double *e = (double *)calloc((size_t)(nA > 0 ? nA : 1), sizeof(double));
    double *yv = (double *)malloc(sizeof(double) * (size_t)(nA > 0 ? nA : 1));
    double *wk = (double *)malloc(sizeof(double) * (size_t)(nA > 0 ? nA : 1));
    for (int32_t c = 0; c < nC; c++) mark[c] = -1;
#pragma omp for schedule(dynamic)
    for (int32_t i = 0; i < N; i++) {
      int r = num_alloc(&s, &F[i]);
      if (!r) r = num_factor(&s, a_vals + (int64_t)i * nnzA, &F[i]);
      if (r) {
        brc[i] = r;
        continue;
      }
      int32_t p0 = b_blockptr[i], p1 = b_blockptr[i + 1];
      cols[i] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(p1 - p0 + 1));
      int32_t k = block_cols(b_col, p0, p1, cols[i], mark, i);
      kcols[i] = k;
      Sloc[i] = (double *)calloc((size_t)k * (size_t)k + 1, sizeof(double));
      tloc[i] = (double *)calloc((size_t)k + 1, sizeof(double));
      /* column a of B_i -> y = A_i^{-1} B_i[:,a]; row b of B_i^T y */
      for (int32_t a = 0; a < k; a++) {
        int32_t ca = cols[i][a];
        for (int32_t p = p0; p < p1; p++)
          if (b_col[p] == ca) e[b_row[p]] += b_vals[p];
        num_solve(&s, &F[i], e, yv, wk);
        for (int32_t p = p0; p < p1; p++)
          if (b_col[p] == ca) e[b_row[p]] = 0.0;
        for (int32_t b = 0; b < k; b++) {
          int32_t cb = cols[i][b];
          double acc = 0.0;
          for (int32_t p = p0; p < p1; p++)
            if (b_col[p] == cb) acc += b_vals[p] * yv[b_row[p]];
          Sloc[i][(int64_t)b * k + a] = acc;
        }
      }
      /* z = A_i^{-1} r_i;  B_i^T z */
      num_solve(&s, &F[i], rhs + (int64_t)i * nA, yv, wk);
      for (int32_t b = 0; b < k; b++) {
        int32_t cb = cols[i][b];
        double acc = 0.0;
        for (int32_t p = p0; p < p1; p++)
          if (b_col[p] == cb) acc += b_vals[p] * yv[b_row[p]];
        tloc[i][b] = acc;
      }
    }
    free(mark);
    free(e);
    free(yv);
    free(wk);
  }
  for (int32_t i = 0; i < N; i++)
    if (brc[i]) {
      rc = brc[i];
      goto done;
    }

  /* reduction in block order: S = C - sum S_i, t = r_g - sum B_i^T z_i */
  if (c_kind == 0) {
    for (int32_t c = 0; c < nC; c++) S[(int64_t)c * nC + c] = c_vals[c];
  } else {
    for (int64_t q = 0; q < (int64_t)nC * nC; q++) S[q] = c_vals[q];
  }
  for (int32_t c = 0; c < nC; c++) t[c] = rhs[(int64_t)N * nA + c];
  for (int32_t i = 0; i < N; i++) {
    int32_t k = kcols[i];
    for (int32_t b = 0; b < k; b++) {
      for (int32_t a = 0; a < k; a++)
        S[(int64_t)cols[i][b] * nC + cols[i][a]] -= Sloc[i][(int64_t)b * k + a];
      t[cols[i][b]] -= tloc[i][b];
    }
  }
  if (S_out) memcpy(S_out, S, sizeof(double) * (size_t)nC * (size_t)nC);
  if (t_out) memcpy(t_out, t, sizeof(double) * (size_t)nC);

  /* part 4 above: S = L_s D_s L_s^T, x_g = S^{-1} t */
  {
    int64_t in_s[3] = {0, 0, 0};
    rc = orc_dense_ldlt(nC, S, in_s);
    if (rc) goto done;
    double *xg = x + (int64_t)N * nA;
    memcpy(xg, t, sizeof(double) * (size_t)nC);
    dense_ldlt_solve(nC, S, xg);
    if (inertia) {
      inertia[0] = in_s[0];
      inertia[1] = in_s[1];
      inertia[2] = in_s[2];
    }
  }

  /* part 5 above: x_i = A_i^{-1} (r_i - B_i x_g) */
  {
    const double *xg = x + (int64_t)N * nA;
#pragma omp parallel
    {
      double *v = (double *)malloc(sizeof(double) * (size_t)(nA > 0 ? nA : 1));
      double *wk = (double *)malloc(sizeof(double) * (size_t)(nA > 0 ? nA : 1));
#pragma omp for schedule(dynamic)
      for (int32_t i = 0; i < N; i++) {
        memcpy(v, rhs + (int64_t)i * nA, sizeof(double) * (size_t)nA);
        for (int32_t p = b_blockptr[i]; p < b_blockptr[i + 1]; p++)
          v[b_row[p]] -= b_vals[p] * xg[b_col[p]];
        num_solve(&s, &F[i], v, x + (int64_t)i * nA, wk);
      }
      free(v);
      free(wk);
    }
  }

  /* part 6 above: inertia of K = sum of block inertias + inertia of S */
  if (inertia) {
    for (int32_t i = 0; i < N; i++)
      for (int32_t j = 0; j < nA; j++) {
        double d = F[i].D[j];
        inertia[d > 0 ? 0 : (d < 0 ? 1 : 2)]++;
      }
  }

done:
  for (int32_t i = 0; i < N; i++) {
    num_free(&F[i]);
    free(Sloc[i]);
    free(tloc[i]);
    free(cols[i]);
  }
  free(F);
  free(kcols);
  free(S);
  free(t);
  free(Sloc);
  free(tloc);
  free(cols);
  free(brc);
  sym_free(&s);
  return rc;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
