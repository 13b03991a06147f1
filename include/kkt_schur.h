/*
 * kkt_schur.h -- C ABI of the GB300 Schur-complement solver for
 * block-arrowhead KKT systems (Kardos, Kourounis, Schenk,
 * "Structure-Exploiting Interior Point Methods", Sec. 4).
 *
 * The system (eq. hessianPerm, written with B on the right):
 *
 *     K = [ A_0                B_0 ]     x = [x_0; ...; x_{N-1}; x_g]
 *         [      ...           ... ]     r = [r_0; ...; r_{N-1}; r_g]
 *         [          A_{N-1}   B_{N-1}]
 *         [ B_0^T ... B_{N-1}^T  C ]
 *
 * is solved by Schur-complement decomposition (eqs. SCform, SCsolve,
 * SCsolve1; Algorithm 1):
 *
 *     A_i = P L_i D_i L_i^T P^T                      (block factors)
 *     S   = C - sum_i B_i^T A_i^{-1} B_i              (Schur assembly, eq. SCform)
 *     t   = r_g - sum_i B_i^T A_i^{-1} r_i            (RHS reduction, eq. SCsolve)
 *     S   = L_s D_s L_s^T,  x_g = S^{-1} t            (dense factor and solve of S)
 *     x_i = A_i^{-1} (r_i - B_i x_g)                  (local solves, eq. SCsolve1)
 *
 * followed by FP64 iterative refinement on the full K (Sec. 2.1: refinement
 * improves the accuracy of the direct solve).
 *
 * All indices are 0-based int32.  All functions return a kkt_status; none
 * aborts the process.  Device-side numerical events (perturbed pivots,
 * refinement that stalls) are reported through kkt_get_info.
 */
#ifndef KKT_SCHUR_H
#define KKT_SCHUR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kkt_handle kkt_handle; /* opaque; owns every device buffer it allocates */

typedef enum {
  KKT_OK = 0,
  KKT_ERR_INVALID = 1,       /* malformed pattern, sizes or arguments */
  KKT_ERR_OOM = 2,           /* a device or host allocation failed */
  KKT_ERR_CUDA = 3,          /* a CUDA runtime call failed (message in kkt_last_error) */
  KKT_ERR_ZERO_PIVOT = 4,    /* a pivot was exactly zero and pivot_eps is 0 */
  KKT_ERR_INERTIA = 5,       /* inertia differs from (N*nP + nC, N*(nA-nP), 0) */
  KKT_ERR_NOT_CONVERGED = 6, /* refinement did not reach refine_tol */
  KKT_ERR_TIMEOUT = 7,       /* a bounded device wait ran out */
  KKT_ERR_STATE = 8,         /* call out of order (e.g. solve before factor) */
  KKT_ERR_NONFINITE = 9      /* a NaN or Inf in the values of K or the right-hand side, or a
                                solution that is not finite after the FP64 fallback */
} kkt_status;

/* Arithmetic of the dense factor of S (and of the Schur contraction where
 * noted).  The block factors, the residual and the refinement are FP64 in
 * every mode.
 *   KKT_FP64:          FP64 on the CUDA cores.
 *   KKT_TF32/KKT_BF16: S factored in FP32 with the trailing update on the tensor
 *                      cores (TF32 or BF16 operands, FP32 accumulation); FP64
 *                      refinement on K, FP64-accurate refactor of S if it stalls.
 *   KKT_F64_EMULATED:  FP64-accurate factor of S whose trailing update runs on
 *                      the BF16 tensor cores: operands cut into exact 8-bit
 *                      digit slices, digit products accumulated exactly in FP32
 *                      and recombined in FP64. */
typedef enum { KKT_FP64 = 0, KKT_TF32 = 1, KKT_BF16 = 2, KKT_F64_EMULATED = 3 } kkt_precision;

/* Sparsity of one arrowhead system.  All arrays are host memory, read during
 * kkt_analyze only (copied; the caller keeps ownership).
 *   A (eq. hessianPerm, blocks A_i): every block shares one pattern, given as
 *     the lower triangle in CSR: row r holds columns a_col[a_rowptr[r] ..
 *     a_rowptr[r+1]) in strictly increasing order, each <= r, and the last
 *     one == r (the diagonal must be present).  Rows [0, nP) are primal
 *     variables (positive pivots expected), rows [nP, nA) multipliers
 *     (negative pivots expected).
 *   B: block i's entries are b_blockptr[i] .. b_blockptr[i+1] of b_row
 *     (in [0, nA)) and b_col (in [0, nC)), sorted by (row, col).
 *   C: c_kind 0 = diagonal (nC values), 1 = dense symmetric (nC*nC values,
 *     row-major; only the lower triangle is read).
 *   a_vals_hint: optional (may be NULL) values of one block in the A pattern.
 *     They choose each multiplier's pivot partner: the primal neighbour with
 *     the largest |coupling|, eliminated right before the multiplier.  Without
 *     a hint the best-connected primal neighbour is used. */
typedef struct {
  int32_t N, nA, nP, nC;
  const int32_t* a_rowptr;
  const int32_t* a_col;
  const int32_t* b_blockptr;
  const int32_t* b_row;
  const int32_t* b_col;
  int32_t c_kind;
  const double* a_vals_hint;
} kkt_pattern;

typedef struct {
  kkt_precision prec;  /* arithmetic of the Schur contraction and the factor of S */
  double refine_tol;   /* target normwise backward error of the refined solution (1e-10) */
  int32_t max_refine;  /* refinement steps at most (10); after an FP64 fallback the refinement on the
                          FP64-accurate factor has max_refine steps of its own */
  double pivot_eps;    /* |d| < pivot_eps * ||A_i||_max is replaced by +-pivot_eps * ||A_i||_max
                          with the expected sign and counted; 0 turns the perturbation off */
  int32_t use_graphs;  /* capture the device work of kkt_factor after the input copies as a CUDA
                          graph at the handle's first kkt_factor and replay it on later calls (the
                          solve and its refinement launch directly).  Default 1. */
  int32_t fp64_fallback; /* refactor S in FP64 when refinement stalls in a reduced mode */
  int32_t reduced_contraction; /* KKT_TF32/KKT_BF16 only: also run the Schur contraction
                                  G_i = W_i^T D_i^{-1} W_i on the tensor cores in that precision
                                  (0, the default: FP64 contraction).  On a stall the fallback then
                                  recomputes G in FP64 and reassembles S before refactoring it. */
  int32_t structured_s; /* 0 (default): S dense, factored and solved whole.
                           1: limit the dense factor of S and its solves to S's row envelope
                           (LDL^T without pivoting creates no fill outside it): the same
                           arithmetic on every entry that can be nonzero, the exact zeros outside
                           skipped.  For the adjacent-period coupling S is block-tridiagonal and
                           the cost drops from n_C^3/3 to ~ n_C (2 n_stor)^2.
                           2: the paper's structured S for its cumulative MPOPF coupling (Sec. 4.3,
                           eqs. LocalSchurBs, LocalSchurBs3, GlobalSchur): the coupling variables
                           are ordered by period, n_s = n_C / N per period, block i's coupling
                           columns of period m are zero for m < i and equal (pattern and values)
                           for all m > i, and C is diagonal (c_kind 0); kkt_analyze returns
                           KKT_ERR_INVALID for a pattern without that structure.  S is then
                           kept as two block vectors (S_d: N diagonal n_s x n_s blocks, S_o: the
                           block repeated below the diagonal in each block column), assembled
                           from the N local blocks, factored by N partial LDL^T steps of order
                           2 n_s (O(N n_s^3) flops; FP32 in the TF32/BF16 modes, with FP64
                           refinement on K and the FP64 steps as the fallback, FP64 otherwise) and
                           solved by two chains of N n_s x n_s products.  The analysis builds no
                           per-entry gather lists of S.  B's values are checked on the device at
                           every factor: values that do not repeat make the next kkt_solve
                           return KKT_ERR_INVALID.  Default 0. */
  int32_t dense_tail;   /* factor the top of the elimination tree (a suffix of the supernodes,
                           whose rows are all tail columns) as one dense lower triangle per block
                           with the blocked dense kernels of the factor of S, instead of
                           supernode by supernode.  Chosen at analysis: the longest suffix whose
                           dense flops are at most r times its exact sparse flops (r: tail_ratio,
                           else 1.5, else the autotuner's) and whose N triangles fit 24 GiB
                           (mode 1) or 96 GiB (mode 2).  The same static-pivot rule applies; the
                           factor is scattered back into the supernodal panels.
                           0: off; 1: trailing updates in FP64 on the CUDA cores; 2: trailing
                           updates in emulated FP64 on the tensor cores (7 base-256 digit
                           slices per operand, as in KKT_F64_EMULATED); -1 (default): 2 in the
                           KKT_TF32, KKT_BF16 and KKT_F64_EMULATED modes, 1 in KKT_FP64 (all its
                           arithmetic stays FP64 on the CUDA cores). */
  int32_t autotune;     /* choose the size of the dense tail by timing: the tail is the longest suffix
                           whose dense flops are at most r times its sparse flops; with autotune the
                           distinct tails of r in {1, 1.25, 1.5, 2, 3} are analysed and timed once each
                           (one kkt_factor on the values hint in every block, B = 0, C = I) and the
                           fastest is kept.  The candidates share the first analysis (ordering,
                           supernodes, reach).  Needs a_vals_hint; adds those factorizations to
                           kkt_analyze; ignored when tail_ratio is set.  Default 0 (r = 1.5). */
  int32_t early_solve;  /* the first application of kkt_solve after a kkt_factor starts its front half
                           (forward block solves, right-hand-side reduction), which needs only the
                           block factors, as soon as that factor's Schur assembly has finished, on a
                           stream of the handle, while the dense factor of S still runs.  The
                           right-hand side is then read on that stream: a right-hand side on the
                           device must be complete when kkt_factor is called.  Default 0. */
  int32_t time_kernels; /* record CUDA events around every launch of the dominant kernel families
                           (also inside the factor's CUDA graph) and keep each launch's algorithmic
                           work, for kkt_kernel_stats.  Default 0. */
  double tail_ratio;    /* the cost ratio r of the dense tail (above); 0, the default, takes 1.5 or,
                           with autotune, the autotuner's choice.  Negative values are rejected. */
  int32_t refine_mode;  /* 0 (default): iterative refinement, x += K~^{-1}(r - Kx) while the backward
                           error falls at least by half per step; 1: GMRES refinement (FP64 GMRES on K,
                           right-preconditioned by the factorization K~, restarted every gmres_restart
                           iterations), which converges where the plain iteration stalls on a
                           reduced-precision factor of an ill-conditioned S.  Both stop at refine_tol,
                           count one step per application of K~^{-1} (at most max_refine) and, in the
                           TF32/BF16 modes, refactor S FP64-accurately when they stop short. */
  int32_t gmres_restart; /* Krylov vectors per GMRES cycle (default 8) */
  int32_t device_refine; /* refine_mode 0 only: run kkt_solve's application of the factorization and its
                            refinement loop as one CUDA graph whose loop is a device-side conditional
                            (WHILE) node: a one-thread kernel evaluates the convergence test, and the host
                            reads the outcome once, after the loop, instead of a residual norm per step.
                            The arithmetic is kkt_solve's own, step for step, so the solution is the same
                            bit for bit.  When the loop stops above refine_tol in the TF32/BF16 modes,
                            the FP64 fallback and its refinement run as without this option.  Not used for
                            the first solve after a factor with early_solve.  Default 0. */
} kkt_options;

typedef struct {
  int64_t n_pos, n_neg, n_zero; /* inertia of K from the pivots of all D_i and of the current
                                   factor of S (in KKT_TF32/KKT_BF16 mode that factor is FP32 and
                                   its pivot signs can be wrong for an ill-conditioned S) */
  int64_t n_perturbed;          /* pivots replaced under pivot_eps */
  int32_t refine_steps;         /* refinement steps taken by the last kkt_solve */
  int32_t fell_back_fp64;       /* 1 if the last solve refactored S in FP64 */
  double rel_residual;          /* eta = ||r-Kx||_inf / (||K||_inf ||x||_inf + ||r||_inf) */
  double ms_analyze, ms_factor, ms_solve; /* host wall times of the last calls */
  int64_t nnz_l;                /* strictly lower nonzeros of one block factor */
  int64_t panel_doubles;        /* stored factor values per block (supernodal panels) */
  int32_t n_supernodes, n_levels;
  int32_t k_coupling_rows;      /* k: distinct rows of A carrying a nonzero of B */
  int32_t w_rows;               /* rows of the elimination-tree reach of those rows */
  double factor_flops;          /* block-factor flops per block */
  int64_t device_bytes;         /* device memory held by the handle */
  /* device times (CUDA events on the call's stream) of the last kkt_factor,
   * per phase: (a) block factors, (b) Schur assembly, (c) dense factor of S */
  double ms_block_factor, ms_schur_assembly, ms_dense_factor;
  double ms_solve_device;       /* device time of the last kkt_solve, refinement included */
  int64_t n_launches;           /* kernels launched by this handle since kkt_analyze */
  int32_t dense_tail_cols;      /* columns of the dense tail of each block factor (0 = none) */
  int32_t tail_augmented;       /* 1 if the tail factor also forms the tail's rows of W and its
                                   share of G (the k coupling rows appended to it) */
  double tail_ratio;            /* cost ratio r the dense tail was chosen with (0 without a tail) */
  int32_t autotune_candidates;  /* distinct tails timed by the autotuner (0 without autotune) */
  int32_t schur_block;          /* n_s of the structured S (structured_s = 2), else 0 */
} kkt_info;

/* Default options: FP64, refine_tol 1e-10, max_refine 10, pivot_eps 1e-20,
 * graphs on, FP64 fallback on, dense tail chosen by the mode (-1). */
void kkt_default_options(kkt_options* opt);

/* Symbolic analysis of the pattern: ordering of the shared A pattern,
 * elimination tree, supernodes, reach of B's rows, gather maps for S and t;
 * uploads the index structures and allocates every device buffer that the
 * numeric calls use.  Runs on the current CUDA device.  On success *out owns
 * all of it until kkt_destroy. */
kkt_status kkt_analyze(const kkt_pattern* pattern, const kkt_options* opt, kkt_handle** out);

/* Numeric factorization (Algorithm 1 up to the factor of S): block factors,
 * Schur complement S = C - sum_i B_i^T A_i^{-1} B_i, dense LDL^T of S.
 *   a_vals: N * nnz(A) doubles, block i at offset i * nnz(A), in the pattern's
 *           CSR order;  b_vals: nnz(B) doubles in the pattern's entry order;
 *   c_vals: nC (c_kind 0) or nC*nC (c_kind 1) doubles.
 *   on_device: 0 = host pointers (copied on `stream`, pageable or pinned),
 *              1 = device pointers (read until `stream` passes this work).
 *   stream: a cudaStream_t (NULL = legacy default stream).
 * The call is asynchronous with respect to the host for device inputs; the
 * inertia and perturbation counts are read by kkt_get_info. */
kkt_status kkt_factor(kkt_handle* h, const double* a_vals, const double* b_vals,
                      const double* c_vals, int32_t on_device, void* stream);

/* ---- inertia correction (Sec. 2, inertia correction and curvature detection) ----
 * The IPM needs K with inertia (N*nP + nC, N*(nA - nP), 0): positive pivots for
 * the primal rows of every block and for the coupling variables, negative ones
 * for the multipliers (coupling_dual below: the coupling variables count as
 * multipliers).  When the factor shows another inertia, the diagonal is
 * shifted, K + diag(dw I on the primal rows of every A_i and on C, -dc I on the
 * dual rows), and refactored with growing dw until the inertia is right.  The
 * trial values follow the usual interior-point rule (the paper names the rule,
 * not its constants; these are the defaults below):
 *   first trial after the unshifted factor: dw = delta_w_init, or, once a call
 *     on this handle has succeeded with dw > 0, max(delta_w_min, shrink * last dw);
 *   dc = delta_c when a pivot of a block factor or of S was zero, or a block
 *     pivot was replaced under pivot_eps (a singular or nearly singular
 *     Jacobian), else 0;
 *   next trials: dw *= grow_first while no call on the handle has needed a
 *     shift, dw *= grow afterwards; give up when dw > delta_w_max or after
 *     max_trials factorizations (KKT_ERR_INERTIA; the handle then holds the
 *     last trial's factor).
 * The inertia of S counts: in KKT_TF32 / KKT_BF16 mode a factor of S with the
 * wrong count is first redone FP64-accurately (as the refinement fallback
 * does), since its reduced-precision pivot signs can be wrong on an
 * ill-conditioned S. */
typedef struct {
  double delta_w_init; /* 1e-4 */
  double delta_w_min;  /* 1e-20 */
  double delta_w_max;  /* 1e40 */
  double grow_first;   /* 100 */
  double grow;         /* 8 */
  double shrink;       /* 1/3 */
  double delta_c;      /* 1e-8 */
  int32_t max_trials;  /* 40 */
  int32_t coupling_dual; /* 0 (default): the coupling variables are primal (expected inertia
                            (N*nP + nC, N*nD, 0), C shifted by +dw); 1: they are multipliers, as
                            in the paper's own MPOPF coupling (expected (N*nP, N*nD + nC, 0), C
                            shifted by -dc) */
} kkt_inertia_options;

typedef struct {
  double delta_w, delta_c; /* the shifts of the factor the handle holds */
  int32_t trials;          /* factorizations done (1: the unshifted factor was right) */
  int32_t reserved;
} kkt_inertia_result;

void kkt_default_inertia_options(kkt_inertia_options* opt);

/* kkt_factor with inertia correction (above).  Arguments as kkt_factor, plus
 * opt (NULL: defaults) and result (may be NULL).  Synchronizes `stream` after
 * every trial (the inertia is read on the host).  kkt_solve afterwards solves
 * the shifted system, whose matrix the refinement's residual also uses. */
kkt_status kkt_factor_inertia(kkt_handle* h, const double* a_vals, const double* b_vals,
                              const double* c_vals, int32_t on_device, void* stream,
                              const kkt_inertia_options* opt, kkt_inertia_result* result);

/* Solve K x = rhs for nrhs right-hand sides (stacked, each N*nA + nC long)
 * with the current factorization, refined in FP64 to opt.refine_tol.
 * rhs and x: host (on_device 0) or device (1) arrays.  Returns
 * KKT_ERR_NOT_CONVERGED when refinement stops above refine_tol (x then holds
 * the best iterate).  The convergence test sees every NaN and Inf: a
 * non-finite ||K||_inf or ||rhs||_inf (a NaN or Inf among the values) returns
 * KKT_ERR_NONFINITE at once; a non-finite iterate first takes the FP64-accurate
 * refactor of S in the reduced modes and, if it stays non-finite, returns
 * KKT_ERR_NONFINITE (rel_residual is then NaN).  Synchronizes `stream` (the
 * refinement reads its residual norm on the host). */
kkt_status kkt_solve(kkt_handle* h, const double* rhs, double* x, int32_t nrhs, int32_t on_device,
                     void* stream);

/* Statistics of the handle and of the last factor/solve (synchronizes the
 * handle's last stream). */
kkt_status kkt_get_info(kkt_handle* h, kkt_info* info);

/* Frees every device and host buffer of the handle.  NULL is accepted. */
kkt_status kkt_destroy(kkt_handle* h);

/* Static string for a status code. */
const char* kkt_status_string(kkt_status s);

/* Text of the last error on this thread ("" if none). */
const char* kkt_last_error(void);

/* One application of the current factorization to a device right-hand side,
 * allocating nothing.  The paper has no counterpart: this exists for callers
 * that cannot call cudaMalloc while they solve (a serving process that gives
 * all device memory to its own pool up front and must stay inside that
 * budget, or a latency-critical loop that cannot take the device-wide
 * synchronization an allocation may imply).
 *   rhs, x: device arrays of N*nA + nC doubles (caller-owned; rhs is read,
 *           x is written).  No refinement: x = (factored K)^{-1} rhs.  The
 *           call applies the same factorization as kkt_solve with its own
 *           kernels on the static work vectors (level solves over every
 *           supernode, a column-by-column solve with the factor of S), so x
 *           agrees with the first application inside kkt_solve to rounding,
 *           within the conditioning bound of K, not bit for bit.
 *   Work vectors come from one file-scope device array of 2^21 doubles
 *   (16 MiB) that every GPU loading this library holds until process exit;
 *   systems with N*nA + 2*N*k + 2*nC above that (k: rows of A carrying B's
 *   nonzeros, see kkt_info) are rejected with KKT_ERR_INVALID.
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device current); make that first call before any
 *   stream capture.  All calls share the array and it keeps the last call's
 *   contents: calls whose kernels overlap on the GPU (different streams,
 *   different handles) race on it and must be serialized by the caller.
 *   Needs an FP64-accurate factor of S (handles in KKT_FP64 or
 *   KKT_F64_EMULATED mode); otherwise returns KKT_ERR_STATE.
 *   Asynchronous with respect to the host; errors of the launches, and an
 *   error left pending on this thread by an earlier launch, are returned as
 *   KKT_ERR_CUDA. */
kkt_status kkt_solve_noalloc(kkt_handle* h, const double* rhs, double* x, void* stream);

/* ---- the steps of Algorithm 1 one at a time (Sec. 4.2), for a solve whose
 * blocks are spread over processes, one GPU each ----
 * Process p holds a handle analysed for its own blocks i in N_p (its share of
 * the periods) and the coupling columns they touch, c0 .. c0 + nC_p - 1
 * (re-indexed from 0); the root holds every coupling column and C, the others
 * a zero C.  Then (Algorithm 1):
 *   every p:  kkt_factor_blocks     A_i = L_i D_i L_i^T and S_p = C_p - sum B_i^T A_i^{-1} B_i
 *   reduce:   the root adds each S_p into the window (c0, c0) of its own S
 *             (kkt_schur_matrix, kkt_accumulate);
 *   root:     kkt_factor_schur      S = L_s D_s L_s^T
 *   every p:  kkt_solve_front       t_p = r_g,p - sum B_i^T A_i^{-1} r_i (r_g,p = 0 off the root)
 *   reduce:   the root adds each t_p into its t window (kkt_accumulate);
 *   root:     kkt_solve_coupling    x_g = S^{-1} t;  broadcast x_g
 *   every p:  kkt_solve_back        x_i = A_i^{-1} (r_i - B_i x_g) with its window of x_g.
 * FP64 refinement on the distributed K uses kkt_residual (the coupling rows
 * of each process's residual are its part of r_g - C x_g - sum B_i^T x_i, added
 * up at the root like t), kkt_abs_rowsums (the rows of |K|, for ||K||_inf) and
 * kkt_norm_inf.  The collectives are the caller's (torch.distributed in the
 * Python layer).  All arrays are device arrays of the handle's device, all
 * calls asynchronous on `stream` except kkt_norm_inf.  A handle with the
 * structured S (structured_s = 2) has no dense S: kkt_factor_blocks,
 * kkt_schur_matrix, kkt_factor_schur and kkt_schur_factor_copy return
 * KKT_ERR_INVALID for it; kkt_solve_front, kkt_solve_coupling and
 * kkt_solve_back work after kkt_factor. */

/* kkt_factor without the factor of S: block factors and the assembled S of
 * the handle's blocks (Algorithm 1: block factorization, local Schur
 * contributions and their accumulation; eq. SCform).  The Schur contraction
 * is FP64 in every mode.  kkt_solve needs kkt_factor_schur afterwards. */
kkt_status kkt_factor_blocks(kkt_handle* h, const double* a_vals, const double* b_vals, const double* c_vals,
                             int32_t on_device, void* stream);
/* The handle's S buffer: nC x nC doubles, column-major with leading dimension
 * *ld = nC, lower triangle (the strictly upper part is zero after
 * kkt_factor_blocks).  Owned by the handle until kkt_destroy.  After
 * kkt_factor_schur in the KKT_FP64 and KKT_F64_EMULATED modes it holds the
 * factor (L strictly below the diagonal, D on it); the TF32 and BF16 modes
 * factor a copy and keep S. */
kkt_status kkt_schur_matrix(kkt_handle* h, double** S, int64_t* ld);
/* Dense LDL^T of the handle's current S in its precision mode (Algorithm 1,
 * factorization of S; eq. SCsolve); needs kkt_factor_blocks first. */
kkt_status kkt_factor_schur(kkt_handle* h, void* stream);
/* The current factor of S as nC x nC doubles (device out; column-major, L
 * strictly below the diagonal, D on it, the upper part unspecified): the FP32
 * factor converted in the TF32 and BF16 modes. */
kkt_status kkt_schur_factor_copy(kkt_handle* h, double* out, void* stream);
/* The structured S (structured_s = 2; Sec. 4.3, eq. GlobalSchur) of the last
 * kkt_factor: its diagonal blocks S_d[0..N-1] into Sd and its subdiagonal
 * blocks S_o[0..N-2] (the block repeated in every row below the diagonal of
 * block column j) into So; each block n_s x n_s column-major, the blocks one
 * after another (device arrays, N n_s^2 and (N-1) n_s^2 doubles).
 * KKT_ERR_STATE before a kkt_factor, KKT_ERR_INVALID for a handle without the
 * structured S. */
kkt_status kkt_schur_blocks(kkt_handle* h, double* Sd, double* So, void* stream);
/* dst[i + j ld_dst] += src[i + j ld_src] for i < rows, j < cols (device
 * arrays; a vector is cols = 1).  The reduce of Algorithm 1 on the root. */
kkt_status kkt_accumulate(double* dst, int64_t ld_dst, const double* src, int64_t ld_src, int64_t rows,
                          int64_t cols, void* stream);
/* Front half of one application: z_i = L_i^{-1} P^T r_i for the handle's
 * blocks and t = r_g - sum_i B_i^T A_i^{-1} r_i (eq. SCsolve; rhs: N*nA + nC
 * doubles, t: nC).  Keeps z in the handle for kkt_solve_back. */
kkt_status kkt_solve_front(kkt_handle* h, const double* rhs, double* t, void* stream);
/* x_g = S^{-1} t with the current factor of S (t and xg distinct, nC each). */
kkt_status kkt_solve_coupling(kkt_handle* h, const double* t, double* xg, void* stream);
/* Back half after kkt_solve_front on the same handle: x_i = A_i^{-1} (r_i -
 * B_i x_g) for the handle's blocks (eq. SCsolve1); x (N*nA + nC) also gets
 * xg in its last nC entries. */
kkt_status kkt_solve_back(kkt_handle* h, const double* xg, double* x, void* stream);
/* rho = rhs - K x with the handle's values (block rows r_i - A_i x_i - B_i x_g;
 * coupling rows r_g - C x_g - sum_i B_i^T x_i over the handle's blocks). */
kkt_status kkt_residual(kkt_handle* h, const double* rhs, const double* x, double* rho, void* stream);
/* out (N*nA + nC doubles): the absolute row sums of the handle's K; the
 * coupling rows hold sum |B column| + sum |C row| over the handle's blocks. */
kkt_status kkt_abs_rowsums(kkt_handle* h, double* out, void* stream);
/* *out = max |v_i| over n device doubles (NaN if any entry is NaN);
 * synchronizes `stream`. */
kkt_status kkt_norm_inf(kkt_handle* h, const double* v, int64_t n, double* out, void* stream);

/* ---- slack elimination around the solve (Sec. 2, eqs. SCOPFhessian,
 * SCOPFhessianSymmetric, SCOPFslackAtEnd, SCOPFhessianReduced,
 * SCOPFslackReduction, SCOPFhessianSymmetricRecovery) ----
 * The barrier method's Newton system in (dx, ds, dlE, dlI, dz, dy) is reduced
 * to K by eliminating the bound multipliers z, y and the slacks s of the
 * inequality rows; after the solve the eliminated unknowns are recovered:
 *   A_i: primal diagonals += z/x; inequality-row diagonals = -(s/y) (-L_s^-1,
 *        the base value there is replaced); C's diagonal += z_g/x_g;
 *   rhs: primal rows -(l_a + l_e/x); equality rows -l_c; inequality rows
 *        -(l_d + (s/y)(l_b + l_f/s));
 *   ds = (s/y)(dlI - l_b - l_f/s), dz = -(l_e + z dx)/x, dy = -(l_f + y ds)/s.
 * Every primal variable (the nP primal rows of every block and the nC
 * coupling variables) has a bound with multiplier z; the inequality rows are
 * multiplier rows of A.  The elimination assumes s/y well away from 0 and
 * infinity, as the paper notes.  All arrays are device arrays; the calls are
 * asynchronous on `stream`; each entry is computed by one thread in the order
 * written above, with round-to-nearest and no fused multiply-adds. */
typedef struct kkt_slack kkt_slack;
typedef struct {
  const double *x, *z;   /* N*nP + nC: primal variables (blocks, then coupling) and their bound multipliers, > 0 */
  const double *s, *y;   /* N*n_ineq: slacks of the inequality rows and their bound multipliers, > 0 */
  const double *la, *le; /* N*nP + nC: residuals l_a (stationarity) and l_e (complementarity of x, z) */
  const double *lcd;     /* N*(nA - nP): per block the multiplier rows in row order, l_d on the
                            inequality rows and l_c on the others */
  const double *lb, *lf; /* N*n_ineq: residuals l_b and l_f (complementarity of s, y) */
} kkt_ipm_state;
/* The inequality rows of the handle's pattern: n_ineq increasing rows of A in
 * [nP, nA), the same in every block (host array, copied). */
kkt_status kkt_slack_create(kkt_handle* h, int32_t n_ineq, const int32_t* ineq_rows, kkt_slack** out);
/* a_vals (N*nnzA), c_vals (as kkt_factor) and rhs (N*nA + nC) of the reduced
 * system from the base values (H and J without the bound terms) and the
 * state; a_vals may be a_base and c_vals may be c_base (in place). */
kkt_status kkt_slack_reduce(kkt_slack* sl, const kkt_ipm_state* st, const double* a_base, const double* c_base,
                            double* a_vals, double* c_vals, double* rhs, void* stream);
/* ds, dy (N*n_ineq) and dz (N*nP + nC) from the solution dsol of the reduced
 * system (N*nA + nC). */
kkt_status kkt_slack_recover(kkt_slack* sl, const kkt_ipm_state* st, const double* dsol, double* ds, double* dz,
                             double* dy, void* stream);
kkt_status kkt_slack_destroy(kkt_slack* sl);

/* ---- batching and serving (no counterpart in the paper; the workload's many
 * independent systems of different grids and horizons) ---- */

/* Factor and solve n independent systems, handles[i] with the values and
 * right-hand side of system i (all host or all device arrays, as in kkt_factor
 * and kkt_solve).  Systems are spread round-robin over `streams` CUDA streams
 * (<= 0: 8), one host worker per stream, so the kernels of different systems
 * overlap on the GPU.  statuses (may be NULL) receives each system's status;
 * the return value is the first failure other than KKT_ERR_NOT_CONVERGED, else
 * KKT_ERR_NOT_CONVERGED if any system stopped above refine_tol, else KKT_OK.
 * Every handle must appear at most once. */
kkt_status kkt_batch_factor_solve(kkt_handle* const* handles, int32_t n, const double* const* a_vals,
                                  const double* const* b_vals, const double* const* c_vals,
                                  const double* const* rhs, double* const* x, int32_t on_device,
                                  int32_t streams, kkt_status* statuses);

/* A request loop with continuous batching.  Up to `slots` requests run at once,
 * each on its own stream; a queued request is admitted as soon as a slot is
 * free, its handle is idle, and the device bytes of the handles in flight stay
 * within device_budget_bytes (0 = no budget; a request is always admitted when
 * nothing is in flight).  Handles stay resident: repeated requests on one
 * handle reuse its analysis. */
typedef struct kkt_server kkt_server;
kkt_status kkt_server_create(int32_t slots, int64_t device_budget_bytes, kkt_server** out);
/* Queue one KKT solve (factor + refined solve) on handle h; the arrays must
 * stay valid until the request completes.  *request_id identifies it. */
kkt_status kkt_server_submit(kkt_server* s, kkt_handle* h, const double* a_vals, const double* b_vals,
                             const double* c_vals, const double* rhs, double* x, int32_t on_device,
                             int64_t* request_id);
/* Result of a request: with wait != 0 blocks until it completes; with wait == 0
 * returns KKT_ERR_STATE while it is pending.  *status is the request's status,
 * *latency_ms the time from submit to completion of its solve.  A result is
 * collected once: an id that is neither queued, running nor finished and
 * uncollected gives KKT_ERR_INVALID (instead of waiting forever). */
kkt_status kkt_server_poll(kkt_server* s, int64_t request_id, int32_t wait, kkt_status* status,
                           double* latency_ms);
/* Drains the queue, joins the workers and frees the streams (and the cached handles). */
kkt_status kkt_server_destroy(kkt_server* s);
/* A pattern cache: requests submitted with kkt_server_submit_pattern name a
 * pattern by a caller-chosen key >= 0; the server analyses the pattern (with
 * options opt, NULL for the defaults) at the first request on the key, inside
 * that request's latency, and keeps the handle resident for later requests on
 * the key.  Admission of a new pattern is by free device memory: before an
 * analysis, while cudaMemGetInfo reports less than reserve_bytes free, the
 * idle resident handle used least recently is destroyed; an analysis that
 * still runs out of memory evicts one more and retries, and fails with
 * KKT_ERR_OOM once none is left.  Call before the first pattern request. */
kkt_status kkt_server_set_cache(kkt_server* s, const kkt_options* opt, int64_t reserve_bytes);
/* Queue one KKT solve of the pattern `key` (the pattern's arrays and the
 * values must stay valid until the request completes; the pattern is read only
 * at the key's first request or after an eviction). */
kkt_status kkt_server_submit_pattern(kkt_server* s, int64_t key, const kkt_pattern* pat, const double* a_vals,
                                     const double* b_vals, const double* c_vals, const double* rhs, double* x,
                                     int32_t on_device, int64_t* request_id);
/* Resident patterns, analyses done and handles evicted so far. */
kkt_status kkt_server_cache_info(kkt_server* s, int64_t* resident, int64_t* analyses, int64_t* evictions);

/* ---- per-kernel device times (with kkt_options.time_kernels) ----
 * Families: 0 the emulated-FP64 trailing update (k_tc_update_emu: dense tails
 * of the block factors, and S in KKT_F64_EMULATED or a fallback), 1 the TF32
 * update of S with 256-wide outer panels (k_tc_update_wide), 2 the 64-wide
 * TF32/BF16 update (k_tc_update), 3 the FP64 dense update on the CUDA cores
 * (k_dense_update: S in KKT_FP64, the FP64 tails), 4 the supernodal updates of
 * the block factor (k_factor_update), 5 the dense diagonal blocks of the
 * blocked factors (k_dense_diag_t), 6 the emulated-FP64 update with K = 256
 * of the 256-wide outer panels (k_tc_update_emu_wide), 7 the emulated-FP64
 * panels of those factors (k_tc_panel_emu, timed with the launch that forms
 * its operands: W = L11^{-1} and the digit images of W and A21).  flops: the
 * algorithmic FP64-equivalent flops of the launches (2 per multiply-add on the
 * entries of the lower triangle they update; for a panel, 2 per multiply-add
 * of the row solves it replaces). */
typedef struct {
  int64_t launches;     /* launches of the family in the handle's last factor (and fallback) */
  double ms_total;      /* sum of their device durations (CUDA events on their streams) */
  double ms_max;        /* the longest one */
  double flops;         /* their algorithmic flops */
} kkt_kernel_stat;
/* Statistics of family `family` (0..7); synchronizes the handle. */
kkt_status kkt_kernel_stats(kkt_handle* h, int32_t family, kkt_kernel_stat* out);

/* Measured FP64 FMA throughput of the current device in GFLOP/s (8
 * independent FMA chains per thread, best of 5 launches).  The FP64-bound
 * phases report their roofline fraction against it. */
kkt_status kkt_measure_fp64_peak(double* gflops);

/* Diagnostic: for n device doubles d, recip[i] = the reciprocal the factor
 * kernels take of a pivot d[i] (an FP32 seed and two FP64 Newton-Raphson
 * steps; CUDA's division for |d| outside [1e-36, 1e36]) and quotient[i] =
 * 1.0 / d[i] by CUDA's FP64 division, so that tests can bound the
 * difference.  Device arrays; asynchronous on `stream`. */
kkt_status kkt_probe_pivot_reciprocal(const double* d, int64_t n, double* recip, double* quotient, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* KKT_SCHUR_H */
