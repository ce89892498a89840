/*
 * ddg.h -- C ABI of the GB300 (sm_103a) DDG two-level Schwarz PCG solver.
 *
 * Method: Edwards & Bridson, "The Discretely-Discontinuous Galerkin Coarse
 * Grid for Domain Decomposition" (arXiv 1504.00907).
 *   - Sec. 1: the input is a sparse SPD system A u = f.
 *   - Sec. 4, Fig. 1: the coarse restriction R0 has one row per (subdomain,
 *     generating vector): column j of F restricted to the non-overlapping
 *     subdomain i, orthonormalised per subdomain, rank-deficient columns
 *     dropped; coarse dofs numbered subdomain-major, generator-minor.
 *     A0 = R0 A R0^T (Galerkin projection).
 *   - Sec. 6: overlapping subdomains grow each partition by Delta layers;
 *     local matrices A_i = R~_i A R~_i^T are solved exactly; one pass of
 *     multiplicative Schwarz (pre-smoother), the coarse correction, and the
 *     pass in reverse order (post-smoother) form a symmetric preconditioner.
 *   - Sec. 7: conjugate gradient from u0 = 0 with that preconditioner.
 *
 * Conventions for every entry point:
 *   - Every call returns a ddg_status; nothing throws across the ABI.
 *     ddg_last_error(h) gives a message for the last failing call on h
 *     (ddg_last_error(NULL) for a failing ddg_setup or a failing call that
 *     takes no handle).
 *   - "host" pointers are read during the call only and stay owned by the
 *     caller.  "device" pointers are caller-owned CUDA device memory on the
 *     current device; the library never frees them.  All device work is
 *     enqueued on the stream given to ddg_setup (or ddg_set_stream) and the
 *     calls that return scalars synchronise that stream before returning.
 *   - Vectors are FP64, natural (caller) dof order, length n.  Multi-RHS
 *     blocks are dof-major: entry (dof g, rhs j) at g * m + j.
 *   - One handle must not be used from two host threads at once.  A handle
 *     remembers the device that was current at its setup and makes it
 *     current for the duration of every call on it, so it may be called
 *     from any host thread.
 */
#ifndef DDG_H
#define DDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ddg_handle_s* ddg_handle;   /* opaque, library-owned */

typedef enum {
    DDG_OK = 0,
    DDG_EINVAL = 1,       /* invalid argument (sizes, ids, pointers, options) */
    DDG_ENOMEM = 2,       /* device allocation failed */
    DDG_ENOTSPD = 3,      /* a local or the coarse Cholesky met a non-positive pivot */
    DDG_EBREAKDOWN = 4,   /* CG breakdown: p^T A p <= 0 or a NaN */
    DDG_ENOCONV = 5,      /* maxit reached, or the recurrence met tol but the true
                             residual stayed above it after 3 restarts of CG from the
                             true residual; u holds the last iterate */
    DDG_ETIMEOUT = 6,     /* a bounded device wait ran out (spin_budget_ms); the
                             result is not valid, the handle stays usable */
    DDG_ECUDA = 7         /* a CUDA runtime call failed */
} ddg_status;

/* arithmetic of the preconditioner apply (local solves, coarse solve,
 * restriction/prolongation); the CG recurrence is always FP64 */
enum { DDG_PREC_FP64 = 0, DDG_PREC_FP32 = 1, DDG_PREC_BF16 = 2 };
/* Sec. 6 overlap: GRAPH = graph distance Delta in the graph of A (the
 * paper's definition); BOX = L-infinity grid distance Delta (needs the grid
 * shape in ddg_matrix; dofs must be in natural x-fastest grid order) */
enum { DDG_OVERLAP_GRAPH = 0, DDG_OVERLAP_BOX = 1 };
/* representation of the exact local solves A_i^{-1} (Sec. 6): dense inverses
 * (packed symmetric tiles; overlapping subdomains of at most 3072 dofs) or
 * banded Cholesky factors of A_i in its ascending dof order (any size; the
 * work grows with the half-bandwidth).  AUTO takes the inverses when every
 * block fits them, else the band. */
enum { DDG_LOCAL_AUTO = 0, DDG_LOCAL_INV = 1, DDG_LOCAL_BAND = 2 };
/* tensor-core operands of the batched local solve (Sec. 6's exact local
 * solves as GEMMs over the right-hand sides): none, BF16 or TF32 */
enum { DDG_TC_OFF = 0, DDG_TC_BF16 = 1, DDG_TC_TF32 = 2 };
/* ordering of the exact coarse Cholesky factor of A0 (Sec. 4): the natural
 * subdomain order (a band; its solve is a block-bidiagonal recurrence) or
 * nested dissection of the subdomain graph (a multifrontal factor, far
 * fewer entries on 3D problems, a solve of a few dependent steps per level
 * of the dissection tree) */
enum { DDG_COARSE_BAND = 0, DDG_COARSE_ND = 1 };
/* CG beta: Fletcher-Reeves (textbook) or Polak-Ribiere (flexible) */
enum { DDG_BETA_FR = 0, DDG_BETA_PR = 1, DDG_BETA_AUTO = 2 };
/* optional structure of A that enables a matrix-free SpMV for the FP64
 * CG products; the CSR must still describe the same matrix */
enum {
    DDG_STENCIL_NONE = 0,
    DDG_STENCIL_5PT_2D = 1,   /* [4, -1], Dirichlet, nx x ny */
    DDG_STENCIL_7PT_3D = 2,   /* [6, -1], Dirichlet, nx x ny x nz */
    DDG_STENCIL_13PT_2D = 3,  /* clamped biharmonic (CSR SpMV is used) */
    DDG_STENCIL_VAR7_3D = 4,  /* cell-centred variable coefficient */
    DDG_STENCIL_Q1_ELASTIC = 5 /* trilinear hexahedral linear elasticity on ne^3 elements
                                  of the unit cube, nodes of the x = 0 face clamped:
                                  nx, ny, nz = ne, ne + 1, ne + 1 unclamped nodes,
                                  dofs_per_node = 3 (CSR SpMV is used) */
};

typedef struct {
    int precision;        /* DDG_PREC_*, default DDG_PREC_FP64 */
    int keep_precisions;  /* bitmask of (1 << DDG_PREC_*) local-inverse copies
                             to keep for ddg_set_precision; 0 = `precision` only */
    int overlap_mode;     /* DDG_OVERLAP_*, default GRAPH */
    int beta;             /* DDG_BETA_*, default AUTO (FR for FP64, PR otherwise) */
    int maxit;            /* default 1000 (Sec. 7 stops CG at 1000 iterations) */
    int use_coarse;       /* 1 = two-level (default), 0 = one-level Schwarz */
    double rank_tol;      /* Sec. 4 rank drop: keep column j while |R_jj| >
                             rank_tol * |R_00|; default 1e-10 */
    int chunk_tiles;      /* local-solve work item size in 32x32 tiles; 0 = auto */
    int tensor_cores;     /* DDG_TC_*, default OFF.  BF16: also keep BF16 128x32 slabs
                             of every A_i^{-1}; ddg_solve_batch in DDG_PREC_BF16 then
                             runs its local solves on the tcgen05 tensor cores (BF16 x
                             BF16, FP32 accumulate).  TF32: keep the slabs in FP32
                             rounded to TF32 (twice the bytes); ddg_solve_batch in
                             DDG_PREC_FP32 then runs its local solves as tcgen05 TF32 x
                             TF32 products with FP32 accumulation (the residual is
                             rounded to TF32 too) */
    int dedup_local;      /* 1: subdomains whose local matrices A_i are equal entry for
                             entry (rows and columns in ascending dof order) share one
                             stored inverse (constant-coefficient problems: the
                             interior subdomains); the results do not change; default 0 */
    double spin_budget_ms; /* time limit of every device-side wait (the mbarrier waits
                             of the tensor-core local solve), measured on the GPU's
                             global timer; a wait that runs out makes the call return
                             DDG_ETIMEOUT; default 1000 (0 also means 1000) */
    int autotune;         /* 1: choose the launch shapes of the local solves by timing
                             candidates on this handle's data at setup (warps per CTA
                             4/8, tiles per work item 48/96/192 unless chunk_tiles is
                             set, tile rows per item 8/16) and, for tensor-core batched
                             solves, the operand ring depth 3/4/6 per column count; a
                             choice is kept for the process per (largest block, number
                             of subdomains and colours, columns, precision), so handles
                             of one class share it; results change at rounding level
                             with the shapes; default 0 (8 warps, 96 tiles, 16 rows, 4
                             stages) */
    int local_repr;       /* DDG_LOCAL_*, default AUTO.  With BAND: the BF16 precision
                             uses the FP32 factors, tensor_cores and dedup_local are not
                             available, ddg_solve_batch solves its columns one at a time,
                             and the half-bandwidth must be at most 1024 */
    int coarse_order;     /* DDG_COARSE_*, default ND (the nested-dissection factor is
                             smaller and its solve shorter than the natural-order band
                             on the grids measured; BAND keeps the natural order) */
} ddg_options;

typedef struct {
    int64_t n;               /* rows = columns */
    const int64_t* rowptr;   /* host [n + 1] */
    const int32_t* col;      /* host [nnz], column ids in [0, n), sorted per row */
    const double* val;       /* host [nnz]; A must be symmetric positive definite */
    int dim;                 /* grid dimension (2 or 3) for BOX overlap, else 0 */
    int nx, ny, nz;          /* grid shape (x fastest); nz = 1 in 2D */
    int dofs_per_node;       /* interleaved dofs per grid node (1 for scalars) */
    int stencil_kind;        /* DDG_STENCIL_* */
    const double* coef;      /* host, needed by ddg_grad_coeff: VAR7: cell coefficients
                                kappa[nz][ny][nx]; Q1_ELASTIC: shear modulus per element
                                mu[ne][ne][ne] (x fastest); else NULL */
} ddg_matrix;

typedef struct {
    int64_t n;            /* fine dofs */
    int nsub;             /* subdomains */
    int ncolours;         /* colours of the multiplicative sweep */
    int n0;               /* coarse dimension after rank drop */
    int kmax;             /* generators per subdomain (columns of F) */
    int max_local;        /* largest overlapping subdomain |Omega~_i| */
    int64_t sum_local;    /* sum of |Omega~_i| */
    int64_t local_tiles;  /* size of all packed local inverses in 32x32-tile units (1024 values) */
    int coarse_band;      /* half-bandwidth of A0 in natural coarse order */
    int coarse_blocks;    /* super-blocks of the coarse block-bidiagonal factor */
    double setup_ms;      /* wall time of ddg_setup */
    int precision;        /* current preconditioner precision */
    int local_inverses;   /* stored local inverses: nsub, fewer with dedup_local */
    int graph_solve;      /* 1: the last single-vector solve ran as one CUDA graph launch
                             (its CG loop decided on the device); 0: driven from the host
                             (tracing on, or DDG_NO_GRAPHS set); -1: conditional graphs
                             are unavailable, every solve is driven from the host */
    int ls_warps;         /* warps per CTA of the single-vector local solve */
    int ls_chunk_tiles;   /* tiles per local-solve work item (target) */
    int ls_band_rows;     /* tile rows per local-solve work item (limit) */
    int tc_stages;        /* operand ring depth of the tensor-core local solve */
    int tuned;            /* 1: the shapes above were chosen by the autotuner */
    int local_repr;       /* DDG_LOCAL_INV or DDG_LOCAL_BAND (what setup chose) */
    int local_band;       /* half-bandwidth of the local matrices (BAND), else 0 */
    int64_t local_elems;  /* stored elements of all local operators (one precision) */
    int coarse_order;     /* DDG_COARSE_* */
    int coarse_fronts;    /* ND: fronts of the dissection tree */
    int coarse_levels;    /* ND: levels of the dissection tree */
    int64_t coarse_elems; /* stored elements of the coarse solve (one precision) */
} ddg_info;

/* Fill *opt with the defaults listed above. */
void ddg_default_options(ddg_options* opt);

/*
 * Build the preconditioner for A (Sec. 4 and Sec. 6).
 *   A          host CSR (+ optional grid/stencil description), copied.
 *   partition  host int32[n]: node -> non-overlapping subdomain id; ids
 *              must cover [0, nsub) (empty subdomains are rejected).
 *   F          host FP64 [n * k], column-major (column j at F + j * n): the
 *              generating vectors; 1 <= k <= 96, or k = 0 with use_coarse = 0.
 *              With k > 32, ddg_solve_batch solves its columns one at a time.
 *   overlap    Delta >= 0 layers.
 *   stream     cudaStream_t for all work of this handle (NULL = default).
 *   out        receives the handle.
 * Errors: DDG_EINVAL (bad sizes/ids/options), DDG_ENOTSPD (a local or the
 * coarse factorisation failed), DDG_ENOMEM, DDG_ECUDA.
 */
ddg_status ddg_setup(const ddg_matrix* A, const int32_t* partition, const double* F, int k,
                     int overlap, const ddg_options* opt, void* stream, ddg_handle* out);

/*
 * Three-level V-cycle (Sec. 6): as ddg_setup, but inside the preconditioner
 * the exact coarse solve A0^{-1} is replaced by one application of the
 * two-level method to A0, built from the coarsened generators F0 = R0 F on
 * coarse-level subdomains that group the fine subdomains (no Cholesky factor
 * of A0 is formed; the coarsest matrix A1 = R1 A0 R1^T is factorised).
 *   coarse_partition  host int32[nsub]: fine subdomain -> coarse-level
 *              subdomain id >= 0.  Groups without coarse dofs are dropped
 *              and the rest numbered in ascending id order.
 * The coarse level uses the same overlap Delta, grown by graph distance in
 * the graph of A0, and the same precision, keep_precisions and rank_tol;
 * tensor_cores applies to the fine level only.  Every solve entry point
 * accepts the handle; ddg_solve_batch then solves its columns one at a time.
 * Overlapping coarse-level subdomains are limited to 3072 coarse dofs, like
 * fine ones.
 * Errors: as ddg_setup; DDG_EINVAL also for coarse_partition == NULL or
 * use_coarse == 0; a failure on the coarse level is reported with the
 * prefix "coarse level of the V-cycle: " in ddg_last_error(NULL).
 */
ddg_status ddg_setup_vcycle(const ddg_matrix* A, const int32_t* partition,
                            const int32_t* coarse_partition, const double* F, int k, int overlap,
                            const ddg_options* opt, void* stream, ddg_handle* out);

/*
 * Replace the generators of a built handle (Sec. 4): R0, A0 and its factor
 * are rebuilt from F (host FP64 [n * k], column-major, 1 <= k <= 96); the
 * overlapping subdomains, colouring and local inverses are kept, so a sweep
 * over coarse spaces factorises the local blocks once.  The result equals a
 * handle set up with F from the start.  Also turns the coarse level on for a
 * handle built with use_coarse = 0.  Not for V-cycle handles (DDG_EINVAL).
 * Errors: DDG_EINVAL, DDG_ENOTSPD, DDG_ENOMEM, DDG_ECUDA (the handle then has
 * no usable coarse space and must be destroyed).
 */
ddg_status ddg_set_generators(ddg_handle h, const double* F, int k);

/*
 * Solve A u = f by PCG from u0 = 0 (Sec. 7): stop when the recurrence
 * residual satisfies ||r||_2 <= tol ||f||_2 and the true residual does too
 * (a recurrence that drifts is replaced by the true residual and CG
 * restarts, at most 3 times).  f, u: device FP64 [n], distinct buffers (u is
 * cleared before f is read, so f == u is rejected with DDG_EINVAL).
 * *iters: iterations taken; *relres: true relative residual
 * ||f - A u|| / ||f||.  Either output may be NULL.
 * Errors: DDG_ENOCONV (maxit reached, or the true residual still above tol
 * after the third restart; u is the last iterate and ddg_last_error says
 * which), DDG_EBREAKDOWN, DDG_EINVAL, DDG_ECUDA.
 */
ddg_status ddg_solve(ddg_handle h, const double* f, double* u, double tol, int* iters,
                     double* relres);

/* Same as ddg_solve with host FP64 f and u: the copies to and from the
 * device are part of the call. */
ddg_status ddg_solve_host(ddg_handle h, const double* f_host, double* u_host, double tol,
                          int* iters, double* relres);

/*
 * Multi-RHS solve: F and U are device FP64 [n * m], dof-major.  Each column
 * runs its own CG (own alpha, beta, convergence); the preconditioner is
 * applied to all unconverged columns at once.  iters: host int[m] or NULL;
 * relres: host double[m] or NULL.  With the FP64 preconditioner, a V-cycle
 * handle or more than 32 generators per subdomain the columns are solved
 * one at a time.  Errors: as ddg_solve (the worst column's status), and
 * DDG_ETIMEOUT when a bounded wait of the tensor-core local solve ran out.
 */
ddg_status ddg_solve_batch(ddg_handle h, const double* F, double* U, int m, double tol,
                           int* iters, double* relres);

/*
 * Many independent problems of uneven sizes at once: problem p (handle
 * hs[p], which must be distinct handles, each with its own stream for the
 * problems to overlap on the GPU) solves F[p] (device FP64 [n_p * m[p]],
 * dof-major) into U[p], as ddg_solve_batch would (m[p] = 1: ddg_solve).
 * The problems run concurrently from one host thread each.  iters / relres:
 * host arrays of sum(m) entries (problem-major) or NULL.  Returns the first
 * non-OK status of any problem (its message: ddg_last_error(hs[p])).
 */
ddg_status ddg_solve_many(ddg_handle* hs, int nprob, const double* const* F, double* const* U,
                          const int* m, double tol, int* iters, double* relres);

/* Adjoint solve lambda = A^{-T} g for a loss gradient g = dL/du (device
 * [n], distinct from lambda); A is symmetric, so this reuses the
 * preconditioner and CG.  Statuses as ddg_solve. */
ddg_status ddg_adjoint(ddg_handle h, const double* dLdu, double* lambda, double tol,
                       int* iters, double* relres);

/* Coefficient gradient dL/dc = -lambda^T (dA/dc) u (lambda = A^{-1} dL/du,
 * u = A^{-1} f) for the coefficient array c given at setup: VAR7 handles:
 * c = kappa per cell, dcoef device [n] (chain rule through the harmonic-mean
 * faces); Q1_ELASTIC handles: c = mu per element, dcoef device [ne^3]
 * (dL/dmu_e = -lambda_e^T K^mu_e u_e).  lambda, u: device [n]. */
ddg_status ddg_grad_coeff(ddg_handle h, const double* lambda, const double* u, double* dcoef);

/* One preconditioner application z = M^{-1} r (Sec. 6), r and z device
 * FP64 [n], in the handle's current precision. */
ddg_status ddg_apply_preconditioner(ddg_handle h, const double* r, double* z);

/* Coarse correction alone: z = R0^T A0^{-1} R0 r (Sec. 4). */
ddg_status ddg_coarse_correction(ddg_handle h, const double* r, double* z);

/* y = A x in FP64 (device [n]). */
ddg_status ddg_spmv(ddg_handle h, const double* x, double* y);

/* Test hooks of the bounded device waits (the paper has no counterpart).
 * DDG_DEBUG_TC_NO_COPIES: the producer thread of the tensor-core local solve
 * issues no copies, so no copy is in flight and the MMA thread's first wait
 * runs out after spin_budget_ms; the kernel records the timeout, frees its
 * tensor memory and returns, and ddg_solve_batch returns DDG_ETIMEOUT.
 * flags = 0 restores normal operation. */
enum { DDG_DEBUG_TC_NO_COPIES = 1 };
ddg_status ddg_set_debug(ddg_handle h, int flags);

/* Switch the preconditioner precision (must be among keep_precisions). */
ddg_status ddg_set_precision(ddg_handle h, int precision);
ddg_status ddg_set_stream(ddg_handle h, void* stream);
ddg_status ddg_get_info(ddg_handle h, ddg_info* info);
/* host int32[nsub]: colour of every subdomain (sweep order = colour-major,
 * ids ascending inside a colour; the post-smoother is the exact reverse). */
ddg_status ddg_get_colouring(ddg_handle h, int32_t* colour);
/* host int32[nsub + 1]: coarse dof offsets per subdomain (after rank drop). */
ddg_status ddg_get_coarse_offsets(ddg_handle h, int32_t* offsets);
/* host double[max_len]: recurrence residual history ||r_k|| / ||f|| of the
 * last single-RHS solve, k = 0..iters; returns the count in *len. */
ddg_status ddg_get_history(ddg_handle h, double* hist, int max_len, int* len);

/* Sec. 7: the CG coefficients of the last single-vector solve on h
 * (ddg_solve, ddg_solve_host, ddg_adjoint), of its longest stretch without
 * a true-residual restart (the whole solve when there was none):
 * alpha_j for j < *len and beta_j for j < *len - 1 (beta_j forms
 * p_{j+1} = z_{j+1} + beta_j p_j).  Host arrays of max_len entries; *len
 * receives the number of alphas (both arrays may be NULL to query it). */
ddg_status ddg_get_cg_coefficients(ddg_handle h, double* alpha, double* beta, int max_len, int* len);

/* Sec. 7: condition estimate from m >= 1 CG steps (host only, no handle, no
 * GPU).  The Lanczos tridiagonal of CG has diagonal 1/alpha_0 and
 * 1/alpha_j + beta_{j-1}/alpha_{j-1}, off-diagonal sqrt(beta_j)/alpha_j; its
 * extreme eigenvalues (bisection on Sturm counts, to a relative 1e-14)
 * estimate those of M^{-1} A.  iter_bound (may be NULL) receives the CG
 * bound ln(2/tol) / ln((sqrt(k)+1)/(sqrt(k)-1)) for k = lambda_max/lambda_min
 * (0 when k <= 1), the iterations that reduce the A-norm error by tol.
 * Errors: DDG_EINVAL for m < 1, NULL arrays or outputs, tol outside (0, 1),
 * or a non-positive alpha or negative beta. */
ddg_status ddg_condition_estimate(const double* alpha, const double* beta, int m, double tol,
                                  double* lambda_min, double* lambda_max, double* iter_bound);

/* ---- tracing: per kernel class, launches are always counted; CUDA-event
 * timing of each launch (on the handle's stream) is on for the classes in
 * the mask given to ddg_profile.  bytes are the algorithmic bytes of the
 * timed launches (local solve: the packed upper triangle of every A_i^{-1}
 * of the colour, n_i (n_i + 1) / 2 elements, plus the local residual read and
 * z read + write; no tile padding counted). */
enum {
    DDG_K_LOCAL_SOLVE = 0,    /* packed-inverse GEMV + scatter, one per colour */
    DDG_K_LOCAL_RESIDUAL = 1, /* (r - A z) gathered on the colour's subdomains */
    DDG_K_COARSE = 2,         /* restrict, block-bidiagonal solves, prolong */
    DDG_K_SPMV = 3,           /* FP64 SpMV of the CG recurrence */
    DDG_K_CG = 4,             /* CG vector updates, dots, conversions */
    DDG_K_COUNT = 5
};
typedef struct {
    int64_t launches;   /* kernels launched since the last ddg_profile(h, mask) */
    int64_t timed;      /* launches that were timed with CUDA events */
    double ms;          /* summed event durations of the timed launches */
    double bytes;       /* algorithmic bytes of the timed launches */
} ddg_kernel_stat;
/* Reset all counters and time the classes whose bit (1 << DDG_K_*) is set. */
ddg_status ddg_profile(ddg_handle h, int timed_mask);
/* stats: host ddg_kernel_stat[DDG_K_COUNT]; synchronises the stream. */
ddg_status ddg_get_kernel_stats(ddg_handle h, ddg_kernel_stat* stats);

/* ---- no-allocation entry point (the paper has no counterpart) ----
 * y = A x and xAx = x^T A x for a caller-owned FP64 CSR matrix, without a
 * handle and without allocating device memory: for callers that cannot call
 * cudaMalloc (a host framework's caching allocator owns the device memory, a
 * fixed memory budget set at start-up, a caller inside another library's
 * critical section).  Same arithmetic as the library's CSR SpMV with the
 * fused dot of the CG recurrence (deterministic block-order reduction).
 *   n       rows, 0 <= n <= DDG_NOALLOC_MAX_ROWS, else DDG_EINVAL
 *   rowptr, col, val, x   device inputs (int64 [n+1], int32 [nnz], FP64 [nnz], FP64 [n])
 *   y       device output FP64 [n];  xAx  device output, one FP64
 *   stream  cudaStream_t (NULL = default stream)
 * Scratch: one file-scope static device array (32 KB of block partial sums
 * plus a ticket counter) that every GPU loading the library holds until the
 * process exits.  The first call on a device looks up that array's device
 * address (which may load the module): make that first call before any
 * stream capture.  All calls share the array, so calls whose kernels
 * overlap on the GPU (different streams, different threads) race; each call
 * clears the ticket it needs at zero on its stream.  Errors: DDG_EINVAL (size
 * or null pointer), DDG_ECUDA; the message is in ddg_last_error(NULL). */
#define DDG_NOALLOC_MAX_ROWS 1048576
ddg_status ddg_spmv_dot_noalloc(int64_t n, const int64_t* rowptr, const int32_t* col,
                                const double* val, const double* x, double* y, double* xAx,
                                void* stream);

ddg_status ddg_destroy(ddg_handle h);
const char* ddg_last_error(ddg_handle h);
const char* ddg_status_string(ddg_status s);

#ifdef __cplusplus
}
#endif
#endif /* DDG_H */
