/*
 * wd.h — C ABI of the GB300 sparse direct solver for wavelet-compressed
 * nonlocal operators (Harbrecht & Multerer, "A fast direct solver for nonlocal
 * operators in wavelet coordinates").
 *
 * The operation: given the symmetric positive definite compressed system
 * matrix A (Theorem 3.1), compute a nested-dissection permutation P and the
 * Cholesky factor P A P^T = L L^T (Section 4, Lemma and the block form of
 * P A P^T), then apply the exact inverse of the compressed matrix to
 * right-hand sides, log det A, and Gaussian random field samples P^T L z
 * (Section 5.3, Eq. CholFastField with an orthonormal basis, G = I).
 *
 * Conventions for every call:
 *  - A is passed as its LOWER triangle in compressed sparse column form,
 *    0-based, diagonal first in every column, row indices strictly
 *    increasing: colptr[n+1] (int64), rowidx[nnz] (int32), values[nnz]
 *    (double, same order as rowidx).
 *  - Dense blocks (right-hand sides, samples) are column-major with a leading
 *    dimension, in the ORIGINAL (unpermuted) index order.
 *  - Pointers are borrowed for the duration of the call; the library copies
 *    what it keeps.  The handle owns all internal host and device memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls are ordered on that stream; every call documented as
 *    synchronous synchronizes it before returning.
 *  - Calls come in the order create -> analyze -> factor -> {solve, logdet,
 *    apply_L, selinv}; out of order calls return WD_ERR_STATE.  A new
 *    wd_factor on the same pattern reuses the analysis.
 *  - Errors leave the handle usable; an error in wd_factor leaves no factor.
 *  - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef WD_H
#define WD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wd_ctx *wd_handle;

typedef enum {
    WD_OK = 0,
    WD_ERR_INVALID_ARG = 1,     /* null pointer, negative size, bad option   */
    WD_ERR_PATTERN = 2,         /* malformed CSC (unsorted, missing diagonal,
                                   out of range, duplicate)                  */
    WD_ERR_STATE = 3,           /* call out of order                          */
    WD_ERR_NOT_SPD = 4,         /* a pivot <= 0; wd_status_detail gives the
                                   smallest failing column (permuted order)  */
    WD_ERR_OOM = 5,             /* host or device allocation failed           */
    WD_ERR_CUDA = 6,            /* a CUDA runtime error (message in detail)   */
    WD_ERR_TIMEOUT = 7,         /* a bounded device wait expired              */
    WD_ERR_NO_CONVERGENCE = 8   /* iterative refinement did not reach the
                                   requested backward error                   */
} wd_status;

typedef enum {
    WD_FP64 = 0,       /* fronts, factor and solves in FP64                     */
    WD_MIXED = 1       /* fronts and solves in FP32 (Schur updates on tensor
                          cores where available), FP64 residuals and iterative
                          refinement to the requested backward error           */
} wd_precision;

typedef struct {
    int32_t nd_leaf;        /* ND stops at <= nd_leaf vertices (default 128)     */
    int32_t relax_k;        /* amalgamation: merge while width <= relax_k (64)   */
    int32_t relax_pct;      /* ... or explicit zeros <= relax_pct % (10)         */
    int32_t ir_max_iter;    /* refinement steps in WD_MIXED (default 10)         */
    double ir_tol;          /* target normwise backward error (default 1e-12)    */
    int32_t use_graphs;     /* capture factor/solve launch sequences (1)         */
    int32_t symbolic_only;  /* 1: host-only handle, no GPU is touched; only
                               wd_analyze, wd_symbolic_export and wd_get_info
                               are available (numeric calls: WD_ERR_STATE) (0) */
    int32_t profile;        /* 1: bracket every kernel launch of wd_factor and
                               wd_solve with CUDA events on the caller's stream
                               and accumulate per-kernel times (0)            */
    int32_t diag64_min_k;   /* WD_MIXED: the diagonal blocks of supernodes of
                               width >= diag64_min_k are factored (Cholesky and
                               inverse of the 64 x 64 block) in FP64, then
                               rounded to FP32; 0: none (default 0)           */
    int32_t wait_limit;     /* polls before a bounded device wait gives up
                               (WD_ERR_TIMEOUT); 0: the default (2^26)        */
    int32_t test_closed_gate; /* test hook, 1: every tensor-core update CTA
                               also waits for a device word that nothing sets,
                               so the bounded wait must expire (0)            */
    int32_t test_fail_alloc; /* test hook, k > 0: the handle's k-th device
                               allocation fails as if memory ran out
                               (WD_ERR_OOM); counts from wd_create (0)        */
    int32_t solve_simt;     /* WD_MIXED, more than 8 right-hand sides: 1 runs
                               the solves' products on the FP32 SIMT pipes
                               instead of the tensor cores (0)                */
    int32_t fp64_tc_schur;  /* WD_FP64: 1 runs the Schur updates (C -= L21
                               L21^T, Section 4) on the tensor cores with the
                               FP64 values split into eight bf16 slices of 7
                               bits per 64-column block and row (products
                               accumulated exactly, combined in FP64; error
                               within FP64's own bound for these sums); the
                               panels, diagonal blocks and solves stay FP64.
                               0: FP64 on the SIMT pipes (0)                 */
    int32_t step_launches;  /* WD_MIXED: 1 factors each level's pivot columns
                               with two launches per 64-column pivot block
                               (panel, then update); 0: one launch per level
                               whose CTAs take the blocks' tasks in dependency
                               order and wait (bounded) for what they read (0).
                               diag64_min_k > 0 implies 1                    */
} wd_options;

/* Optional geometry for the nested-dissection ordering.  Per vertex (basis
   function) lambda: its level j = |lambda| (Section 2), the lower corner and
   side of the axis-aligned box supp psi_lambda in integer finest-cell units
   of its parameter domain.  box_lo is n x dim row-major.  patch (may be
   NULL): for a surface made of several parameter domains (e.g. the six
   faces of a cubed sphere), the domain of each vertex, 0..31; boxes are then
   in their own domain's units, and the dissection first cuts along domain
   boundaries (lowest two domains against the rest, then one against the
   other) before cutting boxes inside a domain. */
typedef struct {
    int32_t dim;                 /* 1, 2 or 3                                  */
    const int32_t *level;        /* [n]                                        */
    const int32_t *box_lo;       /* [n * dim]                                  */
    const int32_t *box_side;     /* [n]                                        */
    const int32_t *patch;        /* [n] or NULL                                */
} wd_geometry;

typedef struct {
    int64_t n;
    int64_t nnz_A_lower;
    int64_t nnz_L;              /* structural nonzeros of L (incl. diagonal)   */
    int64_t nnz_L_stored;       /* stored entries incl. amalgamation zeros     */
    double flops_factor;        /* sum_j c_j^2 (structural)                    */
    int32_t nsuper;
    int32_t nlevels;            /* height of the supernodal tree               */
    int32_t max_front;          /* largest front order m_s                     */
    int32_t max_width;          /* widest supernode k_s                        */
    int64_t front_bytes;        /* device bytes of the front pool (FP64)       */
    int64_t factor_launches;    /* kernels launched per wd_factor              */
    double analyze_seconds;
} wd_info;

typedef struct {
    int32_t iterations;         /* refinement steps taken (0 in WD_FP64)       */
    double backward_error;      /* max over columns of
                                   ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf),
                                   residual in FP64; -1 if not computed        */
} wd_solve_info;

/* Fill *opt with the defaults listed above. */
void wd_default_options(wd_options *opt);

/* Create a handle bound to the current CUDA device.  opt may be NULL. */
wd_status wd_create(wd_handle *h, const wd_options *opt);

/* Free the handle and all its memory.  NULL is ignored. */
void wd_destroy(wd_handle h);

/* Symbolic analysis (host): validate the lower CSC pattern, compute the
   nested-dissection permutation (Section 4), the elimination tree, column
   counts, supernodes with relaxed amalgamation, extend-add maps and the level
   schedule, and upload the index arrays.  Synchronous.  colptr/rowidx are
   host arrays.  geom may be NULL: then the identity order is used.  Limits:
   n < 2^31 - 1 and at most 2^31 - 1 entries in the full symmetric matrix
   (2 nnz - n), else WD_ERR_INVALID_ARG; the same for a batch's total. */
wd_status wd_analyze(wd_handle h, int64_t n, const int64_t *colptr, const int32_t *rowidx,
                     const wd_geometry *geom);

/* Batch of independent systems (Section 5's many-instance use, one GPU):
   count instances, instance i with its own lower CSC pattern (n[i], colptr[i],
   rowidx[i]) and optional geometry geom[i] (geom may be NULL for none).  The
   handle then holds the block-diagonal matrix diag(A_0, ..., A_{count-1}):
   its analysis is the union of the instances' analyses, and every later call
   works on it as one matrix, so one launch per tree level covers all
   instances.  wd_factor takes the instances' values concatenated in instance
   order (instance i's values in its rowidx order); wd_solve / wd_apply_L take
   right-hand sides whose rows are the instances' rows concatenated (sum n[i]
   rows).  Refinement, and the backward error reported by wd_solve, use each
   instance's own normwise backward error (the largest over instances and
   columns is reported).  Instances given with identical pointers (n, colptr,
   rowidx and geometry arrays) are analyzed once.  Host, multithreaded. */
wd_status wd_analyze_batch(wd_handle h, int32_t count, const int64_t *n, const int64_t *const *colptr,
                           const int32_t *const *rowidx, const wd_geometry *geom);

/* log det A_i of every instance of a batch (host array of count doubles). */
wd_status wd_logdet_batch(wd_handle h, double *out);

/* Copy the symbolic result into caller-allocated host arrays (any may be
   NULL): perm[n] (perm[new] = old), parent[n] (elimination tree of P A P^T,
   -1 for roots), colcount[n] (nonzeros of column j of L incl. diagonal),
   super_first[nsuper+1], super_rowptr[nsuper+1] and super_rows[...] (sorted
   row indices of each supernode's front, its own columns first). */
wd_status wd_symbolic_export(wd_handle h, int32_t *perm, int32_t *parent, int64_t *colcount,
                             int32_t *super_first, int64_t *super_rowptr, int32_t *super_rows);

wd_status wd_get_info(wd_handle h, wd_info *info);

/* Numeric factorization P A P^T = L L^T (multifrontal, on the GPU).
   values: nnz doubles in the order of the analyzed rowidx, on the host
   (values_on_device = 0) or on the device (1).  Synchronous: returns
   WD_ERR_NOT_SPD if a pivot is not positive. */
wd_status wd_factor(wd_handle h, const double *values, int values_on_device, wd_precision prec,
                    void *stream);

/* B := A^-1 B for nrhs columns of leading dimension ldb >= n, original
   order.  B on the device (B_on_device = 1) or the host (0).  In WD_MIXED the
   solve is refined in FP64 until the backward error is <= ir_tol
   (WD_ERR_NO_CONVERGENCE after ir_max_iter steps).  In WD_FP64 the backward
   error is computed only if info is not NULL.  Synchronous. */
wd_status wd_solve(wd_handle h, double *B, int64_t nrhs, int64_t ldb, int B_on_device,
                   void *stream, wd_solve_info *info);

/* The mass matrix G of a non-orthonormal basis for wd_theta_step (Section
   5, Eq. (theta); its pattern lies inside the system matrix's, Section 6):
   gvalues are its nnz lower-CSC values in the order of the analyzed rowidx
   (zero where G has no entry), on the host (on_device = 0) or the device
   (1); they are copied.  NULL restores G = I.  Needs wd_analyze; stays in
   effect until the next wd_analyze.  Synchronous. */
wd_status wd_set_mass(wd_handle h, const double *gvalues, int on_device);

/* One step of the theta-scheme for a parabolic problem (Section 5,
   Eq. (theta)): the factored matrix is M = G + theta dt K (K the compressed
   operator, positive semidefinite; G = I for an orthonormal basis, else the
   matrix given to wd_set_mass), and the step is
     U := M^-1 [ (1/theta) G U - ((1 - theta)/theta) M U + dt F ],
   i.e. (G + theta dt K) U_new = (G - (1 - theta) dt K) U_old + dt F, with
   F = (1 - theta) f(t_i) + theta f(t_{i+1}) given by the caller (NULL: no
   source).  The products M U and G U are formed to FP64 accuracy from the
   matrices' values (as in wd_backward_error); the solve is wd_solve's,
   refinement included.
   U (in/out) and F: n x nrhs, column-major, leading dimension ld >= n,
   original order, both on the device (on_device = 1) or both on the host (0).
   0 < theta <= 1 (theta = 1: implicit Euler, no product), dt finite and
   >= 0; otherwise WD_ERR_INVALID_ARG.  Needs a successful wd_factor of M;
   info as for wd_solve.  Synchronous.  Not in the paper as an interface: the
   paper states the scheme and factors M once for all steps. */
wd_status wd_theta_step(wd_handle h, double *U, const double *F, int64_t nrhs, int64_t ld, double theta,
                        double dt, int on_device, void *stream, wd_solve_info *info);

/* Normwise backward error of given solutions, the test that stops the
   refinement: *be = max over columns of
     ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)
   X, B: n x nrhs, column-major, leading dimension ld, original order, device
   (1) or host (0).  The residual is formed from A's FP64 values: in FP64 for
   up to 8 columns, in double-float arithmetic (about 48 bits) for more.  For
   a batch, the largest of the instances' own backward errors.  Needs a
   successful wd_factor (for ||A||_inf).  Synchronous. */
wd_status wd_backward_error(wd_handle h, const double *X, const double *B, int64_t nrhs, int64_t ld,
                            int on_device, void *stream, double *be);

/* log det A = 2 sum_j log L_jj (compensated sum).  Synchronous. */
wd_status wd_logdet(wd_handle h, double *out);

/* S := P^T L Z, both n x nrhs with leading dimension ld; Z is indexed in the
   factor's (permuted) order, S in the original order.  Gaussian random field
   samples for Z ~ N(0, I) (Section 5.3).  Device (1) or host (0) arrays.
   Synchronous. */
wd_status wd_apply_L(wd_handle h, const double *Z, double *S, int64_t nrhs, int64_t ld,
                     int on_device, void *stream);

/* Selected inverse: out[e] = (A^-1)(i, j) for every stored lower entry e = (i, j)
   of A, in the order of the analyzed rowidx.  Computed from the FP64 factor by
   Takahashi's recurrences in supernodal form, top-down over the supernodal
   tree (for supernode columns J and rows R below them: W = L_RJ L_JJ^-1,
   Z_RJ = -Z_RR W, Z_JJ = L_JJ^-T L_JJ^-1 - W^T Z_RJ).  This is the gradient of
   log det A with respect to the stored entries (off-diagonal entries stand for
   both (i, j) and (j, i): multiply them by 2).  Needs a WD_FP64 factorization
   (WD_ERR_STATE otherwise).  out on the device (1) or the host (0).  The
   first call allocates the workspace (about twice the factor's memory).
   Synchronous. */
wd_status wd_selinv(wd_handle h, double *out, int on_device, void *stream);

/* Pattern part of the gradient of x^T A^-1 y-type terms: for every stored lower
   entry e = (i, j) of A (analyzed order)
     out[e] = sum_c U(i, c) V(j, c) + U(j, c) V(i, c)   (i != j)
     out[e] = sum_c U(i, c) V(i, c)                     (i == j)
   U, V: n x ncols, column-major, leading dimension ld, original order; device
   (1) or host (0) arrays; ncols may be 0 (U and V may then be NULL).  Needs
   wd_analyze only.  Synchronous. */
wd_status wd_sym_pattern_outer(wd_handle h, const double *U, const double *V, int64_t ncols,
                               int64_t ld, double *out, int on_device, void *stream);

/* Gradient of a loss l with respect to the stored values of A, for a loss that
   depends on A through log det A and X = A^-1 B:
     out[e] = g_logdet * w_e * (A^-1)(i, j) - (G(i,:) . X(j,:) + G(j,:) . X(i,:))   (i != j)
     out[e] = g_logdet * (A^-1)(i, i)       -  G(i,:) . X(i,:)                      (i == j)
   with w_e = 2 (an off-diagonal value stands for both (i, j) and (j, i)),
   g_logdet = dl/d(log det A), G = A^-1 (dl/dX) (the caller's solve).  This
   is dl/dA = g_logdet A^-1 - G X^T restricted to the pattern (the adjoint of
   the factorization of Section 4 and of the solves).  X, G: n x ncols,
   column-major, leading dimension ld, original order; out: one value per
   stored lower entry, analyzed order; all on the device (1) or the host (0).
   g_logdet != 0 needs a WD_FP64 factorization (WD_ERR_STATE otherwise).
   ncols may be 0 (X and G may then be NULL).  Synchronous. */
wd_status wd_value_gradient(wd_handle h, double g_logdet, const double *X, const double *G,
                            int64_t ncols, int64_t ld, double *out, int on_device, void *stream);

/* Copy the stored factor (supernodal panels, FP64) to a host array of
   info.nnz_L_stored doubles: for each supernode s, its m_s x k_s lower
   panel, column-major (ld m_s), rows as in super_rows.  Entries above the
   diagonal of the panel are zero.  Synchronous. */
wd_status wd_export_L(wd_handle h, double *panels);

/* Allocation-free variant of wd_export_L.  The paper has no counterpart: this
   call exists for callers that cannot allocate device memory while it runs,
   e.g. when another allocator (a framework's caching allocator, a memory cap)
   holds the device memory so that wd_export_L's factor-sized cudaMalloc would
   fail, or when the device-wide synchronization of cudaMalloc / cudaFree
   would stall the caller's other streams.
   Writes the same panels as wd_export_L (info.nnz_L_stored doubles, same
   layout) into the caller's DEVICE buffer `panels`, enqueued on `stream`,
   and returns without waiting; launch errors are returned, errors of the
   running kernels surface at the caller's next synchronization.
   Allocates nothing: the only scratch (the panels' offsets) is a static
   device array of WD_NOALLOC_MAX_SUPERNODES + 1 int64 values (512 KiB), one
   per device.  More supernodes than that: WD_ERR_INVALID_ARG, nothing
   enqueued.  Nothing in the scratch has to start at zero (every call rewrites
   the offsets before reading them).  The first call on a device looks up the
   array's address (cudaGetSymbolAddress), which may load the module: make
   that first call during set-up, before any stream capture.  The address is
   cached per device for the life of the process: it does not survive
   cudaDeviceReset (every handle is invalid after a reset anyway).  Calls
   whose executions overlap (unordered streams, several host threads) share
   the scratch and race: order them.  The handle's own later calls that
   rewrite or free the fronts (wd_factor, wd_analyze, wd_destroy) wait for
   this call's copy to finish (an event recorded on `stream`; not when
   `stream` is capturing a CUDA graph, whose launches the caller orders: the
   call can be captured, it makes no allocation or synchronizing call).  The caller's
   current device is restored before returning.  Needs a successful
   wd_factor. */
#define WD_NOALLOC_MAX_SUPERNODES 65536
wd_status wd_export_L_noalloc(wd_handle h, double *panels, void *stream);

/* LU factorization without pivoting of a NONSYMMETRIC matrix with the
   analyzed (symmetric) pattern: P A P^T = L U, L unit lower triangular, on
   the same nested-dissection ordering and supernodes as the Cholesky path
   (Section 4, where Cholesky and LU share the ordering and U has the pattern
   of L transposed; Section 6, the double-layer operator of the PCM example).
   lower[e] = A[r][c] and upper[e] = A[c][r] for every stored lower entry e =
   (r, c) of the analyzed lower CSC (nnz doubles each; the diagonal is taken
   from lower), both on the host (on_device = 0) or the device (1).  FP64.
   No pivoting: a zero pivot gives WD_ERR_NOT_SPD with its column (permuted
   order, wd_status_detail); a matrix whose symmetric part is positive
   definite always factors.  Replaces any Cholesky factor of the handle
   (wd_solve / wd_logdet need a new wd_factor).  Synchronous. */
wd_status wd_factor_lu(wd_handle h, const double *lower, const double *upper, int on_device, void *stream);

/* B := A^-1 B with the LU factor: x = P^T U^-1 L^-1 P b (forward
   substitution with the unit lower L, backward with U), FP64, nrhs columns of
   leading dimension ldb >= n, original order, on the device (B_on_device =
   1) or the host (0).  Needs wd_factor_lu.  Synchronous. */
wd_status wd_solve_lu(wd_handle h, double *B, int64_t nrhs, int64_t ldb, int B_on_device, void *stream);

/* log |det A| = sum_j log |U_jj| (*logabs) and the sign of det A (*sign, +1
   or -1), from the LU factor.  Synchronous. */
wd_status wd_logdet_lu(wd_handle h, double *logabs, int32_t *sign);

/* Schedule of the mixed-precision factorization's pivot columns, one flag per
   elimination-tree level (info.nlevels, deepest level first): 0 = one launch
   of dependency-ordered tasks for the level, 1 = a (panel, update) launch
   pair per 64-column pivot block.  Both compute P A P^T = L L^T (Section 4)
   with the same arithmetic; the choice only changes the time, and a tuner
   picks it by measurement.  Set after wd_analyze (which resets every flag
   to 0); takes effect at the next wd_factor.  With wd_options.step_launches
   = 1 or diag64_min_k > 0 every level uses launch pairs and
   wd_get_level_schedule reports 1 for all.  WD_ERR_INVALID_ARG for a wrong
   count or a flag other than 0 / 1; synchronous. */
wd_status wd_set_level_schedule(wd_handle h, const int8_t *step, int32_t nlevels);
wd_status wd_get_level_schedule(wd_handle h, int8_t *step, int32_t nlevels);

/* LDL^T without pivoting of a SYMMETRIC matrix that need not be positive
   definite: P A P^T = L D L^T, L unit lower triangular on the analyzed
   pattern, D diagonal.  The paper factors the compressed matrix by a Cholesky
   decomposition or, more generally, an LU decomposition on the same ordering
   (Introduction; Section 4); for a symmetric matrix the LU decomposition
   without pivoting is L (D L^T), so this runs the LU factorization of
   wd_factor_lu on the values given once (lower CSC, nnz doubles, host or
   device as on_device) and keeps U = D L^T.  FP64.  A zero pivot gives
   WD_ERR_NOT_SPD with its column (permuted order); a negative pivot does
   not stop it.  Solve with wd_solve_lu, log |det A| and its sign with
   wd_logdet_lu, the inertia with wd_inertia, the factors with wd_export_LU
   (L, and D on the diagonal of U^T).  Replaces any other factor of the
   handle.  Synchronous. */
wd_status wd_factor_ldlt(wd_handle h, const double *values, int on_device, void *stream);

/* Inertia of A from the pivots of the last wd_factor_ldlt (Sylvester's law:
   the numbers of positive and negative entries of D are those of A's
   eigenvalues; no pivot is zero after a successful factorization).  Host
   outputs, each may be NULL.  WD_ERR_STATE without an LDL^T factor.
   Synchronous. */
wd_status wd_inertia(wd_handle h, int64_t *npos, int64_t *nneg);

/* The LU factor as two host arrays of info.nnz_L_stored doubles each, in the
   layout of wd_export_L (per supernode an m_s x k_s panel, column-major, rows
   as in super_rows): lpanels holds L (unit diagonal, zero above it),
   utpanels U^T (entry (r, c) = U[c][row r], zero above the diagonal).
   Synchronous. */
wd_status wd_export_LU(wd_handle h, double *lpanels, double *utpanels);

/* Per-kernel statistics accumulated while wd_options.profile = 1: name (the
   kernel and its precision), launches, summed event time, and the
   algorithmic flops and bytes of those launches (flops of the arithmetic the
   method needs on the stored fronts; bytes of the front, update-matrix and
   A entries each launch must read or write once).  Up to cap entries are
   written to out; *count receives the number of kernels.  reset != 0 clears
   the statistics after copying. */
typedef struct {
    char name[40];
    int64_t launches;
    double milliseconds;
    double flops;
    double bytes;
} wd_kernel_stat;

wd_status wd_kernel_stats(wd_handle h, wd_kernel_stat *out, int32_t cap, int32_t *count,
                          int reset);

/* Number of CUDA kernels this handle has launched (all calls); reset != 0
   sets the counter back to zero after reading it. */
wd_status wd_launch_count(wd_handle h, int64_t *count, int reset);

/* Detail of the last error: failing column (or -1) and a message. */
wd_status wd_status_detail(wd_handle h, int64_t *column, char *msg, size_t len);

const char *wd_status_string(wd_status s);

#ifdef __cplusplus
}
#endif

#endif /* WD_H */
