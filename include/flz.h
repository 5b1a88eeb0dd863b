/*
 * flz.h -- C ABI of a GB300 (sm_103a) filtered Lanczos eigensolver.
 *
 * The library computes all eigenpairs (lambda, x) of a real sparse symmetric
 * matrix A with lambda in a user interval [alpha, beta] by the filtered
 * Lanczos procedure of arXiv 2409.15053 (Cucheb): a Chebyshev filter
 * polynomial p built from the closed-form coefficients of the indicator of
 * [alpha, beta] (Section 2.2), block Lanczos with full reorthogonalization on
 * p(A) (Sections 2.3, 3.2.2), and Rayleigh quotients of the Ritz vectors
 * (eq. rayleigh).
 *
 * Conventions for every entry point:
 *  - Every function returns flz_status; FLZ_OK is 0. No exception crosses the
 *    ABI. After a failure, flz_last_error() returns a message for the calling
 *    thread (valid until that thread's next failing call).
 *  - "Device" pointers are CUDA global-memory addresses on the current device;
 *    "host" pointers are ordinary CPU memory. The library never frees memory
 *    it did not allocate. Handles own every device buffer they allocate until
 *    their destroy call.
 *  - Blocks of vectors are n x r, row-major (row i's r entries contiguous,
 *    leading dimension r), FP64, unless stated otherwise.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Calls that take a stream are asynchronous with respect to the
 *    host unless stated otherwise; calls without one synchronize the device.
 */
#ifndef FLZ_H
#define FLZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum flz_status {
  FLZ_OK = 0,
  FLZ_ERR_INVALID_ARG = 1,    /* null pointer, size out of range, bad enum */
  FLZ_ERR_NOT_SYMMETRIC = 2,  /* a_ij != a_ji for a stored entry (Section 3.2.1 requires symmetry) */
  FLZ_ERR_BAD_CSR = 3,        /* rowptr not monotone / not ending at nnz, column out of range or unsorted */
  FLZ_ERR_EMPTY_INTERVAL = 4, /* [alpha, beta] misses [lambda_min, lambda_max] (Section 3.2.2 validity check) */
  FLZ_ERR_NOT_CONVERGED = 5,  /* basis capacity reached first; partial results remain readable */
  FLZ_ERR_OUT_OF_MEMORY = 6,  /* a device or host allocation failed */
  FLZ_ERR_CUDA = 7,           /* a CUDA runtime call or kernel launch failed */
  FLZ_ERR_TIMEOUT = 8,        /* a bounded device-side wait expired */
  FLZ_ERR_CAPACITY = 9,       /* a caller-provided output buffer is too small */
  FLZ_ERR_NO_INTERVAL = 10,   /* flz_solve before flz_solver_set_interval */
  FLZ_ERR_NOT_SOLVED = 11     /* a result getter before a successful or partial solve */
} flz_status;

typedef enum flz_dtype { FLZ_F64 = 0, FLZ_F32 = 1, FLZ_BF16 = 2 } flz_dtype;
typedef enum flz_memspace { FLZ_HOST = 0, FLZ_DEVICE = 1 } flz_memspace;

/* Arithmetic of the filter recurrence (p(A) applied to a block); the rest of
 * the solver (reorthogonalization, Rayleigh-Ritz, Rayleigh quotients,
 * residuals) is FP64 in every mode.
 * FP64: IEEE FP64 storage and arithmetic (the paper's setting).
 * FP32: matrix values and recurrence vectors stored and combined in FP32. The
 *       filtered Lanczos relation then holds to FP32 rounding, which bounds
 *       the attainable residual (about 1e-7 relative); eigenvalues come from
 *       FP64 Rayleigh quotients and are far more accurate than that.
 * BF16: as FP32 with values and vectors stored in bfloat16, FP32 sums
 *       (attainable residual 1e-4 to 1e-2: the rounded matrix values alone
 *       perturb A by up to 2^-9 of its row sums).
 * DF64: double-FP32: every value is a pair of FP32 words (hi + lo, about 48
 *       significant bits, the same 8 bytes as FP64) combined on the FP32 pipes
 *       with error-free transformations; residuals reach the FP64 range on
 *       GPUs whose FP64 rate is a small fraction of their FP32 rate. The single
 *       solver also keeps its Krylov basis in double-FP32 (reorthogonalization
 *       on the FP32 pipes); a batch uses the double-FP32 filter with an FP64
 *       basis.
 * FX64: 64-bit fixed point on the integer pipes (forward recurrence only):
 *       the recurrence vectors and the running sum are integers in units of
 *       2^-60 of a power-of-two scale near each column's 2-norm, the entries
 *       of 2 Ahat and the coefficients integers in units of 2^-61; every row
 *       sum of products is formed in 96-bit integers and rounded once, so each
 *       degree adds one rounding of 2^-61 (relative to the column's norm) per
 *       entry where FP64 adds one of 2^-53 relative per partial sum. Needs
 *       the spectrum of Ahat inside [-1, 1] (a recurrence value above 1.25 of
 *       its column scale is reported as FLZ_ERR_INVALID_ARG instead of
 *       overflowing) and rows of 2 Ahat with absolute sums at most 3.9; block
 *       widths 1, 2, 3, 4, 8, 16. Where these do not hold the filter runs in
 *       FP64 (flz_stats.filter_precision says which ran). */
typedef enum flz_precision { FLZ_PREC_FP64 = 0, FLZ_PREC_FP32 = 1, FLZ_PREC_BF16 = 2, FLZ_PREC_DF64 = 3,
                             FLZ_PREC_FX64 = 4 } flz_precision;

/* How p_m(Ahat) V is evaluated; both give the same polynomial and differ
 * only in rounding.
 * FORWARD:  three-term recurrence T_{i+1} = 2 z T_i - T_{i-1} (eq. def:cheb1)
 *           with the running sum in the same pass: per degree one pass over A
 *           and five vector streams (gathered T_i, T_{i-1}, T_{i+1}, sum in/out).
 * CLENSHAW: the backward recurrence B_k = b_k V + 2 Ahat B_{k+1} - B_{k+2}
 *           the paper uses (Section 2.2): four vector streams (V, gathered
 *           B_{k+1}, B_{k+2}, B_k) and no running sum. */
typedef enum flz_recurrence { FLZ_REC_FORWARD = 0, FLZ_REC_CLENSHAW = 1 } flz_recurrence;

/* Where the full reorthogonalization of an FP64 basis runs (classical
 * Gram-Schmidt twice against the whole basis, Section 3.2.2).
 * CUDA_CORES: FP64 inner products and updates on the FP64 pipes.
 * TENSOR:     the basis is also held as eight base-256 digits per value
 *             (64-bit fixed point in 2^-62 units; the FP64 basis is rounded
 *             to the same grid, so both copies hold the same numbers), each
 *             digit an integer that BF16 represents exactly. The projections
 *             Q^T W and the updates W - Q H run as BF16 tcgen05 MMAs whose
 *             FP32 accumulations stay exact integers (at most 256 products of
 *             at most 2^14 between drains of tensor memory) and are
 *             recombined exactly. The inner products are exact up to the
 *             rounding of W (or H) to 62 fractional bits of its column scale
 *             and a final FP64 rounding, i.e. more accurate than FP64
 *             arithmetic. 16 bytes per basis value of device memory
 *             besides the FP64 basis.
 * AUTO:       TENSOR where it applies (FP64 basis, enough device memory for
 *             the digit copy at the basis capacity), else CUDA_CORES. The double-FP32 precision keeps its
 *             own basis and always uses the FP32 pipes. */
typedef enum flz_ortho { FLZ_ORTHO_AUTO = 0, FLZ_ORTHO_CUDA_CORES = 1, FLZ_ORTHO_TENSOR = 2 } flz_ortho;

/* How a solve uses start vectors (flz_solver_set_start_vectors); both are
 * additions of this library for sequences of related problems.
 * KRYLOV:   filtered block Lanczos from a start block of random combinations
 *           of the start vectors (plus 1 % noise).
 * SUBSPACE: filtered subspace iteration (Chebyshev-filtered subspace
 *           iteration, the scheme of the dense-sequence solvers that the
 *           paper's Section 5 points to) on the start vectors plus guard and
 *           extra columns: the first sweep applies the solve's filter at half
 *           its degree to the (random) extra columns, later sweeps to all
 *           columns a Chebyshev polynomial damping the
 *           spectrum beyond the block (windows at an end of the spectrum) or
 *           the solve's filter (interior windows), each followed by
 *           Rayleigh-Ritz on A in FP64. It ends when every Ritz pair in
 *           [alpha, beta] has residual <= tol and at least `guard` of the
 *           block's Ritz values lie outside it. It gives up and the solve
 *           falls back to KRYLOV after 12 sweeps, when a sweep does not halve
 *           the largest residual, when the sweeps' rate extrapolated to tol
 *           needs more than 3 (cols + guard) m products of A with a vector
 *           (about what filtered Lanczos takes), or when the block loses rank.
 *           It pays where the window's edge is well separated from the
 *           block's further eigenvalues; in a dense part of the spectrum the
 *           Krylov space's polynomial acceleration wins. */
typedef enum flz_start_mode { FLZ_START_KRYLOV = 0, FLZ_START_SUBSPACE = 1 } flz_start_mode;

typedef struct flz_matrix flz_matrix;
typedef struct flz_solver flz_solver;
typedef struct flz_batch flz_batch;

/* Solver parameters; fill with flz_params_default() then override. */
typedef struct flz_params {
  int32_t block_size;   /* r, block width of block Lanczos (Section 2.3); default 3 as in Section 4; 1..16 */
  int32_t degree;       /* filter degree m; 0 = automatic by eq. (optimaldegree); default 0 */
  double degree_eps;    /* epsilon of eq. (optimaldegree); default 0.3123 */
  int32_t max_degree;   /* cap on the automatic degree; default 2000 */
  double tol;           /* converged when ||Ax - lambda x|| / ||A|| <= tol; default 1e-10 */
  int32_t check_every;  /* block steps between convergence checks (Section 3.2.2: "periodically"); default 30 */
  int32_t max_basis;    /* Krylov basis capacity in vectors; 0 = automatic; rounded down to a multiple of r */
  int32_t guard;        /* Ritz pairs outside [alpha,beta] that must also converge; 0 = max(r, 3) */
  int32_t precision;    /* flz_precision; default FLZ_PREC_FP64 */
  int32_t bounds_steps; /* Lanczos vectors for the spectrum bounds (Section 2.2); default 60 */
  uint64_t seed;        /* seed of the random start blocks; default 1 */
  double lmin, lmax;    /* if lmin < lmax these bounds are used and no estimate is made */
  int32_t damping;      /* 0: plain truncation (Section 2.2, default); 1: Jackson damping g_k b_k;
                           2: Lanczos sigma damping sigma_k b_k (flz_lanczos_sigma_factors) */
  int32_t recurrence;   /* flz_recurrence; default FLZ_REC_FORWARD; batches use FORWARD only */
  double transition;    /* 0: the indicator of [alpha, beta] (Section 2.2, default); > 0: the least-squares
                           smoothed step with linear ramps this wide (mapped units), see
                           flz_smoothed_step_coefficients */
  int32_t ortho;        /* flz_ortho; default FLZ_ORTHO_AUTO */
  int32_t refine;       /* FP32 / BF16 precision only. 0 (default): the solve stops at tol or at the
                           filter's rounding floor. 1: the filtered Lanczos procedure runs to
                           max(tol, 1e-5) (FP32) or max(tol, 1e-2) (BF16), then its wanted, guard and
                           extra Ritz pairs are refined to tol by filtered subspace iteration with the
                           FX64 filter (FP64 where it does not apply) and Rayleigh-Ritz on A in FP64: the
                           mixed-precision form (not in the paper). See flz_stats.refine_sweeps. In a
                           batch the lockstep phase stops at the same floor and every converged problem
                           is refined on its own matrix from its found eigenvectors (plus guard and
                           random extra columns), up to eight problems at a time on host threads. */
  int32_t start_mode;   /* flz_start_mode, used when start vectors are set; default FLZ_START_KRYLOV */
  int32_t persistent;   /* batches with the fixed-point filter only. 0 (default): one launch per degree
                           step, the steps of a block step replayed as a CUDA graph. 1: every degree of a
                           filter application in one cooperative launch whose CTAs meet at a grid barrier
                           between degrees (bounded: a wait beyond the limit of flz_set_wait_limit ends
                           the solve with FLZ_ERR_TIMEOUT). Other solves ignore it. */
  int32_t tile_rows;    /* batches with the fixed-point filter: rows per CTA of the degree step, 128 or
                           256; 0 (default) times both at the batch handle's first flz_batch_solve and
                           keeps the faster. Other solves ignore it. */
} flz_params;

/* One convergence check of a solve (Section 3.2.2's periodic Rayleigh-Ritz
 * test): after `block_steps` steps, the walk down the Ritz pairs ranked by
 * their p(A) Ritz value visited `walked` pairs, `inside` of them in
 * [alpha, beta] with residual <= tol and `outside` outside it; all_small = 1
 * if every visited pair passed; converged = 1 if this check ended the solve
 * (all passed, the guard pairs met and the count equal to the previous
 * check's). */
typedef struct flz_check {
  int64_t block_steps;
  int64_t inside;
  int32_t walked;
  int32_t outside;
  int32_t all_small;
  int32_t converged;
} flz_check;

/* Per-solve statistics (the columns of Tables 2 and 3, plus bounds). */
typedef struct flz_stats {
  int64_t iters;        /* block Lanczos steps taken (Table 2 "iters") */
  int64_t matvecs;      /* r * m * iters (Table 2 "MV") */
  int64_t count;        /* eigenpairs found in [alpha, beta] */
  int32_t degree;       /* m */
  int32_t block_size;   /* r */
  int32_t converged;    /* 1 if the convergence test passed */
  int32_t checks;       /* convergence checks made */
  double lmin, lmax;    /* spectrum bounds used for eq. (transf) */
  double c, e;          /* centre and half-width of eq. (transf) */
  double alpha_mapped, beta_mapped;
  double max_residual;  /* max ||Ax - lambda x|| / ||A|| over the returned pairs */
  double ms_bounds;     /* bound estimation ("PREPROC" of Table 3) */
  double ms_filter;     /* p(A) applications ("MV" of Table 3) */
  double ms_orth;       /* full reorthogonalization and block QR ("ORTH" of Table 3) */
  double ms_check;      /* Rayleigh-Ritz, Ritz vectors, residuals */
  double ms_total;      /* wall time of flz_solve */
  int64_t basis_vectors;/* final Krylov basis size */
  int64_t kernel_launches; /* CUDA kernels this solve launched */
  int32_t ortho;        /* flz_ortho the reorthogonalization ran on (CUDA_CORES or TENSOR) */
  int32_t filter_precision; /* flz_precision the filter ran in (FX64 requested may run as FP64) */
  int32_t refine_sweeps;    /* refinement sweeps (params.refine), 0 if none */
  int32_t refine_degree;    /* largest filter degree of a refinement sweep */
  double ms_refine;         /* refinement or subspace-start time (included in ms_total) */
  int64_t sweep_matvecs;    /* products of A with a vector in the subspace sweeps (columns x degree) */
  int32_t start_used;       /* 0: random start block; 1: Krylov start from the start vectors;
                               2: the subspace start converged (no block Lanczos steps) */
  int32_t tile_rows;        /* batches with the fixed-point filter: rows per CTA of its degree step
                               (128 or 256); 0 otherwise */
} flz_stats;

/* ---- status and parameters ------------------------------------------------ */

/* Static English name of a status code; never NULL. */
const char* flz_status_string(flz_status s);
/* Message of the calling thread's last failure ("" if none); never NULL. */
const char* flz_last_error(void);
/* Writes the defaults listed in flz_params into *p. INVALID_ARG if p is NULL. */
flz_status flz_params_default(flz_params* p);

/* ---- matrices (Section 3.2.1: symmetric, CSR with both triangles, no symmetry exploited) ---- */

/* Creates a matrix handle by COPYING a CSR matrix.
 * n >= 1 rows; nnz >= 0 stored entries; rowptr int32[n+1] with rowptr[0] = 0,
 * non-decreasing, rowptr[n] = nnz; col int32[nnz] in [0, n), strictly
 * increasing within a row; val[nnz] of type val_type (FLZ_F64 or FLZ_F32).
 * `where` says whether the three arrays are host or device memory. If
 * check_symmetry is nonzero every stored a_ij must have a stored a_ji with
 * |a_ij - a_ji| <= 1e-14 max(|a_ij|, |a_ji|), else FLZ_ERR_NOT_SYMMETRIC.
 * The structure is always validated (FLZ_ERR_BAD_CSR). n and nnz must fit in
 * int32. On success *out owns device copies (values kept in FP64, plus FP32
 * and BF16 copies made on first use by a reduced-precision filter). */
flz_status flz_matrix_create_csr(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                                 const void* val, flz_dtype val_type, flz_memspace where,
                                 int32_t check_symmetry, flz_matrix** out);
/* Frees the handle and its device memory. NULL is a no-op. */
flz_status flz_matrix_destroy(flz_matrix* A);
/* n, nnz and the Gershgorin interval [glo, ghi] (any pointer may be NULL). */
flz_status flz_matrix_info(const flz_matrix* A, int64_t* n, int64_t* nnz, double* glo, double* ghi);

/* The filter's storage of A (an addition of this library; the paper uses plain
 * CSR): *sell = 1 if the SELL-32 layout (sliced ELLPACK, 32 rows per slice)
 * was built because its padding is below 30 % of the stored entries (regular
 * stencils; the filter then uses it for r in {1, 2, 3, 4, 8, 16}, in FP64
 * only when the padding is at most 10 %), *sell_entries its
 * stored entries with padding, *long_rows the rows above 256 entries that a
 * CTA-per-row kernel filters. Any pointer may be NULL. */
flz_status flz_matrix_format(const flz_matrix* A, int32_t* sell, int64_t* sell_entries, int32_t* long_rows);

/* ---- the hot path: p_m((A - cI)/e) applied to a block --------------------- */

/* W = p_m(Ahat) V with Ahat = (A - cI)/e (eq. transf) and
 * p_m = sum_{i=0..m} coeffs[i] T_i (Section 2.2), evaluated by the recurrence
 * `recurrence` selects (flz_recurrence): one kernel pass over A per degree.
 * V, W: device FP64, n x r row-major, must not overlap; 1 <= r <= 16;
 * coeffs: host FP64[degree+1]; degree >= 0; e > 0. precision selects the
 * recurrence arithmetic (flz_precision); W is always FP64. Scratch of
 * 2 n r elements (plus n r FP32 for reduced precision, 3 n r 64-bit integers
 * for FX64) is owned by the matrix handle and reused across calls, so calls
 * on one matrix must not overlap in time. Asynchronous on `stream`, except
 * FX64, which synchronizes it to report a range overflow (INVALID_ARG); FX64
 * with the Clenshaw recurrence is INVALID_ARG. */
flz_status flz_filter_apply(flz_matrix* A, double c, double e, const double* coeffs, int32_t degree,
                            int32_t r, const double* V, double* W, int32_t precision, int32_t recurrence,
                            void* stream);

/* The same FP64 filter for callers that cannot allocate device memory. (The
 * paper has no counterpart; this is an addition of this library.) Callers
 * whose device memory belongs to another allocator (a framework pool that has
 * reserved the GPU, an embedding application with a fixed budget) or that
 * cannot afford the device-wide synchronization of cudaMalloc/cudaFree pass
 * the CSR arrays and V, W as device pointers they already own; nothing is
 * allocated and no matrix handle is needed. The two recurrence buffers come
 * from a fixed 16 MiB static device array held by every GPU that loads the
 * library until exit, so n * r must be <= 1,048,576 (FLZ_ERR_CAPACITY
 * otherwise). rowptr int32[n+1], col int32[nnz], val FP64[nnz] must be a valid
 * CSR matrix (not validated here); V, W device FP64 n x r row-major, not
 * overlapping; coeffs host FP64[degree+1]. The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) and should come before
 * any stream capture. All calls share the array: calls that overlap in time
 * on the GPU race and must be ordered by the caller. Asynchronous on
 * `stream`. */
flz_status flz_filter_apply_noalloc(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                                    const double* val, double c, double e, const double* coeffs, int32_t degree,
                                    int32_t r, const double* V, double* W, void* stream);

/* Closed-form Chebyshev coefficients of the indicator of [alpha, beta] within
 * [-1, 1] (Section 2.2): out[0] = (acos a - acos b)/pi, out[i] =
 * 2 (sin(i acos a) - sin(i acos b))/(i pi). Host only; out has degree+1 slots.
 * Requires -1 <= alpha < beta <= 1. */
flz_status flz_filter_coefficients(double alpha, double beta, int32_t degree, double* out);
/* Least-squares filter with a transition band (not in the paper; a filter in
 * the spirit of FILTLAN's, the paper's CPU comparison): the truncated
 * Chebyshev series -- the best degree-`degree` approximation in the weighted
 * Chebyshev 2-norm of eq. (optimaldegree) -- of the smoothed step that is 1 on
 * [alpha, beta], falls linearly to 0 over a width delta on each side and is 0
 * elsewhere on [-1, 1]. delta = 0 gives flz_filter_coefficients. Host only;
 * requires -1 <= alpha < beta <= 1, delta >= 0. */
flz_status flz_smoothed_step_coefficients(double alpha, double beta, double delta, int32_t degree, double* out);
/* Jackson damping factors g_0..g_degree (host; out has degree+1 slots):
 * g_k = ((m-k+1) cos(k pi/(m+1)) + sin(k pi/(m+1)) cot(pi/(m+1))) / (m+1).
 * The paper truncates without damping; damping (params.damping = 1) removes
 * the Gibbs overshoot of the filter at the cost of a wider transition. */
flz_status flz_jackson_factors(int32_t degree, double* out);
/* Lanczos sigma factors sigma_0..sigma_degree (host; out has degree+1 slots):
 * sigma_0 = 1, sigma_k = sin(k pi/(m+1)) / (k pi/(m+1)). params.damping = 2
 * multiplies the coefficients by them: the Gibbs overshoot shrinks (to about
 * 1 % at high degree) with a narrower transition than Jackson's. */
flz_status flz_lanczos_sigma_factors(int32_t degree, double* out);
/* The damping polynomial of the mixed-precision refinement (params.refine;
 * not in the paper): Chebyshev coefficients out[0..degree] (host) in z on
 * [-1, 1] of p(z) = T_d(a z + b) / T_d(b - a), where z -> a z + b maps
 * [zc, 1] onto [-1, 1] (d = degree). p(-1) = 1, |p| <= 1 on [-1, 1], and
 * |p| <= 1 / |T_d(b - a)| on [zc, 1]: it damps the spectrum above zc relative
 * to the pairs below it. Requires -1 < zc < 1. */
flz_status flz_damping_coefficients(double zc, int32_t degree, double* out);
/* Eq. (optimaldegree): least m >= 1 with ||p_m - phi|| < eps ||phi|| in the
 * weighted Chebyshev 2-norm. Host only. CAPACITY if no m <= max_degree fits. */
flz_status flz_filter_degree(double alpha, double beta, double eps, int32_t max_degree, int32_t* degree);

/* Spectrum bounds (Section 2.2, after eq. transf): block Lanczos with full
 * reorthogonalization on A over `steps` vectors (block width r), extreme Ritz
 * values padded by their residual bounds and clamped to the Gershgorin
 * interval. Synchronizes `stream`. */
flz_status flz_spectrum_bounds(flz_matrix* A, int32_t steps, int32_t r, uint64_t seed,
                               double* lmin, double* lmax, void* stream);

/* ---- host utilities: the projected problem of eq. (proj) ------------------- */

/* Eigenvalues (ascending) of a symmetric band matrix: T is K x K, row-major,
 * dense storage, zero outside |i - j| <= b (the block tridiagonal T_k of
 * eq. lanczos has b = r). Orthogonal band-to-tridiagonal reduction by Givens
 * rotations, then implicit QL. Host memory only; theta has K slots. */
flz_status flz_band_eigenvalues(int32_t K, int32_t b, const double* T, double* theta);
/* Unit eigenvectors of the same T for the `count` eigenvalues theta[idx[t]]
 * (theta as returned above), by inverse iteration on the band matrix with
 * partial pivoting; vectors of eigenvalues closer than 1e-3 ||T|| are
 * orthogonalized against each other. Y is K x count, column-major (host). */
flz_status flz_band_eigenvectors(int32_t K, int32_t b, const double* T, const double* theta, int32_t count,
                                 const int32_t* idx, double* Y, uint64_t seed);

/* Dense symmetric eigen-decomposition of the n x n row-major matrix S (host):
 * w[n] ascending eigenvalues, Z[n*n] row-major with column k the unit
 * eigenvector of w[k]. Householder tridiagonalization + implicit QL. */
flz_status flz_sym_eig(int32_t n, const double* S, double* w, double* Z);

/* ---- full reorthogonalization (Section 3.2.2) ------------------------------ */

/* Projection C = Q^T W of the n x r block W (device) on a basis Q of nb
 * blocks (device; block b at Q + b n r, each n x r row-major; K = nb r
 * columns); C is K x r row-major (device), r <= 16. `method` is
 * FLZ_ORTHO_CUDA_CORES or FLZ_ORTHO_TENSOR (see flz_ortho; TENSOR needs |Q| < 1.9, and
 * uses Q rounded to the 2^-62 grid, the rounding a solver's basis already
 * has; Q itself is not modified). Synchronous with respect to `stream`;
 * allocates and frees its own scratch. */
flz_status flz_basis_project(int64_t n, int32_t nb, int32_t r, const double* Q, const double* W, double* C,
                             int32_t method, void* stream);
/* Classical Gram-Schmidt twice of W (device n x r, overwritten) against the
 * same basis: W <- (I - Q Q^T)(I - Q Q^T) W, and C = C_1 + C_2 (K x r,
 * device) the total projection coefficients of the two passes. Same methods
 * and conditions as flz_basis_project. */
flz_status flz_basis_orthogonalize(int64_t n, int32_t nb, int32_t r, const double* Q, double* W, double* C,
                                   int32_t method, void* stream);
/* Combination X = Q H of basis columns (the Ritz vectors of Section 2.3 are
 * X = Q_k Y with Y eigenvectors of T_k): Q as in flz_basis_project (nb device
 * blocks, K = nb r columns), H K x s row-major (device), X n x s row-major
 * (device, overwritten, not overlapping Q or H), 1 <= s <= 16. TENSOR forms
 * the products from the digits of Q (rounded to the 2^-62 grid) and of H
 * (62 fractional bits of each column's scale), summed exactly but for digit
 * pairs below 2^-64 of the column scale, with at most one FP64 rounding per
 * 256 basis columns; CUDA_CORES uses FP64 arithmetic. Synchronous with
 * respect to `stream`; allocates and frees its own scratch. */
flz_status flz_basis_multiply(int64_t n, int32_t nb, int32_t r, const double* Q, const double* H, int32_t s,
                              double* X, int32_t method, void* stream);
/* Measured arithmetic rate of the current device (not in the paper; the
 * denominator of the filter kernels' ALU fractions): kind 0 times FP64 FMAs,
 * kind 1 32-bit integer multiply-adds (the fixed-point filter's limb
 * products), each counted as 2 operations, in *ops_per_s. Independent
 * multiply-add chains on 8 CTAs per SM, timed with CUDA events (fastest of
 * three runs after a warm-up). Synchronizes the device; about 0.1 s. */
flz_status flz_measure_alu_peak(int32_t kind, double* ops_per_s);
/* Limit, in nanoseconds, of every bounded device-side wait of kernels
 * launched after this call (the tensor-core reorthogonalization's and the
 * fixed-point filter's barrier waits; default 2,000,000,000). A wait that
 * reaches it gives up: the kernel drains the work it has in flight, frees
 * its tensor memory and returns, and the call reports FLZ_ERR_TIMEOUT; the
 * device stays usable. A limit of 0 means no waiting at all (a barrier that
 * has not completed at its first, non-blocking test gives up); a tiny limit
 * makes those calls time out, which is how that path is tested, and has no
 * other use. *previous (may be NULL) receives the limit in force before.
 * Process-wide. */
flz_status flz_set_wait_limit(uint64_t ns, uint64_t* previous);
/* Layout check of the tensor-core path: one tcgen05.mma (M = 128, N = n in
 * {16, 32, 64, 128}, K = 16, BF16 operands, FP32 accumulator in tensor memory) of a
 * 128 x 16 A operand and an n x 16 B operand given as shared-memory images
 * (host; a_bytes <= 36864, b_bytes <= 20480, multiples of 16; both K-major
 * unless a_mn_major) and the descriptors' leading and stride byte offsets
 * (multiples of 16 whose reach, under either reading of the two fields, stays
 * inside the images' regions). d (host) receives D as 128 x n row-major FP32.
 * TIMEOUT if the MMA's completion wait expired. Synchronizes the device. */
flz_status flz_tc_mma_probe(const uint16_t* a_img, int64_t a_bytes, const uint16_t* b_img, int64_t b_bytes,
                            int32_t n, int32_t a_mn_major, int32_t a_lbo, int32_t a_sbo, int32_t b_lbo,
                            int32_t b_sbo, float* d);

/* ---- solver (Sections 2.3 and 3.2.2) ---------------------------------------- */

/* Creates a solver bound to A (which must outlive it). params may be NULL
 * (defaults). Device memory for the basis is allocated at flz_solve. */
flz_status flz_solver_create(flz_matrix* A, const flz_params* params, flz_solver** out);
flz_status flz_solver_destroy(flz_solver* s);
/* [alpha, beta] in A's own units (not mapped); alpha < beta. */
flz_status flz_solver_set_interval(flz_solver* s, double alpha, double beta);
/* Warm start for a sequence of related problems (the self-consistent-field
 * iterations of Section 1 solve one eigenproblem per step with a slowly
 * changing potential; an addition of this library): the start block of the
 * solver's following solves is r random combinations of these `cols` vectors
 * plus noise of 1 % of their size, orthonormalized, instead of a random block
 * (params.start_mode KRYLOV), or the vectors themselves start filtered
 * subspace iteration (SUBSPACE, see flz_start_mode). Pass the eigenvectors of
 * the previous problem (flz_get_eigenvectors). With KRYLOV the guard pairs
 * beyond the window still have to be found from the noise, so the step count
 * rarely falls; SUBSPACE needs far fewer products of A with a vector when the
 * problems are close. X is n x cols column-major with leading dimension ld >= n, host or
 * device (`where`); the library copies it. cols = 0 clears it (random start
 * blocks again). Not for the double-FP32 precision (INVALID_ARG). */
flz_status flz_solver_set_start_vectors(flz_solver* s, const double* X, int64_t ld, int32_t cols,
                                        flz_memspace where);
/* Runs the filtered Lanczos procedure: bounds, map, degree, coefficients,
 * block Lanczos on p(A) with full reorthogonalization, periodic Rayleigh-Ritz
 * and residual checks, Rayleigh quotients of the converged Ritz vectors.
 * Synchronous: returns when the result is ready. An interval that covers the
 * whole spectrum makes the filter constant, which cannot separate
 * eigenvectors; that case runs unfiltered block Lanczos (p(z) = z). When the
 * basis spans the whole space (K = n) and every Ritz pair passed, the solve
 * has converged. EMPTY_INTERVAL (outside the Gershgorin interval),
 * NOT_CONVERGED (partial results readable), OUT_OF_MEMORY, CUDA_ERROR. */
flz_status flz_solve(flz_solver* s, void* stream);
/* Spectrum slicing (Section 5 names it as future work): [alpha, beta] is cut
 * into nslices equal-width sub-intervals, solved one after another on the
 * same matrix (bounds estimated once; each slice with its own, smaller
 * Krylov basis and the solver's parameters), and the results are merged in
 * ascending order into this solver's results. A pair found by two adjacent
 * slices (an eigenvalue on a shared endpoint) is kept once: results count as
 * the same pair when their eigenvalues agree to 10 tol ||A|| and their
 * eigenvectors overlap by more than 1/2; when two slices hold different
 * vectors of one multiple eigenspace, the second is orthogonalized against
 * the first. Eigenvectors from different slices come from different Krylov
 * bases: they are orthogonal to within (r_i + r_j) / gap (r the residuals in
 * A's units), not to rounding. nslices = 1 is flz_solve. Stats add
 * up the slices' steps, products and phase times. INVALID_ARG if
 * nslices < 1; otherwise the statuses of flz_solve (NOT_CONVERGED if any
 * slice did not converge; the other slices' results are readable). */
flz_status flz_solve_sliced(flz_solver* s, int32_t nslices, void* stream);
/* Number of eigenpairs found in [alpha, beta]. */
flz_status flz_get_count(const flz_solver* s, int64_t* count);
/* Ascending eigenvalues into host out[cap]; CAPACITY if cap < count. */
flz_status flz_get_eigenvalues(const flz_solver* s, double* out, int64_t cap);
/* Eigenvectors as an n x count column-major array with leading dimension
 * ld >= n, column j matching eigenvalue j, unit 2-norm; `where` says whether
 * out is host or device memory; cap_cols < count gives CAPACITY. */
flz_status flz_get_eigenvectors(const flz_solver* s, double* out, int64_t ld, int64_t cap_cols,
                                flz_memspace where);
/* ||A x_j - lambda_j x_j|| / ||A|| per pair into host out[cap]. */
flz_status flz_get_residuals(const flz_solver* s, double* out, int64_t cap);
flz_status flz_get_stats(const flz_solver* s, flz_stats* out);
/* The convergence checks of the last solve, in order, into host out[cap];
 * *count (may be NULL) receives how many there were (all of them even when
 * cap is smaller; only min(cap, *count) are written). */
flz_status flz_get_checks(const flz_solver* s, flz_check* out, int64_t cap, int64_t* count);

/* ---- batches of independent problems --------------------------------------- */

/* A batch of `count` independent problems (not in the paper, which solves one
 * matrix per call): problem i is all eigenpairs of mats[i] in
 * [alphas[i], betas[i]] (A's units). Every matrix must outlive the batch.
 * params (NULL = defaults) apply to all problems; block_size = 0 picks r in
 * {4, 8, 16} by timing the filter kernel at each width, and tile_rows = 0
 * picks the fixed-point filter's rows per CTA (autotuning; done at the
 * handle's first flz_batch_solve and reused by its later solves). The
 * problems are concatenated into one block-diagonal device matrix and run in
 * lockstep: each kernel of a block Lanczos step serves every problem at once,
 * with per-problem bounds, filter degree and coefficients, and per-problem
 * (segmented) block QR and convergence; the reorthogonalization runs per
 * problem on the tensor cores (params.ortho AUTO or TENSOR) or segmented on
 * the CUDA cores. The kernels of a block step are captured as CUDA graphs and
 * replayed (params.persistent: the fixed-point filter as one cooperative
 * launch instead). Problems stop when they converge. Host arrays
 * alphas/betas have `count` entries. */
flz_status flz_batch_create(int32_t count, flz_matrix* const* mats, const double* alphas, const double* betas,
                            const flz_params* params, flz_batch** out);
flz_status flz_batch_destroy(flz_batch* b);
/* Solves every problem; synchronous like flz_solve. FLZ_ERR_NOT_CONVERGED if
 * any problem did not converge (each problem's stats say which). */
flz_status flz_batch_solve(flz_batch* b, void* stream);
/* Per-problem results, index in [0, count): same meaning and errors as the
 * single-problem getters. */
flz_status flz_batch_get_count(const flz_batch* b, int32_t index, int64_t* count);
flz_status flz_batch_get_eigenvalues(const flz_batch* b, int32_t index, double* out, int64_t cap);
flz_status flz_batch_get_residuals(const flz_batch* b, int32_t index, double* out, int64_t cap);
flz_status flz_batch_get_eigenvectors(const flz_batch* b, int32_t index, double* out, int64_t ld, int64_t cap_cols,
                                      flz_memspace where);
flz_status flz_batch_get_stats(const flz_batch* b, int32_t index, flz_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* FLZ_H */
