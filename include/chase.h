/*
 * chase.h -- C ABI of libchase: Chebyshev Accelerated Subspace iteration
 * Eigensolver (ChASE, Winkelmann, Springer, Di Napoli, arXiv 1805.10121)
 * for dense complex Hermitian matrices on one NVIDIA GB300 GPU (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are column-major complex128 with interleaved (re, im) doubles,
 *   the layout of C99 `double complex` and `std::complex<double>` (the
 *   paper's element type, Listing 1).  Element (i, j) of a matrix with
 *   leading dimension ld sits at index j*ld + i.
 * - H is Hermitian and stored in full (both triangles are read).  It is
 *   never modified: the shift (A - cI) of Alg. 4 is applied inside the
 *   product instead of on A (the paper's Shift() kernel, Listing 1).
 * - Array arguments marked "host or device" may point to host memory or to
 *   device memory of the current CUDA device; the library detects which
 *   (cudaPointerGetAttributes).  Host arrays are staged through device
 *   buffers that the library allocates and frees within the call.  All
 *   arrays of one call must be of the same kind.
 * - The caller owns every array it passes (the paper's ChaseBLAS takes
 *   caller-owned buffers, Listing 2).  Device workspace needed beyond the
 *   caller's arrays is allocated stream-ordered (cudaMallocAsync) on
 *   `stream` and released before the call returns.
 * - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every
 *   call returns after its work on `stream` has completed.
 * - Every entry point returns a CHASE_* status; none aborts or throws.  On a
 *   status other than CHASE_OK or CHASE_NOT_CONVERGED, chase_last_error()
 *   returns a message for the calling thread.
 * - Calls may run at the same time from several host threads on different
 *   streams (each thread keeps its own eigensolver handle); their results
 *   are bit-identical to the same calls run one at a time, whatever else
 *   runs on the device.  Calls that share an output array must be ordered
 *   by the caller.
 */
#ifndef CHASE_H_
#define CHASE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* complex128, interleaved */
typedef struct {
  double re, im;
} chase_c64;

/* complex64, interleaved (single-precision entry points) */
typedef struct {
  float re, im;
} chase_c32;

/* ---- status codes ---- */
#define CHASE_OK 0
#define CHASE_INVALID_ARG 1       /* a size, pointer, degree or option is invalid */
#define CHASE_NOT_CONVERGED 2     /* max_iter reached; outputs hold the current subspace (Sec. 5.3) */
#define CHASE_QR_BREAKDOWN 3      /* orthogonalisation failed even with the shifted retry */
#define CHASE_BOUND_VIOLATION 4   /* a Ritz value exceeded b_sup (Sec. 4.2: the bound must hold) */
#define CHASE_CUDA_ERROR 5        /* a CUDA runtime call failed */
#define CHASE_OUT_OF_MEMORY 6     /* device workspace could not be allocated */
#define CHASE_TIMEOUT 7           /* a bounded wait inside a kernel gave up */
#define CHASE_EIGENSOLVER_ERROR 8 /* the projected eigensolve (Alg. 2 line 3) failed */

/* ---- arithmetic of the filter products (Alg. 4) ---- */
#define CHASE_FP64 0 /* complex128 products on the FP64 tensor pipe (mma.sync f64, ~1 TFLOP/s) */
/* Split-BF16: both operands cut into seven 7-bit integer slices (one power-
 * of-two scale per row of H without its diagonal and per column of the
 * block), slice products on the BF16 tensor cores (tcgen05) with exactly
 * accumulated leading levels; the diagonal of H and the recurrence's
 * shift/scale/axpby are applied in FP64.  Each entry of a product is
 * accurate to about 2^-49 max|off-diagonal row of H| max|column| per term.
 * Reads H through its Hermitian symmetry.  QR, Rayleigh-Ritz, residuals
 * and Lanczos stay FP64. */
#define CHASE_SPLIT_BF16 1
/* Split-BF16 filter as above, and the product H Q of Rayleigh-Ritz (Alg. 2
 * line 2, reused for the residuals) on the same split product: each entry
 * carries the same 2^-49 relative bound, against the K u |H||Q| of an FP64
 * GEMM.  The projected eigenproblem, QR, the Gram products and Lanczos stay
 * FP64.  chase_solve and chase_solve_batched only (the filter entry points
 * take CHASE_FP64 or CHASE_SPLIT_BF16). */
#define CHASE_SPLIT_BF16_RR 2
/* Split-BF16 filter whose accuracy follows each column's residual
 * (chase_solve only; the batched solve treats it as CHASE_SPLIT_BF16).  By
 * the model behind Alg. 5 a degree-m filter divides a column's residual by
 * |rho|^m; while that expected residual exceeds 1e-3 h (h = largest |Ritz
 * value|) the column's products keep the leading 3 slices of each operand
 * (about 2^-21 relative), above 1e-6 h 4 slices (2^-28), else all 7
 * (2^-49).  The first filter, before any residual is known, uses 3.  The
 * active block is ordered by (slices, degree), and each run of equal slices
 * is filtered as its own suffix-retiring block.  Rayleigh-Ritz, QR and
 * residuals stay FP64, so the converged pairs meet the same tolerance; a
 * low-precision column only limits how far this filter can reduce its
 * residual, which it could not reduce to the tolerance anyway. */
#define CHASE_SPLIT_BF16_ADAPT 3
/* chase_filter only: split-BF16 products with the leading 4 or 3 slices of
 * each operand (about 2^-28 or 2^-21 relative per product), the reduced
 * precisions CHASE_SPLIT_BF16_ADAPT switches between. */
#define CHASE_SPLIT_BF16_4 4
#define CHASE_SPLIT_BF16_3 5

/* ---- which part of H the solver reads (chase_solve*, via chase_opts) ---- */
#define CHASE_STORAGE_FULL 0  /* both triangles hold H */
/* Only the lower triangle (diagonal included) is read, as a HEMM with
 * uplo = 'L' would (Sec. 5.1); the strict upper triangle may hold anything.
 * The solver forms the full matrix once in a workspace of N x N entries. */
#define CHASE_STORAGE_LOWER 1

/* ---- residual test used for locking (Alg. 3 line 4) ---- */
#define CHASE_CONV_ABS 0 /* Res <= tol (the paper's absolute criterion, Sec. 6.1) */
#define CHASE_CONV_REL 1 /* Res <= tol * h, h = largest |Ritz value| seen (<= ||H||_2) */

/* Configuration: the fields of Table 1 (ChaseConfig) plus build options. */
typedef struct {
  int deg;          /* initial / constant degree (Table 1: 20); rounded up to even */
  int optim;        /* 1: per-column optimised degrees (Alg. 5); 0: constant deg (Table 1: false) */
  int deg_extra;    /* DEGEXTRA of Alg. 5 line 5 (Table 1: 2) */
  int deg_max;      /* DEGMAX of Alg. 5 line 5 (Table 1: 36; with a split-BF16 filter
                       higher caps, e.g. 64, trade cheap filter steps for FP64
                       iterations; the cap also guards rank deficiency of the
                       filtered block, Sec. 4.1.3) */
  int max_iter;     /* cap on the while loop of Alg. 1 (Table 1: 25) */
  int lanczos_iter; /* k, steps of each Lanczos run (Table 1: 25) */
  int num_lanczos;  /* n_vec, density runs of Alg. 6 (Table 1: 4) */
  int approx;       /* 1: V and Lambda hold an approximate solution (Sec. 3.3) */
  double dos_sigma; /* Gaussian width of Eq. 10 in the variable mapped to [-1, 1] (Sec. 4.2: 0.25) */
  int conv_mode;    /* CHASE_CONV_ABS or CHASE_CONV_REL */
  int precision;    /* CHASE_FP64, CHASE_SPLIT_BF16, _RR or _ADAPT */
  int storage;      /* CHASE_STORAGE_FULL or CHASE_STORAGE_LOWER */
} chase_opts;

/* Counters and per-phase times of one chase_solve call. */
typedef struct {
  int iterations;          /* while-loop iterations of Alg. 1 */
  int nconv;               /* locked pairs */
  long long matvecs;       /* column products with H: filter + RR + Lanczos (Sec. 6.1, footnote 6) */
  long long filter_matvecs;/* column products inside the filter (= sum of the degrees) */
  double b_sup, mu1, mu_nevnex; /* final spectral estimates (Sec. 4.2) */
  double tol_eff;          /* the absolute residual threshold used for locking */
  double flops_filter;     /* 8 N^2 * filter_matvecs (2 N^2 for real problems) */
  double flops_total;      /* all algorithmic FLOPs of the solve */
  double t_total, t_lanczos, t_filter, t_qr, t_rr, t_eigh, t_resid, t_host; /* seconds */
  double t_rr_product;     /* seconds of Rayleigh-Ritz's H Q products (inside t_rr) */
  double flops_rr_product; /* their algorithmic FLOPs (8 N^2 b complex, 2 N^2 b real) */
  int filter_slices_low;   /* iterations in which some column products of the split
                              filter kept fewer than 7 slices (CHASE_SPLIT_BF16_ADAPT;
                              single precision) */
  long long lanczos_matvecs; /* column products with H inside Alg. 6 (k per run) */
  long long filter_matvecs_low; /* filter column products made with fewer than 7 slices */
} chase_stats;

/* Tile choice of the grouped FP64 filter: time the candidates on the first
 * degree step (result cached per batch shape), or 0..3 for a fixed shape
 * (0: 64 x 16, 1: 64 x 32, 2: 128 x 16, 3: 64 x 8 rows x complex columns). */
#define CHASE_TILE_AUTO (-1)

/* Counters and times of one chase_filter_batched call. */
typedef struct {
  int problems;            /* problems with work (N > 0 and b > 0) */
  int steps;               /* degree steps (the largest degree of the batch; summed over
                              the iterations of chase_solve_batched) */
  int tile_config;         /* FP64 tile shape used (see CHASE_TILE_AUTO); -1 for split */
  int launches;            /* kernel launches of the call (graph nodes counted once) */
  long long matvecs;       /* column products with H over all problems (sum of the degrees) */
  double flops;            /* 8 N^2 per column product, summed over problems */
  double t_autotune;       /* host seconds spent choosing the tile shape (0 when cached) */
  double t_graph_build;    /* host seconds to capture and instantiate the step graph */
  double t_steps;          /* device seconds of the step graph (every degree step) */
  double t_product;        /* device seconds of the grouped product launches alone */
  double t_total;          /* host seconds of the whole call */
  /* chase_solve_batched: device seconds of Alg. 1's other phases, all
   * problems together (Cholesky QR; Rayleigh-Ritz with residuals, the
   * batched projected eigensolves included; locking, degrees and the
   * reordering of the blocks) */
  double t_qr, t_rr, t_eigh, t_lock;
} chase_batch_stats;

/* Fill `opts` with the defaults of Table 1 (double precision column):
 * deg 20, optim 1 (the paper's default is false; this library's default is
 * the optimised filter of Sec. 4.1), deg_extra 2, deg_max 36, max_iter 25,
 * lanczos_iter 25, num_lanczos 4, approx 0, dos_sigma 0.25,
 * conv_mode CHASE_CONV_REL, precision CHASE_FP64.
 * Returns CHASE_INVALID_ARG if opts is NULL. */
int chase_opts_default(chase_opts* opts);

/* Message describing the last failure on the calling thread ("" if none).
 * The string stays valid until the thread's next call into the library. */
const char* chase_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (all entry points, all threads).  Instrumentation; never fails. */
long long chase_kernel_launches(void);

/* Number of device memory allocations (stream-ordered workspace and error
 * flags) this library has requested in the process so far, all threads.
 * Instrumentation (the paper has no counterpart); never fails. */
long long chase_device_allocations(void);

/* Kernel timing, for benchmarks (the paper has no counterpart).  While
 * timing is on, the library records a pair of CUDA events on the launching
 * stream around the launches of its products with H:
 *   CHASE_TIMED_SPLIT_PRODUCT  the split-BF16 tensor-core product kernel
 *                              (zgemm_split_kernel; the slicing of the block
 *                              and the K-segment combine are outside);
 *   CHASE_TIMED_FP64_PRODUCT   the FP64 product with H of the filter and of
 *                              Rayleigh-Ritz (DMMA tile kernel, or the
 *                              few-column kernel for at most 6 columns).
 * chase_kernel_timing(1) clears the record and starts; (0) stops.
 * chase_kernel_timing_read waits for the recorded events of one kind and
 * returns their summed duration (seconds), the kernel launches they cover,
 * the algorithmic FLOPs (8 N^2 per complex column, 2 N^2 per real column)
 * and the executed tensor FLOPs (split: slice pairs x algorithmic; FP64: 6
 * of every 8 algorithmic complex FLOPs, the 3M form).  flops and
 * tensor_flops are nullable.  Recording adds two event records per product
 * call and no synchronisation.  Errors: CHASE_INVALID_ARG, CHASE_CUDA_ERROR. */
/* Failure detection (the paper has no counterpart): every wait of the
 * library's pipelined kernels on an mbarrier (TMA stages, MMA completion,
 * flush handshakes) gives up after a cycle budget (about one second), sets
 * a device error flag and lets the kernel return, so that a stuck pipeline
 * ends as CHASE_TIMEOUT with a usable context instead of a hung GPU.  This
 * call runs that wait alone: one thread waits on an mbarrier that nothing
 * arrives at, for budget_cycles SM cycles (0 .. 2e9), with no copy or MMA
 * in flight, and the call returns the status the host derives from the
 * flag: CHASE_TIMEOUT.  Errors: CHASE_INVALID_ARG (budget out of range),
 * CHASE_CUDA_ERROR. */
int chase_wait_selftest(long long budget_cycles, void* stream);

#define CHASE_TIMED_SPLIT_PRODUCT 0
#define CHASE_TIMED_FP64_PRODUCT 1
#define CHASE_TIMED_KINDS 2
int chase_kernel_timing(int enable);
int chase_kernel_timing_read(int kind, double* seconds, long long* launches, double* flops,
                             double* tensor_flops);

/* Chebyshev filter with per-column degrees: Alg. 4 with the three-term
 * recurrence of Eq. 7, c = (b_sup + mu_nevnex)/2, e = (b_sup - mu_nevnex)/2,
 * sigma_1 = e / (mu1 - c).  Column a of V is replaced by p_{m_a}(H) v_a with
 * p_m the normalised Chebyshev polynomial of Eq. 5 (p_m(mu1) = 1).
 *
 * H        N x N, leading dimension ldh >= N (host or device)
 * V        N x b, leading dimension ldv >= N, in/out (host or device);
 *          columns keep the caller's order
 * degrees  b ints, each even and in [2, 1024], any order (host or device).
 *          Even degrees are required because the recurrence double-buffers
 *          (Sec. 4.1.3, Alg. 5 line 6).  Internally the columns are sorted by
 *          degree so that every product acts on a contiguous suffix; a column
 *          leaves the products once it reaches its degree (Alg. 4 lines 12-14).
 * precision  CHASE_FP64, CHASE_SPLIT_BF16, CHASE_SPLIT_BF16_4 or CHASE_SPLIT_BF16_3.
 * work     N x b device workspace with leading dimension N, or NULL (the
 *          library allocates it); ignored for host V.
 * Requires mu1 < mu_nevnex < b_sup.  b == 0 or N == 0 is a no-op.
 * Errors: CHASE_INVALID_ARG (sizes, bounds, odd or out-of-range degree,
 * misaligned pointer), CHASE_OUT_OF_MEMORY, CHASE_CUDA_ERROR, CHASE_TIMEOUT. */
int chase_filter(const chase_c64* H, int64_t N, int64_t ldh, chase_c64* V, int64_t ldv, int b,
                 const int* degrees, double b_sup, double mu1, double mu_nevnex, int precision,
                 chase_c64* work, void* stream);

/* Alg. 4 with a precision per column (Sec. 3.2: the filter only needs to be
 * as accurate as the residual it can reach; the paper filters every column
 * in one precision): column a is filtered with its degree degrees[a] on the
 * split-BF16 product that keeps the leading slices[a] slices of each
 * operand, slices[a] in {3, 4, 7} (about 2^-21, 2^-28 and 2^-49 relative
 * per product).  The columns are ordered by (slices, degree) inside the
 * call and each run of equal slices is filtered as its own suffix-retiring
 * block of the same recurrence; V returns in the caller's column order.
 * H, V, work: as chase_filter (complex128, column-major, host or device).
 * degrees, slices: b ints each, host or device.
 * Errors: CHASE_INVALID_ARG (sizes, NULL arrays, bounds out of order, an odd
 * or out-of-range degree, slices outside {3, 4, 7}, non-finite H or V),
 * CHASE_OUT_OF_MEMORY, CHASE_CUDA_ERROR, CHASE_TIMEOUT. */
int chase_filter_mixed(const chase_c64* H, int64_t N, int64_t ldh, chase_c64* V, int64_t ldv,
                       int b, const int* degrees, const int* slices, double b_sup, double mu1,
                       double mu_nevnex, chase_c64* work, void* stream);

/* Spectral estimates by Lanczos (Alg. 6, Sec. 4.2).
 * starts   N x (1 + nvec) start vectors, leading dimension N (host or device);
 *          column 0 drives the bound run of Alg. 6 line 2, columns 1..nvec
 *          the density runs of line 8.  They need not be normalised.
 * k        Lanczos steps per run (1 <= k <= N).
 * approx   1: only b_sup is computed (Alg. 6 lines 4-6); 0: also mu1,
 *          mu_nevnex from the density of states of Eq. 10 (integral equal to
 *          (nev+nex)/N, Gaussian width dos_sigma in the variable mapping
 *          [mu1, b_sup] to [-1, 1]), and, if V is not NULL, the Ritz vectors
 *          of the first density run whose Ritz value lies below mu_nevnex
 *          overwrite the leading columns of V (Alg. 6 line 13).
 * V        N x (nev + nex), leading dimension ldv, in/out, or NULL.
 * b_sup    out: max over the runs of ||f_k|| + max Ritz value (Alg. 6 line 3).
 * mu1, mu_nevnex, theta_absmax  out (host doubles; mu values untouched when approx).
 * Errors: CHASE_INVALID_ARG, CHASE_OUT_OF_MEMORY, CHASE_CUDA_ERROR. */
int chase_lanczos(const chase_c64* H, int64_t N, int64_t ldh, int k, int nvec, int approx, int nev,
                  int nex, double dos_sigma, const chase_c64* starts, chase_c64* V, int64_t ldv,
                  double* b_sup, double* mu1, double* mu_nevnex, double* theta_absmax,
                  void* stream);

/* Optimised degrees (Alg. 5, Eq. 8), host arrays only:
 * t = (ritz_a - c)/e, |rho| = max|t -+ sqrt(t^2 - 1)|,
 * deg = ceil(|log(resid_a / tol) / log|rho||), deg = min(deg + deg_extra, deg_max),
 * degrees_out[a] = deg + mod(deg, 2); lowered by 2 if that exceeds an odd deg_max.
 * When |rho| <= 1 (Ritz value inside the damped interval) or the quotient is
 * not finite the degree is deg_max before the even rounding.
 * Errors: CHASE_INVALID_ARG (NULL array with b > 0, e <= 0, tol <= 0, deg_max < 2). */
int chase_degrees(int b, const double* resid, const double* ritz, double c, double e, double tol,
                  int deg_extra, int deg_max, int* degrees_out);

/* Deflation and locking rule (Alg. 3), host arrays only: writes in order_out
 * the stable permutation that sorts ritz ascending (line 2) and in *n_lock
 * the length of the leading run of that order whose residual is <= tol
 * (line 4 stops at the first residual above tol).
 * Errors: CHASE_INVALID_ARG. */
int chase_lock(int b, const double* ritz, const double* resid, double tol, int* order_out,
               int* n_lock);

/* Eigen-decomposition of a real symmetric tridiagonal matrix, host arrays
 * only: the Lanczos matrix T_k of Alg. 6 (diag[k] on the diagonal, off[k-1]
 * beside it).  Writes the eigenvalues ascending in w[k] and the normalised
 * eigenvectors column-major in z[k*k] (column j belongs to w[j]); the
 * Eq. 10 weights are the squared first components z[j*k]^2.  Implicit QR
 * sweeps with Wilkinson shifts.
 * Errors: CHASE_INVALID_ARG, CHASE_EIGENSOLVER_ERROR (no convergence). */
int chase_tridiag_eigh(int k, const double* diag, const double* off, double* w, double* z);

/* mu_nev+nex of Alg. 6 line 11 from Lanczos Ritz data, host arrays only:
 * the value t at which the integral of the density estimate of Eq. 10
 * (Sec. 4.2) reaches `target` (= (nev + nex) / N in the solver).
 * nruns    number of density runs (n_vec), >= 1.
 * steps    nruns run lengths (>= 1 each).
 * theta    the Ritz values of run 0, then run 1, ... (sum of steps values).
 * weights  the matching weights |Z_1i|^2 (first eigenvector components
 *          squared), same layout; each run's weights sum to 1.
 * The estimate is the average over the runs of sum_i w_i Phi((t -
 * theta_i) / s), s = dos_sigma (b_sup - mu1) / 2 (dos_sigma itself when the
 * interval has collapsed).  The paper leaves its safeguards unpublished;
 * this library keeps the result strictly inside (mu1, b_sup) by a margin
 * of 1e-6 (b_sup - mu1): it halves s, at most 40 times, and failing that
 * returns mu1 + (b_sup - mu1) min(max(target, 1e-3), 0.5), the quantile of
 * a uniform density.
 * mu_out        out: the estimate.
 * halvings_out  out (nullable): halvings taken, or -1 for the uniform fallback.
 * Errors: CHASE_INVALID_ARG (NULL array, a run length < 1, target outside
 * (0, 1), non-finite bounds, mu1 > b_sup, dos_sigma <= 0). */
int chase_dos_estimate(int nruns, const int* steps, const double* theta, const double* weights,
                       double target, double mu1, double b_sup, double dos_sigma, double* mu_out,
                       int* halvings_out);

/* Orthonormalise V against the locked block Y and within itself (Alg. 1
 * line 5, QR of [Y V], keeping Y): block Gram-Schmidt against Y followed by
 * Cholesky QR, twice; if a Cholesky pivot is not safely positive the first
 * pass is replaced by shifted Cholesky QR.  On return span(V_out) equals the
 * part of span([Y V_in]) orthogonal to Y and V_out^H V_out = I.
 * Y        N x nconv, leading dimension ldy (nconv may be 0; Y may then be NULL)
 * V        N x b, leading dimension ldv, in/out; b <= N - nconv.
 * Both arrays device, or both host.
 * Errors: CHASE_INVALID_ARG, CHASE_QR_BREAKDOWN, CHASE_OUT_OF_MEMORY, CHASE_CUDA_ERROR. */
int chase_orthonormalize(const chase_c64* Y, int64_t N, int64_t ldy, int nconv, chase_c64* V,
                         int64_t ldv, int b, void* stream);

/* Rayleigh-Ritz (Alg. 2): G = Q^H H Q, (W, ritz) = eigh(G) with ritz
 * ascending, Q <- Q W.  Q must have orthonormal columns.  If resid is not
 * NULL it receives ||H q_a - ritz_a q_a||_2 for the new columns (Alg. 1
 * line 8).
 * H        N x N, ldh (host or device)
 * Q        N x b, ldq, in/out (same kind as H)
 * ritz     b doubles out; resid b doubles out or NULL (host arrays)
 * Errors: CHASE_INVALID_ARG, CHASE_EIGENSOLVER_ERROR, CHASE_OUT_OF_MEMORY, CHASE_CUDA_ERROR. */
int chase_rayleigh_ritz(const chase_c64* H, int64_t N, int64_t ldh, chase_c64* Q, int64_t ldq,
                        int b, double* ritz, double* resid, void* stream);

/* Residuals (Alg. 1 line 8): resid[a] = ||H v_a - lambda_a v_a||_2.
 * H N x N (ldh), V N x b (ldv), lambda b doubles (host), resid b doubles out (host).
 * H and V both host or both device.
 * Errors: CHASE_INVALID_ARG, CHASE_OUT_OF_MEMORY, CHASE_CUDA_ERROR. */
int chase_residuals(const chase_c64* H, int64_t N, int64_t ldh, const chase_c64* V, int64_t ldv,
                    int b, const double* lambda, double* resid, void* stream);

/* Residual norms with no device allocation (the paper has no counterpart:
 * it exists for callers that cannot let a library allocate device memory,
 * e.g. a host framework that owns all device memory through its own budgeted
 * pool, or a latency-critical caller that cannot afford the device-wide
 * synchronisation cudaMalloc/cudaFree may cause).  Same result as
 * chase_residuals: resid[a] = ||H v_a - lambda_a v_a||_2.
 * H        N x N (ldh), device
 * V        N x b (ldv), device
 * lambda   b doubles, device;  resid  b doubles out, device
 * Scratch is a fixed static device array inside the library of 2^21
 * complex128 entries (32 MiB), held by every GPU that loads the library
 * until the process exits: requires N * b <= 2097152, else
 * CHASE_INVALID_ARG.  Calls no cudaMalloc / cudaFree.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  The address is cached for the
 * life of the process: after a cudaDeviceReset by the application it is
 * stale, and this entry point must not be called again on that device.  All
 * calls share the array: calls whose work overlaps on the GPU race.  H, V,
 * lambda and resid must live on the current device.
 * Errors: CHASE_INVALID_ARG (sizes, non-device arrays, arrays on another
 * device than the current one), CHASE_CUDA_ERROR, CHASE_TIMEOUT. */
int chase_residuals_noalloc(const chase_c64* H, int64_t N, int64_t ldh, const chase_c64* V,
                            int64_t ldv, int b, const double* lambda, double* resid, void* stream);

/* Real symmetric problems (Sec. 5.1: the library is templated on the field
 * as well as the precision).  Same arguments, layouts, ownership and errors
 * as chase_filter, chase_residuals and chase_solve, with float64 matrices
 * and real symmetric H (both triangles stored; the split-BF16 slices read
 * row r of H from its column r).  Flop counts use 2 N^2 per column product
 * (8 N^2 for complex).  Leading dimensions need not be even: odd ones are
 * staged through padded device buffers inside the call. */
int chase_filter_real(const double* H, int64_t N, int64_t ldh, double* V, int64_t ldv, int b,
                      const int* degrees, double b_sup, double mu1, double mu_nevnex, int precision,
                      double* work, void* stream);
int chase_residuals_real(const double* H, int64_t N, int64_t ldh, const double* V, int64_t ldv,
                         int b, const double* lambda, double* resid, void* stream);
int chase_solve_real(const double* H, int64_t N, int64_t ldh, int nev, int nex, double tol,
                     double* V, int64_t ldv, double* Lambda, double* resid,
                     const double* lanczos_starts, const chase_opts* opts, chase_stats* stats,
                     void* stream);

/* Single precision (Sec. 5.1 templates the library on the precision too):
 * complex64 (`_c32`) and float32 (`_f32`) versions of chase_filter,
 * chase_residuals and chase_solve with the same arguments, layouts and
 * errors.  Every product with H, the Gram products and the projected
 * eigensolve (cheevd / ssyevd) run in FP32 on the CUDA cores; the
 * orthogonalisation runs in double on widened copies of the block (Cholesky
 * QR squares the condition number of a filtered block, which FP32 cannot
 * hold) and rounds back.  Eigenvalues, residuals, bounds and tolerances are
 * doubles.  Single precision reaches residuals of about 1e-6 ||H||, so tol
 * should be 1e-5 or larger (Table 1's single-precision column).
 * opts->precision: CHASE_FP64 (the default) keeps the FP32 products; any
 * split value runs the solve's filter on the split-BF16 tensor-core product
 * with the leading 4 slices of each operand (about 2^-28 relative per
 * product entry, finer than FP32 rounding) on widened copies of the active
 * block, rounded back to single precision after the filter. */
int chase_filter_c32(const chase_c32* H, int64_t N, int64_t ldh, chase_c32* V, int64_t ldv, int b,
                     const int* degrees, double b_sup, double mu1, double mu_nevnex,
                     chase_c32* work, void* stream);
int chase_filter_f32(const float* H, int64_t N, int64_t ldh, float* V, int64_t ldv, int b,
                     const int* degrees, double b_sup, double mu1, double mu_nevnex, float* work,
                     void* stream);
int chase_residuals_c32(const chase_c32* H, int64_t N, int64_t ldh, const chase_c32* V,
                        int64_t ldv, int b, const double* lambda, double* resid, void* stream);
int chase_residuals_f32(const float* H, int64_t N, int64_t ldh, const float* V, int64_t ldv, int b,
                        const double* lambda, double* resid, void* stream);
int chase_solve_c32(const chase_c32* H, int64_t N, int64_t ldh, int nev, int nex, double tol,
                    chase_c32* V, int64_t ldv, double* Lambda, double* resid,
                    const chase_c32* lanczos_starts, const chase_opts* opts, chase_stats* stats,
                    void* stream);
int chase_solve_f32(const float* H, int64_t N, int64_t ldh, int nev, int nex, double tol, float* V,
                    int64_t ldv, double* Lambda, double* resid, const float* lanczos_starts,
                    const chase_opts* opts, chase_stats* stats, void* stream);

/* Chebyshev filter (Alg. 4, Eq. 7) of many independent problems at once.
 * The paper filters one matrix per call; this entry point has no
 * counterpart there: it runs Alg. 4 on P problems of different sizes with
 * one grouped launch per degree step, every step of every problem in one
 * CUDA graph.  Problem p is exactly chase_filter(H[p], N[p], ldh[p], V[p],
 * ldv[p], b[p], degrees[p], b_sup[p], mu1[p], mu_nevnex[p], precision, NULL,
 * stream): the same products, coefficients and column retirement.
 * P         number of problems (>= 0).
 * H, V      host arrays of P device pointers: H[p] N[p] x N[p] Hermitian
 *           (leading dimension ldh[p] >= N[p]), V[p] N[p] x b[p] in/out
 *           (ldv[p] >= N[p]), column-major complex128, 16-byte aligned.
 *           V[p] doubles as the second buffer of the recurrence.
 * N, ldh, ldv, b, b_sup, mu1, mu_nevnex   host arrays of P entries; every
 *           problem needs mu1 < mu_nevnex < b_sup.  Problems with N == 0 or
 *           b == 0 are skipped.
 * degrees   host array of P host pointers, b[p] ints each, even and in
 *           [2, 1024], any order.
 * precision CHASE_FP64 or CHASE_SPLIT_BF16.
 * tile      CHASE_TILE_AUTO or a fixed FP64 tile shape (ignored for split).
 * stats     out, or NULL.
 * Workspace: N[p] x b[p] per problem (FP64), plus the slices of every H
 * (28 N[p]^2 bytes) for split; released before return.
 * Errors: CHASE_INVALID_ARG (sizes, bounds, degrees, host H or V),
 * CHASE_OUT_OF_MEMORY, CHASE_CUDA_ERROR, CHASE_TIMEOUT.  On error V may hold
 * partial results. */
int chase_filter_batched(int P, const chase_c64* const* H, const int64_t* N, const int64_t* ldh,
                         chase_c64* const* V, const int64_t* ldv, const int* b,
                         const int* const* degrees, const double* b_sup, const double* mu1,
                         const double* mu_nevnex, int precision, int tile, chase_batch_stats* stats,
                         void* stream);

/* The ChASE eigensolver (Alg. 1) for the nev smallest eigenpairs of H.
 * H        N x N Hermitian, ldh (host or device)
 * V        N x (nev + nex), ldv, in/out (same kind as H).  In: random
 *          start vectors when opts->approx == 0, approximate eigenvectors
 *          when approx == 1 (Sec. 3.3).  Out: Ritz vectors, ascending.
 * Lambda   nev + nex doubles, in/out (host).  In (approx == 1): approximate
 *          eigenvalues; their min and max give mu1 and mu_nevnex.  Out: Ritz
 *          values ascending; the first nev are converged on CHASE_OK.
 * resid    nev + nex doubles out (host): ||H v_a - lambda_a v_a||_2.
 * lanczos_starts  N x (1 + num_lanczos), leading dimension N (same kind as
 *          H): start vectors of the Lanczos runs (random numbers are inputs).
 * opts     NULL for chase_opts_default().
 * stats    out, or NULL.
 * Requires 1 <= nev, 0 <= nex, nev + nex <= N, tol > 0.
 * Returns CHASE_OK, or CHASE_NOT_CONVERGED after max_iter iterations with
 * the current subspace in V, Lambda, resid (Sec. 5.3), or an error status. */
int chase_solve(const chase_c64* H, int64_t N, int64_t ldh, int nev, int nex, double tol,
                chase_c64* V, int64_t ldv, double* Lambda, double* resid,
                const chase_c64* lanczos_starts, const chase_opts* opts, chase_stats* stats,
                void* stream);

/* ChASE (Alg. 1) on P independent problems with the filter of every
 * iteration grouped: each iteration runs Alg. 4 for all problems that are
 * still iterating as one grouped launch per degree step (one CUDA graph, as
 * chase_filter_batched), then Rayleigh-Ritz, QR, residuals, locking and the
 * degree rule of each problem (lines 5-15).  The paper solves one problem
 * per call; this batching has no counterpart there.  Problem p follows the
 * same steps as chase_solve(H[p], N[p], ldh[p], nev[p], nex[p], tol[p], V[p],
 * ldv[p], Lambda[p], resid[p], lanczos_starts[p], opts, stats + p, stream).
 * H, V, lanczos_starts  host arrays of P device pointers (layouts as in
 *          chase_solve; lanczos_starts[p] has leading dimension N[p]).
 * N, ldh, nev, nex, tol, ldv   host arrays of P entries.
 * Lambda, resid   host arrays of P host pointers (nev[p] + nex[p] doubles).
 * opts     shared by every problem (NULL: chase_opts_default).
 * status   out, P ints: each problem's chase_solve status.
 * stats    out, P entries, or NULL; t_filter is the grouped filter's time
 *          shared out by FLOPs, t_total the whole call.
 * bstats   out (sums over all grouped filter calls), or NULL.
 * Returns CHASE_OK when every problem converged, else the first problem
 * status that is not CHASE_OK, or an error status of the call
 * (CHASE_INVALID_ARG, CHASE_OUT_OF_MEMORY, CHASE_CUDA_ERROR, CHASE_TIMEOUT,
 * CHASE_QR_BREAKDOWN, CHASE_EIGENSOLVER_ERROR), after which status is not
 * written. */
int chase_solve_batched(int P, const chase_c64* const* H, const int64_t* N, const int64_t* ldh,
                        const int* nev, const int* nex, const double* tol, chase_c64* const* V,
                        const int64_t* ldv, double* const* Lambda, double* const* resid,
                        const chase_c64* const* lanczos_starts, const chase_opts* opts,
                        int* status, chase_stats* stats, chase_batch_stats* bstats, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CHASE_H_ */
