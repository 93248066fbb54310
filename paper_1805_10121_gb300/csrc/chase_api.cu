// Entry points of libchase and the ChASE driver (Alg. 1) on one GPU.
//
// The driver keeps H, the search block V (locked prefix + active suffix,
// the buffer layout of Sec. 5.1.1) and all workspace in device memory.  Per
// iteration only nev+nex Ritz values and residuals come back to the host,
// where the locking rule (Alg. 3), the spectral updates (Alg. 1 lines
// 10-11) and the degree rule (Alg. 5) run; the resulting column permutation
// goes back to the device as one gather.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <condition_variable>
#include <functional>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "chase.h"
#include "common.cuh"
#include "context.hpp"

namespace chase {

namespace {

constexpr int kMaxDegAllowed = 1024;
constexpr int kBatchWorkers = 8;  // host threads for the per-problem phases of a batched solve
constexpr int kBatchStreams = 16;  // streams the batched QR / Rayleigh-Ritz launches spread over

// Scalar types of the solver: complex128 and float64 (the default), complex64
// and float32 (the single-precision entry points; Sec. 5.1 templates the
// library on both the field and the precision).
template <class T>
constexpr bool is_cplx = std::is_same<T, chase_c64>::value || std::is_same<T, chase_c32>::value;
template <class T>
constexpr bool is_single = std::is_same<T, chase_c32>::value || std::is_same<T, float>::value;

// Rounding unit, Cholesky pivot threshold (double precision: the single-
// precision solver orthogonalises in double) and Lanczos breakdown threshold.
template <class T>
struct Prec {
  static constexpr double u = 1.1102230246251565e-16;
  static constexpr double chol_tol = 1e-12;
  static constexpr double lanczos_tiny = 1e-13;
};
template <>
struct Prec<chase_c32> {
  static constexpr double lanczos_tiny = 1e-6;
};
template <>
struct Prec<float> {
  static constexpr double lanczos_tiny = 1e-6;
};

// Real float64 problems: every matrix handed to the TMA product has an even
// leading dimension (TMA strides are multiples of 16 bytes), so internal
// buffers pad their rows to even; complex128 columns are already 16-byte
// multiples, and the single-precision products do not use TMA.
template <class T>
int64_t ld_pad(int64_t n) {
  return std::is_same<T, double>::value ? std::max<int64_t>((n + 1) / 2 * 2, 2)
                                        : std::max<int64_t>(n, 1);
}
template <class T>
T from_real(double v);
template <>
chase_c64 from_real<chase_c64>(double v) {
  return chase_c64{v, 0.0};
}
template <>
double from_real<double>(double v) {
  return v;
}
template <>
chase_c32 from_real<chase_c32>(double v) {
  return chase_c32{static_cast<float>(v), 0.f};
}
template <>
float from_real<float>(double v) {
  return static_cast<float>(v);
}

// Events bracketing the phases of one call, accumulated into seconds.
struct PhaseTimer {
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  double* acc = nullptr;
  explicit PhaseTimer(cudaStream_t s) : st(s) {}
  ~PhaseTimer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  void begin(double* target) {
    if (!a && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)) {
      cudaGetLastError();
      return;
    }
    acc = target;
    cudaEventRecord(a, st);
  }
  void end() {
    if (!a || !b) return;
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (acc) *acc += 1e-3 * ms;
  }
};

// A product with H on the FP64 path, recorded for
// chase_kernel_timing as one launch.  Executed FLOPs: the DMMA tile kernel
// forms complex products in the 3M form (6 of 8 real FLOPs); the few-column
// kernel and real products execute all of them.
template <class T>
int timed_h_product(Dev& d, const T* H, int64_t N, int64_t ldh, const T* X, int64_t ldx, int b,
                    T* Y, int64_t ldy, int j0, double alpha, double beta, double shift) {
  if constexpr (is_single<T>) return gemm(d, N, N, H, ldh, X, ldx, b, Y, ldy, j0, b, alpha, beta, shift);
  KernelTimer kt(d.st, CHASE_TIMED_FP64_PRODUCT);
  CHASE_TRY(gemm(d, N, N, H, ldh, X, ldx, b, Y, ldy, j0, b, alpha, beta, shift));
  const int w = b - j0;
  const double alg = (is_cplx<T> ? 8.0 : 2.0) * static_cast<double>(N) * static_cast<double>(N) * w;
  kt.end(w > 0 ? 1 : 0, alg, is_cplx<T> && w > kFewColMax ? 0.75 * alg : alg);
  return CHASE_OK;
}

// Alg. 4 on a block whose columns are sorted by ascending degree.
// X (N x b, ldx) holds the input and receives the output; Wk (N x b, ldw)
// is the second buffer of the double buffering.  start[i] = number of
// columns with degree < i for i = 0 .. maxdeg + 1 (columns with degree < i
// have retired before step i).  Returns the column-product count.
// One filter product: the FP64 DMMA kernel, or the split-BF16 tensor-core
// kernel when slices of H are given.
template <class T>
int filter_product(Dev& d, const T* H, int64_t N, int64_t ldh, const SplitH* sh, SplitX* sx,
                   const T* X, int64_t ldx, int b, T* Y, int64_t ldy, int j0,
                   double alpha, double beta, double shift, int nslices = 7) {
  if constexpr (!is_single<T>) {
    if (sh) return zgemm_split(d, *sh, *sx, X, ldx, j0, b, Y, ldy, alpha, beta, shift, nslices);
  }
  return timed_h_product(d, H, N, ldh, X, ldx, b, Y, ldy, j0, alpha, beta, shift);
}

// A run of columns [col0, col0 + ncols) of the filter block that share one
// precision (nslices of the split product; 7 = full) and are sorted by
// ascending degree: start[i] (i = 0 .. maxdeg + 1) counts the run's columns
// of degree < i, which have retired before step i (Alg. 4 lines 12-14).
struct FilterGroup {
  int col0 = 0, ncols = 0, nslices = 7;
  std::vector<int> start;
};

// Alg. 4 on a block made of runs of columns, each sorted by degree.  X (N x
// b, ldx) holds the input and receives the output; Wk (N x b, ldw) is the
// second buffer of the double buffering.  Every run is an independent set of
// columns of the same three-term recurrence (the coefficients of Eq. 7 do
// not depend on the column), filtered with its own precision and retiring
// its own finished columns.  Adds the column products to *matvecs and those
// made with fewer than 7 slices to *matvecs_low.
template <class T>
int filter_groups(Dev& d, const T* H, int64_t N, int64_t ldh, T* X, int64_t ldx, T* Wk,
                  int64_t ldw, const std::vector<FilterGroup>& groups, int maxdeg, double b_sup,
                  double mu1, double mu_nn, long long* matvecs, const SplitH* sh = nullptr,
                  SplitX* sx = nullptr, long long* matvecs_low = nullptr) {
  const double c = 0.5 * (b_sup + mu_nn);  // Alg. 4 line 2
  const double e = 0.5 * (b_sup - mu_nn);
  const double sigma1 = e / (mu1 - c);     // line 3
  long long mv = 0, low = 0;
  auto product = [&](const FilterGroup& g, int s, const T* src, int64_t lds, T* dst, int64_t ldd,
                     double alpha, double beta) -> int {
    const int j0 = g.col0 + s, j1 = g.col0 + g.ncols;
    if (j0 >= j1) return CHASE_OK;
    CHASE_TRY(filter_product(d, H, N, ldh, sh, sx, src, lds, j1, dst, ldd, j0, alpha, beta, c,
                             g.nslices));
    mv += j1 - j0;
    if (sh && g.nslices < 7) low += j1 - j0;
    return CHASE_OK;
  };
  // line 4: W = (sigma_1 / e) (H - c I) V
  for (const FilterGroup& g : groups) CHASE_TRY(product(g, 0, X, ldx, Wk, ldw, sigma1 / e, 0.0));
  double sigma = sigma1;  // line 5
  T* Vb = X;
  T* Wb = Wk;
  int64_t ldV = ldx, ldW = ldw;
  for (int i = 2; i <= maxdeg; ++i) {  // line 7
    const double tau = 1.0 / (2.0 / sigma1 - sigma);  // line 8
    // line 9: V[:, s:] = 2 (tau / e) (H - c I) W[:, s:] - tau sigma V[:, s:],
    // s = the first column of each run with degree >= i (lines 12-14)
    for (const FilterGroup& g : groups)
      CHASE_TRY(product(g, g.start[i], Wb, ldW, Vb, ldV, 2.0 * tau / e, -tau * sigma));
    std::swap(Vb, Wb);  // line 10
    std::swap(ldV, ldW);
    sigma = tau;  // line 11
  }
  // With even degrees the last product of every column lands in X (Sec. 4.1.3).
  if (Wb != X) {
    set_error("filter: odd maximum degree");
    return CHASE_INVALID_ARG;
  }
  if (matvecs) *matvecs += mv;
  if (matvecs_low) *matvecs_low += low;
  return CHASE_OK;
}

// Alg. 4 on a block whose columns are all sorted by ascending degree and
// filtered with one precision (start as in FilterGroup).
template <class T>
int filter_sorted(Dev& d, const T* H, int64_t N, int64_t ldh, T* X, int64_t ldx,
                  T* Wk, int64_t ldw, int b, const int* start, int maxdeg, double b_sup,
                  double mu1, double mu_nn, long long* matvecs, const SplitH* sh = nullptr,
                  SplitX* sx = nullptr, int nslices = 7) {
  std::vector<FilterGroup> one(1);
  one[0].ncols = b;
  one[0].nslices = nslices;
  one[0].start.assign(start, start + maxdeg + 2);
  return filter_groups(d, H, N, ldh, X, ldx, Wk, ldw, one, maxdeg, b_sup, mu1, mu_nn, matvecs,
                       sh, sx);
}

void starts_from_sorted(const int* m, int b, int maxdeg, std::vector<int>& start) {
  start.assign(maxdeg + 2, 0);
  int s = 0;
  for (int i = 0; i <= maxdeg + 1; ++i) {
    while (s < b && m[s] < i) ++s;
    start[i] = s;
  }
}

// ---------------------------------------------------------------------------
// Orthogonalisation (Alg. 1 line 5): block Gram-Schmidt against the locked
// block Y and Cholesky QR, twice; shifted Cholesky QR first when a pivot is
// not safely positive.
// ---------------------------------------------------------------------------
template <class T>
struct OrthWork {
  T* P = nullptr;     // nconv x b, leading dimension ld_pad(nconv)
  T* G = nullptr;     // b x b, leading dimension ld_pad(b)
  T* Rinv = nullptr;  // panel workspace of the blocked Cholesky / solve, >= 32 b
  double* nrm = nullptr;  // b
};

template <class T>
int orth_alloc(Dev& d, int64_t N, int nconv, int b, OrthWork<T>& w) {
  (void)N;
  CHASE_TRY(d.alloc(&w.P, static_cast<size_t>(ld_pad<T>(std::max(nconv, 1))) * b));
  CHASE_TRY(d.alloc(&w.G, static_cast<size_t>(ld_pad<T>(b)) * b));
  CHASE_TRY(d.alloc(&w.Rinv, static_cast<size_t>(std::max(b, 32)) * b));
  CHASE_TRY(d.alloc(&w.nrm, static_cast<size_t>(b)));
  return CHASE_OK;
}

// One Cholesky QR pass in two halves: cholqr_launch projects V against Y
// and factors its Gram matrix (a breakdown sets KERR_CHOL_BREAKDOWN in d.err,
// read at the caller's next synchronisation); cholqr_finish applies the
// factor, V <- V L^-H.
template <class T>
int cholqr_launch(Dev& d, int64_t N, const T* Y, int64_t ldy, int nconv, T* V, int64_t ldv,
                  int b, OrthWork<T>& w, double shift, double* flops) {
  const int64_t ldp = ld_pad<T>(nconv), ldg = ld_pad<T>(b);
  if (nconv > 0) {  // V <- V - Y (Y^H V)
    CHASE_TRY(gram(d, N, Y, ldy, nconv, V, ldv, b, w.P, ldp));
    CHASE_TRY(gemm(d, N, nconv, Y, ldy, w.P, ldp, b, V, ldv, 0, b, -1.0, 1.0, 0.0));
    *flops += (is_cplx<T> ? 16.0 : 4.0) * N * nconv * b;
  }
  CHASE_TRY(gram(d, N, V, ldv, b, V, ldv, b, w.G, ldg, /*lower=*/true));  // the factor reads only it
  return cholesky_blocked(d, w.G, ldg, b, Prec<T>::chol_tol, shift, w.nrm, w.Rinv);
}

template <class T>
int cholqr_finish(Dev& d, int64_t N, T* V, int64_t ldv, int b, OrthWork<T>& w, double* flops) {
  // V <- V L^-H (= V R^-1 with R = L^H), in place
  CHASE_TRY(trsm_right_lh(d, V, ldv, N, w.G, ld_pad<T>(b), b, w.Rinv));
  *flops += (is_cplx<T> ? 1.0 : 0.25) *
            (8.0 * N * b * b + 4.0 * N * b * b + 8.0 * b * b * b / 3.0);
  return CHASE_OK;
}

template <class T>
int cholqr_pass(Dev& d, int64_t N, const T* Y, int64_t ldy, int nconv, T* V,
                int64_t ldv, int b, OrthWork<T>& w, double shift, double* flops) {
  CHASE_TRY(cholqr_launch(d, N, Y, ldy, nconv, V, ldv, b, w, shift, flops));
  int st = d.sync_check("cholesky");
  if (st != CHASE_OK) {
    cudaMemsetAsync(d.err, 0, sizeof(int), d.st);
    return st;
  }
  return cholqr_finish(d, N, V, ldv, b, w, flops);
}

template <class T>
int orth_core(Dev& d, int64_t N, const T* Y, int64_t ldy, int nconv, T* V,
              int64_t ldv, int b, OrthWork<T>& w, double* flops) {
  if (b == 0) return CHASE_OK;
  // QR of V D equals QR of V for any positive diagonal D: normalise columns.
  CHASE_TRY(launch_col_norms(d, V, ldv, N, b, w.nrm));
  CHASE_TRY(launch_col_inv_scale(d, V, ldv, N, b, w.nrm));
  int st = cholqr_pass(d, N, Y, ldy, nconv, V, ldv, b, w, 0.0, flops);
  if (st == CHASE_QR_BREAKDOWN) {
    // Shifted Cholesky QR: ||G||_2 <= trace(G) <= b for columns of norm <= 1.
    const double u = Prec<T>::u;
    const double shift = 11.0 * (static_cast<double>(N) * b + static_cast<double>(b) * (b + 1)) * u * b;
    CHASE_TRY(launch_col_norms(d, V, ldv, N, b, w.nrm));
    CHASE_TRY(launch_col_inv_scale(d, V, ldv, N, b, w.nrm));
    st = cholqr_pass(d, N, Y, ldy, nconv, V, ldv, b, w, shift, flops);
    if (st == CHASE_QR_BREAKDOWN) {
      set_error("orthonormalisation: shifted Cholesky QR broke down");
      return CHASE_QR_BREAKDOWN;
    }
    CHASE_TRY(st);
    st = cholqr_pass(d, N, Y, ldy, nconv, V, ldv, b, w, 0.0, flops);
  }
  CHASE_TRY(st);
  st = cholqr_pass(d, N, Y, ldy, nconv, V, ldv, b, w, 0.0, flops);
  if (st == CHASE_QR_BREAKDOWN) set_error("orthonormalisation: Cholesky QR broke down");
  return st;
}

// Single precision: the orthogonalisation runs in double on widened copies
// (Cholesky QR squares the condition number of a filtered block, which FP32
// would not hold), then the block is rounded back.
template <class T>
int orth_widened(Dev& d, int64_t N, const T* Y, int64_t ldy, int nconv, T* V, int64_t ldv, int b,
                 double* flops) {
  using D = typename std::conditional<std::is_same<T, chase_c32>::value, chase_c64, double>::type;
  if (b == 0) return CHASE_OK;
  const int64_t lD = ld_pad<D>(N);
  D *Yd = nullptr, *Vd = nullptr;
  if (nconv > 0) {
    CHASE_TRY(d.alloc(&Yd, static_cast<size_t>(lD) * nconv));
    CHASE_TRY(launch_convert(d, Y, ldy, Yd, lD, N, nconv));
  }
  CHASE_TRY(d.alloc(&Vd, static_cast<size_t>(lD) * b));
  CHASE_TRY(launch_convert(d, V, ldv, Vd, lD, N, b));
  OrthWork<D> w;
  CHASE_TRY(orth_alloc(d, N, nconv, b, w));
  CHASE_TRY(orth_core(d, N, Yd, lD, nconv, Vd, lD, b, w, flops));
  return launch_convert(d, Vd, lD, V, ldv, N, b);
}

template <class T>
int orth_any(Dev& d, int64_t N, const T* Y, int64_t ldy, int nconv, T* V, int64_t ldv, int b,
             OrthWork<T>& w, double* flops) {
  if constexpr (is_single<T>)
    return orth_widened(d, N, Y, ldy, nconv, V, ldv, b, flops);
  else
    return orth_core(d, N, Y, ldy, nconv, V, ldv, b, w, flops);
}

// ---------------------------------------------------------------------------
// Rayleigh-Ritz (Alg. 2) with residuals (Alg. 1 line 8)
// ---------------------------------------------------------------------------
template <class T>
struct RRWork {
  T* HQ = nullptr;  // N x b (leading dimension ld_pad(N) here and below)
  T* T2 = nullptr;  // N x b
  T* T3 = nullptr;  // N x b
  T* G = nullptr;   // b x b, leading dimension ld_pad(b)
};

template <class T>
int rr_alloc(Dev& d, int64_t N, int b, RRWork<T>& w) {
  const size_t nb = static_cast<size_t>(ld_pad<T>(N)) * b;
  CHASE_TRY(d.alloc(&w.HQ, nb));
  CHASE_TRY(d.alloc(&w.T2, nb));
  CHASE_TRY(d.alloc(&w.T3, nb));
  CHASE_TRY(d.alloc(&w.G, static_cast<size_t>(ld_pad<T>(b)) * b));
  return CHASE_OK;
}

// Alg. 2 in three parts: rr_pre forms H Q (FP64, or the split product for
// CHASE_SPLIT_BF16_RR) and the lower triangle of G = Q^H (H Q) mirrored to
// the upper one; the eigensolve of G follows (one problem: eigh_device, a
// batch: eigh_batched); rr_post forms Q W, the residuals from (H Q) W, and
// copies Q W into Q.
template <class T>
int rr_pre(Dev& d, const T* H, int64_t N, int64_t ldh, const T* Q, int64_t ldq, int b,
           RRWork<T>& w, const SplitH* sh = nullptr, SplitX* sx = nullptr,
           double* t_hq = nullptr) {
  const int64_t lN = ld_pad<T>(N), lg = ld_pad<T>(b);
  PhaseTimer tq(d.st);  // the product alone (synchronises only when timed)
  if (t_hq) tq.begin(t_hq);
  bool on_split = false;
  if constexpr (!is_single<T>) {
    if (sh) {  // H Q on the split product (CHASE_SPLIT_BF16_RR)
      CHASE_TRY(zgemm_split(d, *sh, *sx, Q, ldq, 0, b, w.HQ, lN, 1.0, 0.0, 0.0));
      on_split = true;
    }
  }
  if (!on_split) CHASE_TRY(timed_h_product(d, H, N, ldh, Q, ldq, b, w.HQ, lN, 0, 1.0, 0.0, 0.0));
  if (t_hq) tq.end();
  // G = Q^H H Q is Hermitian up to rounding: form its lower triangle (the one
  // the eigensolver reads) and take the upper one from it
  CHASE_TRY(gram(d, N, Q, ldq, b, w.HQ, lN, b, w.G, lg, /*lower=*/true));
  return launch_fill_upper_hermitian(d, w.G, lg, b);
}

template <class T>
int rr_post(Dev& d, int64_t N, T* Q, int64_t ldq, int b, const double* w_dev, double* res_dev,
            RRWork<T>& w, double* flops) {
  const int64_t lN = ld_pad<T>(N), lg = ld_pad<T>(b);
  CHASE_TRY(gemm(d, N, b, Q, ldq, w.G, lg, b, w.T2, lN, 0, b, 1.0, 0.0, 0.0));  // Q W
  if (res_dev) {
    // H (Q W) = (H Q) W: the residual reuses the product with H
    CHASE_TRY(gemm(d, N, b, w.HQ, lN, w.G, lg, b, w.T3, lN, 0, b, 1.0, 0.0, 0.0));
    CHASE_TRY(launch_resid_norms(d, w.T3, lN, w.T2, lN, N, b, w_dev, res_dev));
  }
  CHASE_TRY(copy_block(d, Q, ldq, w.T2, lN, N, b, cudaMemcpyDeviceToDevice));
  *flops += (is_cplx<T> ? 1.0 : 0.25) * (8.0 * N * N * b + 8.0 * N * b * b * (res_dev ? 3.0 : 2.0));
  return CHASE_OK;
}

template <class T>
int rr_core(Dev& d, const T* H, int64_t N, int64_t ldh, T* Q, int64_t ldq, int b,
            double* w_dev, double* res_dev, RRWork<T>& w, double* t_eigh, double* flops,
            const SplitH* sh = nullptr, SplitX* sx = nullptr, double* t_hq = nullptr) {
  if (b == 0) return CHASE_OK;
  const int64_t lg = ld_pad<T>(b);
  CHASE_TRY(rr_pre(d, H, N, ldh, Q, ldq, b, w, sh, sx, t_hq));
  PhaseTimer tm(d.st);
  tm.begin(t_eigh);
  CHASE_TRY(eigh_device(d, w.G, lg, b, w_dev));  // (W, Lambda) = TSOLVE(G)
  tm.end();
  return rr_post(d, N, Q, ldq, b, w_dev, res_dev, w, flops);
}

// ---------------------------------------------------------------------------
// Lanczos (Alg. 6)
// ---------------------------------------------------------------------------
struct LanczosOut {
  double b_sup = 0, mu1 = 0, mu_nn = 0, theta_absmax = 0;
  long long matvecs = 0;
};

// starts: N x r device (ld N), r = 1 (approx) or 1 + nvec.  V: N x ncolv
// device or NULL.
template <class T>
int lanczos_core(Dev& d, const T* H, int64_t N, int64_t ldh, int k, int nvec, bool approx,
                 int nev, int nex, double dos_sigma, const T* starts, int64_t lds, T* V,
                 int64_t ldv, int ncolv, LanczosOut& out) {
  const int r = approx ? 1 : 1 + nvec;
  const int64_t lN = ld_pad<T>(N);
  T* U = nullptr;   // N x (k r), leading dimension lN: vector j of run c is column j r + c
  T* Wt = nullptr;  // N x r
  double *alpha = nullptr, *beta = nullptr;
  CHASE_TRY(d.alloc(&U, static_cast<size_t>(lN) * k * r));
  CHASE_TRY(d.alloc(&Wt, static_cast<size_t>(lN) * r));
  CHASE_TRY(d.alloc(&alpha, static_cast<size_t>(k) * r));
  CHASE_TRY(d.alloc(&beta, static_cast<size_t>(k) * r));
  CHASE_TRY(copy_block(d, U, lN, starts, lds, N, r, cudaMemcpyDeviceToDevice));
  CHASE_TRY(launch_normalize_cols(d, U, lN, N, r));
  for (int j = 0; j < k; ++j) {
    T* Vj = U + static_cast<size_t>(j) * r * lN;
    const T* Vp = j > 0 ? U + static_cast<size_t>(j - 1) * r * lN : nullptr;
    T* Vn = j + 1 < k ? U + static_cast<size_t>(j + 1) * r * lN : nullptr;
    CHASE_TRY(gemm(d, N, N, H, ldh, Vj, lN, r, Wt, lN, 0, r, 1.0, 0.0, 0.0));  // A v_j
    CHASE_TRY(launch_lanczos_step(d, N, lN, r, j, Vj, Vp, Wt, Vn, alpha, beta,
                                  Prec<T>::lanczos_tiny));
  }
  std::vector<double> ha(static_cast<size_t>(k) * r), hb(static_cast<size_t>(k) * r);
  CHASE_CUDA(cudaMemcpyAsync(ha.data(), alpha, ha.size() * sizeof(double), cudaMemcpyDeviceToHost, d.st));
  CHASE_CUDA(cudaMemcpyAsync(hb.data(), beta, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, d.st));
  CHASE_TRY(d.sync_check("lanczos"));
  out.matvecs = static_cast<long long>(k) * r;  // column products with H

  // per run: truncate at the first step whose beta is rounding noise
  std::vector<std::vector<double>> theta(r), Z(r);
  std::vector<int> steps(r);
  std::vector<double> fnorm(r);
  for (int c = 0; c < r; ++c) {
    int st = k;
    double scale = 0.0;
    for (int j = 0; j < k; ++j) {
      const double a = ha[static_cast<size_t>(j) * r + c], bj = hb[static_cast<size_t>(j) * r + c];
      scale = std::max(scale, std::max(std::fabs(a), bj));
      if (!(bj > Prec<T>::lanczos_tiny * scale)) {
        st = j + 1;
        break;
      }
    }
    steps[c] = st;
    std::vector<double> dg(st), of(std::max(st - 1, 0));
    for (int j = 0; j < st; ++j) dg[j] = ha[static_cast<size_t>(j) * r + c];
    for (int j = 0; j + 1 < st; ++j) of[j] = hb[static_cast<size_t>(j) * r + c];
    fnorm[c] = hb[static_cast<size_t>(st - 1) * r + c];
    theta[c].resize(st);
    Z[c].resize(static_cast<size_t>(st) * st);
    if (!tridiag_eigh(st, dg.data(), of.data(), theta[c].data(), Z[c].data())) {
      set_error("lanczos: tridiagonal eigensolve did not converge");
      return CHASE_EIGENSOLVER_ERROR;
    }
  }
  double bsup = fnorm[0] + theta[0].back();  // Alg. 6 line 3
  double absmax = 0.0;
  for (int c = 0; c < r; ++c) {
    bsup = std::max(bsup, fnorm[c] + theta[c].back());
    for (double t : theta[c]) absmax = std::max(absmax, std::fabs(t));
  }
  out.b_sup = bsup;
  out.theta_absmax = absmax;
  if (approx) return CHASE_OK;

  // density runs are c = 1 .. nvec
  double mu1 = theta[1][0];
  for (int c = 2; c < r; ++c) mu1 = std::min(mu1, theta[c][0]);  // Alg. 6 line 12
  // Eq. 10 over the density runs, quantile of line 11 with its safeguard
  std::vector<int> dsteps(steps.begin() + 1, steps.end());
  std::vector<double> dtheta, dw;
  for (int c = 1; c < r; ++c)
    for (int i = 0; i < steps[c]; ++i) {
      const double z0 = Z[c][static_cast<size_t>(i) * steps[c]];
      dtheta.push_back(theta[c][i]);
      dw.push_back(z0 * z0);
    }
  const double target = static_cast<double>(nev + nex) / static_cast<double>(N);  // line 11
  const double mu_nn =
      dos_estimate(nvec, dsteps.data(), dtheta.data(), dw.data(), target, mu1, bsup, dos_sigma,
                   nullptr, nullptr);
  out.mu1 = mu1;
  out.mu_nn = mu_nn;

  if (V && ncolv > 0) {  // line 13: Ritz vectors of the first density run
    const int st = steps[1];
    std::vector<int> sel;
    for (int i = 0; i < st && static_cast<int>(sel.size()) < ncolv; ++i)
      if (theta[1][i] < out.mu_nn) sel.push_back(i);
    if (!sel.empty()) {
      const int ns = static_cast<int>(sel.size());
      const int64_t lz = ld_pad<T>(st);
      std::vector<T> zs(static_cast<size_t>(lz) * ns, from_real<T>(0.0));
      for (int a = 0; a < ns; ++a)
        for (int i = 0; i < st; ++i)
          zs[static_cast<size_t>(a) * lz + i] = from_real<T>(Z[1][static_cast<size_t>(sel[a]) * st + i]);
      T* dz = nullptr;
      CHASE_TRY(d.alloc(&dz, zs.size()));
      CHASE_CUDA(cudaMemcpyAsync(dz, zs.data(), zs.size() * sizeof(T),
                                 cudaMemcpyHostToDevice, d.st));
      // U_1 Z_sel: basis of run 1 is columns j r + 1, i.e. leading dimension r lN
      CHASE_TRY(gemm(d, N, st, U + lN, static_cast<int64_t>(r) * lN, dz, lz, ns, V, ldv, 0, ns,
                     1.0, 0.0, 0.0));
      CHASE_TRY(d.sync_check("lanczos ritz vectors"));
    }
  }
  return CHASE_OK;
}

// Stage an array that may live on the host into device memory.  Real
// device arrays whose leading dimension is odd are staged too (the TMA
// products need even leading dimensions).
template <class T>
bool needs_stage(bool on_dev, int64_t ld) {
  return !on_dev || (std::is_same<T, double>::value && (ld & 1));
}

template <class T>
int stage_in(Dev& d, bool on_dev, const T* src, int64_t ld, int64_t rows, int64_t cols, T** dst,
             int64_t* ldd) {
  if (!needs_stage<T>(on_dev, ld)) {
    *dst = const_cast<T*>(src);
    *ldd = ld;
    return CHASE_OK;
  }
  const int64_t lp = ld_pad<T>(rows);
  CHASE_TRY(d.alloc(dst, static_cast<size_t>(lp) * std::max<int64_t>(cols, 1)));
  *ldd = lp;
  return copy_block(d, *dst, lp, src, ld, rows, cols,
                    on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
}

bool ld_ok(int64_t ld, int64_t n) { return ld >= std::max<int64_t>(1, n); }

// One ChASE solve (Alg. 1) as a sequence of phases, so that the filter of
// many solves can run as one grouped launch: setup (staging, workspace,
// line 1-2), then per iteration begin_iteration (line 3 and the bound
// check), the filter (line 4), after_filter (lines 5-15), and finally
// finish (ascending output).
// Inputs must be finite: a NaN or Inf in H or a block would otherwise run
// through every step and surface, if at all, as a breakdown far from its
// cause.  One pass of the column-norm kernel per array (a norm that
// overflows, |entries| above about 1e154, is rejected too); `what` names
// the array in the message.
template <class T>
int check_finite(Dev& d, const T* X, int64_t ld, int64_t rows, int64_t cols, const char* where,
                 const char* what) {
  if (rows == 0 || cols == 0) return CHASE_OK;
  double* nrm = nullptr;
  CHASE_TRY(d.alloc(&nrm, static_cast<size_t>(cols)));
  CHASE_TRY(launch_col_norms(d, X, ld, rows, static_cast<int>(cols), nrm));
  std::vector<double> h(static_cast<size_t>(cols));
  CHASE_CUDA(cudaMemcpyAsync(h.data(), nrm, sizeof(double) * cols, cudaMemcpyDeviceToHost, d.st));
  CHASE_TRY(d.sync_check(where));
  for (int64_t j = 0; j < cols; ++j)
    if (!std::isfinite(h[static_cast<size_t>(j)])) {
      set_error("%s: %s holds a non-finite entry (or one beyond 1e154) in column %lld", where,
                what, static_cast<long long>(j));
      return CHASE_INVALID_ARG;
    }
  return CHASE_OK;
}

template <class T>
struct Solver {
  // arguments
  const T* H = nullptr;
  int64_t N = 0, ldh = 0;
  int nev = 0, nex = 0, nx = 0;
  double tol = 0;
  T* V = nullptr;
  int64_t ldv = 0;
  double* Lambda = nullptr;
  double* resid = nullptr;
  const T* starts = nullptr;
  chase_opts o{};
  bool dev = true;
  // device state
  T *dH = nullptr, *dV = nullptr, *dS = nullptr, *Wk = nullptr;
  int64_t lh = 0, lv = 0, ls = 0, lw = 0;
  OrthWork<T> ow;
  RRWork<T> rw;
  SplitH sh;
  SplitX sx;
  // single precision with CHASE_SPLIT_BF16: the filter runs on widened FP64
  // copies of the active block (Dv, Dw), the product with 4 slices
  using Wide = typename std::conditional<is_cplx<T>, chase_c64, double>::type;
  Wide *Dv = nullptr, *Dw = nullptr;
  int64_t lD = 0;
  bool split = false;
  bool split_rr = false;            // H Q of Rayleigh-Ritz on the split product too
  const SplitH* rr_slices = nullptr;  // the slices of H used there
  SplitX* rr_sx = nullptr;
  double *dw = nullptr, *dres = nullptr;
  int* dperm = nullptr;
  // host state
  double N2 = 0, b_sup = 0, mu1 = 0, mu_nn = 0, h = 0, tol_eff = 0;
  int d0 = 0, nconv = 0, iter = 0, status = CHASE_OK, maxdeg = 0;
  bool grouped = false;  // the batched solve filters through the grouped kernels
  std::vector<int> m, order, perm, start;
  // slices of the split product per column (7 = full precision; the FP64
  // filter ignores it), and the runs of equal precision the filter works on
  std::vector<int> cls;
  std::vector<FilterGroup> groups;
  std::vector<double> ritz, res, ra, rr;
  chase_stats S{};

  // FLOPs per entry of a product with H: complex multiply-add 8, real 2
  static constexpr double kMv = is_cplx<T> ? 8.0 : 2.0;

  // active block of the current iteration
  int b() const { return nx - nconv; }
  T* Va() const { return dV + static_cast<size_t>(nconv) * lv; }
  bool more() const { return status == CHASE_OK && nconv < nev && iter < o.max_iter; }

  // Everything before the loop of Alg. 1; `grouped_split` leaves the slices
  // of H to the caller.
  int setup(Dev& d, bool grouped_split) {
    std::memset(&S, 0, sizeof(S));
    nx = nev + nex;
    PhaseTimer tm(d.st);
    const int r = o.approx ? 1 : 1 + o.num_lanczos;
    CHASE_TRY(stage_in(d, dev, H, ldh, N, N, &dH, &lh));
    if (o.storage == CHASE_STORAGE_LOWER) {  // the full matrix from its lower triangle
      T* full = nullptr;
      const int64_t lf = ld_pad<T>(N);
      CHASE_TRY(d.alloc(&full, static_cast<size_t>(lf) * N));
      CHASE_TRY(launch_hermitian_from_lower(d, dH, lh, full, lf, N));
      dH = full;
      lh = lf;
    }
    CHASE_TRY(stage_in(d, dev, V, ldv, N, nx, &dV, &lv));
    CHASE_TRY(stage_in(d, dev, starts, N, N, r, &dS, &ls));
    CHASE_TRY(check_finite(d, dH, lh, N, N, "chase_solve", "H"));
    CHASE_TRY(check_finite(d, dV, lv, N, nx, "chase_solve", "V"));
    CHASE_TRY(check_finite(d, dS, ls, N, r, "chase_solve", "lanczos_starts"));
    lw = ld_pad<T>(N);
    CHASE_TRY(d.alloc(&Wk, static_cast<size_t>(lw) * nx));  // filter double buffer / permutation scratch
    CHASE_TRY(orth_alloc(d, N, nx, nx, ow));
    CHASE_TRY(rr_alloc(d, N, nx, rw));
    // single precision: every product in FP32 on the CUDA cores, or with
    // CHASE_SPLIT_BF16 the filter's products on the split tensor-core
    // product (4 slices, about 2^-28 relative: finer than FP32 rounding)
    split = is_single<T> ? o.precision != CHASE_FP64
                         : (o.precision == CHASE_SPLIT_BF16 || o.precision == CHASE_SPLIT_BF16_RR ||
                            o.precision == CHASE_SPLIT_BF16_ADAPT);
    split_rr = !is_single<T> && o.precision == CHASE_SPLIT_BF16_RR;
    if (split && !grouped_split) {  // slices of H once per solve, slice workspace for the block
      CHASE_TRY(split_prepare_h(d, dH, N, lh, sh));
      CHASE_TRY(split_alloc_x(d, N, nx, sx, is_cplx<T>));
      rr_slices = &sh;
      rr_sx = &sx;
      if constexpr (is_single<T>) {
        lD = ld_pad<Wide>(N);
        CHASE_TRY(d.alloc(&Dv, static_cast<size_t>(lD) * nx));
        CHASE_TRY(d.alloc(&Dw, static_cast<size_t>(lD) * nx));
      }
    }
    CHASE_TRY(d.alloc(&dw, nx));
    CHASE_TRY(d.alloc(&dres, nx));
    CHASE_TRY(d.alloc(&dperm, nx));
    N2 = static_cast<double>(N) * static_cast<double>(N);
    // Alg. 1 line 1: constant initial degree, rounded up to even
    d0 = std::min(o.deg + o.deg % 2, kMaxDegAllowed);
    m.assign(nx, d0);
    grouped = grouped_split;
    cls.assign(nx, initial_slices());
    // line 2: bounds (and start vectors when approx == 0)
    LanczosOut lz;
    tm.begin(&S.t_lanczos);
    CHASE_TRY(lanczos_core(d, dH, N, lh, o.lanczos_iter, o.num_lanczos, o.approx != 0, nev, nex,
                           o.dos_sigma, dS, ls, o.approx ? nullptr : dV, lv, o.approx ? 0 : nx,
                           lz));
    tm.end();
    S.matvecs += lz.matvecs;
    S.lanczos_matvecs += lz.matvecs;
    S.flops_total += kMv * N2 * lz.matvecs;
    b_sup = lz.b_sup;
    if (!std::isfinite(lz.b_sup) || (!o.approx && !(std::isfinite(lz.mu1) && std::isfinite(lz.mu_nn)))) {
      set_error("chase_solve: the Lanczos bounds are not finite (b_sup=%g)", lz.b_sup);
      return CHASE_BOUND_VIOLATION;
    }
    if (o.approx) {
      for (int a = 0; a < nx; ++a)
        if (!std::isfinite(Lambda[a])) {
          set_error("chase_solve: Lambda[%d] is not finite (approx = 1 reads it)", a);
          return CHASE_INVALID_ARG;
        }
      mu1 = *std::min_element(Lambda, Lambda + nx);
      mu_nn = *std::max_element(Lambda, Lambda + nx);
    } else {
      mu1 = lz.mu1;
      mu_nn = lz.mu_nn;
    }
    h = lz.theta_absmax;
    ritz.assign(nx, 0.0);
    res.assign(nx, HUGE_VAL);
    ra.assign(nx, 0.0);
    rr.assign(nx, 0.0);
    order.assign(nx, 0);
    perm.assign(nx, 0);
    tol_eff = o.conv_mode == CHASE_CONV_REL ? tol * h : tol;
    return CHASE_OK;
  }

  // Line 3 of an iteration; false when the bounds are out of order.
  bool begin_iteration() {
    ++iter;
    if (!(mu1 < mu_nn && mu_nn < b_sup)) {
      set_error("chase_solve: spectral estimates out of order (mu1=%g, mu_nevnex=%g, b_sup=%g)",
                mu1, mu_nn, b_sup);
      status = CHASE_BOUND_VIOLATION;
      return false;
    }
    // line 4: the active columns form runs of equal precision, each sorted
    // by degree (line 15)
    maxdeg = *std::max_element(m.begin() + nconv, m.end());
    groups.clear();
    for (int r0 = nconv; r0 < nx;) {
      int r1 = r0 + 1;
      while (r1 < nx && cls[r1] == cls[r0]) ++r1;
      FilterGroup g;
      g.col0 = r0 - nconv;
      g.ncols = r1 - r0;
      g.nslices = cls[r0];
      starts_from_sorted(m.data() + r0, r1 - r0, maxdeg, g.start);
      groups.push_back(std::move(g));
      r0 = r1;
    }
    start = groups.size() == 1 ? groups[0].start : std::vector<int>(maxdeg + 2, 0);
    return true;
  }

  // Slices of the split product before any residual is known: 3 with
  // CHASE_SPLIT_BF16_ADAPT (the first filter starts from random vectors),
  // 4 for single precision, else 7.  The batched solve's grouped filter
  // takes one precision for all columns (7).
  int initial_slices() const {
    if constexpr (is_single<T>) return 4;
    if (o.precision == CHASE_SPLIT_BF16_ADAPT && !grouped) return 3;
    return 7;
  }

  // CHASE_SPLIT_BF16_ADAPT: slices of the split product for one column in the
  // next filter (Sec. 3.2: the filter only has to beat the residual it can
  // reach).  By the model behind Alg. 5 a degree-m filter divides the
  // residual by |rho|^m; while that expected residual stays above 1e-3 h the
  // column's products keep 3 slices (about 2^-21 relative), above 1e-6 h 4
  // slices (2^-28), else all 7 (2^-49).  Columns whose degree was chosen to
  // reach the tolerance therefore run in full precision, and only those
  // that cannot converge in this filter (degree capped at DEGMAX, or a Ritz
  // value inside the damped interval) run on fewer slices.
  int column_slices(double res_a, double ritz_a, int m_a, double c, double e) const {
    if constexpr (is_single<T>) return 4;
    if (o.precision != CHASE_SPLIT_BF16_ADAPT || grouped || !(e > 0.0)) return 7;
    const double t = (ritz_a - c) / e;
    const double rho = std::fabs(t) > 1.0 ? std::fabs(t) + std::sqrt(t * t - 1.0) : 1.0;
    const double expect = res_a * std::pow(rho, -static_cast<double>(m_a));
    if (!(expect <= 1e-3 * h)) return 3;
    if (!(expect <= 1e-6 * h)) return 4;
    return 7;
  }

  // The filter of this solve alone (line 4).
  int filter(Dev& d) {
    PhaseTimer tm(d.st);
    long long fm = 0, low = 0;
    tm.begin(&S.t_filter);
    if constexpr (is_single<T>) {
      if (split) {  // widen, filter on the split product, round back
        CHASE_TRY(launch_convert(d, Va(), lv, Dv, lD, N, b()));
        CHASE_TRY(filter_groups(d, static_cast<const Wide*>(nullptr), N, lD, Dv, lD, Dw, lD,
                                groups, maxdeg, b_sup, mu1, mu_nn, &fm, &sh, &sx, &low));
        CHASE_TRY(launch_convert(d, Dv, lD, Va(), lv, N, b()));
      } else {
        CHASE_TRY(filter_groups(d, dH, N, lh, Va(), lv, Wk, lw, groups, maxdeg, b_sup, mu1, mu_nn,
                                &fm, nullptr, &sx));
      }
    } else {
      CHASE_TRY(filter_groups(d, dH, N, lh, Va(), lv, Wk, lw, groups, maxdeg, b_sup, mu1, mu_nn,
                              &fm, split ? &sh : nullptr, &sx, &low));
    }
    tm.end();
    S.filter_slices_low += low > 0 ? 1 : 0;
    S.filter_matvecs_low += low;
    count_filter(fm);
    return CHASE_OK;
  }

  // The grouped filter's view of this solve's line 4.
  GroupedFilterInput filter_input() const {
    GroupedFilterInput g;
    g.H = dH;
    g.ldh = lh;
    g.n = static_cast<int>(N);
    g.X = Va();
    g.ldx = lv;
    g.W = Wk;
    g.ldw = lw;
    g.b = b();
    g.start = start.data();
    g.maxdeg = maxdeg;
    g.b_sup = b_sup;
    g.mu1 = mu1;
    g.mu_nn = mu_nn;
    return g;
  }

  long long filter_matvecs() const {
    long long fm = 0;
    for (int i = 1; i <= maxdeg; ++i) fm += b() - start[i];
    return fm;
  }

  void count_filter(long long fm) {
    S.filter_matvecs += fm;
    S.matvecs += fm;
    S.flops_filter += kMv * N2 * fm;
    S.flops_total += kMv * N2 * fm;
  }

  // Lines 5-15 of an iteration.
  int after_filter(Dev& d) {
    PhaseTimer tm(d.st);
    const int nb = b();
    T* va = Va();
    // lines 5-6: orthonormalise the active block against the locked one
    tm.begin(&S.t_qr);
    CHASE_TRY(orth_any(d, N, dV, lv, nconv, va, lv, nb, ow, &S.flops_total));
    tm.end();
    // lines 7-8: Rayleigh-Ritz on the active block, residuals
    tm.begin(&S.t_rr);
    CHASE_TRY(rr_core(d, dH, N, lh, va, lv, nb, dw, dres, rw, &S.t_eigh, &S.flops_total,
                      split_rr ? rr_slices : nullptr, split_rr ? rr_sx : nullptr,
                      &S.t_rr_product));
    S.flops_rr_product += kMv * N2 * nb;
    CHASE_CUDA(cudaMemcpyAsync(ra.data(), dw, sizeof(double) * nb, cudaMemcpyDeviceToHost, d.st));
    CHASE_CUDA(cudaMemcpyAsync(rr.data(), dres, sizeof(double) * nb, cudaMemcpyDeviceToHost, d.st));
    tm.end();
    CHASE_TRY(d.sync_check("chase_solve iteration"));
    S.matvecs += nb;
    const int nconv_new = decide(nb);
    CHASE_CUDA(cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, d.st));
    CHASE_TRY(apply_perm(d, dperm));
    // the host arrays read by the copies above change in the next iteration
    CHASE_TRY(d.sync_check("chase_solve permutation"));
    nconv = nconv_new;
    return CHASE_OK;
  }

  // Lines 9-15 on the host, from this iteration's Ritz values and residuals
  // of the nb active columns (ra, rr): locking, the new bounds, degrees,
  // precision classes, and in perm the column order of the next iteration
  // (locked first in Ritz order, then the rest by precision and degree).
  // Returns the new number of locked columns.
  int decide(int nb) {
    const auto t_host0 = std::chrono::steady_clock::now();
    for (int a = 0; a < nb; ++a) h = std::max(h, std::fabs(ra[a]));
    tol_eff = o.conv_mode == CHASE_CONV_REL ? tol * h : tol;
    if (ra[nb - 1] > b_sup + 1e-10 * std::max(1.0, std::fabs(b_sup))) {
      set_error("chase_solve: Ritz value %g above b_sup %g", ra[nb - 1], b_sup);
      status = CHASE_BOUND_VIOLATION;
    }
    int n_new = 0;
    chase_lock(nb, ra.data(), rr.data(), tol_eff, order.data(), &n_new);  // line 9 (Alg. 3)
    for (int a = 0; a < nb; ++a) {
      ritz[nconv + a] = ra[order[a]];
      res[nconv + a] = rr[order[a]];
    }
    const int nconv_new = nconv + n_new;
    mu1 = *std::min_element(ritz.begin(), ritz.end());  // line 10
    mu_nn = *std::max_element(ritz.begin(), ritz.end());
    const double c = 0.5 * (b_sup + mu_nn);  // line 11
    const double e = 0.5 * (b_sup - mu_nn);
    const int nrest = nx - nconv_new;
    std::vector<int> ord2(nrest);
    if (nrest > 0) {
      if (o.optim && e > 0.0)  // lines 12-14
        chase_degrees(nrest, res.data() + nconv_new, ritz.data() + nconv_new, c, e, tol_eff,
                      o.deg_extra, std::min(o.deg_max, kMaxDegAllowed), m.data() + nconv_new);
      else
        std::fill(m.begin() + nconv_new, m.end(), d0);
      // precision of each column in the next filter (7 unless ADAPT)
      for (int a = 0; a < nrest; ++a)
        cls[nconv_new + a] = column_slices(res[nconv_new + a], ritz[nconv_new + a],
                                           m[nconv_new + a], c, e);
      std::iota(ord2.begin(), ord2.end(), 0);  // line 15: stable sort by degree
      // (within runs of equal precision, so that each run is one suffix-
      // retiring block of Alg. 4)
      std::stable_sort(ord2.begin(), ord2.end(), [&](int x, int y) {
        const int cx = cls[nconv_new + x], cy = cls[nconv_new + y];
        if (cx != cy) return cx < cy;
        return m[nconv_new + x] < m[nconv_new + y];
      });
    }
    // one gather over the active block: locked first (Ritz order), then the
    // rest by degree
    for (int a = 0; a < n_new; ++a) perm[a] = order[a];
    for (int a = 0; a < nrest; ++a) perm[n_new + a] = order[n_new + ord2[a]];
    std::vector<double> r2(nrest), s2(nrest);
    std::vector<int> m2(nrest), c2(nrest);
    for (int a = 0; a < nrest; ++a) {
      r2[a] = ritz[nconv_new + ord2[a]];
      s2[a] = res[nconv_new + ord2[a]];
      m2[a] = m[nconv_new + ord2[a]];
      c2[a] = cls[nconv_new + ord2[a]];
    }
    for (int a = 0; a < nrest; ++a) {
      ritz[nconv_new + a] = r2[a];
      res[nconv_new + a] = s2[a];
      m[nconv_new + a] = m2[a];
      cls[nconv_new + a] = c2[a];
    }
    S.t_host += std::chrono::duration<double>(std::chrono::steady_clock::now() - t_host0).count();
    return nconv_new;
  }

  // Gather of the active block into the order of perm (device copy dp).
  int apply_perm(Dev& d, const int* dp) {
    const int nb = b();
    CHASE_TRY(launch_permute_cols(d, Va(), lv, Wk, lw, N, nb, dp, false));
    return copy_block(d, Va(), lv, Wk, lw, N, nb, cudaMemcpyDeviceToDevice);
  }

  // Output: all pairs ascending by Ritz value; returns the solve's status.
  int finish(Dev& d) {
    std::vector<int> fin(nx);
    std::iota(fin.begin(), fin.end(), 0);
    std::stable_sort(fin.begin(), fin.end(), [&](int x, int y) { return ritz[x] < ritz[y]; });
    CHASE_CUDA(cudaMemcpyAsync(dperm, fin.data(), sizeof(int) * nx, cudaMemcpyHostToDevice, d.st));
    CHASE_TRY(launch_permute_cols(d, dV, lv, Wk, lw, N, nx, dperm, false));
    CHASE_TRY(copy_block(d, dV, lv, Wk, lw, N, nx, cudaMemcpyDeviceToDevice));
    if (dV != V)
      CHASE_TRY(copy_block(d, V, ldv, dV, lv, N, nx,
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    CHASE_TRY(d.sync_check("chase_solve output"));
    for (int a = 0; a < nx; ++a) {
      Lambda[a] = ritz[fin[a]];
      resid[a] = res[fin[a]];
    }
    S.iterations = iter;
    S.nconv = nconv;
    S.b_sup = b_sup;
    S.mu1 = mu1;
    S.mu_nevnex = mu_nn;
    S.tol_eff = tol_eff;
    if (status != CHASE_OK) return status;
    return nconv >= nev ? CHASE_OK : CHASE_NOT_CONVERGED;
  }
};


// Host threads, each with its own stream and device context, for the
// per-problem phases of a batched solve (set-up, QR, Rayleigh-Ritz, locking):
// the small launches and host round trips of different problems overlap.
// The threads live as long as the pool; each destroys its cuSOLVER handle
// before it ends.
class WorkerPool {
 public:
  explicit WorkerPool(cudaStream_t main) : main_(main) {}
  WorkerPool(const WorkerPool&) = delete;
  WorkerPool& operator=(const WorkerPool&) = delete;

  int init(int n) {
    for (int w = 0; w < n; ++w) {
      cudaStream_t s = nullptr;
      CHASE_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      streams_.push_back(s);
      devs_.emplace_back(new Dev(s));
      CHASE_TRY(devs_.back()->init());
    }
    nw_ = n;
    rc_.assign(n, CHASE_OK);
    msg_.assign(n, std::string());
    threads_.reserve(n);
    for (int w = 0; w < n; ++w) threads_.emplace_back([this, w] { loop(w); });
    return CHASE_OK;
  }

  ~WorkerPool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : threads_) t.join();
    cudaStreamSynchronize(main_);  // main-stream work may still read worker buffers
    devs_.clear();                 // frees on each worker stream and synchronises it
    for (auto s : streams_) cudaStreamDestroy(s);
  }

  // fn(worker context, item) for every item; each worker takes the next
  // item in list order as soon as it is free (list the costly items first).
  int run(const std::vector<int>& items, std::function<int(Dev&, int)> fn) {
    std::unique_lock<std::mutex> lk(mu_);
    items_ = &items;
    job_ = std::move(fn);
    finished_ = 0;
    next_.store(0);
    ++generation_;
    cv_.notify_all();
    done_.wait(lk, [&] { return finished_ == nw_; });
    for (int w = 0; w < nw_; ++w)
      if (rc_[w] != CHASE_OK) {
        set_error("%s", msg_[w].c_str());
        return rc_[w];
      }
    return CHASE_OK;
  }

 private:
  void loop(int w) {
    int seen = 0;
    for (;;) {
      std::unique_lock<std::mutex> lk(mu_);
      cv_.wait(lk, [&] { return stop_ || generation_ != seen; });
      if (stop_) break;
      seen = generation_;
      const std::vector<int>* items = items_;
      lk.unlock();
      int r = CHASE_OK;
      std::string m;
      for (size_t i = next_.fetch_add(1); i < items->size(); i = next_.fetch_add(1)) {
        r = job_(*devs_[w], (*items)[i]);
        if (r != CHASE_OK) {
          m = chase_last_error();
          break;
        }
      }
      lk.lock();
      rc_[w] = r;
      msg_[w] = m;
      if (++finished_ == nw_) done_.notify_one();
    }
    release_thread_solver();
  }

  cudaStream_t main_;
  std::vector<cudaStream_t> streams_;
  std::vector<std::unique_ptr<Dev>> devs_;
  std::vector<std::thread> threads_;
  std::mutex mu_;
  std::condition_variable cv_, done_;
  std::function<int(Dev&, int)> job_;
  const std::vector<int>* items_ = nullptr;
  int nw_ = 0, generation_ = 0, finished_ = 0;
  std::atomic<size_t> next_{0};
  bool stop_ = false;
  std::vector<int> rc_;
  std::vector<std::string> msg_;
};

// Arguments of one solve, checked as chase_solve does.
bool solve_args_ok(int64_t N, int64_t ldh, int nev, int nex, double tol, int64_t ldv,
                   const void* H, const void* V, const void* Lambda, const void* resid,
                   const void* starts, const chase_opts& o) {
  const int nx = nev + nex;
  return !(N < 1 || nev < 1 || nex < 0 || nx > N || !ld_ok(ldh, N) || !ld_ok(ldv, N) ||
           !(tol > 0.0) || !H || !V || !Lambda || !resid || !starts || o.deg < 1 ||
           o.deg > kMaxDegAllowed - 1 || o.deg_max < 2 || o.deg_max > kMaxDegAllowed ||
           o.deg_extra < 0 || o.max_iter < 0 || o.lanczos_iter < 1 || o.lanczos_iter > N ||
           (!o.approx && o.num_lanczos < 1) ||
           (o.precision != CHASE_FP64 && o.precision != CHASE_SPLIT_BF16 &&
            o.precision != CHASE_SPLIT_BF16_RR && o.precision != CHASE_SPLIT_BF16_ADAPT) ||
           (o.conv_mode != CHASE_CONV_ABS && o.conv_mode != CHASE_CONV_REL) ||
           (o.storage != CHASE_STORAGE_FULL && o.storage != CHASE_STORAGE_LOWER));
}

}  // namespace
}  // namespace chase

using namespace chase;

extern "C" int chase_opts_default(chase_opts* o) {
  if (!o) {
    set_error("chase_opts_default: NULL");
    return CHASE_INVALID_ARG;
  }
  o->deg = 20;
  o->optim = 1;
  o->deg_extra = 2;
  o->deg_max = 36;
  o->max_iter = 25;
  o->lanczos_iter = 25;
  o->num_lanczos = 4;
  o->approx = 0;
  o->dos_sigma = 0.25;
  o->conv_mode = CHASE_CONV_REL;
  o->precision = CHASE_FP64;
  o->storage = CHASE_STORAGE_FULL;
  return CHASE_OK;
}

namespace chase {
namespace {
template <class T>
int filter_impl(const T* H, int64_t N, int64_t ldh, T* V, int64_t ldv, int b, const int* degrees,
                double b_sup, double mu1, double mu_nevnex, int precision, T* work, void* stream) {
  if constexpr (is_single<T>) precision = CHASE_FP64;  // native FP32 products
  if (precision != CHASE_FP64 && precision != CHASE_SPLIT_BF16 &&
      precision != CHASE_SPLIT_BF16_4 && precision != CHASE_SPLIT_BF16_3) {
    set_error("chase_filter: unknown precision %d", precision);
    return CHASE_INVALID_ARG;
  }
  if (N < 0 || b < 0 || !ld_ok(ldh, N) || !ld_ok(ldv, N) || N > (1LL << 30)) {
    set_error("chase_filter: invalid size or leading dimension");
    return CHASE_INVALID_ARG;
  }
  if (N == 0 || b == 0) return CHASE_OK;
  if (!H || !V || !degrees) {
    set_error("chase_filter: NULL array");
    return CHASE_INVALID_ARG;
  }
  if (!(mu1 < mu_nevnex && mu_nevnex < b_sup) || !std::isfinite(b_sup) || !std::isfinite(mu1)) {
    set_error("chase_filter: need mu1 < mu_nevnex < b_sup");
    return CHASE_INVALID_ARG;
  }
  Dev d(stream);
  CHASE_TRY(d.init());
  const bool dev = is_device_ptr(H);
  if (is_device_ptr(V) != dev) {
    set_error("chase_filter: H and V must both be host or both be device arrays");
    return CHASE_INVALID_ARG;
  }
  T *dH = nullptr, *dV = nullptr;
  int64_t lh = 0, lv = 0;
  CHASE_TRY(stage_in(d, dev, H, ldh, N, N, &dH, &lh));
  CHASE_TRY(stage_in(d, dev, V, ldv, N, b, &dV, &lv));
  CHASE_TRY(check_finite(d, dH, lh, N, N, "chase_filter", "H"));
  CHASE_TRY(check_finite(d, dV, lv, N, b, "chase_filter", "V"));
  // the workspace (leading dimension ld_pad(N)) must suit the TMA products
  const int64_t lw = ld_pad<T>(N);
  T* wk = dev && lw == N ? work : nullptr;
  if (!wk) CHASE_TRY(d.alloc(&wk, static_cast<size_t>(lw) * b));
  // degrees -> device, plan on the device (stable sort by degree)
  int *ddeg = nullptr, *dperm = nullptr, *dstart = nullptr, *dinfo = nullptr;
  if (is_device_ptr(degrees)) {
    ddeg = const_cast<int*>(degrees);
  } else {
    CHASE_TRY(d.alloc(&ddeg, b));
    CHASE_CUDA(cudaMemcpyAsync(ddeg, degrees, sizeof(int) * b, cudaMemcpyHostToDevice, d.st));
  }
  CHASE_TRY(d.alloc(&dperm, b));
  CHASE_TRY(d.alloc(&dstart, kMaxDegAllowed + 2));
  CHASE_TRY(d.alloc(&dinfo, 1));
  CHASE_TRY(launch_filter_plan(d, ddeg, b, kMaxDegAllowed, dperm, dstart, dinfo));
  std::vector<int> start(kMaxDegAllowed + 2);
  int maxdeg = 0;
  CHASE_CUDA(cudaMemcpyAsync(start.data(), dstart, sizeof(int) * start.size(), cudaMemcpyDeviceToHost, d.st));
  CHASE_CUDA(cudaMemcpyAsync(&maxdeg, dinfo, sizeof(int), cudaMemcpyDeviceToHost, d.st));
  CHASE_TRY(d.sync_check("chase_filter plan"));
  SplitH sh;
  SplitX sx;
  const bool split = precision != CHASE_FP64;
  const int nslices = precision == CHASE_SPLIT_BF16_4 ? 4 : precision == CHASE_SPLIT_BF16_3 ? 3 : 7;
  if constexpr (!is_single<T>) {
    if (split) {
      CHASE_TRY(split_prepare_h(d, dH, N, lh, sh));
      CHASE_TRY(split_alloc_x(d, N, b, sx, is_cplx<T>));
    }
  }
  // sorted copy into the workspace; V becomes the second buffer
  CHASE_TRY(launch_permute_cols(d, dV, lv, wk, lw, N, b, dperm, false));
  CHASE_TRY(filter_sorted(d, dH, N, lh, wk, lw, dV, lv, b, start.data(), maxdeg, b_sup, mu1,
                          mu_nevnex, nullptr, split ? &sh : nullptr, &sx, nslices));
  CHASE_TRY(launch_permute_cols(d, wk, lw, dV, lv, N, b, dperm, true));
  if (dV != V)
    CHASE_TRY(copy_block(d, V, ldv, dV, lv, N, b,
                         dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
  return d.sync_check("chase_filter");
}
}  // namespace
}  // namespace chase

extern "C" int chase_filter(const chase_c64* H, int64_t N, int64_t ldh, chase_c64* V, int64_t ldv,
                            int b, const int* degrees, double b_sup, double mu1, double mu_nevnex,
                            int precision, chase_c64* work, void* stream) {
  return filter_impl(H, N, ldh, V, ldv, b, degrees, b_sup, mu1, mu_nevnex, precision, work, stream);
}

extern "C" int chase_filter_real(const double* H, int64_t N, int64_t ldh, double* V, int64_t ldv,
                                 int b, const int* degrees, double b_sup, double mu1,
                                 double mu_nevnex, int precision, double* work, void* stream) {
  return filter_impl(H, N, ldh, V, ldv, b, degrees, b_sup, mu1, mu_nevnex, precision, work, stream);
}

extern "C" int chase_filter_c32(const chase_c32* H, int64_t N, int64_t ldh, chase_c32* V,
                                int64_t ldv, int b, const int* degrees, double b_sup, double mu1,
                                double mu_nevnex, chase_c32* work, void* stream) {
  return filter_impl(H, N, ldh, V, ldv, b, degrees, b_sup, mu1, mu_nevnex, CHASE_FP64, work, stream);
}

extern "C" int chase_filter_f32(const float* H, int64_t N, int64_t ldh, float* V, int64_t ldv,
                                int b, const int* degrees, double b_sup, double mu1,
                                double mu_nevnex, float* work, void* stream) {
  return filter_impl(H, N, ldh, V, ldv, b, degrees, b_sup, mu1, mu_nevnex, CHASE_FP64, work, stream);
}


extern "C" int chase_filter_mixed(const chase_c64* H, int64_t N, int64_t ldh, chase_c64* V,
                                  int64_t ldv, int b, const int* degrees, const int* slices,
                                  double b_sup, double mu1, double mu_nevnex, chase_c64* work,
                                  void* stream) {
  using namespace chase;
  if (N < 0 || b < 0 || !ld_ok(ldh, N) || !ld_ok(ldv, N) || N > (1LL << 30)) {
    set_error("chase_filter_mixed: invalid size or leading dimension");
    return CHASE_INVALID_ARG;
  }
  if (N == 0 || b == 0) return CHASE_OK;
  if (!H || !V || !degrees || !slices) {
    set_error("chase_filter_mixed: NULL array");
    return CHASE_INVALID_ARG;
  }
  if (!(mu1 < mu_nevnex && mu_nevnex < b_sup) || !std::isfinite(b_sup) || !std::isfinite(mu1)) {
    set_error("chase_filter_mixed: need mu1 < mu_nevnex < b_sup");
    return CHASE_INVALID_ARG;
  }
  Dev d(stream);
  CHASE_TRY(d.init());
  const bool dev = is_device_ptr(H);
  if (is_device_ptr(V) != dev) {
    set_error("chase_filter_mixed: H and V must both be host or both be device arrays");
    return CHASE_INVALID_ARG;
  }
  // the plan is made on the host: degrees and slices there
  std::vector<int> deg(b), ns(b);
  for (auto [src, dst] : {std::pair<const int*, int*>{degrees, deg.data()},
                          std::pair<const int*, int*>{slices, ns.data()}}) {
    if (is_device_ptr(src))
      CHASE_CUDA(cudaMemcpyAsync(dst, src, sizeof(int) * b, cudaMemcpyDeviceToHost, d.st));
    else
      std::copy(src, src + b, dst);
  }
  CHASE_TRY(d.sync_check("chase_filter_mixed"));
  for (int a = 0; a < b; ++a)
    if (deg[a] < 2 || deg[a] > kMaxDegAllowed || deg[a] % 2 != 0 ||
        (ns[a] != 3 && ns[a] != 4 && ns[a] != 7)) {
      set_error("chase_filter_mixed: column %d: degree %d (even, 2..%d) or slices %d (3, 4, 7)", a,
                deg[a], kMaxDegAllowed, ns[a]);
      return CHASE_INVALID_ARG;
    }
  chase_c64 *dH = nullptr, *dV = nullptr;
  int64_t lh = 0, lv = 0;
  CHASE_TRY(stage_in(d, dev, H, ldh, N, N, &dH, &lh));
  CHASE_TRY(stage_in(d, dev, V, ldv, N, b, &dV, &lv));
  CHASE_TRY(check_finite(d, dH, lh, N, N, "chase_filter_mixed", "H"));
  CHASE_TRY(check_finite(d, dV, lv, N, b, "chase_filter_mixed", "V"));
  const int64_t lw = ld_pad<chase_c64>(N);
  chase_c64* wk = dev && lw == N ? work : nullptr;
  if (!wk) CHASE_TRY(d.alloc(&wk, static_cast<size_t>(lw) * b));
  // columns ordered by (slices, degree): runs of equal precision, each sorted
  // by degree, each filtered as its own suffix-retiring block
  std::vector<int> order(b);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    if (ns[x] != ns[y]) return ns[x] < ns[y];
    return deg[x] < deg[y];
  });
  const int maxdeg = *std::max_element(deg.begin(), deg.end());
  std::vector<int> msorted(b);
  for (int a = 0; a < b; ++a) msorted[a] = deg[order[a]];
  std::vector<FilterGroup> groups;
  for (int r0 = 0; r0 < b;) {
    int r1 = r0 + 1;
    while (r1 < b && ns[order[r1]] == ns[order[r0]]) ++r1;
    FilterGroup g;
    g.col0 = r0;
    g.ncols = r1 - r0;
    g.nslices = ns[order[r0]];
    starts_from_sorted(msorted.data() + r0, r1 - r0, maxdeg, g.start);
    groups.push_back(std::move(g));
    r0 = r1;
  }
  int* dperm = nullptr;
  CHASE_TRY(d.alloc(&dperm, b));
  CHASE_CUDA(cudaMemcpyAsync(dperm, order.data(), sizeof(int) * b, cudaMemcpyHostToDevice, d.st));
  SplitH sh;
  SplitX sx;
  CHASE_TRY(split_prepare_h(d, dH, N, lh, sh));
  CHASE_TRY(split_alloc_x(d, N, b, sx, true));
  CHASE_TRY(launch_permute_cols(d, dV, lv, wk, lw, N, b, dperm, false));
  CHASE_TRY(filter_groups(d, dH, N, lh, wk, lw, dV, lv, groups, maxdeg, b_sup, mu1, mu_nevnex,
                          nullptr, &sh, &sx));
  CHASE_TRY(launch_permute_cols(d, wk, lw, dV, lv, N, b, dperm, true));
  if (dV != V)
    CHASE_TRY(copy_block(d, V, ldv, dV, lv, N, b,
                         dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
  return d.sync_check("chase_filter_mixed");
}

extern "C" int chase_lanczos(const chase_c64* H, int64_t N, int64_t ldh, int k, int nvec, int approx,
                             int nev, int nex, double dos_sigma, const chase_c64* starts,
                             chase_c64* V, int64_t ldv, double* b_sup, double* mu1,
                             double* mu_nevnex, double* theta_absmax, void* stream) {
  if (N < 1 || !ld_ok(ldh, N) || k < 1 || k > N || !H || !starts || !b_sup ||
      (!approx && (nvec < 1 || nev < 1 || nex < 0 || nev + nex > N || !mu1 || !mu_nevnex)) ||
      (V && !ld_ok(ldv, N))) {
    set_error("chase_lanczos: invalid argument");
    return CHASE_INVALID_ARG;
  }
  Dev d(stream);
  CHASE_TRY(d.init());
  const bool dev = is_device_ptr(H);
  if (is_device_ptr(starts) != dev || (V && is_device_ptr(V) != dev)) {
    set_error("chase_lanczos: arrays must all be host or all be device");
    return CHASE_INVALID_ARG;
  }
  const int r = approx ? 1 : 1 + nvec;
  chase_c64 *dH, *dS, *dV = nullptr;
  int64_t lh, ls, lv = ldv;
  CHASE_TRY(stage_in(d, dev, H, ldh, N, N, &dH, &lh));
  CHASE_TRY(stage_in(d, dev, starts, N, N, r, &dS, &ls));
  const int ncolv = V && !approx ? nev + nex : 0;
  if (ncolv) CHASE_TRY(stage_in(d, dev, V, ldv, N, ncolv, &dV, &lv));
  LanczosOut out;
  CHASE_TRY(lanczos_core(d, dH, N, lh, k, nvec, approx != 0, nev, nex, dos_sigma, dS, ls, dV, lv,
                         ncolv, out));
  if (ncolv && !dev) CHASE_TRY(copy_block(d, V, ldv, dV, lv, N, ncolv, cudaMemcpyDeviceToHost));
  CHASE_TRY(d.sync_check("chase_lanczos"));
  *b_sup = out.b_sup;
  if (theta_absmax) *theta_absmax = out.theta_absmax;
  if (!approx) {
    *mu1 = out.mu1;
    *mu_nevnex = out.mu_nn;
  }
  return CHASE_OK;
}

extern "C" int chase_orthonormalize(const chase_c64* Y, int64_t N, int64_t ldy, int nconv,
                                    chase_c64* V, int64_t ldv, int b, void* stream) {
  if (N < 0 || nconv < 0 || b < 0 || nconv + b > N || !ld_ok(ldv, N) ||
      (nconv > 0 && (!Y || !ld_ok(ldy, N))) || (b > 0 && !V)) {
    set_error("chase_orthonormalize: invalid argument");
    return CHASE_INVALID_ARG;
  }
  if (b == 0) return CHASE_OK;
  Dev d(stream);
  CHASE_TRY(d.init());
  const bool dev = is_device_ptr(V);
  if (nconv > 0 && is_device_ptr(Y) != dev) {
    set_error("chase_orthonormalize: Y and V must be of the same kind");
    return CHASE_INVALID_ARG;
  }
  chase_c64 *dY = nullptr, *dV = nullptr;
  int64_t ly = N, lv = 0;
  if (nconv > 0) CHASE_TRY(stage_in(d, dev, Y, ldy, N, nconv, &dY, &ly));
  CHASE_TRY(stage_in(d, dev, V, ldv, N, b, &dV, &lv));
  OrthWork<chase_c64> w;
  CHASE_TRY(orth_alloc(d, N, nconv, b, w));
  double fl = 0.0;
  CHASE_TRY(orth_core(d, N, dY, ly, nconv, dV, lv, b, w, &fl));
  if (!dev) CHASE_TRY(copy_block(d, V, ldv, dV, lv, N, b, cudaMemcpyDeviceToHost));
  return d.sync_check("chase_orthonormalize");
}

extern "C" int chase_rayleigh_ritz(const chase_c64* H, int64_t N, int64_t ldh, chase_c64* Q,
                                   int64_t ldq, int b, double* ritz, double* resid, void* stream) {
  if (N < 0 || b < 0 || b > N || !ld_ok(ldh, N) || !ld_ok(ldq, N) ||
      (b > 0 && (!H || !Q || !ritz))) {
    set_error("chase_rayleigh_ritz: invalid argument");
    return CHASE_INVALID_ARG;
  }
  if (b == 0) return CHASE_OK;
  Dev d(stream);
  CHASE_TRY(d.init());
  const bool dev = is_device_ptr(H);
  if (is_device_ptr(Q) != dev) {
    set_error("chase_rayleigh_ritz: H and Q must be of the same kind");
    return CHASE_INVALID_ARG;
  }
  chase_c64 *dH, *dQ;
  int64_t lh, lq;
  CHASE_TRY(stage_in(d, dev, H, ldh, N, N, &dH, &lh));
  CHASE_TRY(stage_in(d, dev, Q, ldq, N, b, &dQ, &lq));
  RRWork<chase_c64> w;
  CHASE_TRY(rr_alloc(d, N, b, w));
  double *dw = nullptr, *dr = nullptr;
  CHASE_TRY(d.alloc(&dw, b));
  if (resid) CHASE_TRY(d.alloc(&dr, b));
  double te = 0.0, fl = 0.0;
  CHASE_TRY(rr_core(d, dH, N, lh, dQ, lq, b, dw, dr, w, &te, &fl));
  if (!dev) CHASE_TRY(copy_block(d, Q, ldq, dQ, lq, N, b, cudaMemcpyDeviceToHost));
  CHASE_CUDA(cudaMemcpyAsync(ritz, dw, sizeof(double) * b, cudaMemcpyDeviceToHost, d.st));
  if (resid) CHASE_CUDA(cudaMemcpyAsync(resid, dr, sizeof(double) * b, cudaMemcpyDeviceToHost, d.st));
  return d.sync_check("chase_rayleigh_ritz");
}

namespace chase {
namespace {
template <class T>
int residuals_impl(const T* H, int64_t N, int64_t ldh, const T* V, int64_t ldv, int b,
                   const double* lambda, double* resid, void* stream) {
  if (N < 0 || b < 0 || !ld_ok(ldh, N) || !ld_ok(ldv, N) ||
      (b > 0 && (!H || !V || !lambda || !resid))) {
    set_error("chase_residuals: invalid argument");
    return CHASE_INVALID_ARG;
  }
  if (b == 0 || N == 0) return CHASE_OK;
  Dev d(stream);
  CHASE_TRY(d.init());
  const bool dev = is_device_ptr(H);
  if (is_device_ptr(V) != dev) {
    set_error("chase_residuals: H and V must be of the same kind");
    return CHASE_INVALID_ARG;
  }
  T *dH, *dV, *HV = nullptr;
  int64_t lh, lv;
  CHASE_TRY(stage_in(d, dev, H, ldh, N, N, &dH, &lh));
  CHASE_TRY(stage_in(d, dev, V, ldv, N, b, &dV, &lv));
  double *dl = nullptr, *dr = nullptr;
  const int64_t lw = ld_pad<T>(N);
  CHASE_TRY(d.alloc(&HV, static_cast<size_t>(lw) * b));
  CHASE_TRY(d.alloc(&dl, b));
  CHASE_TRY(d.alloc(&dr, b));
  CHASE_CUDA(cudaMemcpyAsync(dl, lambda, sizeof(double) * b, cudaMemcpyHostToDevice, d.st));
  CHASE_TRY(gemm(d, N, N, dH, lh, dV, lv, b, HV, lw, 0, b, 1.0, 0.0, 0.0));
  CHASE_TRY(launch_resid_norms(d, HV, lw, dV, lv, N, b, dl, dr));
  CHASE_CUDA(cudaMemcpyAsync(resid, dr, sizeof(double) * b, cudaMemcpyDeviceToHost, d.st));
  return d.sync_check("chase_residuals");
}
}  // namespace
}  // namespace chase

extern "C" int chase_residuals(const chase_c64* H, int64_t N, int64_t ldh, const chase_c64* V,
                               int64_t ldv, int b, const double* lambda, double* resid,
                               void* stream) {
  return residuals_impl(H, N, ldh, V, ldv, b, lambda, resid, stream);
}

extern "C" int chase_residuals_real(const double* H, int64_t N, int64_t ldh, const double* V,
                                    int64_t ldv, int b, const double* lambda, double* resid,
                                    void* stream) {
  return residuals_impl(H, N, ldh, V, ldv, b, lambda, resid, stream);
}

extern "C" int chase_residuals_c32(const chase_c32* H, int64_t N, int64_t ldh, const chase_c32* V,
                                   int64_t ldv, int b, const double* lambda, double* resid,
                                   void* stream) {
  return residuals_impl(H, N, ldh, V, ldv, b, lambda, resid, stream);
}

extern "C" int chase_residuals_f32(const float* H, int64_t N, int64_t ldh, const float* V,
                                   int64_t ldv, int b, const double* lambda, double* resid,
                                   void* stream) {
  return residuals_impl(H, N, ldh, V, ldv, b, lambda, resid, stream);
}

namespace chase {
namespace {
template <class T>
int solve_impl(const T* H, int64_t N, int64_t ldh, int nev, int nex, double tol, T* V, int64_t ldv,
               double* Lambda, double* resid, const T* lanczos_starts, const chase_opts* opts_in,
               chase_stats* stats, void* stream) {
  chase_opts o;
  if (opts_in)
    o = *opts_in;
  else
    chase_opts_default(&o);
  if (!solve_args_ok(N, ldh, nev, nex, tol, ldv, H, V, Lambda, resid, lanczos_starts, o)) {
    set_error("chase_solve: invalid argument");
    return CHASE_INVALID_ARG;
  }
  Dev d(stream);
  CHASE_TRY(d.init());
  const bool dev = is_device_ptr(H);
  if (is_device_ptr(V) != dev || is_device_ptr(lanczos_starts) != dev) {
    set_error("chase_solve: H, V and lanczos_starts must all be host or all be device");
    return CHASE_INVALID_ARG;
  }
  Solver<T> sv;
  sv.H = H;
  sv.N = N;
  sv.ldh = ldh;
  sv.nev = nev;
  sv.nex = nex;
  sv.tol = tol;
  sv.V = V;
  sv.ldv = ldv;
  sv.Lambda = Lambda;
  sv.resid = resid;
  sv.starts = lanczos_starts;
  sv.o = o;
  sv.dev = dev;
  PhaseTimer total(d.st);
  double t_total = 0.0;
  total.begin(&t_total);
  CHASE_TRY(sv.setup(d, false));
  while (sv.more()) {  // line 3
    if (!sv.begin_iteration()) break;
    CHASE_TRY(sv.filter(d));
    CHASE_TRY(sv.after_filter(d));
  }
  const int st = sv.finish(d);
  if (st != CHASE_OK && st != CHASE_NOT_CONVERGED && st != CHASE_BOUND_VIOLATION) return st;
  total.end();
  sv.S.t_total = t_total;
  if (stats) *stats = sv.S;
  return st;
}
}  // namespace
}  // namespace chase

extern "C" int chase_solve(const chase_c64* H, int64_t N, int64_t ldh, int nev, int nex, double tol,
                           chase_c64* V, int64_t ldv, double* Lambda, double* resid,
                           const chase_c64* lanczos_starts, const chase_opts* opts_in,
                           chase_stats* stats, void* stream) {
  return solve_impl(H, N, ldh, nev, nex, tol, V, ldv, Lambda, resid, lanczos_starts, opts_in, stats,
                    stream);
}

extern "C" int chase_solve_real(const double* H, int64_t N, int64_t ldh, int nev, int nex,
                                double tol, double* V, int64_t ldv, double* Lambda, double* resid,
                                const double* lanczos_starts, const chase_opts* opts_in,
                                chase_stats* stats, void* stream) {
  return solve_impl(H, N, ldh, nev, nex, tol, V, ldv, Lambda, resid, lanczos_starts, opts_in, stats,
                    stream);
}

extern "C" int chase_solve_c32(const chase_c32* H, int64_t N, int64_t ldh, int nev, int nex,
                               double tol, chase_c32* V, int64_t ldv, double* Lambda,
                               double* resid, const chase_c32* lanczos_starts,
                               const chase_opts* opts_in, chase_stats* stats, void* stream) {
  return solve_impl(H, N, ldh, nev, nex, tol, V, ldv, Lambda, resid, lanczos_starts, opts_in, stats,
                    stream);
}

extern "C" int chase_solve_f32(const float* H, int64_t N, int64_t ldh, int nev, int nex, double tol,
                               float* V, int64_t ldv, double* Lambda, double* resid,
                               const float* lanczos_starts, const chase_opts* opts_in,
                               chase_stats* stats, void* stream) {
  return solve_impl(H, N, ldh, nev, nex, tol, V, ldv, Lambda, resid, lanczos_starts, opts_in, stats,
                    stream);
}

namespace chase {
namespace {
// Lines 5-15 of Alg. 1 for every problem of a batch at once.  The steps are
// those of Solver::after_filter, launched for all problems on one stream
// with one synchronisation per phase instead of several per problem, and
// the projected eigenproblems of Alg. 2 solved together (eigh_batched).
// A problem whose first Cholesky QR pass breaks down takes the single-
// problem orthogonalisation (shifted retry, its own synchronisations).
// Adds the phases' times (events on the batch's stream) to t[0] (QR),
// t[1] (Rayleigh-Ritz and residuals), t[2] (the eigensolves) and t[3]
// (locking, degrees and the reordering).
// Problem i's launches go to stream fan[i % fan.size()] (the small kernels
// of different problems then run side by side); the batch's stream d.st
// forks to and joins the fan around each phase.
int batched_after_filter(Dev& d, std::vector<Solver<chase_c64>*>& act,
                         const std::vector<cudaStream_t>& fan, double* t) {
  using T = chase_c64;
  const int P = static_cast<int>(act.size());
  if (P == 0) return CHASE_OK;
  const int S = static_cast<int>(fan.size());
  struct Events {
    std::vector<cudaEvent_t> e;
    ~Events() {
      for (auto x : e) cudaEventDestroy(x);
    }
  } ev;
  ev.e.assign(S + 1, nullptr);
  for (auto& x : ev.e) CHASE_CUDA(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
  auto fork = [&]() -> int {
    CHASE_CUDA(cudaEventRecord(ev.e[S], d.st));
    for (int k = 0; k < S; ++k) CHASE_CUDA(cudaStreamWaitEvent(fan[k], ev.e[S], 0));
    return CHASE_OK;
  };
  auto join = [&]() -> int {
    for (int k = 0; k < S; ++k) {
      CHASE_CUDA(cudaEventRecord(ev.e[k], fan[k]));
      CHASE_CUDA(cudaStreamWaitEvent(d.st, ev.e[k], 0));
    }
    return CHASE_OK;
  };
  int* flags = nullptr;  // per problem: KERR_* bits of its launches
  CHASE_TRY(d.alloc(&flags, P));
  CHASE_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * P, d.st));
  std::vector<std::unique_ptr<Dev>> view(P);
  for (int i = 0; i < P; ++i) {
    view[i].reset(new Dev(S > 0 ? fan[i % S] : d.st));
    view[i]->err = flags + i;
    view[i]->own_err = false;
    view[i]->sync_on_exit = false;
  }
  std::vector<int> hf(P);
  auto read_flags = [&](const char* where) -> int {
    CHASE_TRY(join());
    CHASE_CUDA(cudaMemcpyAsync(hf.data(), flags, sizeof(int) * P, cudaMemcpyDeviceToHost, d.st));
    CHASE_CUDA(cudaStreamSynchronize(d.st));
    for (int i = 0; i < P; ++i)
      if (hf[i] & (KERR_TIMEOUT_FULL | KERR_TIMEOUT_EMPTY)) {
        set_error("%s: a bounded wait in a kernel gave up (problem %d)", where, i);
        return CHASE_TIMEOUT;
      }
    return CHASE_OK;
  };
  PhaseTimer tm(d.st);
  // ---- lines 5-6: Cholesky QR, twice ----
  tm.begin(&t[0]);
  CHASE_TRY(fork());
  for (int i = 0; i < P; ++i) {
    Solver<T>& s = *act[i];
    Dev& v = *view[i];
    const int nb = s.b();
    CHASE_TRY(launch_col_norms(v, s.Va(), s.lv, s.N, nb, s.ow.nrm));
    CHASE_TRY(launch_col_inv_scale(v, s.Va(), s.lv, s.N, nb, s.ow.nrm));
    CHASE_TRY(cholqr_launch(v, s.N, s.dV, s.lv, s.nconv, s.Va(), s.lv, nb, s.ow, 0.0,
                            &s.S.flops_total));
  }
  CHASE_TRY(read_flags("chase_solve_batched QR"));
  std::vector<char> second(P, 0);
  CHASE_TRY(fork());
  for (int i = 0; i < P; ++i) {
    Solver<T>& s = *act[i];
    Dev& v = *view[i];
    if (hf[i] & KERR_CHOL_BREAKDOWN) {  // the single-problem path, with its retry
      CHASE_CUDA(cudaMemsetAsync(flags + i, 0, sizeof(int), d.st));
      CHASE_TRY(orth_core(v, s.N, s.dV, s.lv, s.nconv, s.Va(), s.lv, s.b(), s.ow,
                          &s.S.flops_total));
      continue;
    }
    CHASE_TRY(cholqr_finish(v, s.N, s.Va(), s.lv, s.b(), s.ow, &s.S.flops_total));
    CHASE_TRY(cholqr_launch(v, s.N, s.dV, s.lv, s.nconv, s.Va(), s.lv, s.b(), s.ow, 0.0,
                            &s.S.flops_total));
    second[i] = 1;
  }
  CHASE_TRY(read_flags("chase_solve_batched QR"));
  CHASE_TRY(fork());
  for (int i = 0; i < P; ++i) {
    if (!second[i]) continue;
    Solver<T>& s = *act[i];
    if (hf[i] & KERR_CHOL_BREAKDOWN) {
      set_error("orthonormalisation: Cholesky QR broke down (problem %d of the batch)", i);
      return CHASE_QR_BREAKDOWN;
    }
    CHASE_TRY(cholqr_finish(*view[i], s.N, s.Va(), s.lv, s.b(), s.ow, &s.S.flops_total));
  }
  tm.end();
  // ---- lines 7-8: Rayleigh-Ritz and residuals ----
  tm.begin(&t[1]);
  std::vector<int> off(P + 1, 0);
  for (int i = 0; i < P; ++i) off[i + 1] = off[i] + act[i]->b();
  double* wres = nullptr;  // Ritz values, then residuals, of every problem
  CHASE_TRY(d.alloc(&wres, static_cast<size_t>(2) * off[P]));
  std::vector<EighItem> items(P);
  for (int i = 0; i < P; ++i) {
    Solver<T>& s = *act[i];
    const int nb = s.b();
    CHASE_TRY(rr_pre(*view[i], s.dH, s.N, s.lh, s.Va(), s.lv, nb, s.rw,
                     s.split_rr ? s.rr_slices : nullptr, s.split_rr ? s.rr_sx : nullptr));
    items[i] = EighItem{s.rw.G, ld_pad<T>(nb), nb, wres + off[i]};
  }
  CHASE_TRY(join());
  PhaseTimer te(d.st);
  te.begin(&t[2]);
  int* info = nullptr;
  CHASE_TRY(eigh_batched(d, items, &info));  // (W, Lambda) = TSOLVE(G), every problem
  te.end();
  CHASE_TRY(fork());
  for (int i = 0; i < P; ++i) {
    Solver<T>& s = *act[i];
    const int nb = s.b();
    CHASE_TRY(rr_post(*view[i], s.N, s.Va(), s.lv, nb, wres + off[i], wres + off[P] + off[i], s.rw,
                      &s.S.flops_total));
    s.S.flops_rr_product += s.kMv * s.N2 * nb;
    s.S.matvecs += nb;
  }
  std::vector<double> hw(static_cast<size_t>(2) * off[P]);
  std::vector<int> hinfo(P);
  CHASE_TRY(join());
  CHASE_CUDA(cudaMemcpyAsync(hinfo.data(), info, sizeof(int) * P, cudaMemcpyDeviceToHost, d.st));
  CHASE_CUDA(cudaMemcpyAsync(hw.data(), wres, sizeof(double) * hw.size(), cudaMemcpyDeviceToHost,
                             d.st));
  CHASE_TRY(read_flags("chase_solve_batched Rayleigh-Ritz"));
  tm.end();
  for (int i = 0; i < P; ++i)
    if (hinfo[i] != 0) {
      set_error("batched projected eigensolve returned info = %d", hinfo[i]);
      return CHASE_EIGENSOLVER_ERROR;
    }
  // ---- lines 9-15: locking, bounds, degrees on the host; one reordering ----
  tm.begin(&t[3]);
  std::vector<int> nconv_new(P), hperm(off[P]);
  for (int i = 0; i < P; ++i) {
    Solver<T>& s = *act[i];
    const int nb = s.b();
    std::copy(hw.begin() + off[i], hw.begin() + off[i] + nb, s.ra.begin());
    std::copy(hw.begin() + off[P] + off[i], hw.begin() + off[P] + off[i] + nb, s.rr.begin());
    nconv_new[i] = s.decide(nb);
    std::copy(s.perm.begin(), s.perm.begin() + nb, hperm.begin() + off[i]);
  }
  int* dperm = nullptr;
  CHASE_TRY(d.alloc(&dperm, std::max(off[P], 1)));
  CHASE_CUDA(cudaMemcpyAsync(dperm, hperm.data(), sizeof(int) * off[P], cudaMemcpyHostToDevice,
                             d.st));
  CHASE_TRY(fork());
  for (int i = 0; i < P; ++i) CHASE_TRY(act[i]->apply_perm(*view[i], dperm + off[i]));
  CHASE_TRY(read_flags("chase_solve_batched reordering"));
  tm.end();
  for (int i = 0; i < P; ++i) act[i]->nconv = nconv_new[i];
  return CHASE_OK;
}
}  // namespace
}  // namespace chase

extern "C" int chase_solve_batched(int P, const chase_c64* const* H, const int64_t* N,
                                   const int64_t* ldh, const int* nev, const int* nex,
                                   const double* tol, chase_c64* const* V, const int64_t* ldv,
                                   double* const* Lambda, double* const* resid,
                                   const chase_c64* const* lanczos_starts, const chase_opts* opts_in,
                                   int* status, chase_stats* stats, chase_batch_stats* bstats,
                                   void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  const long long launches0 = chase_kernel_launches();
  if (bstats) *bstats = chase_batch_stats{};
  chase_opts o;
  if (opts_in)
    o = *opts_in;
  else
    chase_opts_default(&o);
  if (P < 0 || (P > 0 && (!H || !N || !ldh || !nev || !nex || !tol || !V || !ldv || !Lambda ||
                          !resid || !lanczos_starts || !status))) {
    set_error("chase_solve_batched: invalid problem count or NULL array");
    return CHASE_INVALID_ARG;
  }
  for (int p = 0; p < P; ++p) {
    if (!solve_args_ok(N[p], ldh[p], nev[p], nex[p], tol[p], ldv[p], H[p], V[p], Lambda[p],
                       resid[p], lanczos_starts[p], o)) {
      set_error("chase_solve_batched: problem %d: invalid argument", p);
      return CHASE_INVALID_ARG;
    }
    if (!is_device_ptr(H[p]) || !is_device_ptr(V[p]) || !is_device_ptr(lanczos_starts[p])) {
      set_error("chase_solve_batched: problem %d: H, V and lanczos_starts must be device arrays", p);
      return CHASE_INVALID_ARG;
    }
  }
  if (P == 0) return CHASE_OK;
  Dev d(stream);
  CHASE_TRY(d.init());
  const bool split = o.precision != CHASE_FP64;
  std::vector<Solver<chase_c64>> sv(P);
  for (int p = 0; p < P; ++p) {
    Solver<chase_c64>& s = sv[p];
    s.H = H[p];
    s.N = N[p];
    s.ldh = ldh[p];
    s.nev = nev[p];
    s.nex = nex[p];
    s.tol = tol[p];
    s.V = V[p];
    s.ldv = ldv[p];
    s.Lambda = Lambda[p];
    s.resid = resid[p];
    s.starts = lanczos_starts[p];
    s.o = o;
    s.dev = true;
  }
  WorkerPool pool(d.st);
  CHASE_TRY(pool.init(std::min(P, kBatchWorkers)));
  // streams for the batched phases (the workspace the workers allocated is
  // released after these finish: the pool synchronises the main stream)
  struct Fan {
    std::vector<cudaStream_t> s;
    ~Fan() {
      for (auto x : s) {
        cudaStreamSynchronize(x);
        cudaStreamDestroy(x);
      }
    }
  } fan;
  for (int k = 0; k < std::min(P, kBatchStreams); ++k) {
    cudaStream_t x = nullptr;
    CHASE_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    fan.s.push_back(x);
  }
  std::vector<int> all(P);  // largest problems first (see WorkerPool::run)
  std::iota(all.begin(), all.end(), 0);
  std::stable_sort(all.begin(), all.end(),
                   [&](int a, int b) {
                     return static_cast<double>(sv[a].N) * (sv[a].nev + sv[a].nex) >
                            static_cast<double>(sv[b].N) * (sv[b].nev + sv[b].nex);
                   });
  // Alg. 1 lines 1-2 of every problem
  CHASE_TRY(pool.run(all, [&](Dev& w, int p) { return sv[p].setup(w, true); }));
  std::vector<GroupedFilterInput> slices(P);  // split: slices of every H, made once
  if (split) {
    std::vector<int> bcap(P);
    for (int p = 0; p < P; ++p) {
      slices[p].H = sv[p].dH;
      slices[p].ldh = sv[p].lh;
      slices[p].n = static_cast<int>(sv[p].N);
      bcap[p] = sv[p].nx;
    }
    CHASE_TRY(grouped_split_prepare(d, slices, bcap));
    for (int p = 0; p < P; ++p) {  // the same slices serve Rayleigh-Ritz's H Q
      Solver<chase_c64>& s = sv[p];
      s.sh.A = slices[p].A;
      s.sh.E = slices[p].E;
      s.sh.Dg = slices[p].Dg;
      s.sh.N = s.N;
      s.sh.Kp = split_k_padded(s.N);
      s.sx.B = slices[p].Bsl;
      s.sx.F = slices[p].F;
      s.sx.cap_cols = slices[p].bcap;
      s.rr_slices = &s.sh;
      s.rr_sx = &s.sx;
    }
  }
  chase_batch_stats bs{};
  bs.problems = P;
  while (true) {  // line 3 of every problem still iterating
    std::vector<int> act;
    for (int p = 0; p < P; ++p)
      if (sv[p].more() && sv[p].begin_iteration()) act.push_back(p);
    if (act.empty()) break;
    std::vector<GroupedFilterInput> in;
    in.reserve(act.size());
    for (int p : act) {
      GroupedFilterInput g = sv[p].filter_input();
      if (split) {
        g.A = slices[p].A;
        g.E = slices[p].E;
        g.Dg = slices[p].Dg;
        g.Bsl = slices[p].Bsl;
        g.F = slices[p].F;
        g.bcap = slices[p].bcap;
      }
      in.push_back(g);
    }
    GroupedFilterTimes tt;
    CHASE_TRY(grouped_filter_sorted(d, in, split, CHASE_TILE_AUTO, &tt));  // line 4, grouped
    bs.steps += tt.steps;
    bs.tile_config = tt.tile_config;
    bs.matvecs += tt.matvecs;
    bs.flops += tt.flops;
    bs.t_autotune += tt.t_autotune;
    bs.t_graph_build += tt.t_graph_build;
    bs.t_steps += tt.t_steps;
    bs.t_product += tt.t_product;
    for (int p : act) {
      Solver<chase_c64>& s = sv[p];
      const long long fm = s.filter_matvecs();
      s.count_filter(fm);
      // the grouped filter's time, shared out by each problem's FLOPs
      if (tt.flops > 0) s.S.t_filter += tt.t_steps * 8.0 * s.N2 * fm / tt.flops;
    }
    // lines 5-15 of every problem at once
    std::vector<Solver<chase_c64>*> ap;
    for (int p : act) ap.push_back(&sv[p]);
    double tph[4] = {0.0, 0.0, 0.0, 0.0};
    CHASE_TRY(batched_after_filter(d, ap, fan.s, tph));
    bs.t_qr += tph[0];
    bs.t_rr += tph[1];
    bs.t_eigh += tph[2];
    bs.t_lock += tph[3];
  }
  int worst = CHASE_OK;
  const double t_total =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  std::vector<int> fin_st(P, CHASE_OK);
  CHASE_TRY(pool.run(all, [&](Dev& w, int p) {
    fin_st[p] = sv[p].finish(w);
    const int st = fin_st[p];
    return (st == CHASE_NOT_CONVERGED || st == CHASE_BOUND_VIOLATION) ? CHASE_OK : st;
  }));
  for (int p = 0; p < P; ++p) {
    const int st = fin_st[p];
    status[p] = st;
    if (worst == CHASE_OK && st != CHASE_OK) worst = st;
    sv[p].S.t_total = t_total;
    if (stats) stats[p] = sv[p].S;
  }
  bs.launches = static_cast<int>(chase_kernel_launches() - launches0);
  bs.t_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (bstats) *bstats = bs;
  return worst;
}
