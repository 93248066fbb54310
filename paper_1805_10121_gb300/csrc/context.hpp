// Per-call device context and the internal launch interface of libchase.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace chase {

// Device context of one ABI call: the stream, a device error flag and the
// stream-ordered workspace allocations, released when the context ends.
struct Dev {
  cudaStream_t st = nullptr;
  int* err = nullptr;  // device int, bit field of KERR_* codes
  std::vector<void*> bufs;

  explicit Dev(void* stream) : st(static_cast<cudaStream_t>(stream)) {}
  Dev(const Dev&) = delete;
  Dev& operator=(const Dev&) = delete;
  ~Dev();

  int init();
  int alloc_bytes(void** p, size_t bytes);
  template <class T>
  int alloc(T** p, size_t count) {
    return alloc_bytes(reinterpret_cast<void**>(p), count * sizeof(T));
  }
  // Synchronise the stream and turn the device error flag into a status.
  int sync_check(const char* where);
};

bool is_device_ptr(const void* p);

// 2-D copies of column-major complex128 blocks (rows x cols).
int copy_block(Dev& d, chase_c64* dst, int64_t ldd, const chase_c64* src, int64_t lds, int64_t rows,
               int64_t cols, cudaMemcpyKind kind);

// ---- kernels.cu ------------------------------------------------------------
// Stable counting sort of the degrees (warp-level match/popc scans):
// perm[pos] = original column at sorted position pos; start[i] = number of
// columns with degree < i (i = 0 .. max_deg + 1); info[0] = max degree.
int launch_filter_plan(Dev& d, const int* deg, int b, int max_allowed, int* perm, int* start,
                       int* info);
// Y[:, j] = X[:, perm[j]]  (gather) or Y[:, perm[j]] = X[:, j] (scatter)
int launch_permute_cols(Dev& d, const chase_c64* X, int64_t ldx, chase_c64* Y, int64_t ldy,
                        int64_t N, int b, const int* perm, bool scatter);
// out[j] = ||X[:, j]||_2
int launch_col_norms(Dev& d, const chase_c64* X, int64_t ldx, int64_t N, int b, double* out);
// X[:, j] *= 1 / s[j]   (s[j] == 0 leaves the column)
int launch_col_inv_scale(Dev& d, chase_c64* X, int64_t ldx, int64_t N, int b, const double* s);
// res[j] = ||HV[:, j] - lam[j] V[:, j]||_2
int launch_resid_norms(Dev& d, const chase_c64* HV, int64_t ldhv, const chase_c64* V, int64_t ldv,
                       int64_t N, int b, const double* lam, double* res);
// G <- (G + G^H) / 2 for a p x p matrix
int launch_hermitize(Dev& d, chase_c64* G, int64_t ldg, int p);
// In-place lower Cholesky G = L L^H (one CTA); sets KERR_CHOL_BREAKDOWN when a
// pivot is not above rel_tol * G_jj.  `shift` is added to the diagonal first.
int launch_cholesky(Dev& d, chase_c64* G, int64_t ldg, int p, double rel_tol, double shift);
// Blocked Cholesky (32-wide panels, trailing updates on the FP64 GEMM); the
// pivot test uses the diagonal of G + shift before any update (diag_ref, p
// doubles of workspace); work holds >= 32 p entries.
int cholesky_blocked(Dev& d, chase_c64* G, int64_t ldg, int p, double rel_tol, double shift,
                     double* diag_ref, chase_c64* work);
// X (N x p) <- X L^-H (blocked right-side triangular solve); work >= 32 p entries.
int trsm_right_lh(Dev& d, chase_c64* X, int64_t ldx, int64_t N, const chase_c64* L, int64_t ldl,
                  int p, chase_c64* work);
// One Lanczos three-term step on r independent runs (one CTA per run):
// alpha = Re(v^H w); w -= alpha v + beta_prev v_prev; beta = ||w||;
// v_next = w / beta (zero when beta is rounding noise).  alpha/beta arrays
// are indexed [step * r + run].
int launch_lanczos_step(Dev& d, int64_t N, int r, int step, const chase_c64* Vj, const chase_c64* Vprev,
                        chase_c64* W, chase_c64* Vnext, double* alpha, double* beta);
// Normalise r columns in place (Lanczos start vectors).
int launch_normalize_cols(Dev& d, chase_c64* X, int64_t ldx, int64_t N, int r);
// Fill the strict lower (lower=true) or upper part of a p x p matrix with zero.
int launch_zero_triangle(Dev& d, chase_c64* A, int64_t lda, int p, bool lower);

// ---- zgemm_split.cu: split-BF16 filter product on the tensor cores --------
// Slices of Ht = [Re H | Im H] (S planes of N x Kp bf16) and row exponents.
struct SplitH {
  void* A = nullptr;
  int* E = nullptr;
  double* Dg = nullptr;  // real diagonal of H, applied in FP64 by the epilogue
  int64_t N = 0, Kp = 0;
};
// Slice workspace for up to max_cols complex columns of the filter block.
struct SplitX {
  void* B = nullptr;
  int* F = nullptr;
  int cap_cols = 0;
  void* P = nullptr;  // FP64 partial products of K segments (grow-only)
  size_t P_cap = 0;   // in complex entries
};
int split_prepare_h(Dev& d, const chase_c64* H, int64_t N, int64_t ldh, SplitH& out);
int split_alloc_x(Dev& d, int64_t N, int max_cols, SplitX& out);
// C[:, j0:j1] = alpha (H X[:, j0:j1] - shift X[:, j0:j1]) + beta C[:, j0:j1]
int zgemm_split(Dev& d, const SplitH& h, SplitX& x, const chase_c64* X, int64_t ldx, int j0, int j1,
                chase_c64* C, int64_t ldc, double alpha, double beta, double shift);

// ---- eigh (cuSOLVER, the small projected eigensolve of Alg. 2 line 3) -----
int eigh_device(Dev& d, chase_c64* G, int64_t ldg, int p, double* w_dev);

// ---- host_alg.cpp ----------------------------------------------------------
// Symmetric tridiagonal eigenproblem (implicit QL with Wilkinson shifts):
// diag[k], off[k-1] -> eigenvalues ascending in w, eigenvectors (k x k,
// column-major) in z.  Returns false if it fails to converge.
bool tridiag_eigh(int k, const double* diag, const double* off, double* w, double* z);

}  // namespace chase
