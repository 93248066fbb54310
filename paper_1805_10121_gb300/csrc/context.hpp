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
  // A view on another context's stream with a flag slot of its own (the
  // per-problem flags of a batch): err is borrowed, and leaving the view
  // does not synchronise (its workspace is released stream-ordered).
  bool own_err = true, sync_on_exit = true;

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

// Records a CUDA event pair on stream `s` around product launches while
// chase_kernel_timing is on (a no-op otherwise).  end() gives the launches
// the range covered and their algorithmic (FP64-equivalent) and executed
// tensor FLOPs; a timer destroyed without end() records nothing.
class KernelTimer {
 public:
  KernelTimer(cudaStream_t s, int kind);
  ~KernelTimer();
  KernelTimer(const KernelTimer&) = delete;
  KernelTimer& operator=(const KernelTimer&) = delete;
  void end(long long launches, double flops, double tensor_flops);

 private:
  cudaStream_t st_;
  int kind_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
  bool active_ = false;
};

// 2-D copies of column-major complex128 blocks (rows x cols).
int copy_block(Dev& d, chase_c64* dst, int64_t ldd, const chase_c64* src, int64_t lds, int64_t rows,
               int64_t cols, cudaMemcpyKind kind);
int copy_block(Dev& d, double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows,
               int64_t cols, cudaMemcpyKind kind);
int copy_block(Dev& d, chase_c32* dst, int64_t ldd, const chase_c32* src, int64_t lds, int64_t rows,
               int64_t cols, cudaMemcpyKind kind);
int copy_block(Dev& d, float* dst, int64_t ldd, const float* src, int64_t lds, int64_t rows,
               int64_t cols, cudaMemcpyKind kind);

// ---- kernels.cu ------------------------------------------------------------
// Element launchers are templates over the scalar T: chase_c64 (Hermitian
// problems) or double (real symmetric ones); both are instantiated.
// Stable counting sort of the degrees (warp-level match/popc scans):
// perm[pos] = original column at sorted position pos; start[i] = number of
// columns with degree < i (i = 0 .. max_deg + 1); info[0] = max degree.
int launch_filter_plan(Dev& d, const int* deg, int b, int max_allowed, int* perm, int* start,
                       int* info);
// Y[:, j] = X[:, perm[j]]  (gather) or Y[:, perm[j]] = X[:, j] (scatter)
template <class T>
int launch_permute_cols(Dev& d, const T* X, int64_t ldx, T* Y, int64_t ldy, int64_t N, int b,
                        const int* perm, bool scatter);
// out[j] = ||X[:, j]||_2
template <class T>
int launch_col_norms(Dev& d, const T* X, int64_t ldx, int64_t N, int b, double* out);
// X[:, j] *= 1 / s[j]   (s[j] == 0 leaves the column)
template <class T>
int launch_col_inv_scale(Dev& d, T* X, int64_t ldx, int64_t N, int b, const double* s);
// res[j] = ||HV[:, j] - lam[j] V[:, j]||_2
template <class T>
int launch_resid_norms(Dev& d, const T* HV, int64_t ldhv, const T* V, int64_t ldv, int64_t N, int b,
                       const double* lam, double* res);
// Upper triangle of the p x p matrix G <- conjugate of its lower triangle,
// diagonal made real: the Hermitian matrix that G's lower triangle defines.
template <class T>
int launch_fill_upper_hermitian(Dev& d, T* G, int64_t ldg, int p);
// In-place lower Cholesky G = L L^H (one CTA); sets KERR_CHOL_BREAKDOWN when a
// pivot is not above rel_tol * G_jj.  `shift` is added to the diagonal first.
template <class T>
int launch_cholesky(Dev& d, T* G, int64_t ldg, int p, double rel_tol, double shift);
// Blocked Cholesky (32-wide panels, trailing updates on the FP64 GEMM); the
// pivot test uses the diagonal of G + shift before any update (diag_ref, p
// doubles of workspace); work holds >= 32 p entries.
template <class T>
int cholesky_blocked(Dev& d, T* G, int64_t ldg, int p, double rel_tol, double shift,
                     double* diag_ref, T* work);
// X (N x p) <- X L^-H (blocked right-side triangular solve); work >= 32 p entries.
template <class T>
int trsm_right_lh(Dev& d, T* X, int64_t ldx, int64_t N, const T* L, int64_t ldl, int p, T* work);
// One Lanczos three-term step on r independent runs (one CTA per run, run c
// in column c of each N x r block, leading dimension ld):
// alpha = Re(v^H w); w -= alpha v + beta_prev v_prev; beta = ||w||;
// v_next = w / beta (zero when beta <= tiny * the run's largest coefficient,
// i.e. rounding noise).  alpha/beta arrays are indexed [step * r + run].
template <class T>
int launch_lanczos_step(Dev& d, int64_t N, int64_t ld, int r, int step, const T* Vj,
                        const T* Vprev, T* W, T* Vnext, double* alpha, double* beta, double tiny);
// Normalise r columns in place (Lanczos start vectors).
template <class T>
int launch_normalize_cols(Dev& d, T* X, int64_t ldx, int64_t N, int r);
// F (n x n, ldf) = the Hermitian (real: symmetric) matrix whose lower
// triangle, diagonal included, is that of L; L's strict upper part is not read.
template <class T>
int launch_hermitian_from_lower(Dev& d, const T* L, int64_t ldl, T* F, int64_t ldf, int64_t n);
// dst (rows x cols, ldd) = src rounded to / widened from single precision.
int launch_convert(Dev& d, const chase_c32* src, int64_t lds, chase_c64* dst, int64_t ldd,
                   int64_t rows, int64_t cols);
int launch_convert(Dev& d, const chase_c64* src, int64_t lds, chase_c32* dst, int64_t ldd,
                   int64_t rows, int64_t cols);
int launch_convert(Dev& d, const float* src, int64_t lds, double* dst, int64_t ldd, int64_t rows,
                   int64_t cols);
int launch_convert(Dev& d, const double* src, int64_t lds, float* dst, int64_t ldd, int64_t rows,
                   int64_t cols);
// Fill the strict lower (lower=true) or upper part of a p x p matrix with zero.
template <class T>
int launch_zero_triangle(Dev& d, T* A, int64_t lda, int p, bool lower);
// Real Gram product C = X^T Y (X N x p, Y N x q) on the FP64 tensor pipe.
int dgram(Dev& d, int64_t N, const double* X, int64_t ldx, int p, const double* Y, int64_t ldy,
          int q, double* C, int64_t ldc, bool lower = false);
inline int gram(Dev& d, int64_t N, const chase_c64* X, int64_t ldx, int p, const chase_c64* Y,
                int64_t ldy, int q, chase_c64* C, int64_t ldc, bool lower = false) {
  return zgram(d, N, X, ldx, p, Y, ldy, q, C, ldc, lower);
}
inline int gram(Dev& d, int64_t N, const double* X, int64_t ldx, int p, const double* Y,
                int64_t ldy, int q, double* C, int64_t ldc, bool lower = false) {
  return dgram(d, N, X, ldx, p, Y, ldy, q, C, ldc, lower);
}
int cgram(Dev& d, int64_t N, const chase_c32* X, int64_t ldx, int p, const chase_c32* Y,
          int64_t ldy, int q, chase_c32* C, int64_t ldc, bool lower = false);
int sgram(Dev& d, int64_t N, const float* X, int64_t ldx, int p, const float* Y, int64_t ldy,
          int q, float* C, int64_t ldc, bool lower = false);
inline int gram(Dev& d, int64_t N, const chase_c32* X, int64_t ldx, int p, const chase_c32* Y,
                int64_t ldy, int q, chase_c32* C, int64_t ldc, bool lower = false) {
  return cgram(d, N, X, ldx, p, Y, ldy, q, C, ldc, lower);
}
inline int gram(Dev& d, int64_t N, const float* X, int64_t ldx, int p, const float* Y,
                int64_t ldy, int q, float* C, int64_t ldc, bool lower = false) {
  return sgram(d, N, X, ldx, p, Y, ldy, q, C, ldc, lower);
}

// ---- zgemm_split.cu: split-BF16 filter product on the tensor cores --------
// Slices of H (S planes of N x Kp bf16) and row exponents: complex H gives
// Ht = [Re H | Im H] (Kp >= 2N), real symmetric H itself (Kp >= N).
struct SplitH {
  void* A = nullptr;
  int* E = nullptr;
  double* Dg = nullptr;  // real diagonal of H, applied in FP64 by the epilogue
  int64_t N = 0, Kp = 0;
  int cplx = 1;
};
// Slice workspace for up to max_cols columns of the filter block.
struct SplitX {
  void* B = nullptr;
  int* F = nullptr;
  int cap_cols = 0;
  int cplx = 1;
  void* P = nullptr;  // FP64 partial products of K segments (grow-only)
  size_t P_cap = 0;   // in units of 16 bytes
};
int split_prepare_h(Dev& d, const chase_c64* H, int64_t N, int64_t ldh, SplitH& out);
int split_prepare_h(Dev& d, const double* H, int64_t N, int64_t ldh, SplitH& out);
// The same slices from a complex64 / float32 H (entries widened exactly).
int split_prepare_h(Dev& d, const chase_c32* H, int64_t N, int64_t ldh, SplitH& out);
int split_prepare_h(Dev& d, const float* H, int64_t N, int64_t ldh, SplitH& out);
int split_alloc_x(Dev& d, int64_t N, int max_cols, SplitX& out, bool cplx = true);
// C[:, j0:j1] = alpha (H X[:, j0:j1] - shift X[:, j0:j1]) + beta C[:, j0:j1]
// with the leading `nslices` slices of each operand (7: full accuracy, about
// 2^-49 relative; 4: about 2^-28; 3: about 2^-21).
int zgemm_split(Dev& d, const SplitH& h, SplitX& x, const chase_c64* X, int64_t ldx, int j0, int j1,
                chase_c64* C, int64_t ldc, double alpha, double beta, double shift,
                int nslices = 7);
int zgemm_split(Dev& d, const SplitH& h, SplitX& x, const double* X, int64_t ldx, int j0, int j1,
                double* C, int64_t ldc, double alpha, double beta, double shift, int nslices = 7);

// ---- grouped filter: many independent problems per launch ----------------
// One problem of a grouped filter, in device memory.  buf0 holds the block
// sorted by degree (the filter's input and final output), buf1 is the second
// buffer of the three-term recurrence; their tensor maps (FP64 path) or the
// slice planes and maps (split path) live in device memory too.
struct GroupedProblem {
  const CUtensorMap* mapA;   // H (FP64) or the slice planes of H (split)
  const CUtensorMap* mapB0;  // FP64: buf0; split: the slices of the active block
  const CUtensorMap* mapB1;  // FP64: buf1
  double2* buf0;
  double2* buf1;
  long long ld0, ld1;
  const int* E;       // split: row exponents of H
  int* F;             // split: column exponents of the active block
  const double* Dg;   // split: real diagonal of H
  void* Bsl;          // split: slice planes of the block [S][2 bcap][Kp]
  long long Kp;       // split: padded K = 2N rounded up to 16
  int n, b, bcap;     // rows, columns of the block, column capacity of Bsl
};
// One active problem of one degree step: columns [s, b) of problem `prob`
// are filtered; its output tiles are CTAs [tile0, next.tile0) and its
// columns [col0, next.col0) of the step's column range.  A step's list ends
// with a sentinel entry holding the totals.
struct GroupedStep {
  int prob, s, tile0, col0;
  double alpha, beta, shift;
};
// FP64 tile shapes of the grouped product (rows x complex columns per CTA).
constexpr int kGroupedFp64Cfgs = 4;
void grouped_fp64_tile(int cfg, int* bm, int* bn);
// One degree step of the FP64 grouped filter: X = parity ? buf1 : buf0,
// Y = the other buffer.
int zgemm_grouped_fp64(Dev& d, int cfg, const GroupedProblem* probs, const GroupedStep* steps,
                       int nact, int ntiles, int parity);
// Kernel attributes (shared memory size) set outside any stream capture.
int zgemm_grouped_fp64_prepare(int cfg);
int zgemm_split_grouped_prepare();
// Split path: slice the active columns of every active problem (one CTA per
// column), then the grouped tensor-core product (one CTA per output tile).
int split_grouped_slice_x(Dev& d, const GroupedProblem* probs, const GroupedStep* steps, int nact,
                          int ncols, int parity);
int zgemm_split_grouped(Dev& d, const GroupedProblem* probs, const GroupedStep* steps, int nact,
                        int ntiles, int parity);
constexpr int kSplitTileRows = 128;      // rows of H per split tile
constexpr int kSplitTileRealCols = 64;   // real columns (32 complex) per split tile
constexpr int kSplitSlices = 7;
constexpr int kSplitStageK = 32;         // K per TMA stage box (64-byte swizzled rows)
int64_t split_k_padded(int64_t N);
// Slices of every problem's H: one CTA per row over all problems; row_prob
// holds the first global row of each problem (P + 1 entries).
struct GroupedSliceH {
  const double2* H;
  long long ldh;
  void* A;
  int* E;
  double* Dg;
  long long Kp;
  int n, row0;
};
int split_grouped_prepare_h(Dev& d, const GroupedSliceH* probs, int P, int total_rows);
// One problem of grouped_filter_sorted: the block X (b columns, sorted by
// ascending degree) is filtered in place with W as the second buffer;
// start[i] (host, i = 0 .. maxdeg + 1) counts the columns of degree < i.
// Split path: the slices of H (A, E, Dg) and a slice workspace of bcap >= b
// columns (Bsl, F), as made by grouped_split_prepare.
struct GroupedFilterInput {
  const chase_c64* H = nullptr;
  int64_t ldh = 0;
  int n = 0;
  chase_c64* X = nullptr;
  int64_t ldx = 0;
  chase_c64* W = nullptr;
  int64_t ldw = 0;
  int b = 0;
  const int* start = nullptr;
  int maxdeg = 0;
  double b_sup = 0, mu1 = 0, mu_nn = 0;
  void* A = nullptr;
  int* E = nullptr;
  double* Dg = nullptr;
  void* Bsl = nullptr;
  int* F = nullptr;
  int bcap = 0;
};
struct GroupedFilterTimes {
  int tile_config = -1, steps = 0, launches = 0;
  long long matvecs = 0;
  double flops = 0, t_autotune = 0, t_graph_build = 0, t_steps = 0, t_product = 0;
};
// Slices of every problem's H and the slice workspace for bcap[q] columns
// (one grouped slicing launch); fills the split fields of `in`.
int grouped_split_prepare(Dev& d, std::vector<GroupedFilterInput>& in, const std::vector<int>& bcap);
// Alg. 4 on every problem of `in` (problems with b == 0 are skipped), one
// grouped launch per degree step, all steps in one CUDA graph.  tile:
// CHASE_TILE_AUTO or a fixed FP64 tile shape.  Synchronises the stream.
int grouped_filter_sorted(Dev& d, const std::vector<GroupedFilterInput>& in, bool split, int tile,
                          GroupedFilterTimes* times);

// Column gather / scatter for many problems: one CTA per column.
struct GroupedPermute {
  const double2* src;
  double2* dst;
  long long lds, ldd;
  const int* perm;
  int n, col0;
};
int launch_grouped_permute(Dev& d, const GroupedPermute* probs, int P, int total_cols, bool scatter);

// ---- eigh (cuSOLVER, the small projected eigensolve of Alg. 2 line 3) -----
int eigh_device(Dev& d, chase_c64* G, int64_t ldg, int p, double* w_dev);
int eigh_device(Dev& d, double* G, int64_t ldg, int p, double* w_dev);
// Single precision (cheevd / ssyevd); eigenvalues returned in double.
int eigh_device(Dev& d, chase_c32* G, int64_t ldg, int p, double* w_dev);
int eigh_device(Dev& d, float* G, int64_t ldg, int p, double* w_dev);
// Many small projected eigenproblems at once (cuSOLVER's batched Hermitian
// eigensolver on buckets of sizes rounded up to 16, each matrix padded as
// diag(G, pad I)): item q's G (p x p, ldg, Hermitian, both triangles) is
// overwritten by its eigenvectors and w (p doubles, device) receives its
// eigenvalues ascending.  *info_dev (device, one int per item in bucket
// order) is nonzero where the eigensolver failed; the caller reads it after
// its next synchronisation.
struct EighItem {
  chase_c64* G;
  long long ldg;
  int p;
  double* w;
};
int eigh_batched(Dev& d, const std::vector<EighItem>& items, int** info_dev);
// Destroy the calling thread's cuSOLVER handle (worker threads, before they end).
void release_thread_solver();

// ---- host_alg.cpp ----------------------------------------------------------
// Symmetric tridiagonal eigenproblem (implicit QL with Wilkinson shifts):
// diag[k], off[k-1] -> eigenvalues ascending in w, eigenvectors (k x k,
// column-major) in z.  Returns false if it fails to converge.
bool tridiag_eigh(int k, const double* diag, const double* off, double* w, double* z);
// Alg. 6 line 11 (Eq. 10 quantile with its width safeguard); see
// chase_dos_estimate in chase.h.  halvings / fallback may be NULL.
double dos_estimate(int nruns, const int* steps, const double* theta, const double* w,
                    double target, double mu1, double b_sup, double dos_sigma, int* halvings,
                    bool* fallback);

}  // namespace chase
