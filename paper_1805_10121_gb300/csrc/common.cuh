// Shared device and host helpers of libchase (sm_103a).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "chase.h"

namespace chase {

// ----------------------------------------------------------------------------
// Error reporting (host)
// ----------------------------------------------------------------------------
void set_error(const char* fmt, ...);
int cuda_status(cudaError_t e, const char* what);
// Count kernel launches issued by the library (chase_kernel_launches()).
void note_launch(int n = 1);

#define CHASE_CUDA(call)                                     \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return ::chase::cuda_status(e_, #call); \
  } while (0)

#define CHASE_TRY(expr)            \
  do {                             \
    int s_ = (expr);               \
    if (s_ != CHASE_OK) return s_; \
  } while (0)

// Kernel error flags written by device code (bit field).
enum : int {
  KERR_TIMEOUT_FULL = 1,    // consumer gave up waiting for a TMA stage
  KERR_TIMEOUT_EMPTY = 2,   // producer gave up waiting for a free stage
  KERR_BAD_DEGREE = 4,      // plan kernel saw an odd / out-of-range degree
  KERR_CHOL_BREAKDOWN = 8,  // Cholesky pivot not safely positive
};

// Upper bound on one bounded wait, in SM clock cycles (~1 s at 2 GHz).
constexpr long long kWaitBudgetCycles = 2000000000LL;

// ----------------------------------------------------------------------------
// Device helpers: mbarrier, TMA, DMMA
// ----------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the phase with the given parity to complete, at most `budget`
// cycles.  Returns false on timeout (the caller records an error and exits).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long budget = kWaitBudgetCycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// 2-D tiled TMA load global -> shared, completion counted on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// D = A(8x4, row) * B(4x8, col) + D on the FP64 tensor pipe.
// Fragment layout: a = A[lane/4][lane%4], b = B[lane%4][lane/4],
// d = {D[lane/4][2*(lane%4)], D[lane/4][2*(lane%4)+1]}.
__device__ __forceinline__ void dmma_8x8x4(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}
#endif  // __CUDACC__

// ----------------------------------------------------------------------------
// Host: tensor maps
// ----------------------------------------------------------------------------
// A complex128 column-major matrix (rows x cols, leading dimension ld) viewed
// as a 2-D float64 tensor {2*rows, cols}; box {2*box_rows, box_cols}.
int make_tmap_c64(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
                  int box_rows, int box_cols);
// A float64 column-major matrix (rows x cols, leading dimension ld) as a 2-D
// tensor {rows, cols}; box {box_rows, box_cols}.
int make_tmap_f64(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
                  int box_rows, int box_cols);
// A 3-D bf16 tensor {d0, d1, d2} with byte strides s1 (dim 1) and s2 (dim 2),
// box {b0, b1, b2}, 32-byte swizzle (b0 * 2 must be 32).
int make_tmap_bf16_3d(CUtensorMap* map, const void* base, int64_t d0, int64_t d1, int64_t d2,
                      int64_t s1, int64_t s2, int b0, int b1, int b2);

// ----------------------------------------------------------------------------
// Host: launch wrappers implemented in the .cu files
// ----------------------------------------------------------------------------
struct Dev;  // per-call device context (stream, error flag, workspace)

// C[:, j0:j1] = alpha * (A * B[:, j0:j1] - shift * B[0:M, j0:j1]) + beta * C[:, j0:j1]
// A: M x K (lda), B: K x ncols (ldb), C: M x ncols (ldc).  shift != 0 needs M == K.
int zgemm(Dev& d, int64_t M, int64_t K, const chase_c64* A, int64_t lda, const chase_c64* B,
          int64_t ldb, int64_t ncols_b, chase_c64* C, int64_t ldc, int j0, int j1, double alpha,
          double beta, double shift);

// The same for real matrices (one DMMA per fragment instead of the 3M form).
int dgemm(Dev& d, int64_t M, int64_t K, const double* A, int64_t lda, const double* B, int64_t ldb,
          int64_t ncols_b, double* C, int64_t ldc, int j0, int j1, double alpha, double beta,
          double shift);
inline int gemm(Dev& d, int64_t M, int64_t K, const chase_c64* A, int64_t lda, const chase_c64* B,
                int64_t ldb, int64_t ncols_b, chase_c64* C, int64_t ldc, int j0, int j1,
                double alpha, double beta, double shift) {
  return zgemm(d, M, K, A, lda, B, ldb, ncols_b, C, ldc, j0, j1, alpha, beta, shift);
}
inline int gemm(Dev& d, int64_t M, int64_t K, const double* A, int64_t lda, const double* B,
                int64_t ldb, int64_t ncols_b, double* C, int64_t ldc, int j0, int j1, double alpha,
                double beta, double shift) {
  return dgemm(d, M, K, A, lda, B, ldb, ncols_b, C, ldc, j0, j1, alpha, beta, shift);
}

// Single precision (complex64 / float32) on the CUDA cores, same contract.
int cgemm(Dev& d, int64_t M, int64_t K, const chase_c32* A, int64_t lda, const chase_c32* B,
          int64_t ldb, int64_t ncols_b, chase_c32* C, int64_t ldc, int j0, int j1, double alpha,
          double beta, double shift);
int sgemm(Dev& d, int64_t M, int64_t K, const float* A, int64_t lda, const float* B, int64_t ldb,
          int64_t ncols_b, float* C, int64_t ldc, int j0, int j1, double alpha, double beta,
          double shift);
inline int gemm(Dev& d, int64_t M, int64_t K, const chase_c32* A, int64_t lda, const chase_c32* B,
                int64_t ldb, int64_t ncols_b, chase_c32* C, int64_t ldc, int j0, int j1,
                double alpha, double beta, double shift) {
  return cgemm(d, M, K, A, lda, B, ldb, ncols_b, C, ldc, j0, j1, alpha, beta, shift);
}
inline int gemm(Dev& d, int64_t M, int64_t K, const float* A, int64_t lda, const float* B,
                int64_t ldb, int64_t ncols_b, float* C, int64_t ldc, int j0, int j1, double alpha,
                double beta, double shift) {
  return sgemm(d, M, K, A, lda, B, ldb, ncols_b, C, ldc, j0, j1, alpha, beta, shift);
}

// Products with at most kFewColMax columns (fewcol.cu), same contract as the
// gemm overloads above; they run on the CUDA cores' FMA pipe without
// workspace, and the gemm overloads route every such product here.
constexpr int kFewColMax = 6;
int fewcol_gemm(Dev& d, int64_t M, int64_t K, const chase_c64* A, int64_t lda, const chase_c64* B,
                int64_t ldb, chase_c64* C, int64_t ldc, int j0, int j1, double alpha, double beta,
                double shift);
int fewcol_gemm(Dev& d, int64_t M, int64_t K, const double* A, int64_t lda, const double* B,
                int64_t ldb, double* C, int64_t ldc, int j0, int j1, double alpha, double beta,
                double shift);
int fewcol_gemm(Dev& d, int64_t M, int64_t K, const chase_c32* A, int64_t lda, const chase_c32* B,
                int64_t ldb, chase_c32* C, int64_t ldc, int j0, int j1, double alpha, double beta,
                double shift);
int fewcol_gemm(Dev& d, int64_t M, int64_t K, const float* A, int64_t lda, const float* B,
                int64_t ldb, float* C, int64_t ldc, int j0, int j1, double alpha, double beta,
                double shift);

// C (p x q, ldc) = X^H Y with X: N x p (ldx), Y: N x q (ldy).  lower: only
// the entries on and below the diagonal are formed (the rest of C is left as
// it was), for Hermitian results of which only the lower triangle is read.
int zgram(Dev& d, int64_t N, const chase_c64* X, int64_t ldx, int p, const chase_c64* Y,
          int64_t ldy, int q, chase_c64* C, int64_t ldc, bool lower = false);

}  // namespace chase
