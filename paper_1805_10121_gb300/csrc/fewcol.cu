// Products with a few right-hand columns (w <= kFewColMax):
//
//   C[:, j] = alpha * (A * B[:, j] - shift * B[0:M, j]) + beta * C[:, j],  j in [j0, j1)
//
// the Lanczos matvecs of Alg. 6 (one vector after a warm start, a block of
// 1 + n_vec otherwise) and the last degree steps of the filter (Alg. 4) when
// only a handful of columns is still active.  A tensor-core tile of 8 or
// more columns would spend most of its work on padding here, and a product
// with so few columns has no operand reuse to exploit, so these run on the
// CUDA cores' FMA pipe: every element of A is read once and multiplied by
// the w entries of B in its row of B^T.
//
// Layout of the work: a warp owns RW consecutive rows of A and splits K over
// KL = 32 / RW lanes (lane = kphase * RW + row), so each load instruction
// reads KL column segments of RW * sizeof(E) = 32 contiguous bytes (one
// sector each).  The KL partial sums of a row are combined by a fixed
// butterfly of shuffles, so the result does not depend on timing.  No
// workspace is needed: the products run inside allocation-free callers.
//
// With one or two columns the FP64 pipe needs A at about 2 TB/s (N = 4000),
// which takes tens of KB of loads in flight per SM: narrow row groups give
// many warps, and each lane keeps kUnroll independent loads of A in flight
// (measured at N = 4000 with one column: 4 rows per warp and 4 loads,
// 310 us and the FP64 pipe 34 % busy, stalled on memory latency; 2 rows and
// 8 loads, 179 us; 16 loads, another 18 % off the Lanczos phase).
#include "common.cuh"
#include "context.hpp"

namespace chase {
namespace {

constexpr int kThreads = 128;  // 4 warps
// independent loads of A in flight per lane: more where the FP64 work per
// loaded element is small
template <int R>
constexpr int kUnroll = R == 1 ? 16 : R <= 2 ? 8 : 4;

template <class E>
struct FC;

template <>
struct FC<double2> {
  using S = double;
  static constexpr int KL = 16;  // 2 rows x 16 B per column segment
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ void fma(double2& c, double2 a, double2 b) {
    c.x = ::fma(a.x, b.x, c.x);
    c.x = ::fma(-a.y, b.y, c.x);
    c.y = ::fma(a.x, b.y, c.y);
    c.y = ::fma(a.y, b.x, c.y);
  }
  static __device__ __forceinline__ double2 shfl_add(double2 v, int m) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, m);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, m);
    return v;
  }
  static __device__ __forceinline__ double2 axpby(double2 acc, double2 bsh, double2 cold, S alpha,
                                                  S beta, S shift, bool use_beta) {
    double2 v = make_double2(alpha * (acc.x - shift * bsh.x), alpha * (acc.y - shift * bsh.y));
    if (use_beta) {
      v.x = ::fma(beta, cold.x, v.x);
      v.y = ::fma(beta, cold.y, v.y);
    }
    return v;
  }
};

template <>
struct FC<double> {
  using S = double;
  static constexpr int KL = 8;  // 4 rows x 8 B per column segment
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ void fma(double& c, double a, double b) { c = ::fma(a, b, c); }
  static __device__ __forceinline__ double shfl_add(double v, int m) {
    return v + __shfl_xor_sync(0xffffffffu, v, m);
  }
  static __device__ __forceinline__ double axpby(double acc, double bsh, double cold, S alpha,
                                                 S beta, S shift, bool use_beta) {
    double v = alpha * (acc - shift * bsh);
    if (use_beta) v = ::fma(beta, cold, v);
    return v;
  }
};

template <>
struct FC<float2> {
  using S = float;
  static constexpr int KL = 8;  // 4 rows x 8 B
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ void fma(float2& c, float2 a, float2 b) {
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(a.y, b.x, c.y);
  }
  static __device__ __forceinline__ float2 shfl_add(float2 v, int m) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, m);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, m);
    return v;
  }
  static __device__ __forceinline__ float2 axpby(float2 acc, float2 bsh, float2 cold, S alpha,
                                                 S beta, S shift, bool use_beta) {
    float2 v = make_float2(alpha * (acc.x - shift * bsh.x), alpha * (acc.y - shift * bsh.y));
    if (use_beta) {
      v.x = fmaf(beta, cold.x, v.x);
      v.y = fmaf(beta, cold.y, v.y);
    }
    return v;
  }
};

template <>
struct FC<float> {
  using S = float;
  static constexpr int KL = 4;  // 8 rows x 4 B
  static __device__ __forceinline__ float zero() { return 0.f; }
  static __device__ __forceinline__ void fma(float& c, float a, float b) { c = fmaf(a, b, c); }
  static __device__ __forceinline__ float shfl_add(float v, int m) {
    return v + __shfl_xor_sync(0xffffffffu, v, m);
  }
  static __device__ __forceinline__ float axpby(float acc, float bsh, float cold, S alpha, S beta,
                                                S shift, bool use_beta) {
    float v = alpha * (acc - shift * bsh);
    if (use_beta) v = fmaf(beta, cold, v);
    return v;
  }
};

template <class E, int R>
__global__ void __launch_bounds__(kThreads)
    fewcol_kernel(const E* __restrict__ A, long long lda, const E* __restrict__ B, long long ldb,
                  E* __restrict__ C, long long ldc, int M, long long K, int j0,
                  typename FC<E>::S alpha, typename FC<E>::S beta, typename FC<E>::S shift) {
  using F = FC<E>;
  constexpr int KL = F::KL, RW = 32 / KL;
  const int lane = threadIdx.x & 31;
  const int row = lane % RW, kp = lane / RW;
  const long long r =
      (static_cast<long long>(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5)) * RW + row;
  const bool live = r < M;

  E acc[R];
#pragma unroll
  for (int j = 0; j < R; ++j) acc[j] = F::zero();

  const E* Ar = A + (live ? r : 0);
  const E* Bj = B + static_cast<long long>(j0) * ldb;
  constexpr int U = kUnroll<R>;
  long long k = kp;
  for (; k + (U - 1) * KL < K; k += U * KL) {
    E h[U];
#pragma unroll
    for (int u = 0; u < U; ++u) h[u] = live ? __ldg(Ar + (k + u * KL) * lda) : F::zero();
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < R; ++j) F::fma(acc[j], h[u], __ldg(Bj + j * ldb + k + u * KL));
  }
  for (; k < K; k += KL) {
    const E h = live ? __ldg(Ar + k * lda) : F::zero();
#pragma unroll
    for (int j = 0; j < R; ++j) F::fma(acc[j], h, __ldg(Bj + j * ldb + k));
  }

  // combine the KL partial sums of each row (lanes differing in kphase)
#pragma unroll
  for (int m = RW; m < 32; m <<= 1)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[j] = F::shfl_add(acc[j], m);

  if (kp != 0 || !live) return;
  const bool use_beta = beta != typename FC<E>::S(0);
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const long long c = j0 + j;
    const E bsh = shift != typename FC<E>::S(0) ? B[c * ldb + r] : F::zero();
    E* cp = C + c * ldc + r;
    *cp = F::axpby(acc[j], bsh, use_beta ? *cp : F::zero(), alpha, beta, shift, use_beta);
  }
}

template <class E, int R>
int launch_r(Dev& d, int64_t M, int64_t K, const E* A, int64_t lda, const E* B, int64_t ldb, E* C,
             int64_t ldc, int j0, double alpha, double beta, double shift) {
  using S = typename FC<E>::S;
  constexpr int rows_per_block = (kThreads / 32) * (32 / FC<E>::KL);
  const unsigned grid = static_cast<unsigned>((M + rows_per_block - 1) / rows_per_block);
  fewcol_kernel<E, R><<<grid, kThreads, 0, d.st>>>(A, lda, B, ldb, C, ldc, static_cast<int>(M), K,
                                                   j0, static_cast<S>(alpha), static_cast<S>(beta),
                                                   static_cast<S>(shift));
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class E>
int launch_any(Dev& d, int64_t M, int64_t K, const E* A, int64_t lda, const E* B, int64_t ldb,
               E* C, int64_t ldc, int j0, int j1, double alpha, double beta, double shift) {
  switch (j1 - j0) {
    case 1: return launch_r<E, 1>(d, M, K, A, lda, B, ldb, C, ldc, j0, alpha, beta, shift);
    case 2: return launch_r<E, 2>(d, M, K, A, lda, B, ldb, C, ldc, j0, alpha, beta, shift);
    case 3: return launch_r<E, 3>(d, M, K, A, lda, B, ldb, C, ldc, j0, alpha, beta, shift);
    case 4: return launch_r<E, 4>(d, M, K, A, lda, B, ldb, C, ldc, j0, alpha, beta, shift);
    case 5: return launch_r<E, 5>(d, M, K, A, lda, B, ldb, C, ldc, j0, alpha, beta, shift);
    case 6: return launch_r<E, 6>(d, M, K, A, lda, B, ldb, C, ldc, j0, alpha, beta, shift);
    default:
      set_error("few-column product: %d columns (at most %d)", j1 - j0, kFewColMax);
      return CHASE_INVALID_ARG;
  }
}

}  // namespace

int fewcol_gemm(Dev& d, int64_t M, int64_t K, const chase_c64* A, int64_t lda, const chase_c64* B,
                int64_t ldb, chase_c64* C, int64_t ldc, int j0, int j1, double alpha, double beta,
                double shift) {
  return launch_any(d, M, K, reinterpret_cast<const double2*>(A), lda,
                    reinterpret_cast<const double2*>(B), ldb, reinterpret_cast<double2*>(C), ldc,
                    j0, j1, alpha, beta, shift);
}

int fewcol_gemm(Dev& d, int64_t M, int64_t K, const double* A, int64_t lda, const double* B,
                int64_t ldb, double* C, int64_t ldc, int j0, int j1, double alpha, double beta,
                double shift) {
  return launch_any(d, M, K, A, lda, B, ldb, C, ldc, j0, j1, alpha, beta, shift);
}

int fewcol_gemm(Dev& d, int64_t M, int64_t K, const chase_c32* A, int64_t lda, const chase_c32* B,
                int64_t ldb, chase_c32* C, int64_t ldc, int j0, int j1, double alpha, double beta,
                double shift) {
  return launch_any(d, M, K, reinterpret_cast<const float2*>(A), lda,
                    reinterpret_cast<const float2*>(B), ldb, reinterpret_cast<float2*>(C), ldc, j0,
                    j1, alpha, beta, shift);
}

int fewcol_gemm(Dev& d, int64_t M, int64_t K, const float* A, int64_t lda, const float* B,
                int64_t ldb, float* C, int64_t ldc, int j0, int j1, double alpha, double beta,
                double shift) {
  return launch_any(d, M, K, A, lda, B, ldb, C, ldc, j0, j1, alpha, beta, shift);
}

}  // namespace chase
