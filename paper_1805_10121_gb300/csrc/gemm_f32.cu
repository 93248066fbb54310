// Single-precision products of the FP32 solver path (complex64 and float32):
//
//   C[:, j] = alpha * (A * B[:, j] - shift * B[0:M, j]) + beta * C[:, j],  j in [j0, j1)
//   C = X^H Y                                                  (Gram, split over K)
//
// The paper's library instantiates the solver in single precision as well
// (Sec. 5.1); on GB300 FP32 runs on the CUDA cores (FFMA, 67 TFLOP/s), so these
// are SIMT kernels: 64 x 64 output tiles, 256 threads with 4 x 4 outputs each,
// operand tiles of 16-wide K staged in shared memory with the next tile
// prefetched into registers.  A complex multiply-add is four FFMAs.  The
// recurrence's shift, scale and axpby (Eq. 7) are applied to the accumulators
// before the single store, as in the FP64 and split-BF16 products.
#include <algorithm>

#include "common.cuh"
#include "context.hpp"

namespace chase {
namespace {

constexpr int TM = 64, TN = 64, TK = 16, NT = 256;

template <class E>
struct Ops;
template <>
struct Ops<float2> {
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ float2 conj(float2 a) { return make_float2(a.x, -a.y); }
  static __device__ __forceinline__ void fma(float2& c, float2 a, float2 b) {
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(a.y, b.x, c.y);
  }
  static __device__ __forceinline__ float2 axpby(float2 acc, float2 bsh, float2 cold, float alpha,
                                                 float beta, float shift, bool use_beta) {
    float2 v = make_float2(alpha * (acc.x - shift * bsh.x), alpha * (acc.y - shift * bsh.y));
    if (use_beta) {
      v.x = fmaf(beta, cold.x, v.x);
      v.y = fmaf(beta, cold.y, v.y);
    }
    return v;
  }
};
template <>
struct Ops<float> {
  static __device__ __forceinline__ float zero() { return 0.f; }
  static __device__ __forceinline__ float conj(float a) { return a; }
  static __device__ __forceinline__ void fma(float& c, float a, float b) { c = fmaf(a, b, c); }
  static __device__ __forceinline__ float axpby(float acc, float bsh, float cold, float alpha,
                                                float beta, float shift, bool use_beta) {
    float v = alpha * (acc - shift * bsh);
    if (use_beta) v = fmaf(beta, cold, v);
    return v;
  }
};

// GRAM = false: C = alpha (A B - shift B) + beta C on the tile (blockIdx.x,
// blockIdx.y) of columns [j0, j1).  GRAM = true: P_z = X^H Y over the K
// chunk z (A = X read transposed and conjugated; C is the partial buffer).
template <class E, bool GRAM>
__global__ void __launch_bounds__(NT)
    f32_gemm_kernel(const E* __restrict__ A, long long lda, const E* __restrict__ B, long long ldb,
                    E* __restrict__ C, long long ldc, int M, long long K, int j0, int j1,
                    float alpha, float beta, float shift, long long kchunk, long long pstride,
                    int lower) {
  // Gram with lower: tiles strictly above the diagonal are not wanted
  if (GRAM && lower && blockIdx.x < blockIdx.y) return;
  __shared__ E As[TK][TM + 1];
  __shared__ E Bs[TK][TN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * TM;
  const int c0 = j0 + blockIdx.y * TN;
  const long long kbeg = GRAM ? blockIdx.z * kchunk : 0;
  const long long kend = GRAM ? min(K, kbeg + kchunk) : K;

  E acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = Ops<E>::zero();

  E ra[4], rb[4];  // the next tile, 4 elements of A and of B per thread
  auto fetch = [&](long long k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + NT * r;
      E va = Ops<E>::zero(), vb = Ops<E>::zero();
      if (GRAM) {  // A[m][k] = conj(X[k, m]): K fastest for coalescing
        const int kk = e % TK, m = e / TK;
        const long long k = k0 + kk;
        if (k < kend && m0 + m < M) va = Ops<E>::conj(A[(long long)(m0 + m) * lda + k]);
      } else {
        const int m = e % TM, kk = e / TM;
        const long long k = k0 + kk;
        if (k < kend && m0 + m < M) va = A[k * lda + m0 + m];
      }
      {
        const int kk = e % TK, n = e / TK;
        const long long k = k0 + kk;
        if (k < kend && c0 + n < j1) vb = B[(long long)(c0 + n) * ldb + k];
      }
      ra[r] = va;
      rb[r] = vb;
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + NT * r;
      if (GRAM)
        As[e % TK][e / TK] = ra[r];
      else
        As[e / TM][e % TM] = ra[r];
      Bs[e % TK][e / TK] = rb[r];
    }
  };

  fetch(kbeg);
  for (long long k0 = kbeg; k0 < kend; k0 += TK) {
    __syncthreads();
    stash();
    __syncthreads();
    if (k0 + TK < kend) fetch(k0 + TK);
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      E a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) Ops<E>::fma(acc[i][j], a[i], b[j]);
    }
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + tx + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + ty + 16 * j;
      if (c >= j1) continue;
      if (GRAM) {
        C[blockIdx.z * pstride + (long long)(c - j0) * ldc + r] = acc[i][j];
      } else {
        const E bsh = shift != 0.f ? B[(long long)c * ldb + r] : Ops<E>::zero();
        E* cp = C + (long long)c * ldc + r;
        const bool use_beta = beta != 0.f;
        *cp = Ops<E>::axpby(acc[i][j], bsh, use_beta ? *cp : Ops<E>::zero(), alpha, beta, shift,
                            use_beta);
      }
    }
  }
}

template <class E>
__global__ void f32_sum_partials_kernel(const E* __restrict__ P, int p, int q, int nsplit,
                                        long long pstride, E* __restrict__ C, long long ldc,
                                        int lower) {
  const long long n = (long long)p * q;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % p, c = e / p;
    if (lower && r < c) continue;
    E s = P[e];
    for (int z = 1; z < nsplit; ++z) {
      const E v = P[z * pstride + e];
      if constexpr (sizeof(E) == 8) {
        reinterpret_cast<float2&>(s).x += reinterpret_cast<const float2&>(v).x;
        reinterpret_cast<float2&>(s).y += reinterpret_cast<const float2&>(v).y;
      } else {
        reinterpret_cast<float&>(s) += reinterpret_cast<const float&>(v);
      }
    }
    C[c * ldc + r] = s;
  }
}

template <class T>
using elem = typename std::conditional<std::is_same<T, chase_c32>::value, float2, float>::type;

template <class T>
int gemm_impl(Dev& d, int64_t M, int64_t K, const T* A, int64_t lda, const T* B, int64_t ldb,
              T* Cm, int64_t ldc, int j0, int j1, double alpha, double beta, double shift) {
  if (j1 <= j0 || M == 0) return CHASE_OK;
  if (K == 0) {
    set_error("single-precision gemm: K == 0 is not supported");
    return CHASE_INVALID_ARG;
  }
  if (shift != 0.0 && M != K) {
    set_error("single-precision gemm: the shifted product needs a square A");
    return CHASE_INVALID_ARG;
  }
  if (j1 - j0 <= kFewColMax)
    return fewcol_gemm(d, M, K, A, lda, B, ldb, Cm, ldc, j0, j1, alpha, beta, shift);
  using E = elem<T>;
  dim3 grid(static_cast<unsigned>((M + TM - 1) / TM), static_cast<unsigned>((j1 - j0 + TN - 1) / TN));
  f32_gemm_kernel<E, false><<<grid, NT, 0, d.st>>>(
      reinterpret_cast<const E*>(A), lda, reinterpret_cast<const E*>(B), ldb,
      reinterpret_cast<E*>(Cm), ldc, static_cast<int>(M), K, j0, j1, static_cast<float>(alpha),
      static_cast<float>(beta), static_cast<float>(shift), 0, 0, 0);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class T>
int gram_impl(Dev& d, int64_t N, const T* X, int64_t ldx, int p, const T* Y, int64_t ldy, int q,
              T* Cm, int64_t ldc, bool lower) {
  if (p == 0 || q == 0) return CHASE_OK;
  using E = elem<T>;
  const int tp = (p + TM - 1) / TM, tq = (q + TN - 1) / TN;
  long long ns = std::max<long long>(1, (4 * 152) / std::max(1, tp * tq));
  ns = std::min<long long>(ns, std::max<long long>(1, N / 256));
  long long kc = (N + ns - 1) / ns;
  kc = (kc + TK - 1) / TK * TK;
  ns = (N + kc - 1) / kc;
  const long long pstride = static_cast<long long>(p) * q;
  E* P = nullptr;
  CHASE_TRY(d.alloc(&P, static_cast<size_t>(pstride * ns)));
  dim3 grid(static_cast<unsigned>(tp), static_cast<unsigned>(tq), static_cast<unsigned>(ns));
  f32_gemm_kernel<E, true><<<grid, NT, 0, d.st>>>(
      reinterpret_cast<const E*>(X), ldx, reinterpret_cast<const E*>(Y), ldy, P, p, p, N, 0, q,
      1.f, 0.f, 0.f, kc, pstride, lower ? 1 : 0);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  const unsigned blocks = static_cast<unsigned>(std::min<long long>((pstride + 255) / 256, 4096));
  f32_sum_partials_kernel<E><<<blocks, 256, 0, d.st>>>(P, p, q, static_cast<int>(ns), pstride,
                                                       reinterpret_cast<E*>(Cm), ldc,
                                                       lower ? 1 : 0);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

}  // namespace

int cgemm(Dev& d, int64_t M, int64_t K, const chase_c32* A, int64_t lda, const chase_c32* B,
          int64_t ldb, int64_t, chase_c32* C, int64_t ldc, int j0, int j1, double alpha,
          double beta, double shift) {
  return gemm_impl(d, M, K, A, lda, B, ldb, C, ldc, j0, j1, alpha, beta, shift);
}

int sgemm(Dev& d, int64_t M, int64_t K, const float* A, int64_t lda, const float* B, int64_t ldb,
          int64_t, float* C, int64_t ldc, int j0, int j1, double alpha, double beta,
          double shift) {
  return gemm_impl(d, M, K, A, lda, B, ldb, C, ldc, j0, j1, alpha, beta, shift);
}

int cgram(Dev& d, int64_t N, const chase_c32* X, int64_t ldx, int p, const chase_c32* Y,
          int64_t ldy, int q, chase_c32* C, int64_t ldc, bool lower) {
  return gram_impl(d, N, X, ldx, p, Y, ldy, q, C, ldc, lower);
}

int sgram(Dev& d, int64_t N, const float* X, int64_t ldx, int p, const float* Y, int64_t ldy,
          int q, float* C, int64_t ldc, bool lower) {
  return gram_impl(d, N, X, ldx, p, Y, ldy, q, C, ldc, lower);
}

}  // namespace chase
