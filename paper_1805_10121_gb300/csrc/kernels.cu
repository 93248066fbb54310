// Supporting kernels of the ChASE iteration on sm_103a: Gram products for
// the orthogonalisation and the Rayleigh quotient, the degree plan of the
// filter, column permutations, norms, residuals, the blocked Cholesky and
// triangular solve of Cholesky QR, and the Lanczos three-term step.  The
// element kernels are templates over the scalar: complex128 (double2) for
// Hermitian problems, double for real symmetric ones (Sec. 5.1: the library
// is templated on the field as well as the precision).
#include <cusolverDn.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "common.cuh"
#include "context.hpp"

namespace chase {

namespace {

constexpr int kRed = 256;  // threads of the reduction kernels

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; result valid in every thread.
__device__ double block_sum(double v, double* scratch /* >= 33 doubles */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double s = 0.0;
  if (warp == 0) {
    s = lane < nw ? scratch[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) scratch[32] = s;
  }
  __syncthreads();
  return scratch[32];
}


// Scalar arithmetic of the element kernels: complex128 or real double.
template <class T>
struct Sc;
template <>
struct Sc<double2> {
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ double2 real(double r) { return make_double2(r, 0.0); }
  static __device__ __forceinline__ double re(double2 a) { return a.x; }
  static __device__ __forceinline__ double abs2(double2 a) { return a.x * a.x + a.y * a.y; }
  static __device__ __forceinline__ double2 scale(double2 a, double f) {
    return make_double2(a.x * f, a.y * f);
  }
  static __device__ __forceinline__ double2 conj(double2 a) { return make_double2(a.x, -a.y); }
  // acc - a conj(b)
  static __device__ __forceinline__ double2 sub_mul_conj(double2 acc, double2 a, double2 b) {
    acc.x -= a.x * b.x + a.y * b.y;
    acc.y -= a.y * b.x - a.x * b.y;
    return acc;
  }
  // Re(conj(a) b)
  static __device__ __forceinline__ double re_dot(double2 a, double2 b) {
    return a.x * b.x + a.y * b.y;
  }
  // a - f b
  static __device__ __forceinline__ double2 sub_scaled(double2 a, double f, double2 b) {
    return make_double2(a.x - f * b.x, a.y - f * b.y);
  }
  static __device__ __forceinline__ void add_re(double2& a, double v) { a.x += v; }
  static __device__ __forceinline__ double2 add(double2 a, double2 b) {
    return make_double2(a.x + b.x, a.y + b.y);
  }
  // (a, b) <- ((a + conj(b)) / 2, conj of that): entries (r, c) and (c, r)
  static __device__ __forceinline__ void hermitize_diag(double2& a) { a.y = 0.0; }
};
template <>
struct Sc<double> {
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double real(double r) { return r; }
  static __device__ __forceinline__ double re(double a) { return a; }
  static __device__ __forceinline__ double abs2(double a) { return a * a; }
  static __device__ __forceinline__ double scale(double a, double f) { return a * f; }
  static __device__ __forceinline__ double conj(double a) { return a; }
  static __device__ __forceinline__ double sub_mul_conj(double acc, double a, double b) {
    return acc - a * b;
  }
  static __device__ __forceinline__ double re_dot(double a, double b) { return a * b; }
  static __device__ __forceinline__ double sub_scaled(double a, double f, double b) {
    return a - f * b;
  }
  static __device__ __forceinline__ void add_re(double& a, double v) { a += v; }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ void hermitize_diag(double&) {}
};

// Single precision: values in FP32, norms and dot products accumulated in
// double by the reductions that call abs2 / re_dot.
template <>
struct Sc<float2> {
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ float2 real(double r) { return make_float2((float)r, 0.f); }
  static __device__ __forceinline__ double re(float2 a) { return a.x; }
  static __device__ __forceinline__ double abs2(float2 a) {
    return (double)a.x * a.x + (double)a.y * a.y;
  }
  static __device__ __forceinline__ float2 scale(float2 a, double f) {
    return make_float2((float)(a.x * f), (float)(a.y * f));
  }
  static __device__ __forceinline__ float2 conj(float2 a) { return make_float2(a.x, -a.y); }
  static __device__ __forceinline__ float2 sub_mul_conj(float2 acc, float2 a, float2 b) {
    acc.x -= a.x * b.x + a.y * b.y;
    acc.y -= a.y * b.x - a.x * b.y;
    return acc;
  }
  static __device__ __forceinline__ double re_dot(float2 a, float2 b) {
    return (double)a.x * b.x + (double)a.y * b.y;
  }
  static __device__ __forceinline__ float2 sub_scaled(float2 a, double f, float2 b) {
    return make_float2((float)(a.x - f * b.x), (float)(a.y - f * b.y));
  }
  static __device__ __forceinline__ void add_re(float2& a, double v) { a.x = (float)(a.x + v); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) {
    return make_float2(a.x + b.x, a.y + b.y);
  }
  static __device__ __forceinline__ void hermitize_diag(float2& a) { a.y = 0.f; }
};
template <>
struct Sc<float> {
  static __device__ __forceinline__ float zero() { return 0.f; }
  static __device__ __forceinline__ float real(double r) { return (float)r; }
  static __device__ __forceinline__ double re(float a) { return a; }
  static __device__ __forceinline__ double abs2(float a) { return (double)a * a; }
  static __device__ __forceinline__ float scale(float a, double f) { return (float)(a * f); }
  static __device__ __forceinline__ float conj(float a) { return a; }
  static __device__ __forceinline__ float sub_mul_conj(float acc, float a, float b) {
    return acc - a * b;
  }
  static __device__ __forceinline__ double re_dot(float a, float b) { return (double)a * b; }
  static __device__ __forceinline__ float sub_scaled(float a, double f, float b) {
    return (float)(a - f * b);
  }
  static __device__ __forceinline__ void add_re(float& a, double v) { a = (float)(a + v); }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
  static __device__ __forceinline__ void hermitize_diag(float&) {}
};

// Device element type of a host scalar type.
template <class T>
struct Dv;
template <>
struct Dv<chase_c32> {
  using type = float2;
};
template <>
struct Dv<float> {
  using type = float;
};
template <>
struct Dv<chase_c64> {
  using type = double2;
};
template <>
struct Dv<double> {
  using type = double;
};
template <class T>
using elem_t = typename Dv<T>::type;
template <class T>
elem_t<T>* dp(T* p) {
  return reinterpret_cast<elem_t<T>*>(p);
}
template <class T>
const elem_t<T>* dp(const T* p) {
  return reinterpret_cast<const elem_t<T>*>(p);
}

// ---------------------------------------------------------------------------
// Gram product C = X^H Y on the FP64 tensor pipe, split over K
// ---------------------------------------------------------------------------
constexpr int GT = 32;  // output tile (p and q)
constexpr int GK = 16;  // K per shared-memory tile

__global__ void __launch_bounds__(128)
    gram_kernel(const double2* __restrict__ X, long long ldx, int p, const double2* __restrict__ Y,
                long long ldy, int q, long long N, long long kchunk, double2* __restrict__ P,
                long long ldp, long long pstride, int lower) {
  // lower: only entries r >= c are wanted; tiles strictly above the diagonal exit
  if (lower && blockIdx.x < blockIdx.y) return;
  __shared__ double2 sX[GT][GK];
  __shared__ double2 sY[GT][GK];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wm = warp & 1, wn = warp >> 1;  // 2 x 2 warps, 16 x 16 each
  const int p0 = blockIdx.x * GT, q0 = blockIdx.y * GT;
  const long long kbeg = blockIdx.z * kchunk;
  const long long kend = min(N, kbeg + kchunk);

  // conj(x) y with three real products: T1 = xr yr, T2 = xi yi,
  // T3 = (xr - xi)(yr + yi); re = T1 + T2, im = T3 - T1 + T2
  double t1[2][2][2] = {}, t2[2][2][2] = {}, t3[2][2][2] = {};
  for (long long k0 = kbeg; k0 < kend; k0 += GK) {
    // load: 32 columns x 16 rows of X and of Y (column-contiguous in k)
    for (int e = threadIdx.x; e < GT * GK; e += 128) {
      const int col = e / GK, kk = e % GK;
      const long long k = k0 + kk;
      double2 xv = make_double2(0.0, 0.0), yv = make_double2(0.0, 0.0);
      if (k < kend) {
        if (p0 + col < p) xv = X[(long long)(p0 + col) * ldx + k];
        if (q0 + col < q) yv = Y[(long long)(q0 + col) * ldy + k];
      }
      sX[col][kk] = xv;
      sY[col][kk] = yv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; kk += 4) {
      double2 a[2], b[2];
      double ad[2], bsum[2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        a[mi] = sX[wm * 16 + mi * 8 + g][kk + t];
        ad[mi] = a[mi].x - a[mi].y;
      }
#pragma unroll
      for (int ni = 0; ni < 2; ++ni) {
        b[ni] = sY[wn * 16 + ni * 8 + g][kk + t];
        bsum[ni] = b[ni].x + b[ni].y;
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) {
          dmma_8x8x4(t1[mi][ni][0], t1[mi][ni][1], a[mi].x, b[ni].x);
          dmma_8x8x4(t2[mi][ni][0], t2[mi][ni][1], a[mi].y, b[ni].y);
          dmma_8x8x4(t3[mi][ni][0], t3[mi][ni][1], ad[mi], bsum[ni]);
        }
    }
    __syncthreads();
  }
  double2* Pz = P + blockIdx.z * pstride;
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = p0 + wm * 16 + mi * 8 + g;
        const int c = q0 + wn * 16 + ni * 8 + 2 * t + h;
        if (r < p && c < q)
          Pz[(long long)c * ldp + r] =
              make_double2(t1[mi][ni][h] + t2[mi][ni][h], t3[mi][ni][h] - t1[mi][ni][h] + t2[mi][ni][h]);
      }
}

// Real Gram product C = X^T Y: one DMMA per fragment.
__global__ void __launch_bounds__(128)
    gram_real_kernel(const double* __restrict__ X, long long ldx, int p, const double* __restrict__ Y,
                     long long ldy, int q, long long N, long long kchunk, double* __restrict__ P,
                     long long ldp, long long pstride, int lower) {
  if (lower && blockIdx.x < blockIdx.y) return;
  __shared__ double sX[GT][GK + 1];
  __shared__ double sY[GT][GK + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wm = warp & 1, wn = warp >> 1;  // 2 x 2 warps, 16 x 16 each
  const int p0 = blockIdx.x * GT, q0 = blockIdx.y * GT;
  const long long kbeg = blockIdx.z * kchunk;
  const long long kend = min(N, kbeg + kchunk);
  double acc[2][2][2] = {};
  for (long long k0 = kbeg; k0 < kend; k0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += 128) {
      const int col = e / GK, kk = e % GK;
      const long long k = k0 + kk;
      double xv = 0.0, yv = 0.0;
      if (k < kend) {
        if (p0 + col < p) xv = X[(long long)(p0 + col) * ldx + k];
        if (q0 + col < q) yv = Y[(long long)(q0 + col) * ldy + k];
      }
      sX[col][kk] = xv;
      sY[col][kk] = yv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; kk += 4) {
      double a[2], b[2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) a[mi] = sX[wm * 16 + mi * 8 + g][kk + t];
#pragma unroll
      for (int ni = 0; ni < 2; ++ni) b[ni] = sY[wn * 16 + ni * 8 + g][kk + t];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) dmma_8x8x4(acc[mi][ni][0], acc[mi][ni][1], a[mi], b[ni]);
    }
    __syncthreads();
  }
  double* Pz = P + blockIdx.z * pstride;
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = p0 + wm * 16 + mi * 8 + g;
        const int c = q0 + wn * 16 + ni * 8 + 2 * t + h;
        if (r < p && c < q) Pz[(long long)c * ldp + r] = acc[mi][ni][h];
      }
}

template <class T>
__global__ void sum_partials_kernel(const T* __restrict__ P, int p, int q, int nsplit,
                                    long long pstride, T* __restrict__ C, long long ldc,
                                    int lower) {
  const long long n = (long long)p * q;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % p, c = e / p;
    if (lower && r < c) continue;
    T acc = Sc<T>::zero();
    for (int z = 0; z < nsplit; ++z) acc = Sc<T>::add(acc, P[z * pstride + e]);
    C[c * ldc + r] = acc;
  }
}

// ---------------------------------------------------------------------------
// Degree plan: stable counting sort by degree with warp match / popc scans
// ---------------------------------------------------------------------------
constexpr int kMaxDeg = 1024;

__global__ void filter_plan_kernel(const int* __restrict__ deg, int b, int max_allowed,
                                   int* __restrict__ perm, int* __restrict__ start,
                                   int* __restrict__ info, int* __restrict__ err) {
  __shared__ int off[kMaxDeg + 2];
  const int lane = threadIdx.x;  // one warp
  for (int i = lane; i < max_allowed + 2; i += 32) off[i] = 0;
  __syncwarp();
  int mx = 0;
  for (int j = lane; j < b; j += 32) {
    int m = deg[j];
    if (m < 2 || m > max_allowed || (m & 1)) {
      atomicOr(err, KERR_BAD_DEGREE);
      m = 2;
    }
    atomicAdd(&off[m], 1);
    mx = max(mx, m);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __syncwarp();
  // exclusive scan of the histogram, 32 degree values per round
  int carry = 0;
  for (int base = 0; base < max_allowed + 2; base += 32) {
    const int i = base + lane;
    const int v = i < max_allowed + 2 ? off[i] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (i < max_allowed + 2) {
      off[i] = carry + incl - v;
      start[i] = carry + incl - v;  // columns with degree < i
    }
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  __syncwarp();
  if (lane == 0) info[0] = mx;
  // stable placement: ranks among equal degrees inside each 32-column chunk
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int base = 0; base < b; base += 32) {
    const int j = base + lane;
    int m = -1;
    if (j < b) {
      m = deg[j];
      if (m < 2 || m > max_allowed || (m & 1)) m = 2;
    }
    const unsigned grp = __match_any_sync(0xffffffffu, m);
    const int rank = __popc(grp & lt_mask);
    if (j < b) perm[off[m] + rank] = j;
    __syncwarp();
    if (j < b && rank == 0) off[m] += __popc(grp);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Column permutations, norms, scaling, residuals
// ---------------------------------------------------------------------------
template <class T>
__global__ void permute_cols_kernel(const T* __restrict__ X, long long ldx, T* __restrict__ Y,
                                    long long ldy, long long N, const int* __restrict__ perm,
                                    int scatter) {
  const int j = blockIdx.y;
  const int src = scatter ? j : perm[j];
  const int dst = scatter ? perm[j] : j;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    Y[(long long)dst * ldy + i] = X[(long long)src * ldx + i];
}

// One column of one problem per CTA: problem by binary search over col0.
__global__ void grouped_permute_kernel(const GroupedPermute* __restrict__ probs, int P, int scatter) {
  const int g = blockIdx.x;
  int lo = 0, hi = P;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (probs[mid].col0 <= g) lo = mid; else hi = mid;
  }
  const GroupedPermute& pr = probs[lo];
  const int j = g - pr.col0;
  const int src = scatter ? j : pr.perm[j];
  const int dst = scatter ? pr.perm[j] : j;
  const double2* x = pr.src + static_cast<long long>(src) * pr.lds;
  double2* y = pr.dst + static_cast<long long>(dst) * pr.ldd;
  for (int i = threadIdx.x; i < pr.n; i += blockDim.x) y[i] = x[i];
}

template <class T>
__global__ void __launch_bounds__(kRed) col_norms_kernel(const T* __restrict__ X, long long ldx,
                                                         long long N, double* __restrict__ out) {
  __shared__ double scratch[33];
  const T* x = X + (long long)blockIdx.x * ldx;
  double s = 0.0;
  for (long long i = threadIdx.x; i < N; i += blockDim.x) s += Sc<T>::abs2(x[i]);
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) out[blockIdx.x] = sqrt(s);
}

template <class T>
__global__ void col_inv_scale_kernel(T* __restrict__ X, long long ldx, long long N,
                                     const double* __restrict__ s) {
  const int j = blockIdx.y;
  const double sj = s[j];
  if (sj == 0.0) return;
  const double f = 1.0 / sj;
  T* x = X + (long long)j * ldx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = Sc<T>::scale(x[i], f);
}

template <class T>
__global__ void __launch_bounds__(kRed)
    resid_norms_kernel(const T* __restrict__ HV, long long ldhv, const T* __restrict__ V,
                       long long ldv, long long N, const double* __restrict__ lam,
                       double* __restrict__ res) {
  __shared__ double scratch[33];
  const int j = blockIdx.x;
  const double l = lam[j];
  const T* hv = HV + (long long)j * ldhv;
  const T* v = V + (long long)j * ldv;
  double s = 0.0;
  for (long long i = threadIdx.x; i < N; i += blockDim.x)
    s += Sc<T>::abs2(Sc<T>::sub_scaled(hv[i], l, v[i]));
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) res[j] = sqrt(s);
}

template <class T>
__global__ void fill_upper_hermitian_kernel(T* __restrict__ G, long long ldg, int p) {
  const long long n = (long long)p * p;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % p), c = (int)(e / p);
    if (r > c) continue;  // the lower triangle is only read
    T* a = G + (long long)c * ldg + r;  // (r, c), upper
    if (r == c)
      Sc<T>::hermitize_diag(*a);
    else
      *a = Sc<T>::conj(G[(long long)r * ldg + c]);  // conj of (c, r)
  }
}

// F = the Hermitian matrix whose lower triangle (diagonal included) is L's:
// F[r, c] = L[r, c] for r >= c, conj(L[c, r]) above; the diagonal is real.
template <class T>
__global__ void hermitian_from_lower_kernel(const T* __restrict__ L, long long ldl,
                                            T* __restrict__ F, long long ldf, long long n) {
  const long long total = n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % n, c = e / n;
    T v = r >= c ? L[c * ldl + r] : Sc<T>::conj(L[r * ldl + c]);
    if (r == c) Sc<T>::hermitize_diag(v);
    F[c * ldf + r] = v;
  }
}

template <class T>
__global__ void zero_triangle_kernel(T* __restrict__ A, long long lda, int p, int lower) {
  const long long n = (long long)p * p;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % p), c = (int)(e / p);
    if (lower ? (r > c) : (r < c)) A[(long long)c * lda + r] = Sc<T>::zero();
  }
}

// ---------------------------------------------------------------------------
// Cholesky (left-looking, one CTA) and triangular inverse
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(1024)
    cholesky_kernel(T* __restrict__ G, long long ld, int p, double rel_tol, double shift,
                    const double* __restrict__ diag_ref, int* __restrict__ err) {
  __shared__ double scratch[33];
  __shared__ double s_ljj;
  __shared__ int s_fail;
  if (threadIdx.x == 0) s_fail = 0;
  if (shift != 0.0)
    for (int j = threadIdx.x; j < p; j += blockDim.x) Sc<T>::add_re(G[(long long)j * ld + j], shift);
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    // pivot: d = G_jj - sum_k |L_jk|^2
    double part = 0.0;
    for (int k = threadIdx.x; k < j; k += blockDim.x) part += Sc<T>::abs2(G[(long long)k * ld + j]);
    part = block_sum(part, scratch);
    if (threadIdx.x == 0) {
      const double gjj = Sc<T>::re(G[(long long)j * ld + j]);
      const double dj = gjj - part;
      const double ref = diag_ref ? diag_ref[j] : gjj;
      const bool bad = !(dj > rel_tol * fabs(ref)) || !isfinite(dj);
      if (bad) {
        s_fail = 1;
        atomicOr(err, KERR_CHOL_BREAKDOWN);
      }
      s_ljj = bad ? 1.0 : sqrt(dj);
      G[(long long)j * ld + j] = Sc<T>::real(s_ljj);
    }
    __syncthreads();
    if (s_fail) return;
    const double inv = 1.0 / s_ljj;
    for (int i = j + 1 + threadIdx.x; i < p; i += blockDim.x) {
      T acc = G[(long long)j * ld + i];
      for (int k = 0; k < j; ++k)  // acc -= L_ik conj(L_jk)
        acc = Sc<T>::sub_mul_conj(acc, G[(long long)k * ld + i], G[(long long)k * ld + j]);
      G[(long long)j * ld + i] = Sc<T>::scale(acc, inv);
    }
    __syncthreads();
  }
}

// Rows of X (nrows x kb, leading dimension ldx) are replaced by the solution y
// of y L^H = x, with L the kb x kb lower factor at (Lp, ldl): thread per row,
// y_j = (x_j - sum_{m<j} y_m conj(L_jm)) / L_jj.  kb <= 32.
template <class T>
__global__ void __launch_bounds__(128)
    row_trsm_lh_kernel(T* __restrict__ X, long long ldx, long long nrows, const T* __restrict__ Lp,
                       long long ldl, int kb) {
  __shared__ T sL[32][33];
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    const int r = e % kb, c = e / kb;
    sL[r][c] = r >= c ? Lp[(long long)c * ldl + r] : Sc<T>::zero();
  }
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nrows;
       i += (long long)gridDim.x * blockDim.x) {
    T y[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j >= kb) break;
      T a = X[(long long)j * ldx + i];
      for (int m = 0; m < j; ++m) a = Sc<T>::sub_mul_conj(a, y[m], sL[j][m]);
      y[j] = Sc<T>::scale(a, 1.0 / Sc<T>::re(sL[j][j]));
      X[(long long)j * ldx + i] = y[j];
    }
  }
}

// dst (cols x rows, leading dimension ldd) = conj(src)^T, src rows x cols (lds)
template <class T>
__global__ void conj_transpose_kernel(const T* __restrict__ src, long long lds, int rows, int cols,
                                      T* __restrict__ dst, long long ldd) {
  const long long n = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % rows), c = (int)(e / rows);
    dst[(long long)r * ldd + c] = Sc<T>::conj(src[(long long)c * lds + r]);
  }
}

template <class T>
__global__ void copy_diag_kernel(const T* __restrict__ G, long long ld, int p,
                                 double* __restrict__ out, double shift) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p; j += gridDim.x * blockDim.x)
    out[j] = Sc<T>::re(G[(long long)j * ld + j]) + shift;
}

template <class T>
__global__ void add_diag_kernel(T* __restrict__ G, long long ld, int p, double shift) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p; j += gridDim.x * blockDim.x)
    Sc<T>::add_re(G[(long long)j * ld + j], shift);
}

// ---------------------------------------------------------------------------
// Lanczos
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kRed)
    lanczos_step_kernel(long long N, long long ld, int r, int step, const T* __restrict__ Vj,
                        const T* __restrict__ Vprev, T* __restrict__ W, T* __restrict__ Vnext,
                        double* __restrict__ alpha, double* __restrict__ beta, double tiny) {
  __shared__ double scratch[33];
  const int c = blockIdx.x;
  const T* v = Vj + (long long)c * ld;
  T* w = W + (long long)c * ld;
  // alpha = Re(v^H w)
  double s = 0.0;
  for (long long i = threadIdx.x; i < N; i += blockDim.x) s += Sc<T>::re_dot(v[i], w[i]);
  const double al = block_sum(s, scratch);
  const double bprev = step > 0 ? beta[(step - 1) * r + c] : 0.0;
  const T* vp = step > 0 ? Vprev + (long long)c * ld : nullptr;
  double nrm = 0.0;
  for (long long i = threadIdx.x; i < N; i += blockDim.x) {
    T b = Sc<T>::sub_scaled(w[i], al, v[i]);
    if (vp) b = Sc<T>::sub_scaled(b, bprev, vp[i]);
    w[i] = b;
    nrm += Sc<T>::abs2(b);
  }
  const double be = sqrt(block_sum(nrm, scratch));
  // beta is rounding noise once the Krylov space is invariant: stop the run
  double scale = fabs(al);
  for (int k = 0; k < step; ++k) scale = fmax(scale, fmax(fabs(alpha[k * r + c]), beta[k * r + c]));
  const bool stop = !(be > tiny * fmax(scale, be));
  if (threadIdx.x == 0) {
    alpha[step * r + c] = al;
    beta[step * r + c] = be;
  }
  if (Vnext) {
    T* vn = Vnext + (long long)c * ld;
    const double f = stop ? 0.0 : 1.0 / be;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) vn[i] = Sc<T>::scale(w[i], f);
  }
}

template <class T>
__global__ void __launch_bounds__(kRed) normalize_cols_kernel(T* __restrict__ X, long long ldx,
                                                              long long N) {
  __shared__ double scratch[33];
  T* x = X + (long long)blockIdx.x * ldx;
  double s = 0.0;
  for (long long i = threadIdx.x; i < N; i += blockDim.x) s += Sc<T>::abs2(x[i]);
  s = block_sum(s, scratch);
  const double f = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  for (long long i = threadIdx.x; i < N; i += blockDim.x) x[i] = Sc<T>::scale(x[i], f);
}

unsigned grid_for(long long n, int threads, unsigned cap = 65535u) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return static_cast<unsigned>(std::min<long long>(g, cap));
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
namespace {
// Gram launch shape: split K so that the grid covers the 152 SMs about four times.
void gram_shape(int64_t N, int p, int q, bool lower, dim3* grid, long long* kchunk,
                long long* nsplit) {
  const int tp = (p + GT - 1) / GT, tq = (q + GT - 1) / GT;
  // tiles that do work: all, or those on and below the diagonal
  const long long tiles = lower ? static_cast<long long>(std::min(tp, tq)) * (std::min(tp, tq) + 1) / 2 +
                                      static_cast<long long>(std::max(0, tp - tq)) * tq
                                : static_cast<long long>(tp) * tq;
  long long ns = std::max<long long>(1, (4 * 152) / std::max<long long>(1, tiles));
  ns = std::min<long long>(ns, std::max<long long>(1, N / 256));
  long long kc = (N + ns - 1) / ns;
  kc = ((kc + GK - 1) / GK) * GK;
  ns = (N + kc - 1) / kc;
  if (ns < 1) ns = 1;
  *grid = dim3(tp, tq, static_cast<unsigned>(ns));
  *kchunk = kc;
  *nsplit = ns;
}

template <class T>
int gram_impl(Dev& d, int64_t N, const T* X, int64_t ldx, int p, const T* Y, int64_t ldy, int q,
              T* C, int64_t ldc, bool lower) {
  if (p == 0 || q == 0) return CHASE_OK;
  using D = elem_t<T>;
  dim3 grid;
  long long kchunk = 0, nsplit = 1;
  gram_shape(N, p, q, lower, &grid, &kchunk, &nsplit);
  D* out = dp(C);
  long long ldo = ldc, pstride = 0;
  D* P = nullptr;
  if (nsplit > 1) {
    pstride = (long long)p * q;
    CHASE_TRY(d.alloc(&P, static_cast<size_t>(pstride * nsplit)));
    out = P;
    ldo = p;
  }
  if constexpr (sizeof(D) == 16)
    gram_kernel<<<grid, 128, 0, d.st>>>(dp(X), ldx, p, dp(Y), ldy, q, N, kchunk, out, ldo, pstride,
                                        lower ? 1 : 0);
  else
    gram_real_kernel<<<grid, 128, 0, d.st>>>(dp(X), ldx, p, dp(Y), ldy, q, N, kchunk, out, ldo,
                                             pstride, lower ? 1 : 0);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  if (nsplit > 1) {
    sum_partials_kernel<D><<<grid_for(pstride, 256, 4096), 256, 0, d.st>>>(
        P, p, q, static_cast<int>(nsplit), pstride, dp(C), ldc, lower ? 1 : 0);
    note_launch();
    CHASE_CUDA(cudaGetLastError());
  }
  return CHASE_OK;
}
}  // namespace

int zgram(Dev& d, int64_t N, const chase_c64* X, int64_t ldx, int p, const chase_c64* Y,
          int64_t ldy, int q, chase_c64* C, int64_t ldc, bool lower) {
  return gram_impl(d, N, X, ldx, p, Y, ldy, q, C, ldc, lower);
}

int dgram(Dev& d, int64_t N, const double* X, int64_t ldx, int p, const double* Y, int64_t ldy,
          int q, double* C, int64_t ldc, bool lower) {
  return gram_impl(d, N, X, ldx, p, Y, ldy, q, C, ldc, lower);
}

int launch_filter_plan(Dev& d, const int* deg, int b, int max_allowed, int* perm, int* start,
                       int* info) {
  if (max_allowed > kMaxDeg) max_allowed = kMaxDeg;
  filter_plan_kernel<<<1, 32, 0, d.st>>>(deg, b, max_allowed, perm, start, info, d.err);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

int launch_grouped_permute(Dev& d, const GroupedPermute* probs, int P, int total_cols, bool scatter) {
  if (total_cols <= 0) return CHASE_OK;
  grouped_permute_kernel<<<static_cast<unsigned>(total_cols), 256, 0, d.st>>>(probs, P,
                                                                               scatter ? 1 : 0);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class T>
int launch_permute_cols(Dev& d, const T* X, int64_t ldx, T* Y, int64_t ldy, int64_t N, int b,
                        const int* perm, bool scatter) {
  if (b == 0 || N == 0) return CHASE_OK;
  if (b > 65535) {
    set_error("permute: too many columns");
    return CHASE_INVALID_ARG;
  }
  dim3 grid(grid_for(N, 256, 64), b);
  permute_cols_kernel<<<grid, 256, 0, d.st>>>(dp(X), ldx, dp(Y), ldy, N, perm, scatter ? 1 : 0);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class T>
int launch_col_norms(Dev& d, const T* X, int64_t ldx, int64_t N, int b, double* out) {
  if (b == 0) return CHASE_OK;
  col_norms_kernel<<<b, kRed, 0, d.st>>>(dp(X), ldx, N, out);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class T>
int launch_col_inv_scale(Dev& d, T* X, int64_t ldx, int64_t N, int b, const double* s) {
  if (b == 0 || N == 0) return CHASE_OK;
  if (b > 65535) {
    set_error("column scaling: too many columns");
    return CHASE_INVALID_ARG;
  }
  dim3 grid(grid_for(N, 256, 64), b);
  col_inv_scale_kernel<<<grid, 256, 0, d.st>>>(dp(X), ldx, N, s);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class T>
int launch_resid_norms(Dev& d, const T* HV, int64_t ldhv, const T* V, int64_t ldv, int64_t N, int b,
                       const double* lam, double* res) {
  if (b == 0) return CHASE_OK;
  resid_norms_kernel<<<b, kRed, 0, d.st>>>(dp(HV), ldhv, dp(V), ldv, N, lam, res);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class T>
int launch_fill_upper_hermitian(Dev& d, T* G, int64_t ldg, int p) {
  if (p == 0) return CHASE_OK;
  fill_upper_hermitian_kernel<<<grid_for((long long)p * p, 256, 4096), 256, 0, d.st>>>(dp(G), ldg,
                                                                                       p);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

namespace {
template <class S, class D>
__global__ void convert_kernel(const S* __restrict__ src, long long lds, D* __restrict__ dst,
                               long long ldd, long long rows, long long cols) {
  const long long total = rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % rows, c = e / rows;
    const S v = src[c * lds + r];
    D o;
    o.x = v.x;
    o.y = v.y;
    dst[c * ldd + r] = o;
  }
}
template <class S, class D>
__global__ void convert_real_kernel(const S* __restrict__ src, long long lds, D* __restrict__ dst,
                                    long long ldd, long long rows, long long cols) {
  const long long total = rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % rows, c = e / rows;
    dst[c * ldd + r] = static_cast<D>(src[c * lds + r]);
  }
}
}  // namespace

int launch_convert(Dev& d, const chase_c32* src, int64_t lds, chase_c64* dst, int64_t ldd,
                   int64_t rows, int64_t cols) {
  if (rows * cols == 0) return CHASE_OK;
  convert_kernel<<<grid_for(rows * cols, 256, 152 * 16), 256, 0, d.st>>>(dp(src), lds, dp(dst), ldd,
                                                                         rows, cols);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}
int launch_convert(Dev& d, const chase_c64* src, int64_t lds, chase_c32* dst, int64_t ldd,
                   int64_t rows, int64_t cols) {
  if (rows * cols == 0) return CHASE_OK;
  convert_kernel<<<grid_for(rows * cols, 256, 152 * 16), 256, 0, d.st>>>(dp(src), lds, dp(dst), ldd,
                                                                         rows, cols);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}
int launch_convert(Dev& d, const float* src, int64_t lds, double* dst, int64_t ldd, int64_t rows,
                   int64_t cols) {
  if (rows * cols == 0) return CHASE_OK;
  convert_real_kernel<<<grid_for(rows * cols, 256, 152 * 16), 256, 0, d.st>>>(src, lds, dst, ldd,
                                                                              rows, cols);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}
int launch_convert(Dev& d, const double* src, int64_t lds, float* dst, int64_t ldd, int64_t rows,
                   int64_t cols) {
  if (rows * cols == 0) return CHASE_OK;
  convert_real_kernel<<<grid_for(rows * cols, 256, 152 * 16), 256, 0, d.st>>>(src, lds, dst, ldd,
                                                                              rows, cols);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class T>
int launch_hermitian_from_lower(Dev& d, const T* L, int64_t ldl, T* F, int64_t ldf, int64_t n) {
  if (n == 0) return CHASE_OK;
  hermitian_from_lower_kernel<<<grid_for(n * n, 256, 152 * 16), 256, 0, d.st>>>(dp(L), ldl, dp(F),
                                                                                 ldf, n);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class T>
int launch_zero_triangle(Dev& d, T* A, int64_t lda, int p, bool lower) {
  if (p == 0) return CHASE_OK;
  zero_triangle_kernel<<<grid_for((long long)p * p, 256, 4096), 256, 0, d.st>>>(dp(A), lda, p,
                                                                                 lower ? 1 : 0);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class T>
int launch_cholesky(Dev& d, T* G, int64_t ldg, int p, double rel_tol, double shift) {
  if (p == 0) return CHASE_OK;
  cholesky_kernel<<<1, 1024, 0, d.st>>>(dp(G), ldg, p, rel_tol, shift, nullptr, d.err);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

namespace {
template <class T>
int launch_row_trsm_lh(Dev& d, T* X, int64_t ldx, int64_t nrows, const T* L, int64_t ldl, int kb) {
  if (nrows <= 0 || kb <= 0) return CHASE_OK;
  if (kb > 32) {
    set_error("row_trsm: block wider than 32");
    return CHASE_INVALID_ARG;
  }
  row_trsm_lh_kernel<<<grid_for(nrows, 128, 152 * 8), 128, 0, d.st>>>(dp(X), ldx, nrows, dp(L),
                                                                       ldl, kb);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class T>
int launch_conj_transpose(Dev& d, const T* src, int64_t lds, int rows, int cols, T* dst,
                          int64_t ldd) {
  if (rows <= 0 || cols <= 0) return CHASE_OK;
  conj_transpose_kernel<<<grid_for((long long)rows * cols, 256, 4096), 256, 0, d.st>>>(
      dp(src), lds, rows, cols, dp(dst), ldd);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}
}  // namespace

// Blocked right-looking Cholesky G = L L^H (lower, in place), 32-wide panels:
// the diagonal block by the one-CTA kernel, the panel below it by row
// triangular solves, the trailing matrix by the FP64 tensor-pipe GEMM.  The
// pivot test compares against the diagonal of G + shift before any update.
template <class T>
int cholesky_blocked(Dev& d, T* G, int64_t ldg, int p, double rel_tol, double shift,
                     double* diag_ref, T* work /* >= 32 * p */) {
  if (p == 0) return CHASE_OK;
  constexpr int nb = 32;
  copy_diag_kernel<<<grid_for(p, 256, 64), 256, 0, d.st>>>(dp(G), ldg, p, diag_ref, shift);
  note_launch();
  if (shift != 0.0) {
    add_diag_kernel<<<grid_for(p, 256, 64), 256, 0, d.st>>>(dp(G), ldg, p, shift);
    note_launch();
  }
  CHASE_CUDA(cudaGetLastError());
  for (int k0 = 0; k0 < p; k0 += nb) {
    const int kb = std::min(nb, p - k0);
    T* Akk = G + static_cast<size_t>(k0) * ldg + k0;
    cholesky_kernel<<<1, 1024, 0, d.st>>>(dp(Akk), ldg, kb, rel_tol, 0.0, diag_ref + k0, d.err);
    note_launch();
    CHASE_CUDA(cudaGetLastError());
    const int m = p - k0 - kb;
    if (m <= 0) break;
    T* Pn = Akk + kb;  // panel rows k0+kb .. p-1, columns k0 .. k0+kb-1
    CHASE_TRY(launch_row_trsm_lh(d, Pn, ldg, m, Akk, ldg, kb));
    // trailing A22 -= Pn Pn^H
    CHASE_TRY(launch_conj_transpose(d, Pn, ldg, m, kb, work, kb));
    T* A22 = Akk + static_cast<size_t>(kb) * ldg + kb;
    CHASE_TRY(gemm(d, m, kb, Pn, ldg, work, kb, m, A22, ldg, 0, m, -1.0, 1.0, 0.0));
  }
  return CHASE_OK;
}

// X (N x p) <- X L^-H with L the lower Cholesky factor (p x p): blocked
// right-side triangular solve, column blocks of 32.
template <class T>
int trsm_right_lh(Dev& d, T* X, int64_t ldx, int64_t N, const T* L, int64_t ldl, int p,
                  T* work /* >= 32 * p */) {
  constexpr int nb = 32;
  for (int k0 = 0; k0 < p; k0 += nb) {
    const int kb = std::min(nb, p - k0);
    T* Xk = X + static_cast<size_t>(k0) * ldx;
    if (k0 > 0) {
      // X[:, k0:k0+kb] -= X[:, 0:k0] R[0:k0, k0:k0+kb],  R = L^H
      CHASE_TRY(launch_conj_transpose(d, L + k0, ldl, kb, k0, work, k0));
      CHASE_TRY(gemm(d, N, k0, X, ldx, work, k0, kb, Xk, ldx, 0, kb, -1.0, 1.0, 0.0));
    }
    CHASE_TRY(launch_row_trsm_lh(d, Xk, ldx, N, L + static_cast<size_t>(k0) * ldl + k0, ldl, kb));
  }
  return CHASE_OK;
}

template <class T>
int launch_lanczos_step(Dev& d, int64_t N, int64_t ld, int r, int step, const T* Vj,
                        const T* Vprev, T* W, T* Vnext, double* alpha, double* beta, double tiny) {
  lanczos_step_kernel<<<r, kRed, 0, d.st>>>(N, ld, r, step, dp(Vj), dp(Vprev), dp(W), dp(Vnext),
                                            alpha, beta, tiny);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class T>
int launch_normalize_cols(Dev& d, T* X, int64_t ldx, int64_t N, int r) {
  if (r == 0) return CHASE_OK;
  normalize_cols_kernel<<<r, kRed, 0, d.st>>>(dp(X), ldx, N);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

#define CHASE_INSTANTIATE_ELEMENT_LAUNCHERS(T)                                                     \
  template int launch_permute_cols<T>(Dev&, const T*, int64_t, T*, int64_t, int64_t, int,         \
                                      const int*, bool);                                           \
  template int launch_col_norms<T>(Dev&, const T*, int64_t, int64_t, int, double*);                \
  template int launch_col_inv_scale<T>(Dev&, T*, int64_t, int64_t, int, const double*);            \
  template int launch_resid_norms<T>(Dev&, const T*, int64_t, const T*, int64_t, int64_t, int,     \
                                     const double*, double*);                                      \
  template int launch_fill_upper_hermitian<T>(Dev&, T*, int64_t, int);                             \
  template int launch_zero_triangle<T>(Dev&, T*, int64_t, int, bool);                              \
  template int launch_hermitian_from_lower<T>(Dev&, const T*, int64_t, T*, int64_t, int64_t);      \
  template int launch_cholesky<T>(Dev&, T*, int64_t, int, double, double);                         \
  template int cholesky_blocked<T>(Dev&, T*, int64_t, int, double, double, double*, T*);           \
  template int trsm_right_lh<T>(Dev&, T*, int64_t, int64_t, const T*, int64_t, int, T*);           \
  template int launch_lanczos_step<T>(Dev&, int64_t, int64_t, int, int, const T*, const T*, T*,    \
                                      T*, double*, double*, double);                               \
  template int launch_normalize_cols<T>(Dev&, T*, int64_t, int64_t, int);
CHASE_INSTANTIATE_ELEMENT_LAUNCHERS(chase_c64)
CHASE_INSTANTIATE_ELEMENT_LAUNCHERS(double)
CHASE_INSTANTIATE_ELEMENT_LAUNCHERS(chase_c32)
CHASE_INSTANTIATE_ELEMENT_LAUNCHERS(float)
#undef CHASE_INSTANTIATE_ELEMENT_LAUNCHERS

// ---------------------------------------------------------------------------
// Projected eigensolve (Alg. 2 line 3): cuSOLVER zheevd, eigenvalues ascending
// ---------------------------------------------------------------------------
namespace {
thread_local cusolverDnHandle_t t_solver = nullptr;
}

void release_thread_solver() {
  if (t_solver) {
    cusolverDnDestroy(t_solver);
    t_solver = nullptr;
  }
}

namespace {
int solver_handle(Dev& d) {
  if (!t_solver) {
    if (cusolverDnCreate(&t_solver) != CUSOLVER_STATUS_SUCCESS) {
      t_solver = nullptr;
      set_error("cusolverDnCreate failed");
      return CHASE_EIGENSOLVER_ERROR;
    }
    // Deterministic results are cuSOLVER's default; stated here so that a
    // change of that default cannot make two identical solves diverge.
    if (cusolverDnSetDeterministicMode(t_solver, CUSOLVER_DETERMINISTIC_RESULTS) !=
        CUSOLVER_STATUS_SUCCESS) {
      cusolverDnDestroy(t_solver);
      t_solver = nullptr;
      set_error("cusolverDnSetDeterministicMode failed");
      return CHASE_EIGENSOLVER_ERROR;
    }
  }
  if (cusolverDnSetStream(t_solver, d.st) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnSetStream failed");
    return CHASE_EIGENSOLVER_ERROR;
  }
  return CHASE_OK;
}

int eigh_info(Dev& d, int* info, const char* what) {
  int h_info = 0;
  CHASE_CUDA(cudaMemcpyAsync(&h_info, info, sizeof(int), cudaMemcpyDeviceToHost, d.st));
  CHASE_CUDA(cudaStreamSynchronize(d.st));
  if (h_info != 0) {
    set_error("%s returned info = %d", what, h_info);
    return CHASE_EIGENSOLVER_ERROR;
  }
  return CHASE_OK;
}
}  // namespace

// Real symmetric projected eigenproblem: cuSOLVER dsyevd.
int eigh_device(Dev& d, double* G, int64_t ldg, int p, double* w_dev) {
  if (p == 0) return CHASE_OK;
  CHASE_TRY(solver_handle(d));
  int lwork = 0;
  if (cusolverDnDsyevd_bufferSize(t_solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, p, G,
                                  static_cast<int>(ldg), w_dev, &lwork) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnDsyevd_bufferSize failed");
    return CHASE_EIGENSOLVER_ERROR;
  }
  double* work = nullptr;
  int* info = nullptr;
  CHASE_TRY(d.alloc(&work, static_cast<size_t>(std::max(lwork, 1))));
  CHASE_TRY(d.alloc(&info, 1));
  if (cusolverDnDsyevd(t_solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, p, G,
                       static_cast<int>(ldg), w_dev, work, lwork, info) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnDsyevd failed to launch");
    return CHASE_EIGENSOLVER_ERROR;
  }
  return eigh_info(d, info, "dsyevd");
}

namespace {
__global__ void widen_kernel(const float* __restrict__ w, int p, double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p; j += gridDim.x * blockDim.x)
    out[j] = w[j];
}
}  // namespace

// Single-precision projected eigenproblems: cuSOLVER cheevd / ssyevd, the
// eigenvalues widened to double for the host decisions.
int eigh_device(Dev& d, chase_c32* G, int64_t ldg, int p, double* w_dev) {
  if (p == 0) return CHASE_OK;
  CHASE_TRY(solver_handle(d));
  float* wf = nullptr;
  CHASE_TRY(d.alloc(&wf, static_cast<size_t>(p)));
  int lwork = 0;
  if (cusolverDnCheevd_bufferSize(t_solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, p,
                                  reinterpret_cast<cuComplex*>(G), static_cast<int>(ldg), wf,
                                  &lwork) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnCheevd_bufferSize failed");
    return CHASE_EIGENSOLVER_ERROR;
  }
  cuComplex* work = nullptr;
  int* info = nullptr;
  CHASE_TRY(d.alloc(&work, static_cast<size_t>(std::max(lwork, 1))));
  CHASE_TRY(d.alloc(&info, 1));
  if (cusolverDnCheevd(t_solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, p,
                       reinterpret_cast<cuComplex*>(G), static_cast<int>(ldg), wf, work, lwork,
                       info) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnCheevd failed to launch");
    return CHASE_EIGENSOLVER_ERROR;
  }
  widen_kernel<<<grid_for(p, 256, 64), 256, 0, d.st>>>(wf, p, w_dev);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return eigh_info(d, info, "cheevd");
}

int eigh_device(Dev& d, float* G, int64_t ldg, int p, double* w_dev) {
  if (p == 0) return CHASE_OK;
  CHASE_TRY(solver_handle(d));
  float* wf = nullptr;
  CHASE_TRY(d.alloc(&wf, static_cast<size_t>(p)));
  int lwork = 0;
  if (cusolverDnSsyevd_bufferSize(t_solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, p, G,
                                  static_cast<int>(ldg), wf, &lwork) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnSsyevd_bufferSize failed");
    return CHASE_EIGENSOLVER_ERROR;
  }
  float* work = nullptr;
  int* info = nullptr;
  CHASE_TRY(d.alloc(&work, static_cast<size_t>(std::max(lwork, 1))));
  CHASE_TRY(d.alloc(&info, 1));
  if (cusolverDnSsyevd(t_solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, p, G,
                       static_cast<int>(ldg), wf, work, lwork, info) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnSsyevd failed to launch");
    return CHASE_EIGENSOLVER_ERROR;
  }
  widen_kernel<<<grid_for(p, 256, 64), 256, 0, d.st>>>(wf, p, w_dev);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return eigh_info(d, info, "ssyevd");
}

int eigh_device(Dev& d, chase_c64* G, int64_t ldg, int p, double* w_dev) {
  if (p == 0) return CHASE_OK;
  CHASE_TRY(solver_handle(d));
  int lwork = 0;
  if (cusolverDnZheevd_bufferSize(t_solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, p,
                                  reinterpret_cast<cuDoubleComplex*>(G), static_cast<int>(ldg),
                                  w_dev, &lwork) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnZheevd_bufferSize failed");
    return CHASE_EIGENSOLVER_ERROR;
  }
  cuDoubleComplex* work = nullptr;
  int* info = nullptr;
  CHASE_TRY(d.alloc(&work, static_cast<size_t>(std::max(lwork, 1))));
  CHASE_TRY(d.alloc(&info, 1));
  if (cusolverDnZheevd(t_solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, p,
                       reinterpret_cast<cuDoubleComplex*>(G), static_cast<int>(ldg), w_dev, work,
                       lwork, info) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnZheevd failed to launch");
    return CHASE_EIGENSOLVER_ERROR;
  }
  return eigh_info(d, info, "zheevd");
}

}  // namespace chase

// ---------------------------------------------------------------------------
// Projected eigenproblems of a batch (Alg. 2 line 3), many at once
// ---------------------------------------------------------------------------
namespace chase {
namespace {
// Item q of a bucket: G (p x p, ld), padded into slot q of the bucket
// (n x n, column-major) as diag(G, pad I) with pad = 1 + 2 ||G||_F, above
// every eigenvalue of G, so that the p lowest eigenpairs of the slot are
// those of G with eigenvectors [w; 0].
__global__ void eigh_pack_kernel(const EighItem* __restrict__ items, int n,
                                 double2* __restrict__ A) {
  __shared__ double scratch[33];
  const EighItem it = items[blockIdx.x];
  const double2* G = reinterpret_cast<const double2*>(it.G);
  double s = 0.0;
  for (long long e = threadIdx.x; e < (long long)it.p * it.p; e += blockDim.x) {
    const double2 v = G[(e / it.p) * it.ldg + e % it.p];
    s += v.x * v.x + v.y * v.y;
  }
  s = block_sum(s, scratch);
  const double pad = 1.0 + 2.0 * sqrt(s);
  double2* slot = A + (long long)blockIdx.x * n * n;
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    const int i = static_cast<int>(e % n), j = static_cast<int>(e / n);
    double2 v = make_double2(0.0, 0.0);
    if (i < it.p && j < it.p)
      v = G[(long long)j * it.ldg + i];
    else if (i == j)
      v = make_double2(pad, 0.0);
    slot[e] = v;
  }
}

// The p lowest eigenpairs of slot q back to item q: eigenvectors into G
// (columns, first p rows), eigenvalues into w.
__global__ void eigh_unpack_kernel(const EighItem* __restrict__ items, int n,
                                   const double2* __restrict__ A, const double* __restrict__ W) {
  const EighItem it = items[blockIdx.x];
  double2* G = reinterpret_cast<double2*>(it.G);
  const double2* slot = A + (long long)blockIdx.x * n * n;
  for (long long e = threadIdx.x; e < (long long)it.p * it.p; e += blockDim.x) {
    const int i = static_cast<int>(e % it.p), j = static_cast<int>(e / it.p);
    G[(long long)j * it.ldg + i] = slot[(long long)j * n + i];
  }
  for (int j = threadIdx.x; j < it.p; j += blockDim.x) it.w[j] = W[(long long)blockIdx.x * n + j];
}
}  // namespace

int eigh_batched(Dev& d, const std::vector<EighItem>& items, int** info_dev) {
  if (items.empty()) return CHASE_OK;
  CHASE_TRY(solver_handle(d));
  cusolverDnParams_t prm = nullptr;
  if (cusolverDnCreateParams(&prm) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnCreateParams failed");
    return CHASE_EIGENSOLVER_ERROR;
  }
  struct ParamsGuard {
    cusolverDnParams_t p;
    ~ParamsGuard() { cusolverDnDestroyParams(p); }
  } guard{prm};
  // buckets of matrix sizes rounded up to a multiple of 16; matrices above
  // kBatchedEighMax take the one-matrix solver
  constexpr int kBatchedEighMax = 256;
  std::map<int, std::vector<int>> buckets;
  int* info = nullptr;
  CHASE_TRY(d.alloc(&info, items.size()));
  CHASE_CUDA(cudaMemsetAsync(info, 0, sizeof(int) * items.size(), d.st));
  int off = 0;
  for (size_t q = 0; q < items.size(); ++q) {
    if (items[q].p > kBatchedEighMax)
      CHASE_TRY(eigh_device(d, items[q].G, items[q].ldg, items[q].p, items[q].w));
    else if (items[q].p > 0)
      buckets[(items[q].p + 15) / 16 * 16].push_back(static_cast<int>(q));
  }
  for (auto& [n, idx] : buckets) {
    const int c = static_cast<int>(idx.size());
    std::vector<EighItem> sub(c);
    for (int k = 0; k < c; ++k) sub[k] = items[idx[k]];
    EighItem* dsub = nullptr;
    double2* A = nullptr;
    double* W = nullptr;
    CHASE_TRY(d.alloc(&dsub, c));
    CHASE_TRY(d.alloc(&A, static_cast<size_t>(c) * n * n));
    CHASE_TRY(d.alloc(&W, static_cast<size_t>(c) * n));
    CHASE_CUDA(cudaMemcpyAsync(dsub, sub.data(), sizeof(EighItem) * c, cudaMemcpyHostToDevice, d.st));
    eigh_pack_kernel<<<c, 256, 0, d.st>>>(dsub, n, A);
    note_launch();
    CHASE_CUDA(cudaGetLastError());
    size_t wd = 0, wh = 0;
    if (cusolverDnXsyevBatched_bufferSize(t_solver, prm, CUSOLVER_EIG_MODE_VECTOR,
                                          CUBLAS_FILL_MODE_LOWER, n, CUDA_C_64F, A, n, CUDA_R_64F, W,
                                          CUDA_C_64F, &wd, &wh, c) != CUSOLVER_STATUS_SUCCESS) {
      set_error("cusolverDnXsyevBatched_bufferSize failed (n = %d, batch = %d)", n, c);
      return CHASE_EIGENSOLVER_ERROR;
    }
    void* work = nullptr;
    CHASE_TRY(d.alloc_bytes(&work, std::max<size_t>(wd, 16)));
    std::vector<char> hwork(std::max<size_t>(wh, 16));
    if (cusolverDnXsyevBatched(t_solver, prm, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                               CUDA_C_64F, A, n, CUDA_R_64F, W, CUDA_C_64F, work, wd, hwork.data(),
                               wh, info + off, c) != CUSOLVER_STATUS_SUCCESS) {
      set_error("cusolverDnXsyevBatched failed to launch (n = %d, batch = %d)", n, c);
      return CHASE_EIGENSOLVER_ERROR;
    }
    eigh_unpack_kernel<<<c, 256, 0, d.st>>>(dsub, n, A, W);
    note_launch();
    CHASE_CUDA(cudaGetLastError());
    if (wh > 0) CHASE_CUDA(cudaStreamSynchronize(d.st));  // the host workspace is in use until here
    off += c;
  }
  if (info_dev) *info_dev = info;
  return CHASE_OK;
}

}  // namespace chase

// ---------------------------------------------------------------------------
// Failure detection: the bounded wait of the pipelined kernels, on its own
// ---------------------------------------------------------------------------
namespace chase {
namespace {
// One thread waits on an mbarrier that nothing ever arrives at, for at most
// `budget` cycles, then records the timeout flag exactly as the product
// kernels' producers and consumers do.  No copy or MMA is in flight.
__global__ void wait_selftest_kernel(long long budget, int* __restrict__ err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_barrier_init();
  if (!mbar_wait_bounded(&bar, 0, budget)) atomicOr(err, KERR_TIMEOUT_FULL);
}
}  // namespace
}  // namespace chase

extern "C" int chase_wait_selftest(long long budget_cycles, void* stream) {
  if (budget_cycles < 0 || budget_cycles > chase::kWaitBudgetCycles) {
    chase::set_error("chase_wait_selftest: budget must be in [0, %lld] cycles",
                     chase::kWaitBudgetCycles);
    return CHASE_INVALID_ARG;
  }
  chase::Dev d(stream);
  CHASE_TRY(d.init());
  chase::wait_selftest_kernel<<<1, 32, 0, d.st>>>(budget_cycles, d.err);
  chase::note_launch();
  CHASE_CUDA(cudaGetLastError());
  return d.sync_check("chase_wait_selftest");
}
