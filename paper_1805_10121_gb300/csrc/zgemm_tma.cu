// Complex FP64 GEMM with the Chebyshev-recurrence epilogue fused in:
//
//   C[:, j] = alpha * (A * B[:, j] - shift * B[0:M, j]) + beta * C[:, j],  j in [j0, j1)
//
// With A = H, B = the current filter block, shift = c, alpha = 2 tau / e and
// beta = -tau sigma this is one step of the three-term recurrence (Eq. 7,
// Alg. 4 line 9); the first step (Alg. 4 line 4) is alpha = sigma_1 / e,
// beta = 0.  Restricting j to the active suffix [j0, j1) is the column
// retirement of Alg. 4 lines 12-14.  The same kernel with shift = 0 forms H Q
// for Rayleigh-Ritz and the block products of the orthogonalisation.
//
// GB300 mapping.  Every FP64 product runs on the FP64 tensor pipe through
// mma.sync.m8n8k4.f64 (there is no f64 kind of tcgen05.mma).  On GB300 that
// pipe delivers about 1 TFLOP/s, roughly 0.15 FLOP per byte of HBM
// bandwidth, so every tile shape used here is compute bound by a wide margin;
// the design goal is to keep the DMMA pipe of all 152 SMs busy:
//  * operand tiles are streamed by TMA (cp.async.bulk.tensor) into a ring
//    of shared-memory stages guarded by mbarriers; one producer warp issues
//    the copies, four consumer warps issue DMMAs, so address generation and
//    copies never occupy the math warps;
//  * a complex product is three real DMMAs (the 3M / Gauss form:
//    T1 = ar br, T2 = ai bi, T3 = (ar + ai)(br + bi), re = T1 - T2,
//    im = T3 - T1 - T2) on the interleaved (re, im) operands read as 16-byte
//    pairs from shared memory: 6 N^2 b executed FLOPs per 8 N^2 b of the
//    complex product, still all FP64;
//  * the shift, scale and axpby of the recurrence are applied while the
//    accumulators are still in registers, so the filter makes one pass over
//    its output per degree step;
//  * the tile shape (64 x 32, 128 x 16, 64 x 16 or 64 x 8 outputs) is the one
//    with the least work on the busiest SM: one CTA already keeps an SM's
//    FP64 pipe busy, so narrow blocks want narrow tiles on more SMs
//    (measured, N = 8000: one column 14.4 ms with 64 x 32, 4.0 ms with
//    64 x 8; 100 columns 56.7 ms and 40.5 ms); products of at most six
//    columns skip the tensor pipe altogether (fewcol.cu);
//  * every mbarrier wait is bounded; a wait that gives up records an error
//    flag that the host turns into CHASE_TIMEOUT, and the producer drains
//    its own copies in flight before the CTA exits.
#include "common.cuh"
#include "context.hpp"

namespace chase {

namespace {

template <int BM_, int BN_, int BK_, int STAGES_, int WARPS_M_, int ES_ = 16>
struct Cfg {
  static constexpr int ES = ES_;  // element bytes: 16 complex128, 8 float64
  static constexpr int BM = BM_, BN = BN_, BK = BK_, STAGES = STAGES_;
  static constexpr int WARPS_M = WARPS_M_;
  static constexpr int WARPS_N = 4 / WARPS_M_;
  static constexpr int kConsumerWarps = 4;
  static constexpr int kThreads = (kConsumerWarps + 1) * 32;
  static constexpr int WTM = BM / WARPS_M;
  static constexpr int WTN = BN / WARPS_N;
  static constexpr int MI = WTM / 8;
  static constexpr int NI = WTN / 8;
  static constexpr int A_BYTES = BM * BK * ES;
  static constexpr int B_BYTES = BK * BN * ES;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 2 * STAGES * 8 + 128;
  static_assert(MI >= 1 && NI >= 1, "warp tile too small");
  static_assert(WTM % 8 == 0 && WTN % 8 == 0, "warp tile must be a multiple of 8");
  static_assert(BK % 4 == 0, "BK must be a multiple of 4");
  static_assert((ES / 8) * BM <= 256 && (ES / 8) * BK <= 256 && BN <= 256, "TMA box limit");
};

// One output tile: its operand maps and coordinates and its epilogue.
struct Fp64Tile {
  const CUtensorMap* mapA;
  const CUtensorMap* mapB;
  int maps_in_global;  // maps live in global memory: acquire them for the async proxy
  int row0, col0;      // first row of A / first (absolute) column of B of the tile
  int M, K, j1;        // rows of A, K extent, columns >= j1 are outside the block
  const double2* Bsh;  // B again, for the shift term
  long long ldb;
  double2* Cout;
  long long ldc;
  double alpha, beta, shift;
};

__device__ __forceinline__ void acquire_tmap_global(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(
                   reinterpret_cast<uint64_t>(map))
               : "memory");
}

template <class C>
__device__ __forceinline__ void zgemm_tile_body(const Fp64Tile& T, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  double2* sA = reinterpret_cast<double2*>(smem);                         // [STAGES][BK][BM]
  double2* sB = reinterpret_cast<double2*>(smem + C::STAGES * C::A_BYTES);  // [STAGES][BN][BK]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int row0 = T.row0;
  const int col0 = T.col0;
  const int M = T.M;
  const int nk = (T.K + C::BK - 1) / C::BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], C::kConsumerWarps);
    }
    fence_barrier_init();
  }
  __syncthreads();

  if (warp == C::kConsumerWarps) {
    // ---------------- producer: one thread issues every TMA copy ----------
    if (lane == 0) {
      if (T.maps_in_global) {
        acquire_tmap_global(T.mapA);
        acquire_tmap_global(T.mapB);
      }
      prefetch_tmap(T.mapA);
      prefetch_tmap(T.mapB);
      int issued = 0;
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % C::STAGES;
        if (kt >= C::STAGES) {
          if (!mbar_wait_bounded(&empty[s], ((kt / C::STAGES) & 1) ^ 1)) {
            atomicOr(err, KERR_TIMEOUT_EMPTY);
            break;
          }
        }
        mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
        tma_load_2d(sA + s * C::BK * C::BM, T.mapA, 2 * row0, kt * C::BK, &full[s]);
        tma_load_2d(sB + s * C::BN * C::BK, T.mapB, 2 * kt * C::BK, col0, &full[s]);
        ++issued;
      }
      // Drain: no copy of this CTA may still be landing when it exits.
      for (int kt = (issued > C::STAGES ? issued - C::STAGES : 0); kt < issued; ++kt) {
        if (!mbar_wait_bounded(&full[kt % C::STAGES], (kt / C::STAGES) & 1))
          atomicOr(err, KERR_TIMEOUT_FULL);
      }
    }
    return;
  }

  // ---------------- consumers: DMMA on the staged tiles ---------------------
  const int wm = warp % C::WARPS_M;
  const int wn = warp / C::WARPS_M;
  const int g = lane >> 2;  // fragment row (A, C) / column (B)
  const int t = lane & 3;   // fragment k index (A, B) / column pair (C)

  double t1[C::MI][C::NI][2];  // sum ar br
  double t2[C::MI][C::NI][2];  // sum ai bi
  double t3[C::MI][C::NI][2];  // sum (ar + ai)(br + bi)
#pragma unroll
  for (int mi = 0; mi < C::MI; ++mi)
#pragma unroll
    for (int ni = 0; ni < C::NI; ++ni) {
      t1[mi][ni][0] = t1[mi][ni][1] = 0.0;
      t2[mi][ni][0] = t2[mi][ni][1] = 0.0;
      t3[mi][ni][0] = t3[mi][ni][1] = 0.0;
    }

  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt % C::STAGES;
    if (!mbar_wait_bounded(&full[s], (kt / C::STAGES) & 1)) {
      if (lane == 0) atomicOr(err, KERR_TIMEOUT_FULL);
      return;
    }
    const double2* a_s = sA + s * C::BK * C::BM;
    const double2* b_s = sB + s * C::BN * C::BK;
#pragma unroll
    for (int kk = 0; kk < C::BK; kk += 4) {
      double2 af[C::MI], bf[C::NI];
      double as[C::MI], bs[C::NI];
#pragma unroll
      for (int mi = 0; mi < C::MI; ++mi) {
        af[mi] = a_s[(kk + t) * C::BM + wm * C::WTM + mi * 8 + g];
        as[mi] = af[mi].x + af[mi].y;
      }
#pragma unroll
      for (int ni = 0; ni < C::NI; ++ni) {
        bf[ni] = b_s[(wn * C::WTN + ni * 8 + g) * C::BK + kk + t];
        bs[ni] = bf[ni].x + bf[ni].y;
      }
#pragma unroll
      for (int mi = 0; mi < C::MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < C::NI; ++ni) {
          dmma_8x8x4(t1[mi][ni][0], t1[mi][ni][1], af[mi].x, bf[ni].x);
          dmma_8x8x4(t2[mi][ni][0], t2[mi][ni][1], af[mi].y, bf[ni].y);
          dmma_8x8x4(t3[mi][ni][0], t3[mi][ni][1], as[mi], bs[ni]);
        }
    }
    // The stage was read through the generic proxy and the producer's next
    // TMA copy overwrites it through the async proxy: order the reads first.
    // Without this fence a copy could land before the last loads of a warp
    // had returned whenever the SM's load pipe was busy (other kernels on the
    // device), corrupting 8 x 8 fragments of the product.
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }

  // ---------------- fused epilogue: shift, scale, axpby ---------------------
#pragma unroll
  for (int mi = 0; mi < C::MI; ++mi) {
    const int r = row0 + wm * C::WTM + mi * 8 + g;
    if (r >= M) continue;
#pragma unroll
    for (int ni = 0; ni < C::NI; ++ni) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = col0 + wn * C::WTN + ni * 8 + 2 * t + h;
        if (c >= T.j1) continue;
        double vr = t1[mi][ni][h] - t2[mi][ni][h];
        double vi = t3[mi][ni][h] - t1[mi][ni][h] - t2[mi][ni][h];
        if (T.shift != 0.0) {
          const double2 bv = T.Bsh[static_cast<long long>(c) * T.ldb + r];
          vr -= T.shift * bv.x;
          vi -= T.shift * bv.y;
        }
        vr *= T.alpha;
        vi *= T.alpha;
        double2* cp = T.Cout + static_cast<long long>(c) * T.ldc + r;
        if (T.beta != 0.0) {
          const double2 cv = *cp;
          vr += T.beta * cv.x;
          vi += T.beta * cv.y;
        }
        *cp = make_double2(vr, vi);
      }
    }
  }
}

// The real (float64) tile: one DMMA per fragment pair, same pipeline and
// epilogue as the complex tile.
template <class C>
__device__ __forceinline__ void dgemm_tile_body(const Fp64Tile& T, int* __restrict__ err) {
  static_assert(C::ES == 8, "real configuration expected");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  double* sA = reinterpret_cast<double*>(smem);                         // [STAGES][BK][BM]
  double* sB = reinterpret_cast<double*>(smem + C::STAGES * C::A_BYTES);  // [STAGES][BN][BK]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  const double* Bsh = reinterpret_cast<const double*>(T.Bsh);
  double* Cout = reinterpret_cast<double*>(T.Cout);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int row0 = T.row0;
  const int col0 = T.col0;
  const int M = T.M;
  const int nk = (T.K + C::BK - 1) / C::BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], C::kConsumerWarps);
    }
    fence_barrier_init();
  }
  __syncthreads();

  if (warp == C::kConsumerWarps) {
    if (lane == 0) {  // producer
      if (T.maps_in_global) {
        acquire_tmap_global(T.mapA);
        acquire_tmap_global(T.mapB);
      }
      prefetch_tmap(T.mapA);
      prefetch_tmap(T.mapB);
      int issued = 0;
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % C::STAGES;
        if (kt >= C::STAGES) {
          if (!mbar_wait_bounded(&empty[s], ((kt / C::STAGES) & 1) ^ 1)) {
            atomicOr(err, KERR_TIMEOUT_EMPTY);
            break;
          }
        }
        mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
        tma_load_2d(sA + s * C::BK * C::BM, T.mapA, row0, kt * C::BK, &full[s]);
        tma_load_2d(sB + s * C::BN * C::BK, T.mapB, kt * C::BK, col0, &full[s]);
        ++issued;
      }
      for (int kt = (issued > C::STAGES ? issued - C::STAGES : 0); kt < issued; ++kt) {
        if (!mbar_wait_bounded(&full[kt % C::STAGES], (kt / C::STAGES) & 1))
          atomicOr(err, KERR_TIMEOUT_FULL);
      }
    }
    return;
  }

  const int wm = warp % C::WARPS_M;
  const int wn = warp / C::WARPS_M;
  const int g = lane >> 2;
  const int t = lane & 3;
  double acc[C::MI][C::NI][2];
#pragma unroll
  for (int mi = 0; mi < C::MI; ++mi)
#pragma unroll
    for (int ni = 0; ni < C::NI; ++ni) acc[mi][ni][0] = acc[mi][ni][1] = 0.0;

  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt % C::STAGES;
    if (!mbar_wait_bounded(&full[s], (kt / C::STAGES) & 1)) {
      if (lane == 0) atomicOr(err, KERR_TIMEOUT_FULL);
      return;
    }
    const double* a_s = sA + s * C::BK * C::BM;
    const double* b_s = sB + s * C::BN * C::BK;
#pragma unroll
    for (int kk = 0; kk < C::BK; kk += 4) {
      double af[C::MI], bf[C::NI];
#pragma unroll
      for (int mi = 0; mi < C::MI; ++mi) af[mi] = a_s[(kk + t) * C::BM + wm * C::WTM + mi * 8 + g];
#pragma unroll
      for (int ni = 0; ni < C::NI; ++ni) bf[ni] = b_s[(wn * C::WTN + ni * 8 + g) * C::BK + kk + t];
#pragma unroll
      for (int mi = 0; mi < C::MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < C::NI; ++ni) dmma_8x8x4(acc[mi][ni][0], acc[mi][ni][1], af[mi], bf[ni]);
    }
    // The stage was read through the generic proxy and the producer's next
    // TMA copy overwrites it through the async proxy: order the reads first.
    // Without this fence a copy could land before the last loads of a warp
    // had returned whenever the SM's load pipe was busy (other kernels on the
    // device), corrupting 8 x 8 fragments of the product.
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }

#pragma unroll
  for (int mi = 0; mi < C::MI; ++mi) {
    const int r = row0 + wm * C::WTM + mi * 8 + g;
    if (r >= M) continue;
#pragma unroll
    for (int ni = 0; ni < C::NI; ++ni) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = col0 + wn * C::WTN + ni * 8 + 2 * t + h;
        if (c >= T.j1) continue;
        double v = acc[mi][ni][h];
        if (T.shift != 0.0) v -= T.shift * Bsh[static_cast<long long>(c) * T.ldb + r];
        v *= T.alpha;
        double* cp = Cout + static_cast<long long>(c) * T.ldc + r;
        if (T.beta != 0.0) v += T.beta * *cp;
        *cp = v;
      }
    }
  }
}

template <class C>
__global__ void __launch_bounds__(C::kThreads)
    dgemm_tma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     int M, int K, int j0, int j1, const double* __restrict__ Bsh, long long ldb,
                     double* __restrict__ Cout, long long ldc, double alpha, double beta,
                     double shift, int* __restrict__ err) {
  Fp64Tile T;
  T.mapA = &tmA;
  T.mapB = &tmB;
  T.maps_in_global = 0;
  T.row0 = blockIdx.x * C::BM;
  T.col0 = j0 + blockIdx.y * C::BN;
  T.M = M;
  T.K = K;
  T.j1 = j1;
  T.Bsh = reinterpret_cast<const double2*>(Bsh);
  T.ldb = ldb;
  T.Cout = reinterpret_cast<double2*>(Cout);
  T.ldc = ldc;
  T.alpha = alpha;
  T.beta = beta;
  T.shift = shift;
  dgemm_tile_body<C>(T, err);
}

template <class C>
__global__ void __launch_bounds__(C::kThreads)
    zgemm_tma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     int M, int K, int j0, int j1, const double2* __restrict__ Bsh, long long ldb,
                     double2* __restrict__ Cout, long long ldc, double alpha, double beta,
                     double shift, int* __restrict__ err) {
  Fp64Tile T;
  T.mapA = &tmA;
  T.mapB = &tmB;
  T.maps_in_global = 0;
  T.row0 = blockIdx.x * C::BM;
  T.col0 = j0 + blockIdx.y * C::BN;
  T.M = M;
  T.K = K;
  T.j1 = j1;
  T.Bsh = Bsh;
  T.ldb = ldb;
  T.Cout = Cout;
  T.ldc = ldc;
  T.alpha = alpha;
  T.beta = beta;
  T.shift = shift;
  zgemm_tile_body<C>(T, err);
}

// Grouped: one CTA per output tile of every active problem of one degree
// step of the filter; X = parity ? buf1 : buf0, Y = the other buffer.
template <class C>
__global__ void __launch_bounds__(C::kThreads)
    zgemm_grouped_kernel(const GroupedProblem* __restrict__ probs,
                         const GroupedStep* __restrict__ steps, int nact, int parity,
                         int* __restrict__ err) {
  const int bid = blockIdx.x;
  int lo = 0, hi = nact;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (steps[mid].tile0 <= bid) lo = mid; else hi = mid;
  }
  const GroupedStep stp = steps[lo];
  const GroupedProblem& pr = probs[stp.prob];
  const int local = bid - stp.tile0;
  const int ncol_tiles = (pr.b - stp.s + C::BN - 1) / C::BN;
  Fp64Tile T;
  T.mapA = pr.mapA;
  T.mapB = parity ? pr.mapB1 : pr.mapB0;
  T.maps_in_global = 1;
  T.row0 = (local / ncol_tiles) * C::BM;
  T.col0 = stp.s + (local % ncol_tiles) * C::BN;
  T.M = pr.n;
  T.K = pr.n;
  T.j1 = pr.b;
  T.Bsh = parity ? pr.buf1 : pr.buf0;
  T.ldb = parity ? pr.ld1 : pr.ld0;
  T.Cout = parity ? pr.buf0 : pr.buf1;
  T.ldc = parity ? pr.ld0 : pr.ld1;
  T.alpha = stp.alpha;
  T.beta = stp.beta;
  T.shift = stp.shift;
  zgemm_tile_body<C>(T, err);
}

template <class C>
int launch_cfg(Dev& d, int64_t M, int64_t K, const chase_c64* A, int64_t lda, const chase_c64* B,
               int64_t ldb, int64_t ncols_b, chase_c64* Cm, int64_t ldc, int j0, int j1,
               double alpha, double beta, double shift) {
  CUtensorMap tmA, tmB;
  CHASE_TRY(make_tmap_c64(&tmA, A, M, K, lda, C::BM, C::BK));
  CHASE_TRY(make_tmap_c64(&tmB, B, K, ncols_b, ldb, C::BK, C::BN));
  // once per instantiation; function-local static initialisation is thread safe
  static const cudaError_t attr_rc = cudaFuncSetAttribute(
      zgemm_tma_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  CHASE_CUDA(attr_rc);
  dim3 grid(static_cast<unsigned>((M + C::BM - 1) / C::BM),
            static_cast<unsigned>((j1 - j0 + C::BN - 1) / C::BN));
  zgemm_tma_kernel<C><<<grid, C::kThreads, C::SMEM, d.st>>>(
      tmA, tmB, static_cast<int>(M), static_cast<int>(K), j0, j1,
      reinterpret_cast<const double2*>(B), ldb, reinterpret_cast<double2*>(Cm), ldc, alpha, beta,
      shift, d.err);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class C>
int launch_cfg_real(Dev& d, int64_t M, int64_t K, const double* A, int64_t lda, const double* B,
                    int64_t ldb, int64_t ncols_b, double* Cm, int64_t ldc, int j0, int j1,
                    double alpha, double beta, double shift) {
  CUtensorMap tmA, tmB;
  CHASE_TRY(make_tmap_f64(&tmA, A, M, K, lda, C::BM, C::BK));
  CHASE_TRY(make_tmap_f64(&tmB, B, K, ncols_b, ldb, C::BK, C::BN));
  // once per instantiation; function-local static initialisation is thread safe
  static const cudaError_t attr_rc = cudaFuncSetAttribute(
      dgemm_tma_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  CHASE_CUDA(attr_rc);
  dim3 grid(static_cast<unsigned>((M + C::BM - 1) / C::BM),
            static_cast<unsigned>((j1 - j0 + C::BN - 1) / C::BN));
  dgemm_tma_kernel<C><<<grid, C::kThreads, C::SMEM, d.st>>>(
      tmA, tmB, static_cast<int>(M), static_cast<int>(K), j0, j1, B, ldb, Cm, ldc, alpha, beta,
      shift, d.err);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

using CfgWide = Cfg<64, 32, 16, 2, 2>;    // 64 x 32 tile, warps 2 x 2 (32 x 16 each)
using CfgMid = Cfg<64, 16, 16, 2, 4>;     // 64 x 16 tile, warps 4 x 1 (16 x 16 each)
using CfgNarrow = Cfg<64, 8, 16, 2, 4>;   // 64 x 8 tile, warps 4 x 1 (16 x 8 each)
using CfgTall = Cfg<128, 16, 16, 2, 4>;   // 128 x 16 tile, warps 4 x 1 (32 x 16 each)
using RCfgWide = Cfg<64, 32, 16, 3, 2, 8>;    // real tiles: same shapes, float64 elements
using RCfgMid = Cfg<64, 16, 16, 3, 4, 8>;
using RCfgNarrow = Cfg<64, 8, 16, 3, 4, 8>;

template <class C>
int grouped_attr() {
  // once per instantiation; function-local static initialisation is thread safe
  static const cudaError_t attr_rc = cudaFuncSetAttribute(
      zgemm_grouped_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  CHASE_CUDA(attr_rc);
  return CHASE_OK;
}

template <class C>
int launch_grouped(Dev& d, const GroupedProblem* probs, const GroupedStep* steps, int nact,
                   int ntiles, int parity) {
  CHASE_TRY(grouped_attr<C>());
  zgemm_grouped_kernel<C><<<static_cast<unsigned>(ntiles), C::kThreads, C::SMEM, d.st>>>(
      probs, steps, nact, parity, d.err);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

int sm_count() {
  static const int v = [] {  // thread-safe one-time initialisation
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 152;
    cudaGetLastError();
    return n;
  }();
  return v;
}

// Predicted time of an M x w product with tile shape C, in units of
// output-tile area: one CTA of four DMMA warps already keeps an SM's FP64
// pipe busy (measured: two to six co-resident CTAs run no faster per
// output), so the product takes as long as the busiest SM's tiles, i.e.
// ceil(tiles / SMs) x tile area.  Fits the measured times of all four
// shapes at N = 1200 - 8000 and 1 - 480 columns to within a few percent.
template <class C>
double tile_cost(int64_t M, int w) {
  const int64_t tiles = ((M + C::BM - 1) / C::BM) * ((w + C::BN - 1) / C::BN);
  const int64_t per_sm = (tiles + sm_count() - 1) / sm_count();
  return static_cast<double>(per_sm) * C::BM * C::BN;
}
}  // namespace

// Candidate tile shapes of the grouped FP64 filter, in autotuning order.
void grouped_fp64_tile(int cfg, int* bm, int* bn) {
  switch (cfg) {
    case 0: *bm = CfgMid::BM; *bn = CfgMid::BN; break;
    case 1: *bm = CfgWide::BM; *bn = CfgWide::BN; break;
    case 2: *bm = CfgTall::BM; *bn = CfgTall::BN; break;
    default: *bm = CfgNarrow::BM; *bn = CfgNarrow::BN; break;
  }
}

int zgemm_grouped_fp64_prepare(int cfg) {
  switch (cfg) {
    case 0: return grouped_attr<CfgMid>();
    case 1: return grouped_attr<CfgWide>();
    case 2: return grouped_attr<CfgTall>();
    default: return grouped_attr<CfgNarrow>();
  }
}

int zgemm_grouped_fp64(Dev& d, int cfg, const GroupedProblem* probs, const GroupedStep* steps,
                       int nact, int ntiles, int parity) {
  if (ntiles <= 0) return CHASE_OK;
  switch (cfg) {
    case 0: return launch_grouped<CfgMid>(d, probs, steps, nact, ntiles, parity);
    case 1: return launch_grouped<CfgWide>(d, probs, steps, nact, ntiles, parity);
    case 2: return launch_grouped<CfgTall>(d, probs, steps, nact, ntiles, parity);
    default: return launch_grouped<CfgNarrow>(d, probs, steps, nact, ntiles, parity);
  }
}

int zgemm(Dev& d, int64_t M, int64_t K, const chase_c64* A, int64_t lda, const chase_c64* B,
          int64_t ldb, int64_t ncols_b, chase_c64* Cm, int64_t ldc, int j0, int j1, double alpha,
          double beta, double shift) {
  if (j1 <= j0 || M == 0) return CHASE_OK;
  if (K == 0) {
    set_error("zgemm: K == 0 is not supported");
    return CHASE_INVALID_ARG;
  }
  if (shift != 0.0 && M != K) {
    set_error("zgemm: the shifted product needs a square A");
    return CHASE_INVALID_ARG;
  }
  const int w = j1 - j0;
  if (w <= kFewColMax)
    return fewcol_gemm(d, M, K, A, lda, B, ldb, Cm, ldc, j0, j1, alpha, beta, shift);
  // the tile shape with the least work on the busiest SM (ties: the wider
  // tile, which re-reads A fewer times)
  const double cost[4] = {tile_cost<CfgWide>(M, w), tile_cost<CfgTall>(M, w),
                          tile_cost<CfgMid>(M, w), tile_cost<CfgNarrow>(M, w)};
  int best = 0;
  for (int c = 1; c < 4; ++c)
    if (cost[c] < 0.97 * cost[best]) best = c;
  if (best == 0) return launch_cfg<CfgWide>(d, M, K, A, lda, B, ldb, ncols_b, Cm, ldc, j0, j1, alpha, beta, shift);
  if (best == 1) return launch_cfg<CfgTall>(d, M, K, A, lda, B, ldb, ncols_b, Cm, ldc, j0, j1, alpha, beta, shift);
  if (best == 2) return launch_cfg<CfgMid>(d, M, K, A, lda, B, ldb, ncols_b, Cm, ldc, j0, j1, alpha, beta, shift);
  return launch_cfg<CfgNarrow>(d, M, K, A, lda, B, ldb, ncols_b, Cm, ldc, j0, j1, alpha, beta, shift);
}

int dgemm(Dev& d, int64_t M, int64_t K, const double* A, int64_t lda, const double* B, int64_t ldb,
          int64_t ncols_b, double* Cm, int64_t ldc, int j0, int j1, double alpha, double beta,
          double shift) {
  if (j1 <= j0 || M == 0) return CHASE_OK;
  if (K == 0) {
    set_error("dgemm: K == 0 is not supported");
    return CHASE_INVALID_ARG;
  }
  if (shift != 0.0 && M != K) {
    set_error("dgemm: the shifted product needs a square A");
    return CHASE_INVALID_ARG;
  }
  const int w = j1 - j0;
  if (w <= kFewColMax)
    return fewcol_gemm(d, M, K, A, lda, B, ldb, Cm, ldc, j0, j1, alpha, beta, shift);
  // as for complex: the least work on the busiest SM, ties to the wider tile
  const double cost[3] = {tile_cost<RCfgWide>(M, w), tile_cost<RCfgMid>(M, w),
                          tile_cost<RCfgNarrow>(M, w)};
  int best = 0;
  for (int c = 1; c < 3; ++c)
    if (cost[c] < 0.97 * cost[best]) best = c;
  if (best == 2)
    return launch_cfg_real<RCfgNarrow>(d, M, K, A, lda, B, ldb, ncols_b, Cm, ldc, j0, j1, alpha,
                                       beta, shift);
  if (best == 1)
    return launch_cfg_real<RCfgMid>(d, M, K, A, lda, B, ldb, ncols_b, Cm, ldc, j0, j1, alpha, beta,
                                    shift);
  return launch_cfg_real<RCfgWide>(d, M, K, A, lda, B, ldb, ncols_b, Cm, ldc, j0, j1, alpha, beta,
                                   shift);
}

}  // namespace chase
