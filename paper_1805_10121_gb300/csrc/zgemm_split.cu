// Complex GEMM with the Chebyshev-recurrence epilogue on the BF16 tensor cores
// (tcgen05), accurate to about 1e-11 relative: the "split-BF16" filter product.
//
//   C[:, j] = alpha * (H X[:, j] - shift * X[:, j]) + beta * C[:, j],  j in [j0, j1)
//
// Why.  GB300 runs FP64 at about 1 TFLOP/s and BF16 at about 2 PFLOP/s.  The
// filter product is exact integer arithmetic once both operands are cut into
// 7-bit integer slices with one power-of-two scale per row of H and per column
// of X, so it can run on the BF16 tensor pipe without giving up accuracy:
//
//   Ht[r, :] = [Re H[r, :], Im H[r, :]] = 2^E_r  sum_s a_s[r, :] 2^-7(s+1)
//   Xt[:, 2c] = [Re X[:, c]; -Im X[:, c]],  Xt[:, 2c+1] = [Im X[:, c]; Re X[:, c]]
//             = 2^F_c sum_t b_t[:, .] 2^-7(t+1)
//   (H X)(r, c) = 2^(E_r + F_c - 14) sum_d 2^-7d L_d,   L_d = sum_{s+t=d} a_s b_t
//
// with a_s, b_t integers in [-127, 127] (exact in BF16).  S = 7 slices per
// operand keep the 28 pairs with s + t <= 6; truncation and the dropped pairs
// leave a relative error near 2^-49 of max|row| max|column| per entry.
//
// Diagonal.  The slices carry H without its (real) diagonal: the diagonal of
// a Hermitian matrix is often far larger than its other entries (it holds
// the mean eigenvalue), and a row scale set by it would waste the slices'
// bits on every other entry.  The epilogue adds (H_rr - shift) X[r, c] in
// FP64, next to the recurrence's own shift.
//
// Exactness.  Products of slices are integers below 2^14, so a level-d sum is
// exact in an FP32 accumulator while it stays below 2^24: levels 0-2 are
// flushed from TMEM into exact int32 sums (in the flush warps' registers) every 256 K
// (3 * 256 * 127^2 < 2^24); levels 3-6, already scaled by 2^-21 or less,
// accumulate in FP32 over the whole K.  The int32 sums bound one launch's K
// below 44380; longer K (N > 22000), and narrow blocks that would leave SMs
// idle, are split into K segments whose FP64 partial products a combine
// kernel sums before the epilogue.
//
// Structure (one CTA = 128 rows of H x 32 complex columns, 320 threads):
//  * warp 0: TMA producer, one 3-D box per operand per stage loads all S
//    slices of a 32-wide K range (64-byte rows, SWIZZLE_64B: the TMA unit
//    moves one box row per cycle, so 32-byte rows would leave it as slow as
//    the tensor pipe), 2-stage mbarrier ring;
//  * warp 1: allocates 512 TMEM columns (7 levels x 64 FP32 columns) and one
//    thread issues the MMAs of each 16-wide K block: per slice s of H one
//    tcgen05.mma (M = 128, K = 16) against the slices t of the block whose
//    levels s + t belong to the pass, N = 64 x (their count).  The B planes
//    are consecutive rows of the B tile and the levels consecutive TMEM
//    columns, so the 28 slice pairs take 10 MMAs (N up to 256), which read
//    each slice of H from shared memory once instead of 7 - s times.  At a
//    chunk boundary the tail levels go first, so the flush overlaps them;
//    stages are committed back to the producer and chunks to the flush
//    warps;
//  * warps 2-9 (two per TMEM lane quarter, 32 columns each): flush the exact
//    levels every chunk into int32 registers, then combine all levels and
//    apply the diagonal, shift, scale and axpby (Eq. 7) while writing the
//    FP64 output.
// Every wait is bounded; a wait that gives up sets the error flag.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "context.hpp"

namespace chase {
namespace split {
constexpr int S = 7;                 // 7-bit slices per operand (full accuracy)
constexpr int BM = 128;              // rows per CTA (TMEM lanes)
constexpr int BN = 64;               // real columns of the product per CTA (32 complex)
constexpr int BK = 16;               // K per MMA (a K block)
constexpr int KPS = 2;               // K blocks per stage: 32 K, one 64-byte swizzle row
constexpr int BX = BK * KPS;         // K per stage
constexpr int NSTAGE = 2;
constexpr int CHUNK = 16;            // k-blocks per exact chunk (256 K)
constexpr int A_TILE = BM * BX * 2;  // 8192 B per slice
constexpr int B_TILE = BN * BX * 2;  // 4096 B per slice
constexpr int STAGE_A = S * A_TILE;
constexpr int STAGE_B = S * B_TILE;
constexpr int STAGE_BYTES = STAGE_A + STAGE_B;
constexpr int kFlushWarps = 8;       // two per TMEM lane quarter, 32 columns each
constexpr int kThreads = (2 + kFlushWarps) * 32;
constexpr int SMEM = 1024 + NSTAGE * STAGE_BYTES + 256;

// A product that keeps only the leading NS slices of each operand (pairs
// s + t < NS): the truncation error becomes about 2^-(7 NS) of the scales
// instead of 2^-49, for (NS (NS + 1) / 2) / 28 of the tensor work.  The stage
// ring and the TMEM allocation shrink with NS.
template <int NS>
struct Slices {
  static constexpr int S = NS;
  static constexpr int NEXACT = NS < 3 ? NS : 3;
  static constexpr int STAGE_A = NS * A_TILE;
  static constexpr int STAGE_B = NS * B_TILE;
  static constexpr int STAGE_BYTES = STAGE_A + STAGE_B;
  static constexpr int NSTAGE = NS <= 4 ? 4 : 2;
  static constexpr int TMEM_COLS = NS * BN <= 256 ? 256 : 512;
  static constexpr int SMEM = 1024 + NSTAGE * STAGE_BYTES + 256;
  static_assert(SMEM <= 232448, "shared memory per CTA");
};

// K-major operand with 64-byte swizzled rows: 8-row atoms of 512 B stacked
// along M (SBO); the second K block of a row starts 32 bytes in.
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // LBO (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;        // SBO: 8 rows x 64 B
  d |= (uint64_t)1 << 46;                 // version
  d |= (uint64_t)4 << 61;                 // SWIZZLE_64B
  return d;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

#define TMEM_LD32(taddr, r)                                                                          \
  asm volatile(                                                                                      \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15," \
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"                   \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),         \
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),      \
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),   \
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),   \
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])                                           \
      : "r"(taddr))

#define TMEM_LD8(taddr, r)                                                                           \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"          \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), \
                 "=r"(r[7])                                                                          \
               : "r"(taddr))

#define TMEM_LD16(taddr, r)                                                                          \
  asm volatile(                                                                                      \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}," \
      " [%16];\n"                                                                                    \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),         \
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),      \
        "=r"(r[14]), "=r"(r[15])                                                                     \
      : "r"(taddr))

// 2^e as a double from its exponent bits, for -1022 <= e <= 1023.
__device__ __forceinline__ double pow2_normal(int e) {
  return __longlong_as_double(static_cast<long long>(e + 1023) << 52);
}

// One output tile of the split product: where its operands are (tensor maps
// and coordinates) and where its result goes.  Columns are counted in the
// B map: real column 2c / 2c+1 of the product belong to complex column c,
// whose exponent is F[c] and whose output column is c + joff.
struct SplitTile {
  const CUtensorMap* mapA;
  const CUtensorMap* mapB;
  int maps_in_global;  // maps live in global memory: acquire them for the async proxy
  int cplx;            // 1: complex operands (B rows 2c, 2c+1 per column); 0: real
  int arow;            // first row of H (A map row) of the tile
  int brow;            // first B map row (real product column) of the tile
  int cend;            // complex columns >= cend are outside the block
  int joff;            // output / shift column = complex column + joff
  int kb0, nkb;        // K blocks of this launch
  int M;               // rows of H
  const int* E;
  const int* F;
  const double* Dg;
  const double2* X;
  long long ldx;
  double2* Y;
  long long ldy;
  double alpha, beta, shift;
  double2* P;  // K-segment partial products (nullptr: fused epilogue)
  long long ldp;
};

__device__ __forceinline__ void acquire_tmap(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(
                   reinterpret_cast<uint64_t>(map))
               : "memory");
}

// The FP64 epilogue of one output tile: combine the exact int32 level sums
// of this thread's row (32 columns, half hf of the tile) with the FP32 tail
// levels read from TMEM, scale, and apply the diagonal, shift, scale and
// axpby of Eq. 7 (or store the raw K-segment partial product).
template <int NS>
__device__ __forceinline__ void split_epilogue(const SplitTile& T, uint32_t tbase,
                                               const int (&sums)[Slices<NS>::NEXACT][32], int row,
                                               int hf) {
  constexpr int S = Slices<NS>::S;
  constexpr int NEXACT = Slices<NS>::NEXACT;
  const int row0 = T.arow, colr0 = T.brow, M = T.M;
  {
    const int grow = row0 + row;
    const bool in_rows = grow < M;
    const int er = in_rows ? T.E[grow] : 0;
    const bool raw = T.P != nullptr;  // one K segment: the combine kernel finishes
    const double alpha = raw ? 1.0 : T.alpha;
    const double adsh = raw ? 0.0 : T.alpha * ((T.Dg && in_rows ? T.Dg[grow] : 0.0) - T.shift);
#pragma unroll
    for (int c0 = 0; c0 < 32; c0 += 8) {
      float t[8];
      if constexpr (S > NEXACT) {
        uint32_t r[8];
        TMEM_LD8(tbase + (S - 1) * BN + c0, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int j = 0; j < 8; ++j) t[j] = __uint_as_float(r[j]);
#pragma unroll 1
        for (int d = S - 2; d >= NEXACT; --d) {
          TMEM_LD8(tbase + d * BN + c0, r);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int j = 0; j < 8; ++j) t[j] = fmaf(t[j], 0.0078125f, __uint_as_float(r[j]));
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) t[j] = 0.f;  // no tail levels
      }
      if (in_rows && T.cplx) {
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          const int cc = (colr0 + hf * 32 + c0 + j) >> 1;  // complex column (B map)
          if (cc >= T.cend) continue;
          const int ex = er + T.F[cc] - 28;
          const bool normal = ex >= -1022 && ex <= 1023;
          const double sc = normal ? pow2_normal(ex) * alpha : alpha;
          double v[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const long long Sx = (static_cast<long long>(sums[0][c0 + j + h]) << 14) +
                                 (static_cast<long long>(sums[1][c0 + j + h]) << 7) +
                                 static_cast<long long>(sums[2][c0 + j + h]);
            v[h] = (static_cast<double>(Sx) + static_cast<double>(t[j + h] * 0.0078125f)) * sc;
            if (!normal) v[h] = ldexp(v[h], ex);  // subnormal or overflowing scale
          }
          if (raw) {
            T.P[static_cast<long long>(cc) * T.ldp + grow] = make_double2(v[0], v[1]);
            continue;
          }
          const long long jc = cc + T.joff;
          if (adsh != 0.0) {
            const double2 xv = T.X[jc * T.ldx + grow];
            v[0] = fma(adsh, xv.x, v[0]);
            v[1] = fma(adsh, xv.y, v[1]);
          }
          double2* yp = T.Y + jc * T.ldy + grow;
          if (T.beta != 0.0) {
            const double2 yv = *yp;
            v[0] = fma(T.beta, yv.x, v[0]);
            v[1] = fma(T.beta, yv.y, v[1]);
          }
          *yp = make_double2(v[0], v[1]);
        }
      } else if (in_rows) {  // real operands: one B-map row per column
        const double* Xr = reinterpret_cast<const double*>(T.X);
        double* Yr = reinterpret_cast<double*>(T.Y);
        double* Pr = reinterpret_cast<double*>(T.P);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int cc = colr0 + hf * 32 + c0 + j;
          if (cc >= T.cend) continue;
          const int ex = er + T.F[cc] - 28;
          const bool normal = ex >= -1022 && ex <= 1023;
          const double sc = normal ? pow2_normal(ex) * alpha : alpha;
          const long long Sx = (static_cast<long long>(sums[0][c0 + j]) << 14) +
                               (static_cast<long long>(sums[1][c0 + j]) << 7) +
                               static_cast<long long>(sums[2][c0 + j]);
          double v = (static_cast<double>(Sx) + static_cast<double>(t[j] * 0.0078125f)) * sc;
          if (!normal) v = ldexp(v, ex);
          if (raw) {
            Pr[static_cast<long long>(cc) * T.ldp + grow] = v;
            continue;
          }
          const long long jc = cc + T.joff;
          if (adsh != 0.0) v = fma(adsh, Xr[jc * T.ldx + grow], v);
          double* yp = Yr + jc * T.ldy + grow;
          if (T.beta != 0.0) v = fma(T.beta, *yp, v);
          *yp = v;
        }
      }
    }
  }
}

// The split product over a list of output tiles, persistent: each CTA
// allocates its TMEM and initialises its barriers once, then takes tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ... (tile(t, T) describes tile t).
// Barrier phases run on across tiles (global stage and chunk counters).
// While the flush warps run a tile's epilogue, the producer already loads
// the next tile's first stages; the MMA issuer starts the next tile once
// the epilogue has read TMEM (tmem_free).  CTAs that start their k-th tile
// together stream the same K ranges of neighbouring tiles, so the L2 serves
// each slab once to all of them.
template <int NS, class TileFn>
__device__ __forceinline__ void split_tiles_body(const TileFn& tile, int ntiles,
                                                 int* __restrict__ err) {
  static_assert(NS >= 3 && NS <= 7, "3 to 7 slices");
  using C = Slices<NS>;
  constexpr int S = C::S;
  constexpr int NEXACT = C::NEXACT;
  constexpr int NSTAGE = C::NSTAGE;
  constexpr int STAGE_A = C::STAGE_A;
  constexpr int STAGE_B = C::STAGE_B;
  constexpr int STAGE_BYTES = C::STAGE_BYTES;
  constexpr int TMEM_COLS = C::TMEM_COLS;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* sA = sm;
  unsigned char* sB = sm + NSTAGE * STAGE_A;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + NSTAGE * STAGE_BYTES);
  uint64_t* full = bars;                 // [NSTAGE]
  uint64_t* empty = bars + NSTAGE;       // [NSTAGE]
  uint64_t* chunk_full = bars + 2 * NSTAGE;
  uint64_t* chunk_empty = chunk_full + 1;
  uint64_t* done = chunk_full + 2;
  uint64_t* tmem_free = chunk_full + 3;  // the epilogue has read the tile's TMEM
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(chunk_full + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(chunk_full, 1);
    mbar_init(chunk_empty, kFlushWarps);
    mbar_init(done, 1);
    mbar_init(tmem_free, kFlushWarps);
    fence_barrier_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // ---------------- TMA producer
      long long g = 0;  // stages issued by this CTA so far
      bool ok = true;
      const CUtensorMap* last_a = nullptr;
      const CUtensorMap* last_b = nullptr;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        SplitTile T;
        tile(t, T);
        if (T.mapA != last_a || T.mapB != last_b) {
          if (T.maps_in_global) {
            acquire_tmap(T.mapA);
            acquire_tmap(T.mapB);
          }
          prefetch_tmap(T.mapA);
          prefetch_tmap(T.mapB);
          last_a = T.mapA;
          last_b = T.mapB;
        }
        const int nst = (T.nkb + KPS - 1) / KPS;  // stages (the last may hold one K block)
        for (int ks = 0; ks < nst; ++ks, ++g) {
          const int st = static_cast<int>(g % NSTAGE);
          if (g >= NSTAGE &&
              !mbar_wait_bounded(&empty[st], static_cast<uint32_t>((g / NSTAGE) & 1) ^ 1u)) {
            atomicOr(err, KERR_TIMEOUT_EMPTY);
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[st], STAGE_BYTES);
          tma_load_3d(smem_u32(sA + st * STAGE_A), T.mapA, (T.kb0 + ks * KPS) * BK, T.arow, 0,
                      smem_u32(&full[st]));
          tma_load_3d(smem_u32(sB + st * STAGE_B), T.mapB, (T.kb0 + ks * KPS) * BK, T.brow, 0,
                      smem_u32(&full[st]));
        }
      }
      // no copy may be in flight when the CTA ends
      for (long long k = (g > NSTAGE ? g - NSTAGE : 0); k < g; ++k)
        if (!mbar_wait_bounded(&full[k % NSTAGE], static_cast<uint32_t>((k / NSTAGE) & 1)))
          atomicOr(err, KERR_TIMEOUT_FULL);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------- MMA issuer
      // kind::f16 instruction descriptor without N: FP32 D, BF16 A and B, K-major, M = 128
      const uint32_t idesc_base = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BM >> 4) << 24);
      bool ok = true;
      long long g = 0, gc = 0;  // stages and exact chunks consumed so far
      int tk = 0;               // tiles started
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tk) {
        SplitTile T;
        tile(t, T);
        const int nkb = T.nkb;
        const int nst = (nkb + KPS - 1) / KPS;
        const int nchunks = (nkb + CHUNK - 1) / CHUNK;
        // the previous tile's epilogue must have read TMEM before it is overwritten
        if (tk > 0 && !mbar_wait_bounded(tmem_free, static_cast<uint32_t>((tk - 1) & 1))) {
          atomicOr(err, KERR_TIMEOUT_FULL);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        for (int ks = 0; ks < nst && ok; ++ks, ++g) {
          const int st = static_cast<int>(g % NSTAGE);
          if (!mbar_wait_bounded(&full[st], static_cast<uint32_t>((g / NSTAGE) & 1))) {
            atomicOr(err, KERR_TIMEOUT_FULL);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          for (int kh = 0; kh < KPS && ok; ++kh) {
            const int kb = ks * KPS + kh;
            if (kb >= nkb) break;
            const int ch = kb / CHUNK, kin = kb % CHUNK;
            const uint32_t a0 = smem_u32(sA + st * STAGE_A) + kh * (BK * 2);
            const uint32_t b0 = smem_u32(sB + st * STAGE_B) + kh * (BK * 2);
            // At a chunk boundary the tail levels (3-6) go first: they do not touch
            // the exact levels that the flush warps are still reading, so the
            // tensor pipe works while the flush runs.
            const bool boundary = (kin == 0 && ch > 0);
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
              const bool exact_pass = (pass == 1);
              if (boundary && exact_pass &&
                  !mbar_wait_bounded(chunk_empty, static_cast<uint32_t>((gc + ch - 1) & 1))) {
                atomicOr(err, KERR_TIMEOUT_FULL);
                ok = false;
                break;
              }
#pragma unroll
              for (int s = 0; s < S; ++s) {
                // Slice s of H against the slices t of the block that feed the levels
                // d = s + t of this pass, as one MMA: the B planes t are consecutive
                // rows of the B tile and the levels consecutive TMEM columns, so
                // N = 64 x (number of levels).
                const uint64_t da = desc_sw64(a0 + s * A_TILE);
                const int d0 = exact_pass ? s : (s < NEXACT ? NEXACT : s);
                const int nlev = exact_pass ? NEXACT - s : S - d0;
                if (nlev <= 0) continue;
                // first contribution to these levels in this accumulation window?
                const bool first = (s == 0) && (exact_pass ? kin == 0 : kb == 0);
                const uint32_t idn = idesc_base | ((uint32_t)((nlev * BN) >> 3) << 17);
                umma_bf16(tmem + d0 * BN, da, desc_sw64(b0 + (d0 - s) * B_TILE), idn,
                          first ? 0u : 1u);
              }
            }
            if (!ok) break;
            if (kin == CHUNK - 1 || kb == nkb - 1) umma_commit(smem_u32(chunk_full));
          }
          if (!ok) break;
          umma_commit(smem_u32(&empty[st]));
        }
        gc += nchunks;
      }
      umma_commit(smem_u32(done));  // every MMA of this CTA has completed when this fires
      if (!mbar_wait_bounded(done, 0)) atomicOr(err, KERR_TIMEOUT_FULL);
    }
  } else {
    // ---------------- flush and epilogue (warps 2..9): warp w reads TMEM
    // lanes 32 (w % 4) .. +31 (one row each) and 32 columns, half hf.
    const int q = warp & 3;
    const int hf = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    const uint32_t tbase = tmem + (static_cast<uint32_t>(q * 32) << 16) + hf * 32;
    int sums[NEXACT][32];  // exact level sums of this row, 32 columns
    bool ok = true;
    long long gc = 0;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      SplitTile T;
      tile(t, T);
      const int nchunks = (T.nkb + CHUNK - 1) / CHUNK;
      for (int ch = 0; ch < nchunks; ++ch) {
        if (!mbar_wait_bounded(chunk_full, static_cast<uint32_t>((gc + ch) & 1))) {
          if (lane == 0) atomicOr(err, KERR_TIMEOUT_FULL);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
        for (int d = 0; d < NEXACT; ++d) {
          uint32_t r[32];
          TMEM_LD32(tbase + d * BN, r);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int v = __float2int_rn(__uint_as_float(r[j]));
            sums[d][j] = (ch == 0) ? v : sums[d][j] + v;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(chunk_empty);
      }
      if (!ok) break;
      // The last chunk_full covers every MMA of the tile, tail levels included.
      split_epilogue<NS>(T, tbase, sums, row, hf);
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(tmem_free);
      gc += nchunks;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
}

// Output tiles in groups of kRasterRows row tiles: CTA b takes row tile
// (b mod the group's rows) of the group and column tile (b / the group's
// rows), so the CTAs resident at one time cover a block of about 8 row
// tiles x 19 column tiles instead of 3 x all column tiles.  Resident CTAs
// stream the same K range, so the L2 serves each operand slab to all of
// them once; the compact block cuts the distinct A and B bytes per wave,
// the DRAM traffic of a launch, by about a third at N = 8000-30000.
constexpr int kRasterRows = 8;

__device__ __forceinline__ void raster_tile(int bid, int rtiles, int ctiles, int* rt, int* ct) {
  const int per_group = kRasterRows * ctiles;
  const int g = bid / per_group;
  const int r0 = g * kRasterRows;
  const int gr = min(kRasterRows, rtiles - r0);
  const int in = bid - g * per_group;
  *rt = r0 + in % gr;
  *ct = in / gr;
}

// The tiles of one problem: a base tile description and the raster order.
struct OneProblemTiles {
  SplitTile base;
  int rtiles, ctiles;
  __device__ __forceinline__ void operator()(int t, SplitTile& T) const {
    T = base;
    int rt, ct;
    raster_tile(t, rtiles, ctiles, &rt, &ct);
    T.arow = rt * BM;
    T.brow = ct * BN;
  }
};

// One problem, persistent CTAs over its output tiles (raster_tile order); B
// map over the active block.
template <int NS>
__global__ void __launch_bounds__(kThreads, 1)
    zgemm_split_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                       const int* __restrict__ Erow, const int* __restrict__ Fcol,
                       const double* __restrict__ Dg, int M, int kb0, int nkb, int ncols, int j0,
                       const double2* __restrict__ Xsh, long long ldx, double2* __restrict__ Y,
                       long long ldy, double alpha, double beta, double shift,
                       double2* __restrict__ P, long long ldp, int cplx, int* __restrict__ err) {
  OneProblemTiles src;
  SplitTile& T = src.base;
  T.mapA = &tmA;
  T.mapB = &tmB;
  T.maps_in_global = 0;
  T.cplx = cplx;
  T.arow = 0;
  T.brow = 0;
  T.cend = ncols;
  T.joff = j0;
  T.kb0 = kb0;
  T.nkb = nkb;
  T.M = M;
  T.E = Erow;
  T.F = Fcol;
  T.Dg = Dg;
  T.X = Xsh;
  T.ldx = ldx;
  T.Y = Y;
  T.ldy = ldy;
  T.alpha = alpha;
  T.beta = beta;
  T.shift = shift;
  T.P = P;
  T.ldp = ldp;
  src.ctiles = ((cplx ? 2 : 1) * ncols + BN - 1) / BN;
  src.rtiles = (M + BM - 1) / BM;
  split_tiles_body<NS>(src, src.rtiles * src.ctiles, err);
}

// Problem of CTA `bid` in a grouped step list: the last entry with
// key <= bid (keys ascending; entry nact is the sentinel with the total).
__device__ __forceinline__ int grouped_find(const GroupedStep* __restrict__ steps, int nact, int bid,
                                            bool by_tile) {
  int lo = 0, hi = nact;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    const int key = by_tile ? steps[mid].tile0 : steps[mid].col0;
    if (key <= bid) lo = mid; else hi = mid;
  }
  return lo;
}

// The tiles of every active problem of one degree step of a grouped filter
// (tile t: the problem whose tile range holds t, found by binary search;
// within a problem the column tile runs fastest).
struct GroupedStepTiles {
  const GroupedProblem* probs;
  const GroupedStep* steps;
  int nact, parity;
  __device__ __forceinline__ void operator()(int t, SplitTile& T) const {
    const int e = grouped_find(steps, nact, t, true);
    const GroupedStep stp = steps[e];
    const GroupedProblem& pr = probs[stp.prob];
    const int local = t - stp.tile0;
    const int ncol_tiles = (2 * (pr.b - stp.s) + BN - 1) / BN;
    T.mapA = pr.mapA;
    T.mapB = pr.mapB0;
    T.maps_in_global = 1;
    T.cplx = 1;
    T.arow = (local / ncol_tiles) * BM;
    T.brow = 2 * stp.s + (local % ncol_tiles) * BN;
    T.cend = pr.b;
    T.joff = 0;
    T.kb0 = 0;
    T.nkb = static_cast<int>(pr.Kp / BK);
    T.M = pr.n;
    T.E = pr.E;
    T.F = pr.F;
    T.Dg = pr.Dg;
    T.X = parity ? pr.buf1 : pr.buf0;
    T.ldx = parity ? pr.ld1 : pr.ld0;
    T.Y = parity ? pr.buf0 : pr.buf1;
    T.ldy = parity ? pr.ld0 : pr.ld1;
    T.alpha = stp.alpha;
    T.beta = stp.beta;
    T.shift = stp.shift;
    T.P = nullptr;
    T.ldp = 0;
  }
};

// Many problems in one launch: persistent CTAs over the output tiles of
// every active problem of one degree step (problems ordered by decreasing
// N, so the longest tiles go first).
__global__ void __launch_bounds__(kThreads, 1)
    zgemm_split_grouped_kernel(const GroupedProblem* __restrict__ probs,
                               const GroupedStep* __restrict__ steps, int nact, int parity,
                               int ntiles, int* __restrict__ err) {
  GroupedStepTiles src{probs, steps, nact, parity};
  split_tiles_body<S>(src, ntiles, err);
}

// ---------------------------------------------------------------------------
// Slicing.  For |y| < 1 the slices are the 7-bit digits of y's binary
// fraction with y's sign: a_s = sign(y) floor(|y| 2^(7(s+1))) mod 128, the
// values that a = trunc(128 y), y <- 128 y - a gives (S times, every step
// exact).  They are read off the IEEE bits with integer instructions: this
// GPU's FP64 pipe is narrow, and the scaling y = v 2^-E is an exponent shift.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7FFFFFFFFFFFFFFFull;
}

// Smallest E with m < 2^E for the magnitude m with bits mb (0 for m == 0);
// the order of non-negative doubles is the order of their bit patterns.
__device__ __forceinline__ int exponent_above_bits(unsigned long long mb) {
  if (mb == 0) return 0;
  const int eb = static_cast<int>(mb >> 52);
  if (eb != 0) return eb - 1022;
  return (63 - __clzll(static_cast<long long>(mb))) - 1073;  // subnormal
}

// Digits of |v| 2^-e (< 1) into a[0..S-1], signed like v.
__device__ __forceinline__ void slice7_bits(double v, int e, float* a) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
  const int eb = static_cast<int>((bits >> 52) & 0x7FF);
  unsigned long long m = bits & ((1ull << 52) - 1);
  int ex;  // |v| = m 2^(ex - 52)
  if (eb == 0) {
    ex = -1022;
  } else {
    m |= 1ull << 52;
    ex = eb - 1023;
  }
  // F = floor(|v| 2^-e 2^49) = m 2^(ex - e - 3); |v| < 2^e keeps F < 2^49
  const int sh = e + 3 - ex;
  const unsigned long long F = sh >= 64 ? 0ull : (sh >= 0 ? (m >> sh) : (m << (-sh)));
  const float sg = (bits >> 63) ? -1.0f : 1.0f;
#pragma unroll
  for (int s = 0; s < S; ++s) a[s] = sg * static_cast<float>((F >> (42 - 7 * s)) & 127u);
}

__device__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* scratch) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < static_cast<int>((blockDim.x + 31) >> 5) ? scratch[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long x = __shfl_xor_sync(0xffffffffu, w, o);
      w = x > w ? x : w;
    }
    if (lane == 0) scratch[32] = w;
  }
  __syncthreads();
  return scratch[32];
}

// Entries of H widened to FP64 (exact for complex64 input).
__device__ __forceinline__ double2 widen2(double2 v) { return v; }
__device__ __forceinline__ double2 widen2(float2 v) {
  return make_double2(static_cast<double>(v.x), static_cast<double>(v.y));
}

// Row r of Ht from column r of the Hermitian H (complex128 or complex64):
// Re H[r, k] = Re H[k, r], Im H[r, k] = -Im H[k, r].  A: [S][N][Kp] bf16, E: [N].
template <class C2>
__device__ __forceinline__ void slice_h_row(const C2* __restrict__ col, int r, int N,
                                            __nv_bfloat16* __restrict__ A, long long Kp,
                                            int* __restrict__ E, double* __restrict__ Dg,
                                            unsigned long long* scratch) {
  unsigned long long mb = 0;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    if (k == r) continue;  // the diagonal is applied in FP64 by the epilogue
    const double2 v = widen2(col[k]);
    const unsigned long long x = abs_bits(v.x), y = abs_bits(v.y);
    mb = x > mb ? x : mb;
    mb = y > mb ? y : mb;
  }
  mb = block_max_u64(mb, scratch);
  const int er = exponent_above_bits(mb);
  if (threadIdx.x == 0) {
    E[r] = er;
    Dg[r] = widen2(col[r]).x;
  }
  const long long plane = static_cast<long long>(N) * Kp;
  __nv_bfloat16* row = A + static_cast<long long>(r) * Kp;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const double2 v = k == r ? make_double2(0.0, 0.0) : widen2(col[k]);
    float ar[S], ai[S];
    slice7_bits(v.x, er, ar);
    slice7_bits(-v.y, er, ai);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      row[s * plane + k] = __float2bfloat16_rn(ar[s]);
      row[s * plane + N + k] = __float2bfloat16_rn(ai[s]);
    }
  }
}

template <class C2>
__global__ void __launch_bounds__(256) slice_h_kernel(const C2* __restrict__ H, long long ldh,
                                                      int N, __nv_bfloat16* __restrict__ A,
                                                      long long Kp, int* __restrict__ E,
                                                      double* __restrict__ Dg) {
  __shared__ unsigned long long scratch[33];
  const int r = blockIdx.x;
  slice_h_row(H + static_cast<long long>(r) * ldh, r, N, A, Kp, E, Dg, scratch);
}

// All problems' H at once: CTA g slices global row g (problem by binary
// search over the first rows).
__global__ void __launch_bounds__(256) slice_h_grouped_kernel(const GroupedSliceH* __restrict__ probs,
                                                              int P) {
  __shared__ unsigned long long scratch[33];
  const int g = blockIdx.x;
  int lo = 0, hi = P;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (probs[mid].row0 <= g) lo = mid; else hi = mid;
  }
  const GroupedSliceH& pr = probs[lo];
  const int r = g - pr.row0;
  slice_h_row(pr.H + static_cast<long long>(r) * pr.ldh, r, pr.n,
              static_cast<__nv_bfloat16*>(pr.A), pr.Kp, pr.E, pr.Dg, scratch);
}

// Rows 2c and 2c+1 of Xt^T from column c of X (exponent to *Fc):
// r0 points at row 2c of slice plane 0 of B, planes are `plane` apart.
__device__ __forceinline__ void slice_x_col(const double2* __restrict__ col, int N,
                                            __nv_bfloat16* __restrict__ r0, long long Kp,
                                            long long plane, int* __restrict__ Fc,
                                            unsigned long long* scratch) {
  unsigned long long mb = 0;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const double2 v = col[k];
    const unsigned long long x = abs_bits(v.x), y = abs_bits(v.y);
    mb = x > mb ? x : mb;
    mb = y > mb ? y : mb;
  }
  mb = block_max_u64(mb, scratch);
  const int fc = exponent_above_bits(mb);
  if (threadIdx.x == 0) *Fc = fc;
  __nv_bfloat16* r1 = r0 + Kp;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const double2 v = col[k];
    float sr[S], si[S];
    slice7_bits(v.x, fc, sr);
    slice7_bits(v.y, fc, si);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      r0[s * plane + k] = __float2bfloat16_rn(sr[s]);
      r0[s * plane + N + k] = __float2bfloat16_rn(-si[s]);
      r1[s * plane + k] = __float2bfloat16_rn(si[s]);
      r1[s * plane + N + k] = __float2bfloat16_rn(sr[s]);
    }
  }
}

// Columns c of X in [j0, j0 + ncols) to rows 2c, 2c+1 (c relative to j0):
// B: [S][rows_cap][Kp] bf16, F: [ncols].
__global__ void __launch_bounds__(256) slice_x_kernel(const double2* __restrict__ X, long long ldx,
                                                      int N, int j0, __nv_bfloat16* __restrict__ B,
                                                      long long Kp, long long rows_cap,
                                                      int* __restrict__ F) {
  __shared__ unsigned long long scratch[33];
  const int c = blockIdx.x;
  slice_x_col(X + static_cast<long long>(j0 + c) * ldx, N, B + static_cast<long long>(2 * c) * Kp, Kp,
              rows_cap * Kp, F + c, scratch);
}

// Grouped: the active columns [s, b) of every active problem of a degree
// step, column c to rows 2c, 2c+1 of the problem's slice planes.
__global__ void __launch_bounds__(256) slice_x_grouped_kernel(const GroupedProblem* __restrict__ probs,
                                                              const GroupedStep* __restrict__ steps,
                                                              int nact, int parity) {
  __shared__ unsigned long long scratch[33];
  const int e = grouped_find(steps, nact, blockIdx.x, false);
  const GroupedStep stp = steps[e];
  const GroupedProblem& pr = probs[stp.prob];
  const int c = stp.s + (blockIdx.x - stp.col0);
  const double2* X = parity ? pr.buf1 : pr.buf0;
  const long long ldx = parity ? pr.ld1 : pr.ld0;
  __nv_bfloat16* B = static_cast<__nv_bfloat16*>(pr.Bsl);
  slice_x_col(X + static_cast<long long>(c) * ldx, pr.n, B + static_cast<long long>(2 * c) * pr.Kp,
              pr.Kp, 2LL * pr.bcap * pr.Kp, pr.F + c, scratch);
}

// Real operands (float64 or float32 H): row r of H from its column r (H
// symmetric), K = N.
template <class R>
__global__ void __launch_bounds__(256) slice_h_real_kernel(const R* __restrict__ H, long long ldh,
                                                           int N, __nv_bfloat16* __restrict__ A,
                                                           long long Kp, int* __restrict__ E,
                                                           double* __restrict__ Dg) {
  __shared__ unsigned long long scratch[33];
  const int r = blockIdx.x;
  const R* col = H + static_cast<long long>(r) * ldh;
  unsigned long long mb = 0;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    if (k == r) continue;
    const unsigned long long x = abs_bits(static_cast<double>(col[k]));
    mb = x > mb ? x : mb;
  }
  mb = block_max_u64(mb, scratch);
  const int er = exponent_above_bits(mb);
  if (threadIdx.x == 0) {
    E[r] = er;
    Dg[r] = static_cast<double>(col[r]);
  }
  const long long plane = static_cast<long long>(N) * Kp;
  __nv_bfloat16* row = A + static_cast<long long>(r) * Kp;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    float a[S];
    slice7_bits(k == r ? 0.0 : static_cast<double>(col[k]), er, a);
#pragma unroll
    for (int s = 0; s < S; ++s) row[s * plane + k] = __float2bfloat16_rn(a[s]);
  }
}

// Real block: column c of X (c in [j0, j0 + ncols)) to B row c - j0, K = N.
__global__ void __launch_bounds__(256) slice_x_real_kernel(const double* __restrict__ X, long long ldx,
                                                           int N, int j0,
                                                           __nv_bfloat16* __restrict__ B,
                                                           long long Kp, long long rows_cap,
                                                           int* __restrict__ F) {
  __shared__ unsigned long long scratch[33];
  const int c = blockIdx.x;
  const double* col = X + static_cast<long long>(j0 + c) * ldx;
  unsigned long long mb = 0;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const unsigned long long x = abs_bits(col[k]);
    mb = x > mb ? x : mb;
  }
  mb = block_max_u64(mb, scratch);
  const int fc = exponent_above_bits(mb);
  if (threadIdx.x == 0) F[c] = fc;
  const long long plane = rows_cap * Kp;
  __nv_bfloat16* row = B + static_cast<long long>(c) * Kp;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    float a[S];
    slice7_bits(col[k], fc, a);
#pragma unroll
    for (int s = 0; s < S; ++s) row[s * plane + k] = __float2bfloat16_rn(a[s]);
  }
}

// Sum of the K segments' products plus the FP64 epilogue:
// C[r, j0+c] = alpha (sum_g P_g[r, c] + (H_rr - shift) X[r, j0+c]) + beta C[r, j0+c].
template <class E>
__global__ void split_combine_kernel(const E* __restrict__ P, int nseg, long long pstride,
                                     long long ldp, const double* __restrict__ Dg,
                                     const E* __restrict__ X, long long ldx, int j0, int ncols, int N,
                                     E* __restrict__ C, long long ldc, double alpha, double beta,
                                     double shift) {
  constexpr int W = sizeof(E) / sizeof(double);  // 2 complex, 1 real
  const long long total = static_cast<long long>(N) * ncols;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(e % N);
    const int c = static_cast<int>(e / N);
    double v[W] = {};
    for (int g = 0; g < nseg; ++g) {
      const double* p = reinterpret_cast<const double*>(P + g * pstride + c * ldp + r);
#pragma unroll
      for (int w = 0; w < W; ++w) v[w] += p[w];
    }
    const long long jc = j0 + c;
    const double ds = Dg[r] - shift;
    const double* xv = reinterpret_cast<const double*>(X + jc * ldx + r);
    double* cp = reinterpret_cast<double*>(C + jc * ldc + r);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      double o = alpha * (v[w] + ds * xv[w]);
      if (beta != 0.0) o += beta * cp[w];
      cp[w] = o;
    }
  }
}

}  // namespace split

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {
int64_t k_padded(int64_t N) { return ((2 * N + split::BK - 1) / split::BK) * split::BK; }

// SMs of the current device (persistent grids: one CTA per SM)
int split_sm_count() {
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
static_assert(kSplitTileRows == split::BM && kSplitTileRealCols == split::BN &&
                  kSplitSlices == split::S && kSplitStageK == split::BX,
              "grouped tile constants");
}  // namespace

int64_t split_k_padded(int64_t N) { return k_padded(N); }

namespace {
int64_t k_padded_real(int64_t N) { return ((N + split::BK - 1) / split::BK) * split::BK; }
}  // namespace

namespace {
template <class C2>
int prepare_h_complex(Dev& d, const C2* H, int64_t N, int64_t ldh, SplitH& out) {
  out.N = N;
  out.Kp = k_padded(N);
  out.cplx = 1;
  CHASE_TRY(d.alloc_bytes(&out.A, static_cast<size_t>(split::S) * N * out.Kp * 2));
  CHASE_TRY(d.alloc(&out.E, static_cast<size_t>(N)));
  CHASE_TRY(d.alloc(&out.Dg, static_cast<size_t>(N)));
  split::slice_h_kernel<C2><<<static_cast<unsigned>(N), 256, 0, d.st>>>(
      H, ldh, static_cast<int>(N), static_cast<__nv_bfloat16*>(out.A), out.Kp, out.E, out.Dg);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class R>
int prepare_h_real(Dev& d, const R* H, int64_t N, int64_t ldh, SplitH& out) {
  out.N = N;
  out.Kp = k_padded_real(N);
  out.cplx = 0;
  CHASE_TRY(d.alloc_bytes(&out.A, static_cast<size_t>(split::S) * N * out.Kp * 2));
  CHASE_TRY(d.alloc(&out.E, static_cast<size_t>(N)));
  CHASE_TRY(d.alloc(&out.Dg, static_cast<size_t>(N)));
  split::slice_h_real_kernel<R><<<static_cast<unsigned>(N), 256, 0, d.st>>>(
      H, ldh, static_cast<int>(N), static_cast<__nv_bfloat16*>(out.A), out.Kp, out.E, out.Dg);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}
}  // namespace

int split_prepare_h(Dev& d, const chase_c64* H, int64_t N, int64_t ldh, SplitH& out) {
  return prepare_h_complex(d, reinterpret_cast<const double2*>(H), N, ldh, out);
}

int split_prepare_h(Dev& d, const chase_c32* H, int64_t N, int64_t ldh, SplitH& out) {
  return prepare_h_complex(d, reinterpret_cast<const float2*>(H), N, ldh, out);
}

int split_prepare_h(Dev& d, const double* H, int64_t N, int64_t ldh, SplitH& out) {
  return prepare_h_real(d, H, N, ldh, out);
}

int split_prepare_h(Dev& d, const float* H, int64_t N, int64_t ldh, SplitH& out) {
  return prepare_h_real(d, H, N, ldh, out);
}

int split_alloc_x(Dev& d, int64_t N, int max_cols, SplitX& out, bool cplx) {
  out.cap_cols = max_cols;
  out.cplx = cplx ? 1 : 0;
  const int64_t Kp = cplx ? k_padded(N) : k_padded_real(N);
  const int rows = cplx ? 2 * max_cols : max_cols;
  CHASE_TRY(d.alloc_bytes(&out.B, static_cast<size_t>(split::S) * rows * Kp * 2));
  CHASE_TRY(d.alloc(&out.F, static_cast<size_t>(max_cols)));
  return CHASE_OK;
}

namespace {
// K blocks one launch may cover with exact int32 level sums: level 2 holds
// 3 pairs, 3 * K * 127^2 < 2^31 gives K < 44380.
constexpr int kMaxKBlocksPerSegment = 44000 / split::BK;

// K blocks one launch streams at most (K = 16000).  Resident CTAs share
// operand slabs in L2 only while their K positions stay close, and they
// drift apart over a tile's K range: at K = 30000 per launch (N = 30000,
// 1500 columns) a launch read 18x its algorithmic bytes from DRAM, at
// K = 16000 (N = 8000) 4.6x.  Longer products therefore run as K segments
// of at most this length, their FP64 partial products summed by the
// combine kernel.
constexpr int kStreamKBlocks = 1000;

// nkb K blocks, `tiles` output tiles per segment
int segments_for(int64_t nkb, int64_t tiles) {
  const int64_t cap = std::min<int64_t>(kMaxKBlocksPerSegment, kStreamKBlocks);
  int nseg = static_cast<int>((nkb + cap - 1) / cap);
  // Narrow blocks leave SMs idle: split K until the grid covers the SMs,
  // keeping every segment at least 64 K blocks long.  (Splitting wider
  // grids to trim the last wave costs more in the combine pass and the
  // extra epilogues than it recovers: measured on the N = 8000 solve.)
  while (tiles * nseg < 152 && nkb / (nseg + 1) >= 64 && nseg < 8) ++nseg;
  return nseg;
}

// The split product for complex (E = double2) or real (E = double) operands
// with the leading NS slices of each operand.
template <int NS, class E>
int split_product_ns(Dev& d, const SplitH& h, SplitX& x, const E* X, int64_t ldx, int j0, int j1,
                     E* C, int64_t ldc, double alpha, double beta, double shift) {
  using SC = split::Slices<NS>;
  constexpr bool cplx = sizeof(E) == 16;
  const int ncols = j1 - j0;
  if (ncols <= 0) return CHASE_OK;
  if (ncols > x.cap_cols || h.cplx != (cplx ? 1 : 0) || x.cplx != h.cplx) {
    set_error("split product: %d columns for a workspace of %d, or mixed real/complex slices",
              ncols, x.cap_cols);
    return CHASE_INVALID_ARG;
  }
  const int64_t N = h.N, Kp = h.Kp;
  const int64_t K = cplx ? 2 * N : N;            // real K extent of the product
  const int64_t rows_cap = cplx ? 2LL * x.cap_cols : x.cap_cols;
  const int64_t brows = cplx ? 2LL * ncols : ncols;  // B-map rows of the active block
  if constexpr (cplx)
    split::slice_x_kernel<<<static_cast<unsigned>(ncols), 256, 0, d.st>>>(
        X, ldx, static_cast<int>(N), j0, static_cast<__nv_bfloat16*>(x.B), Kp, rows_cap, x.F);
  else
    split::slice_x_real_kernel<<<static_cast<unsigned>(ncols), 256, 0, d.st>>>(
        X, ldx, static_cast<int>(N), j0, static_cast<__nv_bfloat16*>(x.B), Kp, rows_cap, x.F);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  CUtensorMap tmA, tmB;
  // the maps read the leading NS slice planes
  CHASE_TRY(make_tmap_bf16_3d(&tmA, h.A, K, N, split::S, Kp * 2, Kp * 2 * N, split::BX, split::BM,
                              NS));
  CHASE_TRY(make_tmap_bf16_3d(&tmB, x.B, K, brows, split::S, Kp * 2, Kp * 2 * rows_cap, split::BX,
                              split::BN, NS));
  // once per instantiation; function-local static initialisation is thread safe
  static const cudaError_t attr_rc = cudaFuncSetAttribute(
      split::zgemm_split_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, SC::SMEM);
  CHASE_CUDA(attr_rc);
  const int64_t ctiles = (brows + split::BN - 1) / split::BN;
  const int64_t rtiles = (N + split::BM - 1) / split::BM;
  // persistent CTAs, one per SM at most (raster_tile orders the tiles)
  dim3 grid(static_cast<unsigned>(std::min<int64_t>(ctiles * rtiles, split_sm_count())));
  const int nkb = static_cast<int>(Kp / split::BK);
  const int nseg = segments_for(nkb, ctiles * rtiles);
  const double2* Xd = reinterpret_cast<const double2*>(X);
  double2* Cd = reinterpret_cast<double2*>(C);
  // algorithmic FLOPs (8 N^2 per complex column, 2 N^2 per real one) and the
  // BF16 tensor FLOPs of the NS (NS + 1) / 2 slice pairs
  const double alg = (cplx ? 8.0 : 2.0) * static_cast<double>(N) * static_cast<double>(N) * ncols;
  const double pairs = NS * (NS + 1) / 2.0;
  if (nseg == 1) {
    KernelTimer kt(d.st, CHASE_TIMED_SPLIT_PRODUCT);
    split::zgemm_split_kernel<NS><<<grid, split::kThreads, SC::SMEM, d.st>>>(
        tmA, tmB, h.E, x.F, h.Dg, static_cast<int>(N), 0, nkb, ncols, j0, Xd, ldx, Cd, ldc, alpha,
        beta, shift, nullptr, 0, cplx ? 1 : 0, d.err);
    note_launch();
    CHASE_CUDA(cudaGetLastError());
    kt.end(1, alg, pairs * alg);
    return CHASE_OK;
  }
  // K segments write raw partial products; the combine kernel sums them and
  // applies the diagonal, the shift and the axpby in FP64.
  const long long pstride = static_cast<long long>(N) * ncols;  // elements of E
  const size_t need = static_cast<size_t>(pstride) * nseg * sizeof(E) / sizeof(double2) + 1;
  if (need > x.P_cap) {  // grow-only: released with the call's other workspace
    void* np = nullptr;
    CHASE_TRY(d.alloc_bytes(&np, std::max(need, 2 * x.P_cap) * sizeof(double2)));
    x.P = np;
    x.P_cap = std::max(need, 2 * x.P_cap);
  }
  E* P = static_cast<E*>(x.P);
  int per = (nkb + nseg - 1) / nseg;
  per = (per + split::KPS - 1) / split::KPS * split::KPS;  // segments start on stage boundaries
  KernelTimer kt(d.st, CHASE_TIMED_SPLIT_PRODUCT);
  int launched = 0;
  for (int g = 0; g < nseg; ++g) {
    const int kb0 = g * per;
    const int cnt = std::min(per, nkb - kb0);
    if (cnt <= 0) break;
    split::zgemm_split_kernel<NS><<<grid, split::kThreads, SC::SMEM, d.st>>>(
        tmA, tmB, h.E, x.F, h.Dg, static_cast<int>(N), kb0, cnt, ncols, j0, Xd, ldx, Cd, ldc,
        alpha, beta, shift, reinterpret_cast<double2*>(P + g * pstride), N, cplx ? 1 : 0, d.err);
    note_launch();
    CHASE_CUDA(cudaGetLastError());
    ++launched;
  }
  kt.end(launched, alg, pairs * alg);
  const long long total = pstride;
  const unsigned blocks = static_cast<unsigned>(std::min<long long>((total + 255) / 256, 152 * 16));
  split::split_combine_kernel<E><<<blocks, 256, 0, d.st>>>(P, nseg, pstride, N, h.Dg, X, ldx, j0,
                                                           ncols, static_cast<int>(N), C, ldc,
                                                           alpha, beta, shift);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

template <class E>
int split_product(Dev& d, const SplitH& h, SplitX& x, const E* X, int64_t ldx, int j0, int j1, E* C,
                  int64_t ldc, double alpha, double beta, double shift, int nslices) {
  switch (nslices) {
    case 3:
      return split_product_ns<3>(d, h, x, X, ldx, j0, j1, C, ldc, alpha, beta, shift);
    case 4:
      return split_product_ns<4>(d, h, x, X, ldx, j0, j1, C, ldc, alpha, beta, shift);
    case 7:
      return split_product_ns<7>(d, h, x, X, ldx, j0, j1, C, ldc, alpha, beta, shift);
    default:
      set_error("split product: %d slices (3, 4 or 7 supported)", nslices);
      return CHASE_INVALID_ARG;
  }
}
}  // namespace

int zgemm_split(Dev& d, const SplitH& h, SplitX& x, const chase_c64* X, int64_t ldx, int j0, int j1,
                chase_c64* C, int64_t ldc, double alpha, double beta, double shift, int nslices) {
  return split_product(d, h, x, reinterpret_cast<const double2*>(X), ldx, j0, j1,
                       reinterpret_cast<double2*>(C), ldc, alpha, beta, shift, nslices);
}

int zgemm_split(Dev& d, const SplitH& h, SplitX& x, const double* X, int64_t ldx, int j0, int j1,
                double* C, int64_t ldc, double alpha, double beta, double shift, int nslices) {
  return split_product(d, h, x, X, ldx, j0, j1, C, ldc, alpha, beta, shift, nslices);
}

int split_grouped_prepare_h(Dev& d, const GroupedSliceH* probs, int P, int total_rows) {
  if (total_rows <= 0) return CHASE_OK;
  split::slice_h_grouped_kernel<<<static_cast<unsigned>(total_rows), 256, 0, d.st>>>(probs, P);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

int split_grouped_slice_x(Dev& d, const GroupedProblem* probs, const GroupedStep* steps, int nact,
                          int ncols, int parity) {
  if (ncols <= 0) return CHASE_OK;
  split::slice_x_grouped_kernel<<<static_cast<unsigned>(ncols), 256, 0, d.st>>>(probs, steps, nact,
                                                                                 parity);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

int zgemm_split_grouped_prepare() {
  // once per instantiation; function-local static initialisation is thread safe
  static const cudaError_t attr_rc = cudaFuncSetAttribute(
      split::zgemm_split_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, split::SMEM);
  CHASE_CUDA(attr_rc);
  return CHASE_OK;
}

int zgemm_split_grouped(Dev& d, const GroupedProblem* probs, const GroupedStep* steps, int nact,
                        int ntiles, int parity) {
  if (ntiles <= 0) return CHASE_OK;
  CHASE_TRY(zgemm_split_grouped_prepare());
  split::zgemm_split_grouped_kernel<<<static_cast<unsigned>(std::min(ntiles, split_sm_count())),
                                      split::kThreads, split::SMEM, d.st>>>(probs, steps, nact,
                                                                          parity, ntiles, d.err);
  note_launch();
  CHASE_CUDA(cudaGetLastError());
  return CHASE_OK;
}

}  // namespace chase
