// Host runtime of libchase: error strings, tensor maps, device context,
// pointer kinds and block copies.
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "context.hpp"

namespace chase {

namespace {
thread_local char g_err[512] = "";
std::atomic<long long> g_launches{0};
std::atomic<long long> g_allocs{0};
}

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int cuda_status(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return CHASE_OUT_OF_MEMORY;
  return CHASE_CUDA_ERROR;
}

// ---------------------------------------------------------------------------
// Tensor maps (driver entry point fetched through the runtime, so the library
// needs no link-time dependency on libcuda)
// ---------------------------------------------------------------------------
namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
std::once_flag g_encode_once;
}  // namespace

namespace {
EncodeTiledFn encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  });
  return g_encode;
}

// 2-D float64 tensor {d0, d1} with row stride ld_bytes, box {b0, b1}.
int make_tmap_2d_f64(CUtensorMap* map, const void* base, int64_t d0, int64_t d1, int64_t ld_bytes,
                     int b0, int b1) {
  EncodeTiledFn enc = encoder();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return CHASE_CUDA_ERROR;
  }
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) {
    set_error("TMA operand base address is not 16-byte aligned");
    return CHASE_INVALID_ARG;
  }
  if ((ld_bytes & 15) != 0) {
    set_error("TMA operand leading dimension is not a multiple of 16 bytes");
    return CHASE_INVALID_ARG;
  }
  cuuint64_t gdim[2] = {static_cast<cuuint64_t>(d0), static_cast<cuuint64_t>(d1)};
  cuuint64_t gstride[1] = {static_cast<cuuint64_t>(ld_bytes)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(b0), static_cast<cuuint32_t>(b1)};
  cuuint32_t estride[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(base), gdim, gstride,
                   box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) dims=%lldx%lld ld=%lld B box=%dx%d", (int)r,
              (long long)d0, (long long)d1, (long long)ld_bytes, b0, b1);
    return CHASE_INVALID_ARG;
  }
  return CHASE_OK;
}
}  // namespace

int make_tmap_c64(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
                  int box_rows, int box_cols) {
  return make_tmap_2d_f64(map, base, 2 * rows, cols, ld * 16, 2 * box_rows, box_cols);
}

int make_tmap_f64(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
                  int box_rows, int box_cols) {
  return make_tmap_2d_f64(map, base, rows, cols, ld * 8, box_rows, box_cols);
}

int make_tmap_bf16_3d(CUtensorMap* map, const void* base, int64_t d0, int64_t d1, int64_t d2,
                      int64_t s1, int64_t s2, int b0, int b1, int b2) {
  EncodeTiledFn enc = encoder();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return CHASE_CUDA_ERROR;
  }
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (s1 & 15) != 0 || (s2 & 15) != 0 ||
      (b0 * 2 != 32 && b0 * 2 != 64)) {
    set_error("bf16 tensor map: misaligned base/stride or box");
    return CHASE_INVALID_ARG;
  }
  cuuint64_t gdim[3] = {static_cast<cuuint64_t>(d0), static_cast<cuuint64_t>(d1),
                        static_cast<cuuint64_t>(d2)};
  cuuint64_t gstride[2] = {static_cast<cuuint64_t>(s1), static_cast<cuuint64_t>(s2)};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(b0), static_cast<cuuint32_t>(b1),
                       static_cast<cuuint32_t>(b2)};
  cuuint32_t estride[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), gdim, gstride,
                   box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   b0 * 2 == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (bf16 3-D) failed (%d)", (int)r);
    return CHASE_INVALID_ARG;
  }
  return CHASE_OK;
}

// ---------------------------------------------------------------------------
// Device context
// ---------------------------------------------------------------------------
Dev::~Dev() {
  for (void* p : bufs) cudaFreeAsync(p, st);
  if (err && own_err) cudaFreeAsync(err, st);
  if (sync_on_exit) cudaStreamSynchronize(st);
}

int Dev::init() {
  void* p = nullptr;
  g_allocs.fetch_add(1, std::memory_order_relaxed);
  CHASE_CUDA(cudaMallocAsync(&p, sizeof(int), st));
  err = static_cast<int*>(p);
  CHASE_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  return CHASE_OK;
}

int Dev::alloc_bytes(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return CHASE_OK;
  g_allocs.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaMallocAsync(p, bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device workspace allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    *p = nullptr;
    return CHASE_OUT_OF_MEMORY;
  }
  bufs.push_back(*p);
  return CHASE_OK;
}

int Dev::sync_check(const char* where) {
  int h = 0;
  CHASE_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, where);
  if (h & (KERR_TIMEOUT_FULL | KERR_TIMEOUT_EMPTY)) {
    set_error("%s: a bounded wait in a kernel gave up (flags 0x%x)", where, h);
    return CHASE_TIMEOUT;
  }
  if (h & KERR_BAD_DEGREE) {
    set_error("%s: degrees must be even and in [2, 1024]", where);
    return CHASE_INVALID_ARG;
  }
  if (h & KERR_CHOL_BREAKDOWN) {
    set_error("%s: Cholesky breakdown", where);
    return CHASE_QR_BREAKDOWN;
  }
  return CHASE_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

namespace {
int copy_block_bytes(Dev& d, void* dst, int64_t ldd, const void* src, int64_t lds, int64_t rows,
                     int64_t cols, size_t es, cudaMemcpyKind kind) {
  if (rows == 0 || cols == 0) return CHASE_OK;
  CHASE_CUDA(cudaMemcpy2DAsync(dst, static_cast<size_t>(ldd) * es, src, static_cast<size_t>(lds) * es,
                               static_cast<size_t>(rows) * es, static_cast<size_t>(cols), kind,
                               d.st));
  return CHASE_OK;
}
}  // namespace

int copy_block(Dev& d, chase_c64* dst, int64_t ldd, const chase_c64* src, int64_t lds, int64_t rows,
               int64_t cols, cudaMemcpyKind kind) {
  return copy_block_bytes(d, dst, ldd, src, lds, rows, cols, sizeof(chase_c64), kind);
}

int copy_block(Dev& d, double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows,
               int64_t cols, cudaMemcpyKind kind) {
  return copy_block_bytes(d, dst, ldd, src, lds, rows, cols, sizeof(double), kind);
}

int copy_block(Dev& d, chase_c32* dst, int64_t ldd, const chase_c32* src, int64_t lds, int64_t rows,
               int64_t cols, cudaMemcpyKind kind) {
  return copy_block_bytes(d, dst, ldd, src, lds, rows, cols, sizeof(chase_c32), kind);
}

int copy_block(Dev& d, float* dst, int64_t ldd, const float* src, int64_t lds, int64_t rows,
               int64_t cols, cudaMemcpyKind kind) {
  return copy_block_bytes(d, dst, ldd, src, lds, rows, cols, sizeof(float), kind);
}

// ---------------------------------------------------------------------------
// Kernel timing for benchmarks: event pairs on the launching stream around
// the product launches, read back (and destroyed) by chase_kernel_timing_read
// ---------------------------------------------------------------------------
namespace {
struct TimedRange {
  int kind;
  cudaEvent_t a, b;
  long long launches;
  double flops, tensor_flops;
};
std::mutex g_timing_mu;
std::atomic<bool> g_timing_on{false};
std::vector<TimedRange> g_timed;

void clear_timed_locked() {
  for (auto& r : g_timed) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_timed.clear();
}
}  // namespace

KernelTimer::KernelTimer(cudaStream_t s, int kind) : st_(s), kind_(kind) {
  if (!g_timing_on.load(std::memory_order_relaxed)) return;
  if (cudaEventCreate(&a_) != cudaSuccess || cudaEventCreate(&b_) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  active_ = cudaEventRecord(a_, st_) == cudaSuccess;
}

void KernelTimer::end(long long launches, double flops, double tensor_flops) {
  if (!active_) return;
  active_ = false;
  if (cudaEventRecord(b_, st_) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(a_);
    cudaEventDestroy(b_);
    return;
  }
  std::lock_guard<std::mutex> lk(g_timing_mu);
  g_timed.push_back({kind_, a_, b_, launches, flops, tensor_flops});
}

KernelTimer::~KernelTimer() {
  if (active_) {  // left by an error path: discard
    cudaEventDestroy(a_);
    cudaEventDestroy(b_);
  }
}

}  // namespace chase

extern "C" int chase_kernel_timing(int enable) {
  std::lock_guard<std::mutex> lk(chase::g_timing_mu);
  if (enable) chase::clear_timed_locked();
  chase::g_timing_on.store(enable != 0, std::memory_order_relaxed);
  return CHASE_OK;
}

extern "C" int chase_kernel_timing_read(int kind, double* seconds, long long* launches,
                                        double* flops, double* tensor_flops) {
  if (kind < 0 || kind >= CHASE_TIMED_KINDS || !seconds || !launches) {
    chase::set_error("chase_kernel_timing_read: invalid argument");
    return CHASE_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(chase::g_timing_mu);
  double s = 0.0, f = 0.0, tf = 0.0;
  long long n = 0;
  for (auto& r : chase::g_timed) {
    if (r.kind != kind) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return chase::cuda_status(cudaGetLastError(), "chase_kernel_timing_read");
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
      return chase::cuda_status(cudaGetLastError(), "chase_kernel_timing_read");
    s += 1e-3 * ms;
    n += r.launches;
    f += r.flops;
    tf += r.tensor_flops;
  }
  *seconds = s;
  *launches = n;
  if (flops) *flops = f;
  if (tensor_flops) *tensor_flops = tf;
  return CHASE_OK;
}

extern "C" const char* chase_last_error(void) { return chase::g_err; }

extern "C" long long chase_device_allocations(void) {
  return chase::g_allocs.load(std::memory_order_relaxed);
}

extern "C" long long chase_kernel_launches(void) {
  return chase::g_launches.load(std::memory_order_relaxed);
}
