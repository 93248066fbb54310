// Allocation-free residual norms: chase_residuals_noalloc.
//
// Some callers cannot let a library allocate device memory.  A host
// framework that owns every byte of device memory through its own pool
// (and budgets it) breaks when a library calls cudaMalloc behind its back,
// and cudaMalloc / cudaFree may synchronise the whole device, which a
// latency-critical caller running other streams concurrently cannot
// tolerate.  For them this entry point computes the same residual norms as
// chase_residuals with no allocation at all: the product H V is staged in a
// fixed scratch array that lives in the library's own device image.
//
// Scratch: `g_noalloc_scratch`, a file-scope __device__ array of
// kNoAllocMaxElems complex128 entries (32 MiB) plus an error flag.  Every GPU
// that loads the library holds it until the process exits.  Its address is
// looked up once per device (cudaGetSymbolAddress, with that device current)
// on the first call made on that device; that first call should therefore
// come before any CUDA stream capture.  All calls share the array and it
// keeps the last call's contents: the error flag is cleared on every call,
// and the H V staging area is fully overwritten before it is read.  Calls
// whose work overlaps on the GPU (different streams, or different host
// threads on one device) race on the array.  The cached address assumes the
// device's context lives as long as the process: after a cudaDeviceReset by
// the application it is stale, so this entry point must not be used again
// on that device in that process.
#include <mutex>

#include "common.cuh"
#include "context.hpp"

namespace chase {
namespace {

constexpr size_t kNoAllocMaxElems = size_t(2) << 20;  // complex128 entries of H V (32 MiB)
constexpr size_t kNoAllocFlagOffset = kNoAllocMaxElems * sizeof(double2);
constexpr size_t kNoAllocBytes = kNoAllocFlagOffset + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_scratch_mu;
constexpr int kMaxDevices = 256;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.
int scratch_address(void** out) {
  int dev = 0;
  CHASE_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("chase_residuals_noalloc: device ordinal %d out of range", dev);
    return CHASE_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return CHASE_OK;
}

// The error flag of this entry point lives in the static array, not in the
// allocation pool: detach it from the context before the context releases
// its (empty) workspace.
struct FlagDetach {
  Dev& d;
  ~FlagDetach() { d.err = nullptr; }
};

}  // namespace
}  // namespace chase

using namespace chase;

extern "C" int chase_residuals_noalloc(const chase_c64* H, int64_t N, int64_t ldh,
                                       const chase_c64* V, int64_t ldv, int b,
                                       const double* lambda, double* resid, void* stream) {
  if (N < 0 || b < 0 || ldh < (N > 0 ? N : 1) || ldv < (N > 0 ? N : 1)) {
    set_error("chase_residuals_noalloc: invalid size or leading dimension");
    return CHASE_INVALID_ARG;
  }
  if (N == 0 || b == 0) return CHASE_OK;
  // N b <= max without forming the product (which could wrap for a huge N)
  if (static_cast<size_t>(N) > kNoAllocMaxElems / static_cast<size_t>(b)) {
    set_error("chase_residuals_noalloc: N*b exceeds the fixed scratch of %zu entries (N = %lld, "
              "b = %d)", kNoAllocMaxElems, static_cast<long long>(N), b);
    return CHASE_INVALID_ARG;
  }
  if (!H || !V || !lambda || !resid || !is_device_ptr(H) || !is_device_ptr(V) ||
      !is_device_ptr(lambda) || !is_device_ptr(resid)) {
    set_error("chase_residuals_noalloc: H, V, lambda and resid must be device arrays");
    return CHASE_INVALID_ARG;
  }
  // the scratch looked up below belongs to the current device: every array
  // must live there too
  {
    int cur = 0;
    CHASE_CUDA(cudaGetDevice(&cur));
    for (const void* p : {static_cast<const void*>(H), static_cast<const void*>(V),
                          static_cast<const void*>(lambda), static_cast<const void*>(resid)}) {
      cudaPointerAttributes a;
      CHASE_CUDA(cudaPointerGetAttributes(&a, p));
      if (a.device != cur) {
        set_error("chase_residuals_noalloc: an array lives on device %d, the current device is "
                  "%d", a.device, cur);
        return CHASE_INVALID_ARG;
      }
    }
  }
  void* base = nullptr;
  CHASE_TRY(scratch_address(&base));
  chase_c64* HV = static_cast<chase_c64*>(base);
  Dev d(stream);
  FlagDetach detach{d};
  d.err = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + kNoAllocFlagOffset);
  CHASE_CUDA(cudaMemsetAsync(d.err, 0, sizeof(int), d.st));
  CHASE_TRY(zgemm(d, N, N, H, ldh, V, ldv, b, HV, N, 0, b, 1.0, 0.0, 0.0));
  CHASE_TRY(launch_resid_norms(d, HV, N, V, ldv, N, b, lambda, resid));
  return d.sync_check("chase_residuals_noalloc");
}
