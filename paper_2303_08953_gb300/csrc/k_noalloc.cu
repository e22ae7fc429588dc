// Allocation-free block dot product W = Q^T X.
//
// Some callers cannot call cudaMalloc: services and frameworks that hand
// all device memory out through their own pool allocator and forbid direct
// allocations, programs that fix their device-memory budget at start-up,
// and code paths that must not add the device-wide synchronisation that
// cudaFree implies.  For them, sg_block_dot_noalloc computes the same
// product as sg_block_dot with no handle and no allocation: the split
// partial sums of the reduction live in a file-scope device array of fixed
// size, which every GPU that loads this library holds until the process
// exits.
//
// The array's name is only a host-side stand-in in host code, so the
// device address is looked up with cudaGetSymbolAddress once per device,
// with that device current, on the first call made on it.
#include <cstdio>
#include <mutex>

#include "sg_internal.h"

namespace {

constexpr int64_t kScratchDoubles = SG_NOALLOC_SCRATCH_DOUBLES;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

void put_err(char* err, int32_t cap, const char* msg) {
  if (err && cap > 0) std::snprintf(err, static_cast<size_t>(cap), "%s", msg);
}

}  // namespace

extern "C" sg_status sg_block_dot_noalloc(int64_t n, const double* Q,
                                          int64_t ldq, int32_t i,
                                          const double* X, int64_t ldx,
                                          int32_t s, double* W, int32_t ldw,
                                          void* stream, char* err,
                                          int32_t err_cap) {
  put_err(err, err_cap, "");
  if (n < 0 || i < 0 || s < 0 || ldq < n || ldx < n || ldw < i) {
    put_err(err, err_cap, "sg_block_dot_noalloc: bad sizes or leading dimensions");
    return SG_EINVAL;
  }
  if (static_cast<int64_t>(i) * s > kScratchDoubles) {
    char msg[200];
    std::snprintf(msg, sizeof(msg),
                  "sg_block_dot_noalloc: i*s = %lld exceeds the scratch of %lld "
                  "entries (SG_NOALLOC_SCRATCH_DOUBLES)",
                  static_cast<long long>(i) * s, static_cast<long long>(kScratchDoubles));
    put_err(err, err_cap, msg);
    return SG_EINVAL;
  }
  if (i == 0 || s == 0) return SG_OK;
  if (!Q || !X || !W) {
    put_err(err, err_cap, "sg_block_dot_noalloc: null pointer");
    return SG_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    put_err(err, err_cap, "sg_block_dot_noalloc: no usable current device");
    return SG_ECUDA;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        char msg[200];
        std::snprintf(msg, sizeof(msg), "sg_block_dot_noalloc: cudaGetSymbolAddress: %s",
                      cudaGetErrorString(e));
        put_err(err, err_cap, msg);
        return SG_ECUDA;
      }
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  try {
    sg::block_dot_capped(n, Q, ldq, i, X, ldx, s, W, ldw, scratch,
                         kScratchDoubles, static_cast<cudaStream_t>(stream));
  } catch (const sg::Error& e) {
    put_err(err, err_cap, e.what());
    return e.code;
  }
  return SG_OK;
}
