// dmpt_sp2_response_static: the response solve for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc or hand over a workspace: code that
// runs inside a host framework owning every device allocation (and forbidding
// others), code that must not allocate after start-up so its memory use stays
// fixed, or plug-ins that only receive input and output pointers.  This entry
// point takes its scratch space from one file-scope device array of fixed size
// instead of a caller workspace, so it allocates nothing.
//
// The array, g_dmpt_static_scratch, holds DMPT_STATIC_SCRATCH_BYTES and is
// loaded on every GPU that loads the library; it stays resident until the
// process exits.  It covers n <= DMPT_STATIC_MAX_N and k <= DMPT_STATIC_MAX_K
// in every precision.
//
// In host code the array's name is only a host-side stand-in, not a device
// address.  The device address is obtained once per device with
// cudaGetSymbolAddress, with that device current, on the first call on that
// device; that first call should therefore come before any stream capture.
// All calls share the array and it keeps the previous call's contents; the
// solve clears (or fully overwrites) everything it reads before reading it.
// Calls that overlap on the GPU (other streams, other host threads) race on
// the array and must be serialised by the caller.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "dmpt_internal.cuh"

static __device__ __align__(256) unsigned char g_dmpt_static_scratch[DMPT_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `dev` (looked up once per device).
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_addr[dev]) {
    *out = g_addr[dev];
    return cudaSuccess;
  }
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return e;
  if (prev != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return e;
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_dmpt_static_scratch);
  if (prev != dev) cudaSetDevice(prev);
  if (e != cudaSuccess) return e;
  g_addr[dev] = p;
  *out = p;
  return cudaSuccess;
}

}  // namespace

extern "C" dmpt_status dmpt_sp2_response_static(dmpt_handle h, const double* H,
                                                const double* H1, int k, int64_t n, int64_t ld,
                                                int64_t n_occ, const dmpt_options* o, double* P,
                                                double* P1, dmpt_info* info, void* stream) {
  if (!h) return DMPT_EINVAL;
  if (n > DMPT_STATIC_MAX_N || k > DMPT_STATIC_MAX_K) {
    if (info) info->status = DMPT_EINVAL;
    fprintf(stderr,
            "dmpt_sp2_response_static: n = %lld, k = %d exceeds the static scratch limit "
            "(n <= %d, k <= %d); use dmpt_sp2_response with a workspace\n",
            (long long)n, k, DMPT_STATIC_MAX_N, DMPT_STATIC_MAX_K);
    return DMPT_EINVAL;
  }
  if (o && o->timing) return DMPT_EUNSUPPORTED;  // timing would create CUDA events
  const int dev = dmpt::handle_device(h);
  if (dev < 0 || dev >= kMaxDevices) return DMPT_EINVAL;
  dmpt_options d;
  dmpt_default_options(&d);
  const size_t need = dmpt_workspace_size(n < 1 ? 1 : n, k < 1 ? 1 : k, o ? o : &d);
  if (need > sizeof(g_dmpt_static_scratch)) return DMPT_EINVAL;
  void* ws = nullptr;
  if (scratch_address(dev, &ws) != cudaSuccess) return DMPT_ECUDA;
  return dmpt_sp2_response(h, H, H1, k, n, ld, n_occ, o, P, P1, info, ws,
                           sizeof(g_dmpt_static_scratch), stream);
}
