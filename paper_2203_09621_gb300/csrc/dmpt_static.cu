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
// in every precision, without the S0 tape (ckpt_every = 0).
//
// In host code the array's name is only a host-side stand-in, not a device
// address.  The device address is obtained with cudaGetSymbolAddress, with
// the device current, on the first call on that device (and again when the
// device's context has been replaced, e.g. after cudaDeviceReset); that first
// call should therefore come before any stream capture.
// All calls share the array and it keeps the previous call's contents; the
// solve clears (or fully overwrites) everything it reads before reading it.
// Calls that overlap on the GPU (other streams, other host threads) race on
// the array and must be serialised by the caller.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "dmpt_internal.cuh"

static __device__ __align__(256) unsigned char g_dmpt_static_scratch[DMPT_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};
CUcontext g_ctx[kMaxDevices] = {nullptr};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

// cuCtxGetCurrent through the runtime's driver entry-point lookup (the
// library does not link libcuda); NULL when unavailable.
CtxGetCurrentFn ctx_get_current() {
  static const CtxGetCurrentFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<CtxGetCurrentFn>(p);
    return (CtxGetCurrentFn) nullptr;
  }();
  return fn;
}

// Device address of the scratch array on `dev`, looked up with `dev` current
// once per device and context.  The caller has made `dev` current.
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  CUcontext ctx = nullptr;
  CtxGetCurrentFn get = ctx_get_current();
  if (get && get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  if (g_addr[dev] && ctx && ctx == g_ctx[dev]) {
    *out = g_addr[dev];
    return cudaSuccess;
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_dmpt_static_scratch);
  if (e != cudaSuccess) return e;
  g_addr[dev] = p;
  g_ctx[dev] = ctx;   // NULL (no driver lookup): looked up again on every call
  *out = p;
  return cudaSuccess;
}

dmpt_status refuse(dmpt_handle h, dmpt_info* info, dmpt_status s, const char* msg) {
  if (info) info->status = s;
  fprintf(stderr, "dmpt_sp2_response_static: %s\n", msg);
  return dmpt::report(h, s, msg);
}

}  // namespace

extern "C" dmpt_status dmpt_sp2_response_static(dmpt_handle h, const double* H,
                                                const double* H1, int k, int64_t n, int64_t ld,
                                                int64_t n_occ, const dmpt_options* o, double* P,
                                                double* P1, dmpt_info* info, void* stream) {
  if (info) memset(info, 0, sizeof(*info));
  if (!h) {
    if (info) info->status = DMPT_EINVAL;
    return DMPT_EINVAL;
  }
  char msg[256];
  if (n > DMPT_STATIC_MAX_N || k > DMPT_STATIC_MAX_K) {
    snprintf(msg, sizeof(msg),
             "n = %lld, k = %d exceeds the static scratch limit (n <= %d, k <= %d); use "
             "dmpt_sp2_response with a workspace",
             (long long)n, k, DMPT_STATIC_MAX_N, DMPT_STATIC_MAX_K);
    return refuse(h, info, DMPT_EINVAL, msg);
  }
  if (o && o->timing)
    return refuse(h, info, DMPT_EUNSUPPORTED, "timing = 1 is not supported (it creates CUDA events)");
  if (o && o->autotune)
    return refuse(h, info, DMPT_EUNSUPPORTED,
                  "autotune = 1 is not supported (tuning creates CUDA events and runs probe "
                  "solves); pass the tuned fields instead");
  if (o && o->ckpt_every)
    return refuse(h, info, DMPT_EUNSUPPORTED,
                  "ckpt_every = 1 is not supported: the static scratch keeps no S0 tape, so "
                  "dmpt_sp2_backward cannot follow this call");
  const int dev = dmpt::handle_device(h);
  if (dev < 0 || dev >= kMaxDevices) return refuse(h, info, DMPT_EINVAL, "device out of range");
  dmpt_options d;
  dmpt_default_options(&d);
  const size_t need = dmpt_workspace_size(n < 1 ? 1 : n, k < 1 ? 1 : k, o ? o : &d);
  if (need == 0) return refuse(h, info, DMPT_EINVAL, "invalid arguments or options");
  if (need > sizeof(g_dmpt_static_scratch)) {
    snprintf(msg, sizeof(msg), "needs %zu bytes of scratch, more than the %zu of the static array",
             need, sizeof(g_dmpt_static_scratch));
    return refuse(h, info, DMPT_EINVAL, msg);
  }
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != dev) e = cudaSetDevice(dev);
  void* ws = nullptr;
  if (e == cudaSuccess) e = scratch_address(dev, &ws);
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "scratch address lookup: %s", cudaGetErrorString(e));
    return refuse(h, info, DMPT_ECUDA, msg);
  }
  return dmpt_sp2_response(h, H, H1, k, n, ld, n_occ, o, P, P1, info, ws,
                           sizeof(g_dmpt_static_scratch), stream);
}
