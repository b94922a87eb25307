// hopu_apply_convection_noalloc: the convection apply with its scratch in a static
// device buffer, for callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a region whose
// device memory is owned and accounted by the caller's own pool (a memory budget that
// must not grow behind its back), in a process that pre-reserves all device memory at
// start-up, or in a library-in-a-library setting where only the host application may
// allocate.  hopu_apply_convection keeps per-context scratch that hopu_create
// allocated; this entry point uses none of it.  It needs a context for the mesh and the
// reference tables, created once during set-up, and the caller's input and output
// vectors; the two scratch arrays of the apply (the wind projected to L2 and the
// element-major facet moments) live in the file-scope array below instead.
//
// The array is part of the library image: every GPU that loads libhopu holds
// kNoAllocScratchBytes of device memory until the process exits.  Every call shares it
// and it keeps the contents of the last call; nothing in it has to start at zero (both
// scratch arrays are overwritten completely by every call).  Calls that overlap on the
// GPU -- two streams, two threads, two contexts on one device -- race on it.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/hopu.h"
#include "context.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device.  In host code the symbol is only a
// host-side stand-in, so the address is looked up with cudaGetSymbolAddress with that
// device current: on every call made outside a stream capture, and the last address found
// is reused by calls made while the stream is being captured.
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

hopu_status noalloc_fail(hopu_ctx* c, int code, const std::string& msg) {
  if (c->status == HOPU_OK) {
    c->status = code;
    c->err = msg;
  }
  return (hopu_status)code;
}

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

}  // namespace

extern "C" hopu_status hopu_apply_convection_noalloc(hopu_ctx* c, const void* w_hdiv, const void* u_l2,
                                                     void* y_l2, const int8_t* facet_l) {
  if (!c) return HOPU_EINVAL;
  if (c->status != HOPU_OK) return (hopu_status)c->status;
  if (!w_hdiv || !u_l2 || !y_l2 || y_l2 == u_l2)
    return noalloc_fail(c, HOPU_EINVAL, "apply_convection_noalloc: NULL or aliased vectors");
  if (((reinterpret_cast<uintptr_t>(w_hdiv) | reinterpret_cast<uintptr_t>(u_l2) |
        reinterpret_cast<uintptr_t>(y_l2)) & 15u) != 0)
    return noalloc_fail(c, HOPU_EINVAL, "apply_convection_noalloc: vectors must be 16-byte aligned");

  // scratch layout: [wind in L2][facet moments, element-major]
  const size_t wl_bytes = align256(c->tsize * (size_t)c->n_l2);
  const size_t gam_bytes = c->tsize * (size_t)c->topo.n_elems * (c->dim + 1) * c->ref.nf * c->dim;
  const size_t need = wl_bytes + gam_bytes;
  if (need > kNoAllocScratchBytes)
    return noalloc_fail(c, HOPU_EINVAL,
                        "apply_convection_noalloc: this mesh needs " + std::to_string(need) +
                            " bytes of scratch; the static buffer holds " + std::to_string(kNoAllocScratchBytes) +
                            " (use hopu_apply_convection)");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(c, HOPU_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(c, HOPU_ENOTSUP, "apply_convection_noalloc: device index too large");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(c->stream, &cs);
  if (e != cudaSuccess)
    return noalloc_fail(c, HOPU_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
      // outside a capture the device address of the static buffer is looked up on every
      // call (cheap), so a device reset or a new primary context never leaves a stale one
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return noalloc_fail(c, HOPU_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_ptr[dev] = p;
    } else if (!g_scratch_ptr[dev]) {
      // inside a capture the address of an earlier call on this device is reused
      return noalloc_fail(c, HOPU_EINVAL,
                          "apply_convection_noalloc: the first call on a device must come before any stream capture");
    }
    base = g_scratch_ptr[dev];
  }
  void* wl = base;
  void* gam = static_cast<unsigned char*>(base) + wl_bytes;

  hopu::Combine plain;
  const int8_t* fl = facet_l ? facet_l : c->facet_l;
  hopu::timed(c, HOPU_K_V2L, [&] { c->ops->v2l(c->dm, c->dt, w_hdiv, wl, c->stream); });
  hopu::timed(c, HOPU_K_FACET, [&] { c->ops->facet(c->dm, c->dt, u_l2, wl, c->l, fl, gam, nullptr, c->stream); });
  hopu::timed(c, HOPU_K_VOLUME, [&] { c->ops->volume(c->dm, c->dt, u_l2, wl, gam, plain, y_l2, c->stream); });
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return noalloc_fail(c, HOPU_ECUDA, std::string("apply_convection_noalloc kernels: ") + cudaGetErrorString(e));
  return HOPU_OK;
}
