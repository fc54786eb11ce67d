// vt_static.cu -- vt_voronoi_static: Voronoi labelling with no device allocation
// anywhere, for callers that are not allowed to allocate GPU memory.
//
// vt_voronoi needs a caller-provided workspace.  Some callers cannot obtain
// one: a plugin whose host application owns every device allocation and
// hands it only input and output buffers, or a latency-bound loop that
// cannot afford the device-wide synchronisation cudaMalloc and cudaFree may
// cause.  This entry point runs the unchanged vt_voronoi pipeline on a
// scratch buffer that lives in this file as a static __device__ array of
// kStaticScratchBytes (64 MiB).  Every GPU that loads this part of the library
// keeps those 64 MiB until the process exits.
//
// Host code must not pass `g_vt_scratch` itself to a kernel: in host code that
// name is only a stand-in for the symbol, not a device address.  The device
// address is looked up once per device with cudaGetSymbolAddress (the first
// call on each device does it, with that device current) and cached; a
// cudaDeviceReset ends the context the cached address belongs to, so the
// entry point must not be called again in that process after a reset.
#include <mutex>
#include <string>

#include "vt.h"
#include "vt_internal.cuh"

namespace vt {
void ctx_set_error(vt_ctx* ctx, const std::string& msg);
vt_status ctx_plan_bytes(const vt_ctx* ctx, int kind, int64_t n_sites, size_t* bytes);
}

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_vt_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_vt_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" vt_status vt_voronoi_static(vt_ctx* ctx, int64_t n_sites, const int32_t* d_sites,
                                       int32_t* d_labels, void* stream) {
  if (!ctx) return VT_ERR_ARG;
  // the scratch of the plan this call will run (the context's bin size and
  // margin for this site count), not the autotuner's largest plan
  size_t need = 0;
  vt_status s = vt::ctx_plan_bytes(ctx, VT_VORONOI, n_sites, &need);
  if (s != VT_OK) {
    vt::ctx_set_error(ctx, "vt_voronoi_static: n_sites out of range");
    return s;
  }
  if (need > kStaticScratchBytes) {
    vt::ctx_set_error(ctx, "vt_voronoi_static: this grid and site count need " +
                               std::to_string(need) + " bytes of scratch, more than the " +
                               std::to_string(kStaticScratchBytes) +
                               " bytes of the static buffer; use vt_voronoi with a workspace");
    return VT_ERR_WORKSPACE;
  }
  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    vt::ctx_set_error(ctx, std::string("vt_voronoi_static: cudaGetSymbolAddress: ") +
                               cudaGetErrorString(e));
    return VT_ERR_CUDA;
  }
  // The pipeline clears the part of the scratch that must start at zero (error
  // word, counters, bin histogram) before it uses it.
  return vt_voronoi(ctx, n_sites, d_sites, d_labels, scratch, kStaticScratchBytes, stream);
}
