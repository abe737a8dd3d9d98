// mlps_static.cu -- a forward render that needs no device allocation at all.
//
// Who this is for: callers that cannot allocate device memory where they render. Examples are
// a host application or plug-in whose device memory is owned by someone else's allocator (it
// may not call cudaMalloc behind that allocator's back), and frame loops that must not call
// cudaMalloc / cudaFree because those calls can synchronise the whole device or fail in the
// middle of a frame. The regular entry point asks the caller for `saved` and `scratch`
// buffers; this one uses a fixed workspace that lives in a static device array instead.
//
// The array belongs to this file's module of the library image. With CUDA's lazy module
// loading (the default) that module is loaded on a device, and its kStaticBytes of device memory
// reserved there, by the first call of this entry point on that device (the symbol lookup in
// static_workspace); with eager loading it happens when the library loads. Either way the
// memory stays reserved until the process exits. That first call can therefore fail for lack
// of device memory (MLPS_ERR_CUDA) and can synchronise: make it once, before the frame loop
// and before any stream capture. Later calls reserve nothing.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/mlps.h"

namespace {

constexpr size_t kStaticBytes = 32u << 20;  // 32 MiB: the limit stated in include/mlps.h
constexpr int kMaxDevices = 64;

// The workspace. In host code this symbol is only a stand-in for the device array: its device
// address must be looked up (static_workspace below) and passed to the kernels.
static __device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the array on the current device; looked up once per device, with that
// device current (the lookup loads the module on that device, see above). nullptr (and the
// CUDA error in *err) if the lookup fails.
void* static_workspace(int dev, cudaError_t* err) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_static_ws);
    if (*err != cudaSuccess) return nullptr;
    g_addr[dev] = p;
  }
  *err = cudaSuccess;
  return g_addr[dev];
}

}  // namespace

extern "C" mlps_status mlps_render_forward_static(const mlps_config* cfg, const mlps_scene* scene,
                                                  const mlps_camera* cams, int32_t n_views,
                                                  float* rgb, float* trans, float* feat,
                                                  int32_t* device_status, void* stream) {
  if (!scene) return MLPS_ERR_INVALID_ARGUMENT;
  size_t saved_bytes = 0, scratch_bytes = 0;
  mlps_status s = mlps_workspace_size(cfg, scene->K, cams, n_views, &saved_bytes, &scratch_bytes);
  if (s != MLPS_OK) return s;
  const size_t saved_al = (saved_bytes + 255) & ~size_t(255);
  if (saved_al + scratch_bytes > kStaticBytes) return MLPS_ERR_WORKSPACE_TOO_SMALL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MLPS_ERR_CUDA;
  cudaError_t e;
  unsigned char* ws = static_cast<unsigned char*>(static_workspace(dev, &e));
  if (!ws) return MLPS_ERR_CUDA;
  // The regular forward pass clears the region's header (status word and counters) and every
  // per-call count it relies on before use, so the previous call's contents do no harm.
  s = mlps_render_forward(cfg, scene, cams, n_views, rgb, trans, feat, ws, saved_bytes,
                          ws + saved_al, scratch_bytes, stream);
  if (s != MLPS_OK) return s;  // device_status is left as it was (documented in include/mlps.h)
  if (device_status) {
    // the status word is the first int of the region: hand it to the caller asynchronously
    if (cudaMemcpyAsync(device_status, ws, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                        static_cast<cudaStream_t>(stream)) != cudaSuccess)
      return MLPS_ERR_CUDA;
  }
  return MLPS_OK;
}
