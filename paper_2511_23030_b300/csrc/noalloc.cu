// Chunk frustum cull that allocates nothing.
//
// Some callers cannot allocate device memory when they cull: a program whose
// device memory is entirely owned by its own allocator or pool, or one that
// runs under a fixed memory budget planned in advance (the embedded setting
// of a mapper on a small board), cannot let a library call cudaMalloc, and
// cannot hold a dcg_ctx, whose creation allocates.  For them this file
// offers dcg_cull_chunks_noalloc: the same cull as dcg_cull_chunks, but the
// scratch it needs (the per-chunk union flags) lives in a file-scope
// __device__ array of fixed size that every GPU loading the library holds
// until the process exits, and the cameras travel by value in the kernel's
// parameters.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "kernels.cuh"

namespace {

constexpr int kNoAllocMaxChunks = 1 << 20;  // chunks per call
constexpr int kNoAllocMaxViews = dcg::kMaxViewsApi;  // views per call (16)

// union flags of one call, 1 MiB, shared by every call on a device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocMaxChunks];

// The device address of the array is looked up once per device and primary
// context: after a cudaDeviceReset the next call finds a new context and looks
// the address up again instead of writing through the old one.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
  CUcontext ctx = nullptr;
  unsigned char* addr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];
std::mutex g_scratch_mu;
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn g_ctx_get_current = nullptr;

cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_ctx_get_current) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorSymbolNotFound;
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
  }
  ScratchAddr& sa = g_scratch[dev];
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) == CUDA_SUCCESS && ctx && ctx == sa.ctx && sa.addr) {
    *out = sa.addr;
    return cudaSuccess;
  }
  // first call on this device or in this context: the lookup also makes the
  // runtime's primary context current if it was not yet
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  sa.ctx = ctx;
  sa.addr = static_cast<unsigned char*>(p);
  *out = sa.addr;
  return cudaSuccess;
}

}  // namespace

extern "C" dcg_status dcg_cull_chunks_noalloc(const int32_t* coords, int32_t n_chunks, float chunk_size, float dfar,
                                              const dcg_camera* cams, int32_t n_views, uint8_t* mask_out,
                                              int32_t* list_out, int32_t* n_out, void* stream) {
  if (n_chunks < 0 || (n_chunks > 0 && !coords) || !cams || n_views <= 0 || !list_out || !n_out ||
      !(chunk_size > 0.f))
    return DCG_ERR_ARG;
  if (n_chunks > kNoAllocMaxChunks || n_views > kNoAllocMaxViews) return DCG_ERR_CAPACITY;
  for (int v = 0; v < n_views; ++v)
    if (cams[v].W <= 0 || cams[v].H <= 0 || !(cams[v].fx > 0.f) || !(cams[v].fy > 0.f) || !(cams[v].znear > 0.f) ||
        !(cams[v].zfar > cams[v].znear))
      return DCG_ERR_ARG;
  unsigned char* d_vis = nullptr;
  if (scratch_address(&d_vis) != cudaSuccess) return DCG_ERR_CUDA;
  // the cameras are copied into the launch's parameters here, before return
  dcg::CullCams tab;
  std::memset(&tab, 0, sizeof(tab));
  std::memcpy(tab.c, cams, sizeof(dcg_camera) * n_views);
  // launch_cull clears the union flags left by the previous call before use
  const cudaError_t e = dcg::launch_cull(coords, n_chunks, nullptr, &tab, n_views, chunk_size, dfar, mask_out, d_vis,
                                         list_out, n_out, (cudaStream_t)stream);
  return e == cudaSuccess ? DCG_OK : DCG_ERR_CUDA;
}
