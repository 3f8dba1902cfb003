// Chunk frustum cull that allocates nothing.
//
// Some callers cannot allocate device memory when they cull: a program whose
// device memory is entirely owned by its own allocator or pool, or one that
// runs under a fixed memory budget planned in advance (the embedded setting
// of a mapper on a small board), cannot let a library call cudaMalloc, and
// cannot hold a dcg_ctx, whose creation allocates.  For them this file
// offers dcg_cull_chunks_noalloc: the same cull as dcg_cull_chunks, but the
// scratch it needs (the camera table and the per-chunk union flags) lives in
// a file-scope __device__ array of fixed size that every GPU loading the
// library holds until the process exits.
#include <mutex>

#include "kernels.cuh"

namespace {

constexpr int kNoAllocMaxChunks = 1 << 20;  // chunks per call
constexpr int kNoAllocMaxViews = 16;        // views per call
constexpr size_t kCamBytes = sizeof(dcg_camera) * kNoAllocMaxViews;
constexpr size_t kCamBytesAligned = (kCamBytes + 255) / 256 * 256;

// [camera table | union flags], 1 MiB + 2 KiB, shared by every call on a device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kCamBytesAligned + kNoAllocMaxChunks];

constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (looked up once
// per device; the symbol name itself is only a host-side handle).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
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
  unsigned char* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return DCG_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  dcg_camera* d_cams = reinterpret_cast<dcg_camera*>(base);
  uint8_t* d_vis = base + kCamBytesAligned;
  if (cudaMemcpyAsync(d_cams, cams, sizeof(dcg_camera) * n_views, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return DCG_ERR_CUDA;
  // launch_cull clears the union flags left by the previous call before use
  dcg::launch_cull(coords, n_chunks, d_cams, n_views, chunk_size, dfar, mask_out, d_vis, list_out, n_out, s);
  return cudaGetLastError() == cudaSuccess ? DCG_OK : DCG_ERR_CUDA;
}
