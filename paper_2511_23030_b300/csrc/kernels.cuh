// Kernel launchers of the dcg library (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/dcg.h"

namespace dcg {

typedef unsigned long long u64;

constexpr int kMaxViewsApi = 16;  // views per render call

// Phases timed by the optional profiler (dcg_profile); same order as in dcg.h.
enum Phase { PH_CULL = 0, PH_GATHER, PH_PRE_FWD, PH_BINNING, PH_BLEND_FWD, PH_LOSS, PH_BLEND_BWD, PH_PRE_BWD,
             PH_SCATTER, PH_STALL, PH_SAMPLE, PH_LOOP, PH_COUNT };

// Kernel launches issued by the library in this process (for launch accounting).
extern unsigned long long g_launches;
inline void count_launch(unsigned long long k = 1) { g_launches += k; }

struct ProfHook {
  void* h = nullptr;
  void (*mark)(void* h, int phase, bool begin, cudaStream_t s) = nullptr;
  void operator()(int phase, bool begin, cudaStream_t s) const {
    if (mark) mark(h, phase, begin, s);
  }
};

// device error word bits
constexpr unsigned ERRW_KEY_RANGE_BIT = 1u;
constexpr unsigned ERRW_CAPACITY_BIT = 2u;
constexpr unsigned ERRW_TIMEOUT_BIT = 4u;  // reserved: no kernel waits on another block or a flag
constexpr unsigned ERRW_BOUNDS_BIT = 8u;   // an index outside its buffer (bounds-check build)

// Bounds-check build (compiled with -DDCG_CHECKS=1): dcg_oob(i, n, ew) is true
// when index i is outside a buffer of n elements; it then sets
// ERRW_BOUNDS_BIT in the device error word and the caller skips the access
// (nothing traps); dcg_sync reports DCG_ERR_BOUNDS.  In the normal build it
// is constant false and the guarded branches compile away.
#if defined(DCG_CHECKS) && DCG_CHECKS
__device__ __forceinline__ bool dcg_oob(unsigned long long i, unsigned long long n, unsigned* ew) {
  if (i < n) return false;
  atomicOr(ew, ERRW_BOUNDS_BIT);
  return true;
}
#else
__device__ __forceinline__ bool dcg_oob(unsigned long long, unsigned long long, unsigned*) { return false; }
#endif

// ---------------------------------------------------------------- chunk.cu
void launch_chunk_keys(const float* means, long long row, long long col, long long n, float s, u64* keys,
                       unsigned* errword, int num_sms, cudaStream_t st);
// Cameras of one cull passed by value (kernel parameter space, 1.5 KB).
struct CullCams {
  dcg_camera c[kMaxViewsApi];
};
// Cull of C chunks against V views: the cameras come from device memory
// (cams) or, when tab is not null, by value from *tab.  Clears vis first;
// returns the first error of the clear or the launches.
cudaError_t launch_cull(const int32_t* coords, int C, const dcg_camera* cams, const CullCams* tab, int V, float s,
                        float dfar, uint8_t* mask, uint8_t* vis, int32_t* list, int32_t* n, cudaStream_t st);
// Load verification: adds the checksum of page p of a chunk (cnt rows) to *out.
void launch_page_checksum(const float* page, long long p, long long page_g, int Fp, long long cnt,
                          unsigned long long* out, cudaStream_t st);
void launch_active_map(const long long* off, const int32_t* chunk, int nl, long long n, int32_t* chunk_out,
                       int32_t* row_out, int num_sms, cudaStream_t st);
void launch_page_copy(bool gather, float* pool, long long page_g, int Fp, int c0, int nc, const long long* desc, int nd,
                      float* active, long long stride, cudaStream_t st);

// ---------------------------------------------------------------- loopclosure.cu
// One affected keyframe: pose before the correction (world -> camera), its
// intrinsics and image, the correction x' = C x (3 x 4 row-major) and the
// rotation of C as a unit quaternion (w, x, y, z).
struct LcView {
  float R[9], t[3];
  float fx, fy, cx, cy, znear, zfar;
  int W, H;
  float C[12];
  float q[4];
};
// flags: per row, on return the keyframe (1-based) that moved it, else 0; with
// skip_done a nonzero flag on entry marks a row already moved (left alone, flag cleared).
void launch_loop_transform(float* act, long long stride, long long n, const long long* seg_off, const int* seg_chunk,
                           int nseg, const uint8_t* mask, int C, const LcView* kf, int K, uint32_t* flags, int skip_done,
                           int num_sms, cudaStream_t st);
// Loop-closure redistribution: moved flags (in place of the transformed
// flags, whose count goes to *n_transformed), the moved rows ascending with
// their keys in midx / mkey and their number in *n_moved; then the
// permutation perm (gather form) from the planned destinations.
void launch_lc_moved(uint32_t* flags, const u64* keys, long long n, const long long* seg_off, const u64* seg_key,
                     int nseg, unsigned long long* n_transformed, long long* midx, u64* mkey, u64* part, int P,
                     u64* n_moved, int num_sms, cudaStream_t st);
void launch_lc_dest(const uint32_t* moved, long long n, const long long* seg_off, const long long* seg_base, int nseg,
                    const long long* midx, const long long* mdest, long long nm, long long* perm, int num_sms,
                    cudaStream_t st);
void launch_permute_rows(const float* src, long long sstride, float* dst, long long dstride, const long long* perm,
                         long long n, int rows, int num_sms, cudaStream_t st);
void launch_cap_rows(float* row, long long n, float cap, int num_sms, cudaStream_t st);

// ---------------------------------------------------------------- sampling.cu
// The views of one batched sampling or back-projection call, passed by value
// (kernel parameter space): view v's pixels are the window pixels
// [off, off + W H) of the concatenated buffers, its 32 x 32 penalty tiles
// the grid blocks [tile0, tile0 + ntx nty).
constexpr int kLsMaxViews = 16;
constexpr int kLsTile = 32;
struct LsView {
  LcView cam;  // W, H always; pose and intrinsics for the back-projection
  long long off;
  int tile0, ntx;
};
struct LsViews {
  LsView v[kLsMaxViews];
  int V;
  int n_tiles;
  long long n_pix;
};
cudaError_t log_init();
// Eq. 1 over all views: flags, ordered compaction of window indices into
// idx_out (at most cap), total in *count, per-view counts in vcount (device, V).
void launch_log_sample(const float* img, const float* ren, const LsViews& views, float kappa, const float* u,
                       float* ps_out, uint32_t* flags, int32_t* idx_out, long long cap, u64* part, int Pb, u64* count,
                       u64* vcount, cudaStream_t st);
void launch_backproject(const int32_t* idx, long long n, const float* depth, const float* img, const LsViews& views,
                        float logit, int F, float* out, long long stride, int num_sms, cudaStream_t st);

// ---------------------------------------------------------------- optim.cu
constexpr int kAdamMaxF = 64;
struct AdamArgs {
  float step[kAdamMaxF];  // lr_c / (1 - beta1^t) per component
  float beta1, beta2, isb2, eps;  // isb2 = 1 / sqrt(1 - beta2^t)
};
void launch_adam(float* p, long long ps, const float* g, long long gs, float* m, float* v, long long ms, long long n,
                 int F, const AdamArgs& aa, int num_sms, cudaStream_t st);

// ---------------------------------------------------------------- raster
// Per-view camera constants (built on the host from dcg_camera).
struct DevCam {
  float fx, fy, cx, cy;
  float R[9];
  float t[3];
  float C[3];   // camera centre -R^T t
  float znear, zfar;
  float xlo, xhi, ylo, yhi;  // clamp of x/z and y/z inside the Jacobian
  int W, H;
  int ntx, nty;     // tiles along x / y
  int tile_base;    // global index of tile (0,0) of this view
  int pad;
  long long pix_off;  // pixel offset of this view in the stacked outputs
};

struct DevCounters {
  u64 n_vis;    // visible (view, Gaussian) pairs
  u64 n_inst;   // instances requested (> capacity means overflow)
  u64 n_inst_c; // instances kept (min with capacity)
  u64 n_eval;   // pixel-Gaussian evaluations of the forward blend
  u64 n_blend;  // pixel-Gaussian pairs the forward blend composited (alpha >= 1/255, before termination)
  unsigned tile_queue;
  unsigned tile_queue_bwd;
  unsigned pad[8];
};

struct RasterArgs {
  // inputs
  const float* g;      // planar Gaussians
  long long stride;
  long long n;
  int deg;
  int V;
  const DevCam* cams;
  int tile_w, tile_h, stage;
  int n_tiles;
  long long n_pix;
  int idx_bits;        // bits of the Gaussian index in the depth keys
  int view_bits;
  // per (view, Gaussian) pair: index v * n + i
  float4* rec;
  float* depth;
  uint32_t* touched;
  short4* rect;
  float4* bin;         // per pair, 2 float4: (u, v, A', B'), (C', rect x0|y0 << 16, rect x1|y1 << 16, 0)
  float4* grad2d;
  // lists
  u64* list_a;
  u64* list_b;
  u64* inst_a;
  u64* inst_b;
  long long cap_pairs, cap_inst;
  uint2* ranges;
  float* T_final;
  uint32_t* n_contrib;
  DevCounters* counters;
  u64* part;
  uint32_t* hist;
  int P;
  unsigned* errword;
  int num_sms;
  int bwd_slots;  // 1: backward accumulates per-lane slots instead of warp reductions
  int bwd_pix;    // 1: the half-warp backward keeps pixels on the lanes (one Gaussian per half per step)
  ProfHook prof;
};

// Runs preprocess, depth sort, instance emission, tile sort and ranges; then
// the forward blend.  Returns the sorted instance buffer via *inst_sorted.
void raster_forward(RasterArgs& a, float* rgb, float* depth_out, u64** list_sorted, u64** inst_sorted,
                    cudaStream_t st);
void raster_backward(RasterArgs& a, const u64* inst_sorted, const float* dL_drgb, const float* dL_ddepth,
                     float* grads, long long g_stride, float* dL_dpose, cudaStream_t st);

// ---------------------------------------------------------------- loss
int loss_partials(int num_sms);  // scratch floats the loss needs
void launch_loss_l1(const float* rgb, const float* depth, const float* trgb, const float* tdepth, const DevCam* cams,
                    int V, long long n_pix, float wimg, float lam, float* dr, float* dd, float* loss, float* part,
                    int num_sms, cudaStream_t st);
// loss.cu: SSIM term (16 x 16 tiles of the views in `cams`: W, H, pix_off, ntx, tile_base)
int ssim_tile();
cudaError_t ssim_init();
void launch_ssim(const float* rgb, const float* trgb, const DevCam* cams, int V, int n_tiles, float lam_s, float* dr,
                 float* loss, float* part, cudaStream_t st);

}  // namespace dcg
