// LoG penalty sampling of Eq. 1 and back-projection of the sampled pixels
// (Sec. III-B "Sampling").
//
// P_s = max(P_L - P~, 0): P_L and P~ are the norms (over the three colour
// channels) of the Laplacian-of-Gaussian responses of the input image and of
// the image rendered from the current map.  LoG with sigma = 1 on a 7 x 7
// support, as the sum of two separable terms g2(dx) g(dy) + g(dx) g2(dy)
// (g the normalised Gaussian, g2 its second derivative shifted to sum 0),
// with the nearest edge pixel repeated outside the image.  Pixel p is sampled
// iff u(p) < min(1, kappa P_s(p)) for caller-supplied uniforms u; the sampled
// pixels are compacted in ascending order.
//
// A call covers every view of a keyframe window at once: one penalty grid
// over all views' 32 x 32 tiles (a block finds its view in the table passed
// by value), one ordered compaction over the concatenated pixels (window
// indices: views in order, each ascending), the samples per view by a search
// of the sorted indices, one back-projection.
//
// One block of 256 threads per 32 x 32 output tile takes the six image x
// channel planes one at a time (16 KB of shared memory; its 64 registers
// leave four blocks per SM): it stages the plane on the tile plus a 3-pixel
// halo (38 x 38), runs
// the two horizontal passes (g, g2) as a sliding window (a task is 4
// adjacent outputs of one row from three float4 loads, written as two
// float4), then each thread runs the vertical pass for 4 rows of one column
// from 10 loads per filter and adds the squares to the channel norms it
// keeps in registers.  Bank mapping: the float4 accesses of each 8-lane
// phase are 8 consecutive vectors of one row, the vertical reads are 32
// adjacent columns of one row: no conflicts.
#include <cmath>

#include "device_scan.cuh"
#include "kernels.cuh"

namespace dcg {

namespace {

constexpr int kR = 3;
constexpr int kT = kLsTile;       // output tile side
constexpr int kA = kT + 2 * kR;   // 38: staged side
constexpr int kSP = 40;           // pitch of a staged row (16-byte rows for float4 loads)
constexpr int kHP = 36;           // pitch of a horizontal-result row (16-byte rows for float4 stores)
constexpr int kNC = 6;            // image x channel planes
constexpr int kHT = 4;            // horizontal outputs per task
constexpr int kVR = 4;            // vertical outputs per thread
constexpr int kS = kA * kSP;      // staged floats of one plane
constexpr int kH = 2 * kA * kHP;  // its horizontal results (g and g2)
constexpr float kY00 = 0.28209479177387814f;

__constant__ float c_g[2 * kR + 1], c_g2[2 * kR + 1];

__global__ void __launch_bounds__(256) k_log_penalty(const float* __restrict__ img_all, const float* __restrict__ ren_all,
                                                     const LsViews views, float kappa, const float* __restrict__ u_all,
                                                     float* __restrict__ ps_all, uint32_t* __restrict__ flags_all) {
  __shared__ __align__(16) float s[kS];  // one staged plane [kA][kSP]
  __shared__ __align__(16) float h[kH];  // its horizontal results [2][kA][kHP]
  const int tid = threadIdx.x;
  int v = 0;
  while (v + 1 < views.V && (int)blockIdx.x >= views.v[v + 1].tile0) ++v;
  const int W = views.v[v].cam.W, H = views.v[v].cam.H;
  const long long off = views.v[v].off;
  const int tl = (int)blockIdx.x - views.v[v].tile0;
  const int bx = tl % views.v[v].ntx, by = tl / views.v[v].ntx;
  const float* const img = img_all + 3 * off;
  const float* const ren = ren_all + 3 * off;
  const float* const u = u_all + off;
  float* const ps_out = ps_all ? ps_all + off : nullptr;
  uint32_t* const flags = flags_all + off;
  const int x0 = bx * kT - kR, y0 = by * kT - kR;
  const long long P = (long long)W * H;
  // staging: this thread's elements of the 38 x 38 tile (global offsets, clamped to the image)
  constexpr int kLoads = (kA * kA + 255) / 256;
  int gofs[kLoads];  // a view has fewer than 2^31 pixels
#pragma unroll
  for (int j = 0; j < kLoads; ++j) {
    const int i = tid + 256 * j;
    const int r = i / kA, q = i - r * kA;
    const int gx = min(max(x0 + q, 0), W - 1), gy = min(max(y0 + r, 0), H - 1);
    gofs[j] = gy * W + gx;
  }
  // horizontal tasks (rows x 8 groups of 4 columns) and the vertical column / rows of this thread
  constexpr int kTasks = kA * (kT / kHT);
  const int q = tid & 31, r0 = (tid >> 5) * kVR;
  float n2i[kVR], n2r[kVR];  // squared channel norms of the image's and the rendering's response
#pragma unroll
  for (int o = 0; o < kVR; ++o) n2i[o] = n2r[o] = 0.f;
#pragma unroll 1
  for (int pl = 0; pl < kNC; ++pl) {
    const float* const src = (pl < 3 ? img : ren) + (pl % 3) * P;
#pragma unroll
    for (int j = 0; j < kLoads; ++j) {
      const int i = tid + 256 * j;
      if (i < kA * kA) {
        const int r = i / kA;
        s[r * kSP + (i - r * kA)] = src[gofs[j]];
      }
    }
    __syncthreads();  // staged (and the previous plane's vertical pass is done with h)
    for (int t = tid; t < kTasks; t += 256) {
      const int r = t >> 3, q0 = (t & 7) * kHT;
      const float4* row = reinterpret_cast<const float4*>(s + r * kSP + q0);
      const float4 xa = row[0], xb = row[1], xc = row[2];
      float x[12];
      x[0] = xa.x; x[1] = xa.y; x[2] = xa.z; x[3] = xa.w;
      x[4] = xb.x; x[5] = xb.y; x[6] = xb.z; x[7] = xb.w;
      x[8] = xc.x; x[9] = xc.y; x[10] = xc.z; x[11] = xc.w;
      float a[kHT], b[kHT];
#pragma unroll
      for (int o = 0; o < kHT; ++o) {
        a[o] = 0.f;
        b[o] = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kR; ++k) {
          a[o] += c_g[k] * x[o + k];
          b[o] += c_g2[k] * x[o + k];
        }
      }
      *reinterpret_cast<float4*>(h + r * kHP + q0) = make_float4(a[0], a[1], a[2], a[3]);
      *reinterpret_cast<float4*>(h + (kA + r) * kHP + q0) = make_float4(b[0], b[1], b[2], b[3]);
    }
    __syncthreads();  // horizontal results complete (and the staged plane is free again)
    const float* hg = h + r0 * kHP + q;
    const float* hg2 = h + (kA + r0) * kHP + q;
    float vv[kVR] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int t = 0; t < kVR + 2 * kR; ++t) {
      const float ga = hg[t * kHP], gb = hg2[t * kHP];
#pragma unroll
      for (int o = 0; o < kVR; ++o) {
        const int k = t - o;
        if (k >= 0 && k <= 2 * kR) vv[o] += c_g[k] * gb + c_g2[k] * ga;
      }
    }
    if (pl < 3) {
#pragma unroll
      for (int o = 0; o < kVR; ++o) n2i[o] += vv[o] * vv[o];
    } else {
#pragma unroll
      for (int o = 0; o < kVR; ++o) n2r[o] += vv[o] * vv[o];
    }
  }
  const int px = bx * kT + q;
  if (px >= W) return;
#pragma unroll
  for (int o = 0; o < kVR; ++o) {
    const int py = by * kT + r0 + o;
    if (py >= H) break;
    const float ps = fmaxf(sqrtf(n2i[o]) - sqrtf(n2r[o]), 0.f);
    const long long p = (long long)py * W + px;
    if (ps_out) ps_out[p] = ps;
    flags[p] = u[p] < fminf(1.f, kappa * ps) ? 1u : 0u;
  }
}

struct FlagCount {
  const uint32_t* f;
  __device__ u64 operator()(u64 i) const { return f[i]; }
};
struct IdxEmit {
  int32_t* out;
  u64 cap;
  __device__ void operator()(u64 i, u64 off, u64) const {
    if (off < cap) out[off] = (int32_t)i;
  }
};

// Samples per view: the window indices are ascending, so view v's samples
// are those in [off_v, off_v + W_v H_v).  One warp per view finds both ends
// by a 32-way search (each step tests 32 pivots at once and keeps the span
// between the last one below the key and the next).
__device__ u64 warp_lower_bound(const int32_t* __restrict__ idx, u64 n, long long key, int lane) {
  u64 lo = 0, hi = n;  // the first index with idx >= key lies in [lo, hi]
  while (hi - lo > 32) {
    const u64 step = (hi - lo + 31) / 32;
    const u64 piv = lo + (u64)lane * step;
    const bool below = piv < hi && (long long)idx[piv] < key;
    const int c = __popc(__ballot_sync(0xffffffffu, below));
    const u64 nhi = lo + (u64)c * step < hi ? lo + (u64)c * step : hi;
    lo = c ? lo + (u64)(c - 1) * step + 1 : lo;
    hi = nhi;
  }
  const bool below = lo + (u64)lane < hi && (long long)idx[lo + lane] < key;
  return lo + (u64)__popc(__ballot_sync(0xffffffffu, below));
}

__global__ void k_view_counts(const int32_t* __restrict__ idx, const u64* n_ptr, u64 cap, const LsViews views,
                              u64* __restrict__ vcount) {
  const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (v >= views.V) return;  // whole warps
  const u64 n = *n_ptr < cap ? *n_ptr : cap;
  const long long a = views.v[v].off, b = a + (long long)views.v[v].cam.W * views.v[v].cam.H;
  const u64 lo = warp_lower_bound(idx, n, a, lane), hi = warp_lower_bound(idx, n, b, lane);
  if (lane == 0) vcount[v] = hi - lo;
}

// New Gaussians at the sampled pixels: centre at the pixel's depth along its
// ray, isotropic scale of one pixel footprint (depth / fx), identity
// rotation, the given opacity logit, SH DC from the pixel colour (rest 0).
// idx holds window indices; the view is the last one starting at or before.
__global__ void k_backproject(const int32_t* __restrict__ idx, long long n, const float* __restrict__ depth,
                              const float* __restrict__ img_all, const LsViews views, float logit, int F,
                              float* __restrict__ out, long long stride) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const long long pw = idx[j];
    int v = 0;
    while (v + 1 < views.V && pw >= views.v[v + 1].off) ++v;
    const LcView& cam = views.v[v].cam;
    const long long off = views.v[v].off, p = pw - off;
    const long long P = (long long)cam.W * cam.H;
    const float* const img = img_all + 3 * off;
    const float x = (float)(p % cam.W), y = (float)(p / cam.W);
    const float d = depth[pw];
    const float c0 = d * (x - cam.cx) / cam.fx, c1 = d * (y - cam.cy) / cam.fy, c2 = d;
    const float v0 = c0 - cam.t[0], v1 = c1 - cam.t[1], v2 = c2 - cam.t[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) out[a * stride + j] = cam.R[a] * v0 + cam.R[3 + a] * v1 + cam.R[6 + a] * v2;
    const float ls = logf(d / cam.fx);
    out[3 * stride + j] = ls;
    out[4 * stride + j] = ls;
    out[5 * stride + j] = ls;
    out[6 * stride + j] = 1.f;
    out[7 * stride + j] = 0.f;
    out[8 * stride + j] = 0.f;
    out[9 * stride + j] = 0.f;
    out[10 * stride + j] = logit;
    for (int ch = 0; ch < 3; ++ch) out[(11 + ch) * stride + j] = (img[ch * P + p] - 0.5f) / kY00;
    for (int f = 14; f < F; ++f) out[f * stride + j] = 0.f;
  }
}

}  // namespace

cudaError_t log_init() {
  double g[2 * kR + 1], g2[2 * kR + 1], s = 0.0, m = 0.0;
  for (int k = -kR; k <= kR; ++k) s += (g[k + kR] = std::exp(-0.5 * k * k));
  for (int k = 0; k <= 2 * kR; ++k) g[k] /= s;
  for (int k = -kR; k <= kR; ++k) m += (g2[k + kR] = ((double)k * k - 1.0) * g[k + kR]);
  m /= 2 * kR + 1;
  float gf[2 * kR + 1], g2f[2 * kR + 1];
  for (int k = 0; k <= 2 * kR; ++k) {
    gf[k] = (float)g[k];
    g2f[k] = (float)(g2[k] - m);
  }
  cudaError_t e = cudaMemcpyToSymbol(c_g, gf, sizeof(gf));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_g2, g2f, sizeof(g2f));
  return e;
}

void launch_log_sample(const float* img, const float* ren, const LsViews& views, float kappa, const float* u,
                       float* ps_out, uint32_t* flags, int32_t* idx_out, long long cap, u64* part, int Pb, u64* count,
                       u64* vcount, cudaStream_t st) {
  k_log_penalty<<<views.n_tiles, 256, 0, st>>>(img, ren, views, kappa, u, ps_out, flags);
  part_scan_emit(nullptr, (u64)views.n_pix, FlagCount{flags}, IdxEmit{idx_out, (u64)cap}, part, Pb, count, st);
  k_view_counts<<<1, 32 * kLsMaxViews, 0, st>>>(idx_out, count, (u64)cap, views, vcount);
  count_launch(5);
}

void launch_backproject(const int32_t* idx, long long n, const float* depth, const float* img, const LsViews& views,
                        float logit, int F, float* out, long long stride, int num_sms, cudaStream_t st) {
  if (n <= 0) return;
  const long long blocks = (n + 255) / 256;
  k_backproject<<<(int)(blocks < num_sms * 8ll ? blocks : num_sms * 8ll), 256, 0, st>>>(idx, n, depth, img, views,
                                                                                     logit, F, out, stride);
  count_launch();
}

}  // namespace dcg
