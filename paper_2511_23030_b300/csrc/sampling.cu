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
// One block per 16 x 16 tile loads both images on the tile plus a 3-pixel
// halo, runs the two horizontal passes (g, g2) and the vertical pass for each
// channel and image, and writes P_s and the sample flag.
#include <cmath>

#include "device_scan.cuh"
#include "kernels.cuh"

namespace dcg {

namespace {

constexpr int kR = 3;
constexpr int kT = 16;
constexpr int kA = kT + 2 * kR;  // 22
constexpr float kY00 = 0.28209479177387814f;

__constant__ float c_g[2 * kR + 1], c_g2[2 * kR + 1];

__global__ void __launch_bounds__(256) k_log_penalty(const float* __restrict__ img, const float* __restrict__ ren,
                                                     int W, int H, float kappa, const float* __restrict__ u,
                                                     float* __restrict__ ps_out, uint32_t* __restrict__ flags) {
  __shared__ float s[2][3][kA][kA + 1];
  __shared__ float h[2][3][2][kA][kT + 1];
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * kT - kR, y0 = blockIdx.y * kT - kR;
  const long long P = (long long)W * H;
  for (int i = tid; i < kA * kA; i += 256) {
    const int r = i / kA, q = i - r * kA;
    const int gx = min(max(x0 + q, 0), W - 1), gy = min(max(y0 + r, 0), H - 1);
    const long long k = (long long)gy * W + gx;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      s[0][c][r][q] = img[c * P + k];
      s[1][c][r][q] = ren[c * P + k];
    }
  }
  __syncthreads();
  for (int i = tid; i < 2 * 3 * kA * kT; i += 256) {
    const int q = i % kT, r = (i / kT) % kA, c = (i / (kT * kA)) % 3, m = i / (kT * kA * 3);
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) {
      const float x = s[m][c][r][q + k];
      a += c_g[k] * x;
      b += c_g2[k] * x;
    }
    h[m][c][0][r][q] = a;
    h[m][c][1][r][q] = b;
  }
  __syncthreads();
  const int r = tid / kT, q = tid - r * kT;
  const int px = blockIdx.x * kT + q, py = blockIdx.y * kT + r;
  if (px >= W || py >= H) return;
  float n2[2] = {0.f, 0.f};
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float v = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * kR; ++k) v += c_g[k] * h[m][c][1][r + k][q] + c_g2[k] * h[m][c][0][r + k][q];
      n2[m] += v * v;
    }
  const float ps = fmaxf(sqrtf(n2[0]) - sqrtf(n2[1]), 0.f);
  const long long p = (long long)py * W + px;
  if (ps_out) ps_out[p] = ps;
  flags[p] = u[p] < fminf(1.f, kappa * ps) ? 1u : 0u;
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

// New Gaussians at the sampled pixels: centre at the pixel's depth along its
// ray, isotropic scale of one pixel footprint (depth / fx), identity
// rotation, the given opacity logit, SH DC from the pixel colour (rest 0).
__global__ void k_backproject(const int32_t* __restrict__ idx, long long n, const float* __restrict__ depth,
                              const float* __restrict__ img, int W, int H, LcView cam, float logit, int F,
                              float* __restrict__ out, long long stride) {
  const long long P = (long long)W * H;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const long long p = idx[j];
    const float x = (float)(p % W), y = (float)(p / W);
    const float d = depth[p];
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
  return e == cudaSuccess ? cudaMemcpyToSymbol(c_g2, g2f, sizeof(g2f)) : e;
}

void launch_log_sample(const float* img, const float* ren, int W, int H, float kappa, const float* u, float* ps_out,
                       uint32_t* flags, int32_t* idx_out, long long cap, u64* part, int Pb, u64* count,
                       cudaStream_t st) {
  dim3 grid((unsigned)((W + kT - 1) / kT), (unsigned)((H + kT - 1) / kT));
  k_log_penalty<<<grid, 256, 0, st>>>(img, ren, W, H, kappa, u, ps_out, flags);
  part_scan_emit(nullptr, (u64)W * (u64)H, FlagCount{flags}, IdxEmit{idx_out, (u64)cap}, part, Pb, count, st);
  count_launch(4);
}

void launch_backproject(const int32_t* idx, long long n, const float* depth, const float* img, int W, int H,
                        const LcView& cam, float logit, int F, float* out, long long stride, int num_sms,
                        cudaStream_t st) {
  if (n <= 0) return;
  const long long blocks = (n + 255) / 256;
  k_backproject<<<(int)(blocks < num_sms * 8ll ? blocks : num_sms * 8ll), 256, 0, st>>>(idx, n, depth, img, W, H, cam,
                                                                                     logit, F, out, stride);
  count_launch();
}

}  // namespace dcg
