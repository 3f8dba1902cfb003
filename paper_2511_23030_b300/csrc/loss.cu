// SSIM term of the image loss (Eq. 3): lambda_s (1 - SSIM(I, I_gt)) per view
// and its gradient, fused in one kernel.
//
// SSIM follows the 3DGS reading: 11 x 11 Gaussian window (sigma 1.5, sum 1),
// C1 = 0.01^2, C2 = 0.03^2, windowed means as a same-size correlation with
// zero padding, the mean of the per-pixel SSIM over pixels and channels.
// Per pixel S = A1 A2 / (B1 B2) with A1 = 2 mx my + C1, A2 = 2 sxy + C2,
// B1 = mx^2 + my^2 + C1, B2 = sx^2 + sy^2 + C2.  S depends on the rendered
// image x only through mx = w*x, Sxx = w*(x^2) and Sxy = w*(x y), so
//   dL/dx = w*g_mu + 2 x (w*g_xx) + y (w*g_xy)
// with, per pixel and c = dL/dS = -lambda_s / (3 H W),
//   g_mu = c S (2 my / A1 - 2 my / A2 - 2 mx / B1 + 2 mx / B2),
//   g_xx = -c S / B2,   g_xy = 2 c S / A2
// (the window is symmetric, so the adjoint correlation is the same one).
//
// One block per (16 x 16 output tile, channel): it loads x and y on the tile
// plus a 10-pixel halo (36 x 36), runs the separable window over it for the
// five statistics on the tile plus a 5-pixel halo (26 x 26), forms S and the
// three g maps there (zero outside the image), runs the window over the g
// maps for the tile, and adds the result to dL/dI.  No global scratch; the
// loss partial of each block is reduced in a fixed order.
#include <cmath>

#include "kernels.cuh"

namespace dcg {

namespace {

constexpr int kR = 5;                  // window radius
constexpr int kT = 16;                 // output tile
constexpr int kG = kT + 2 * kR;        // 26: region of S and g
constexpr int kA = kT + 4 * kR;        // 36: region of x and y
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

__constant__ float c_win[2 * kR + 1];

__global__ void __launch_bounds__(256) k_ssim(const float* __restrict__ rgb, const float* __restrict__ trgb,
                                              const DevCam* __restrict__ cams, int V, float lam_s,
                                              float* __restrict__ dr, float* __restrict__ part) {
  __shared__ float sx[kA][kA + 1], sy[kA][kA + 1];
  __shared__ float h[5][kA][kG + 1];
  __shared__ float g3[3][kG][kG + 1];
  __shared__ float hb[3][kG][kT + 1];
  __shared__ float red[8];
  const int tid = threadIdx.x;
  const int gt = blockIdx.x, ch = blockIdx.y;
  int v = 0;
  while (v + 1 < V && gt >= cams[v + 1].tile_base) ++v;
  const DevCam& c = cams[v];
  const int W = c.W, H = c.H;
  const long long P = (long long)W * H;
  const int local = gt - c.tile_base;
  const int ty = local / c.ntx, tx = local - ty * c.ntx;
  const int ax = tx * kT - 2 * kR, ay = ty * kT - 2 * kR;  // origin of the 36 x 36 region
  const float* X = rgb + 3 * c.pix_off + ch * P;
  const float* Y = trgb + 3 * c.pix_off + ch * P;
  float* D = dr + 3 * c.pix_off + ch * P;
  for (int i = tid; i < kA * kA; i += 256) {
    const int r = i / kA, q = i - r * kA;
    const int gx = ax + q, gy = ay + r;
    const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
    const long long k = (long long)gy * W + gx;
    sx[r][q] = in ? X[k] : 0.f;
    sy[r][q] = in ? Y[k] : 0.f;
  }
  __syncthreads();
  // horizontal window pass: rows 0..35, columns 0..25 of the S region
  for (int i = tid; i < kA * kG; i += 256) {
    const int r = i / kG, q = i - r * kG;
    float m0 = 0.f, m1 = 0.f, s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) {
      const float wk = c_win[k], a = sx[r][q + k], b = sy[r][q + k];
      m0 += wk * a;
      m1 += wk * b;
      s0 += wk * (a * a);
      s1 += wk * (b * b);
      s2 += wk * (a * b);
    }
    h[0][r][q] = m0;
    h[1][r][q] = m1;
    h[2][r][q] = s0;
    h[3][r][q] = s1;
    h[4][r][q] = s2;
  }
  __syncthreads();
  // vertical pass, S and the g maps on the 26 x 26 region
  const float coef = -lam_s / (3.f * (float)P);
  float acc = 0.f;
  for (int i = tid; i < kG * kG; i += 256) {
    const int r = i / kG, q = i - r * kG;
    float mx = 0.f, my = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) {
      const float wk = c_win[k];
      mx += wk * h[0][r + k][q];
      my += wk * h[1][r + k][q];
      xx += wk * h[2][r + k][q];
      yy += wk * h[3][r + k][q];
      xy += wk * h[4][r + k][q];
    }
    const int px = ax + kR + q, py = ay + kR + r;
    const bool in = px >= 0 && px < W && py >= 0 && py < H;
    float gmu = 0.f, gxx = 0.f, gxy = 0.f;
    if (in) {
      const float A1 = 2.f * mx * my + kC1, A2 = 2.f * (xy - mx * my) + kC2;
      const float B1 = mx * mx + my * my + kC1, B2 = (xx - mx * mx) + (yy - my * my) + kC2;
      const float iA1 = 1.f / A1, iA2 = 1.f / A2, iB1 = 1.f / B1, iB2 = 1.f / B2;
      const float S = A1 * A2 * iB1 * iB2;
      const float cs = coef * S;
      gmu = cs * (2.f * my * (iA1 - iA2) + 2.f * mx * (iB2 - iB1));
      gxx = -cs * iB2;
      gxy = 2.f * cs * iA2;
      if (r >= kR && r < kR + kT && q >= kR && q < kR + kT) acc += S;
    }
    g3[0][r][q] = gmu;
    g3[1][r][q] = gxx;
    g3[2][r][q] = gxy;
  }
  __syncthreads();
  // backward horizontal pass: rows 0..25, output columns 0..15
  for (int i = tid; i < kG * kT; i += 256) {
    const int r = i / kT, q = i - r * kT;
    float b0 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) {
      const float wk = c_win[k];
      b0 += wk * g3[0][r][q + k];
      b1 += wk * g3[1][r][q + k];
      b2 += wk * g3[2][r][q + k];
    }
    hb[0][r][q] = b0;
    hb[1][r][q] = b1;
    hb[2][r][q] = b2;
  }
  __syncthreads();
  {
    const int r = tid / kT, q = tid - r * kT;  // 256 threads = one output pixel each
    float b0 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) {
      const float wk = c_win[k];
      b0 += wk * hb[0][r + k][q];
      b1 += wk * hb[1][r + k][q];
      b2 += wk * hb[2][r + k][q];
    }
    const int px = tx * kT + q, py = ty * kT + r;
    if (px < W && py < H) {
      const float x = sx[r + 2 * kR][q + 2 * kR], y = sy[r + 2 * kR][q + 2 * kR];
      D[(long long)py * W + px] += b0 + 2.f * x * b1 + y * b2;
    }
  }
  // loss partial of this block: -lambda_s / (3 P) * sum S (fixed-order reduction)
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int w = 0; w < 8; ++w) s += red[w];
    part[(long long)gt * 3 + ch] = coef * s;
  }
}

// *loss += add + sum of the partials, in a fixed order.
__global__ void k_sum_partials(const float* __restrict__ part, long long nb, float add, float* loss) {
  __shared__ float red[32];
  float acc = 0.f;
  for (long long b = threadIdx.x; b < nb; b += blockDim.x) acc += part[b];
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float s2 = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (threadIdx.x == 0) *loss += add + s2;
  }
}

}  // namespace

int ssim_tile() { return kT; }

cudaError_t ssim_init() {
  double w[2 * kR + 1], s = 0.0;
  for (int k = -kR; k <= kR; ++k) s += (w[k + kR] = std::exp(-(double)(k * k) / (2.0 * 1.5 * 1.5)));
  float wf[2 * kR + 1];
  for (int k = 0; k <= 2 * kR; ++k) wf[k] = (float)(w[k] / s);
  return cudaMemcpyToSymbol(c_win, wf, sizeof(wf));
}

void launch_ssim(const float* rgb, const float* trgb, const DevCam* cams, int V, int n_tiles, float lam_s, float* dr,
                 float* loss, float* part, cudaStream_t st) {
  if (n_tiles <= 0) return;
  k_ssim<<<dim3((unsigned)n_tiles, 3), 256, 0, st>>>(rgb, trgb, cams, V, lam_s, dr, part);
  k_sum_partials<<<1, 256, 0, st>>>(part, 3ll * n_tiles, lam_s * (float)V, loss);
  count_launch(2);
}

}  // namespace dcg
