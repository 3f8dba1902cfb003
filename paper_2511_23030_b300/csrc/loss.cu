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

// Sliding window of 2R+1 taps over a run of `RUN` outputs: out[o] for
// o < RUN from in[0 .. RUN + 2R), all in registers.
template <int RUN>
__device__ __forceinline__ void win_run(const float (&in)[RUN + 2 * kR], float (&out)[RUN]) {
#pragma unroll
  for (int o = 0; o < RUN; ++o) {
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) acc += c_win[k] * in[o + k];
    out[o] = acc;
  }
}

constexpr int kRunH = 13;  // outputs per thread in the forward horizontal pass (26 = 2 x 13)
constexpr int kRunV = 13;  // outputs per thread in the forward vertical pass
constexpr int kRunBH = 8;  // outputs per thread in the backward horizontal pass (half a row)
constexpr int kRunBV = 4;  // outputs per thread in the backward vertical pass (a quarter column)

__global__ void __launch_bounds__(256) k_ssim(const float* __restrict__ rgb, const float* __restrict__ trgb,
                                              const DevCam* __restrict__ cams, int V, float lam_s,
                                              float* __restrict__ dr, float* __restrict__ part) {
  __shared__ float sx[kA][kA + 1], sy[kA][kA + 1];
  __shared__ float h[5][kA][kG + 1];
  // vertical-pass statistics st[0..4]; after the S pass st[0..2] hold the g
  // maps and the backward horizontal pass writes hb over st[3..4]
  __shared__ float st_raw[5 * kG * (kG + 1)];
  __shared__ float red[8];
  float(*st)[kG][kG + 1] = reinterpret_cast<float(*)[kG][kG + 1]>(st_raw);
  float(*hb)[kG][kT + 1] = reinterpret_cast<float(*)[kG][kT + 1]>(st_raw + 3 * kG * (kG + 1));
  static_assert(3 * kG * (kT + 1) <= 2 * kG * (kG + 1), "hb fits over st[3..4]");
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
  // horizontal pass: item = (row, half of the 26 columns, group); groups:
  // 0 -> (x, x^2), 1 -> (y, y^2), 2 -> x y
  for (int it = tid; it < kA * 2 * 3; it += 256) {
    const int grp = it / (kA * 2), rem = it - grp * (kA * 2), r = rem >> 1, q0 = (rem & 1) * kRunH;
    float a[kRunH + 2 * kR], o1[kRunH], o2[kRunH];
    if (grp == 0) {
#pragma unroll
      for (int k = 0; k < kRunH + 2 * kR; ++k) a[k] = sx[r][q0 + k];
    } else if (grp == 1) {
#pragma unroll
      for (int k = 0; k < kRunH + 2 * kR; ++k) a[k] = sy[r][q0 + k];
    } else {
#pragma unroll
      for (int k = 0; k < kRunH + 2 * kR; ++k) a[k] = sx[r][q0 + k] * sy[r][q0 + k];
    }
    win_run<kRunH>(a, o1);
    if (grp < 2) {
#pragma unroll
      for (int k = 0; k < kRunH + 2 * kR; ++k) a[k] = a[k] * a[k];
      win_run<kRunH>(a, o2);
    }
    float* d1 = grp == 0 ? &h[0][r][q0] : (grp == 1 ? &h[1][r][q0] : &h[4][r][q0]);
    float* d2 = grp == 0 ? &h[2][r][q0] : &h[3][r][q0];
#pragma unroll
    for (int o = 0; o < kRunH; ++o) d1[o] = o1[o];
    if (grp < 2) {
#pragma unroll
      for (int o = 0; o < kRunH; ++o) d2[o] = o2[o];
    }
  }
  __syncthreads();
  // vertical pass: item = (statistic, column, half of the 26 rows)
  for (int it = tid; it < 5 * kG * 2; it += 256) {
    const int sidx = it / (kG * 2), rem = it - sidx * (kG * 2), q = rem >> 1, r0 = (rem & 1) * kRunV;
    float a[kRunV + 2 * kR], o[kRunV];
#pragma unroll
    for (int k = 0; k < kRunV + 2 * kR; ++k) a[k] = h[sidx][r0 + k][q];
    win_run<kRunV>(a, o);
#pragma unroll
    for (int k = 0; k < kRunV; ++k) st[sidx][r0 + k][q] = o[k];
  }
  __syncthreads();
  // S and the g maps on the 26 x 26 region (g written over the statistics)
  const float coef = -lam_s / (3.f * (float)P);
  float acc = 0.f;
  for (int i = tid; i < kG * kG; i += 256) {
    const int r = i / kG, q = i - r * kG;
    const float mx = st[0][r][q], my = st[1][r][q], xx = st[2][r][q], yy = st[3][r][q], xy = st[4][r][q];
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
    st[0][r][q] = gmu;  // each thread rewrites only its own position
    st[1][r][q] = gxx;
    st[2][r][q] = gxy;
  }
  __syncthreads();
  // backward horizontal pass: item = (g map, row, half of the 16 output columns)
  constexpr int kSegH = kT / kRunBH;
  for (int it = tid; it < 3 * kG * kSegH; it += 256) {
    const int m = it / (kG * kSegH), rem = it - m * (kG * kSegH), r = rem / kSegH, q0 = (rem - r * kSegH) * kRunBH;
    float a[kRunBH + 2 * kR], o[kRunBH];
#pragma unroll
    for (int k = 0; k < kRunBH + 2 * kR; ++k) a[k] = st[m][r][q0 + k];
    win_run<kRunBH>(a, o);
#pragma unroll
    for (int k = 0; k < kRunBH; ++k) hb[m][r][q0 + k] = o[k];
  }
  __syncthreads();
  // backward vertical pass: item = (g map, column, quarter of the 16 output rows);
  // the window sums on the tile go to h[m] rows 0..15
  constexpr int kSegV = kT / kRunBV;
  for (int it = tid; it < 3 * kT * kSegV; it += 256) {
    const int m = it / (kT * kSegV), rem = it - m * (kT * kSegV), q = rem / kSegV, r0 = (rem - q * kSegV) * kRunBV;
    float a[kRunBV + 2 * kR], o[kRunBV];
#pragma unroll
    for (int k = 0; k < kRunBV + 2 * kR; ++k) a[k] = hb[m][r0 + k][q];
    win_run<kRunBV>(a, o);
#pragma unroll
    for (int k = 0; k < kRunBV; ++k) h[m][r0 + k][q] = o[k];
  }
  __syncthreads();
  {
    const int r = tid / kT, q = tid - r * kT;  // 256 threads = one output pixel each
    const int px = tx * kT + q, py = ty * kT + r;
    if (px < W && py < H) {
      const float x = sx[r + 2 * kR][q + 2 * kR], y = sy[r + 2 * kR][q + 2 * kR];
      D[(long long)py * W + px] += h[0][r][q] + 2.f * x * h[1][r][q] + y * h[2][r][q];
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
