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
// One block per (32 x 32 output tile, channel): it stages x and y on the
// tile plus a 10-pixel halo (52 x 52), runs the horizontal window for the
// five statistics (x, y, x^2, y^2, x y) over it, then each thread runs the
// vertical window for 7 pixels of one column of the tile plus a 5-pixel halo
// (42 x 42) for all five statistics in registers and forms S and the three g
// maps there (zero outside the image; written over the staged images), runs
// the horizontal window over the g maps, and each thread finishes 4 pixels
// of one column of the tile (vertical window of all three maps, x and y read
// again from global memory) and adds them to dL/dI.  No global scratch; the
// loss partial of each block is reduced in a fixed order.
#include <cmath>

#include "kernels.cuh"

namespace dcg {

namespace {

constexpr int kR = 5;                  // window radius
constexpr int kT = 32;                 // output tile
constexpr int kG = kT + 2 * kR;        // 42: region of S and g
constexpr int kA = kT + 4 * kR;        // 52: region of x and y
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

constexpr int kRunH = 14;  // forward horizontal: outputs per item (42 = 3 x 14)
constexpr int kRunV = 7;   // forward vertical + S: pixels per item (42 = 6 x 7; 42 x 6 = 252 items)
constexpr int kRunBH = 8;  // backward horizontal: outputs per item (32 = 4 x 8)
constexpr int kRunBV = 4;  // backward vertical: pixels per item (32 = 8 x 4; 32 x 8 = 256 items)
// shared memory: the staged images (later the g maps) and the horizontal
// results (later the backward horizontal results)
constexpr int kXP = kA + 1, kHP = kG + 1, kGP = kG + 1, kBP = kT + 1;
constexpr int kSmX = 2 * kA * kXP;  // sx, sy
constexpr int kSmH = 5 * kA * kHP;  // h[5]
static_assert(3 * kG * kGP <= kSmX, "g maps fit over the staged images");
static_assert(3 * kG * kBP <= kSmH, "backward horizontal results fit over h");
constexpr size_t kSsimSmem = sizeof(float) * (size_t)(kSmX + kSmH);

__global__ void __launch_bounds__(256) k_ssim(const float* __restrict__ rgb, const float* __restrict__ trgb,
                                              const DevCam* __restrict__ cams, int V, float lam_s,
                                              float* __restrict__ dr, float* __restrict__ part) {
  extern __shared__ float sm[];
  float* const sx = sm;               // [kA][kXP]
  float* const sy = sm + kA * kXP;    // [kA][kXP]
  float* const g = sm;                // [3][kG][kGP], after the forward horizontal pass
  float* const h = sm + kSmX;         // [5][kA][kHP]
  float* const hb = sm + kSmX;        // [3][kG][kBP], after the forward vertical pass
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
  const int ax = tx * kT - 2 * kR, ay = ty * kT - 2 * kR;  // origin of the 52 x 52 region
  const float* X = rgb + 3 * c.pix_off + ch * P;
  const float* Y = trgb + 3 * c.pix_off + ch * P;
  float* D = dr + 3 * c.pix_off + ch * P;
  for (int i = tid; i < kA * kA; i += 256) {
    const int r = i / kA, q = i - r * kA;
    const int gx = ax + q, gy = ay + r;
    const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
    const long long k = (long long)gy * W + gx;
    sx[r * kXP + q] = in ? X[k] : 0.f;
    sy[r * kXP + q] = in ? Y[k] : 0.f;
  }
  __syncthreads();
  // forward horizontal pass: item = (group, row, run of 14 columns); groups:
  // 0 -> (x, x^2) into h[0], h[2]; 1 -> (y, y^2) into h[1], h[3]; 2 -> x y into h[4]
  for (int it = tid; it < 3 * kA * 3; it += 256) {
    const int grp = it / (kA * 3), rem = it - grp * (kA * 3), r = rem / 3, q0 = (rem - r * 3) * kRunH;
    float a[kRunH + 2 * kR], o1[kRunH], o2[kRunH];
    const float* rx = sx + r * kXP + q0;
    const float* ry = sy + r * kXP + q0;
    if (grp == 0) {
#pragma unroll
      for (int k = 0; k < kRunH + 2 * kR; ++k) a[k] = rx[k];
    } else if (grp == 1) {
#pragma unroll
      for (int k = 0; k < kRunH + 2 * kR; ++k) a[k] = ry[k];
    } else {
#pragma unroll
      for (int k = 0; k < kRunH + 2 * kR; ++k) a[k] = rx[k] * ry[k];
    }
    win_run<kRunH>(a, o1);
    float* d1 = h + ((grp == 2 ? 4 : grp) * kA + r) * kHP + q0;
#pragma unroll
    for (int o = 0; o < kRunH; ++o) d1[o] = o1[o];
    if (grp < 2) {
#pragma unroll
      for (int k = 0; k < kRunH + 2 * kR; ++k) a[k] = a[k] * a[k];
      win_run<kRunH>(a, o2);
      float* d2 = h + ((2 + grp) * kA + r) * kHP + q0;
#pragma unroll
      for (int o = 0; o < kRunH; ++o) d2[o] = o2[o];
    }
  }
  __syncthreads();
  // forward vertical pass of all five statistics for 7 pixels of one column
  // of the 42 x 42 region, then S and the g maps (written over the staged images)
  const float coef = -lam_s / (3.f * (float)P);
  float acc = 0.f;
  if (tid < kG * (kG / kRunV)) {
    const int q = tid % kG, r0 = (tid / kG) * kRunV;
    float stv[5][kRunV];
#pragma unroll
    for (int sidx = 0; sidx < 5; ++sidx) {
      float a[kRunV + 2 * kR];
      const float* col = h + (sidx * kA + r0) * kHP + q;
#pragma unroll
      for (int k = 0; k < kRunV + 2 * kR; ++k) a[k] = col[k * kHP];
      win_run<kRunV>(a, stv[sidx]);
    }
    const int px = ax + kR + q;
#pragma unroll
    for (int o = 0; o < kRunV; ++o) {
      const int r = r0 + o, py = ay + kR + r;
      const bool in = px >= 0 && px < W && py >= 0 && py < H;
      float gmu = 0.f, gxx = 0.f, gxy = 0.f;
      if (in) {
        const float mx = stv[0][o], my = stv[1][o], xx = stv[2][o], yy = stv[3][o], xy = stv[4][o];
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
      g[(0 * kG + r) * kGP + q] = gmu;
      g[(1 * kG + r) * kGP + q] = gxx;
      g[(2 * kG + r) * kGP + q] = gxy;
    }
  }
  __syncthreads();
  // backward horizontal pass: item = (g map, row, run of 8 output columns)
  for (int it = tid; it < 3 * kG * (kT / kRunBH); it += 256) {
    const int m = it / (kG * (kT / kRunBH)), rem = it - m * (kG * (kT / kRunBH));
    const int r = rem / (kT / kRunBH), q0 = (rem - r * (kT / kRunBH)) * kRunBH;
    float a[kRunBH + 2 * kR], o[kRunBH];
    const float* row = g + (m * kG + r) * kGP + q0;
#pragma unroll
    for (int k = 0; k < kRunBH + 2 * kR; ++k) a[k] = row[k];
    win_run<kRunBH>(a, o);
    float* d = hb + (m * kG + r) * kBP + q0;
#pragma unroll
    for (int k = 0; k < kRunBH; ++k) d[k] = o[k];
  }
  __syncthreads();
  // backward vertical pass of the three maps for 4 pixels of one column of
  // the tile, and dL/dI there
  {
    const int q = tid % kT, r0 = (tid / kT) * kRunBV;
    float wm[3][kRunBV];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      float a[kRunBV + 2 * kR];
      const float* col = hb + (m * kG + r0) * kBP + q;
#pragma unroll
      for (int k = 0; k < kRunBV + 2 * kR; ++k) a[k] = col[k * kBP];
      win_run<kRunBV>(a, wm[m]);
    }
    const int px = tx * kT + q;
    if (px < W) {
#pragma unroll
      for (int o = 0; o < kRunBV; ++o) {
        const int py = ty * kT + r0 + o;
        if (py < H) {
          const long long p = (long long)py * W + px;
          D[p] += wm[0][o] + 2.f * X[p] * wm[1][o] + Y[p] * wm[2][o];
        }
      }
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
  cudaError_t e = cudaMemcpyToSymbol(c_win, wf, sizeof(wf));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ssim, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSsimSmem);
  return e;
}

void launch_ssim(const float* rgb, const float* trgb, const DevCam* cams, int V, int n_tiles, float lam_s, float* dr,
                 float* loss, float* part, cudaStream_t st) {
  if (n_tiles <= 0) return;
  k_ssim<<<dim3((unsigned)n_tiles, 3), 256, kSsimSmem, st>>>(rgb, trgb, cams, V, lam_s, dr, part);
  k_sum_partials<<<1, 256, 0, st>>>(part, 3ll * n_tiles, lam_s * (float)V, loss);
  count_launch(2);
}

}  // namespace dcg
