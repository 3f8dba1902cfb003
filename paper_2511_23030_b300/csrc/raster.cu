// Differentiable tile rasteriser of RGB and depth for the active Gaussians of
// one or several views (Sec. III-E: the visible subset is rasterised and the
// loss of Eq. 2-4 is back-propagated), written for sm_103a.
//
// Forward per render call:
//   1. k_preprocess_fwd   one thread per Gaussian, all views: parameters are
//                         read once per call; per (view, Gaussian) pair the
//                         projection, 2D conic, 3-sigma tile rectangle and SH
//                         colour are written as one 48-byte record.
//   2. compaction         ordered scan over pairs -> keys (view, depth, index)
//   3. depth sort         stable LSD radix sort on the depth bits (the view
//                         bits ride along; the tile sort separates views)
//   4. instance emission  ordered scan of tiles-touched in depth order; each
//                         instance is (half-block mask, global tile id, pair)
//   5. tile sort          stable LSD radix sort on the tile id only: the depth
//                         order inside a tile survives from step 3
//   6. ranges             [start, end) per tile
//   7. k_blend_fwd_h      persistent warps take (tile, warp block) items from a
//                         device queue, compact each half-block's instances in
//                         shared memory, blend front to back
// Backward:
//   8. k_blend_bwd_h      reverse traversal from each pixel's last contributor,
//                         transmittance recomputed by division, per-Gaussian
//                         2D gradients reduced per half-warp (transposed
//                         butterfly), then atomics into the pair's 2D slot
//   9. k_preprocess_bwd   one thread per Gaussian, all views: chain rule to the
//                         parameters (written once) and the pose twist of each
//                         view; it zeroes the 2D slots it consumes, so they are
//                         zero whenever a backward starts
#include <algorithm>
#include <cstdio>

#include "radix.cuh"
#include "kernels.cuh"

namespace dcg {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kPMin = -4.5f * 1.4426950408889634f;  // q <= 9  <=>  p = -(q/2) log2(e) >= -4.5 log2(e)
constexpr float kDilate = 0.3f;

// Real spherical harmonics with Condon-Shortley phase as polynomials of the
// unit direction (x, y, z); constants are K_l^m (times sqrt2 for m != 0) of
// the normalised Legendre form, written out in closed form.
#define SH_C0 0.28209479177387814f   /* 1 / (2 sqrt(pi)) */
#define SH_C1 0.48860251190291992f   /* sqrt(3 / (4 pi)) */
#define SH_C2A 1.0925484305920792f   /* sqrt(15 / pi) / 2 */
#define SH_C2B 0.31539156525252005f  /* sqrt(5 / pi) / 4 */
#define SH_C2C 0.54627421529603959f  /* sqrt(15 / pi) / 4 */
#define SH_C3A -0.59004358992664352f /* -sqrt(35 / (2 pi)) / 4 */
#define SH_C3B 2.8906114426405538f   /* sqrt(105 / pi) / 2 */
#define SH_C3C -0.45704579946446572f /* -sqrt(21 / (2 pi)) / 4 */
#define SH_C3D 0.37317633259011540f  /* sqrt(7 / pi) / 4 */
#define SH_C3E 1.4453057213202769f   /* sqrt(105 / pi) / 4 */

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y) {
  Y[0] = SH_C0;
  if (deg < 1) return;
  Y[1] = -SH_C1 * y;
  Y[2] = SH_C1 * z;
  Y[3] = -SH_C1 * x;
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, yz = y * z, xz = x * z;
  Y[4] = SH_C2A * xy;
  Y[5] = -SH_C2A * yz;
  Y[6] = SH_C2B * (2.f * zz - xx - yy);
  Y[7] = -SH_C2A * xz;
  Y[8] = SH_C2C * (xx - yy);
  if (deg < 3) return;
  Y[9] = SH_C3A * y * (3.f * xx - yy);
  Y[10] = SH_C3B * xy * z;
  Y[11] = SH_C3C * y * (4.f * zz - xx - yy);
  Y[12] = SH_C3D * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = SH_C3C * x * (4.f * zz - xx - yy);
  Y[14] = SH_C3E * z * (xx - yy);
  Y[15] = SH_C3A * x * (xx - 3.f * yy);
}

// Gradient (in R^3) of the basis polynomials above, accumulated as
// g += w_k * grad Y_k for weights w[k].
__device__ __forceinline__ void sh_grad_acc(int deg, float x, float y, float z, const float* w, float* g) {
  if (deg < 1) return;
  g[0] += -SH_C1 * w[3];
  g[1] += -SH_C1 * w[1];
  g[2] += SH_C1 * w[2];
  if (deg < 2) return;
  g[0] += SH_C2A * y * w[4] - 2.f * SH_C2B * x * w[6] - SH_C2A * z * w[7] + 2.f * SH_C2C * x * w[8];
  g[1] += SH_C2A * x * w[4] - SH_C2A * z * w[5] - 2.f * SH_C2B * y * w[6] - 2.f * SH_C2C * y * w[8];
  g[2] += -SH_C2A * y * w[5] + 4.f * SH_C2B * z * w[6] - SH_C2A * x * w[7];
  if (deg < 3) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  g[0] += 6.f * SH_C3A * x * y * w[9] + SH_C3B * y * z * w[10] - 2.f * SH_C3C * x * y * w[11] -
          6.f * SH_C3D * x * z * w[12] + SH_C3C * (4.f * zz - 3.f * xx - yy) * w[13] + 2.f * SH_C3E * x * z * w[14] +
          3.f * SH_C3A * (xx - yy) * w[15];
  g[1] += 3.f * SH_C3A * (xx - yy) * w[9] + SH_C3B * x * z * w[10] + SH_C3C * (4.f * zz - xx - 3.f * yy) * w[11] -
          6.f * SH_C3D * y * z * w[12] - 2.f * SH_C3C * x * y * w[13] - 2.f * SH_C3E * y * z * w[14] -
          6.f * SH_C3A * x * y * w[15];
  g[2] += SH_C3B * x * y * w[10] + 8.f * SH_C3C * y * z * w[11] + SH_C3D * (6.f * zz - 3.f * xx - 3.f * yy) * w[12] +
          8.f * SH_C3C * x * z * w[13] + SH_C3E * (xx - yy) * w[14];
}

// ----------------------------------------------------------------------------
// Double-float (hi + lo) arithmetic from error-free transformations, used for
// the projected centre so that pixel offsets keep ~1e-7 relative precision at
// any image coordinate.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ DF quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
// (r0 m0 + r1 m1 + r2 m2) + t
__device__ __forceinline__ DF df_affine(float r0, float r1, float r2, float m0, float m1, float m2, float t) {
  const DF p0 = two_prod(r0, m0), p1 = two_prod(r1, m1), p2 = two_prod(r2, m2);
  DF s = two_sum(p0.hi, p1.hi);
  float lo = __fadd_rn(s.lo, __fadd_rn(p0.lo, p1.lo));
  DF s2 = two_sum(s.hi, p2.hi);
  lo = __fadd_rn(lo, __fadd_rn(s2.lo, p2.lo));
  DF s3 = two_sum(s2.hi, t);
  lo = __fadd_rn(lo, s3.lo);
  return quick_two_sum(s3.hi, lo);
}
__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const DF p = two_prod(q1, b.hi);
  const float r = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), a.lo), __fmul_rn(q1, b.lo));
  return quick_two_sum(q1, __fdiv_rn(r, b.hi));
}
// f * x + c
__device__ __forceinline__ DF df_scale_add(float f, DF x, float c) {
  const DF p = two_prod(f, x.hi);
  float lo = __fadd_rn(p.lo, __fmul_rn(f, x.lo));
  const DF s = two_sum(p.hi, c);
  lo = __fadd_rn(lo, s.lo);
  return quick_two_sum(s.hi, lo);
}
// (hi + lo) - x0 rounded once to float
__device__ __forceinline__ float df_sub_round(float hi, float lo, float x0) {
  const DF d = two_sum(hi, -x0);
  return __fadd_rn(d.hi, __fadd_rn(d.lo, lo));
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The blend decision shared bit-for-bit by the forward and backward kernels.
// sx = dx * (A' dx), bx = B' dx are per Gaussian and pixel column.
__device__ __forceinline__ float blend_power(float sx, float bx, float Cp, float dy) {
  return __fmaf_rn(dy, __fmaf_rn(Cp, dy, bx), sx);
}

// ----------------------------------------------------------------------------
// Support geometry used by binning.  The support region of a Gaussian is the
// ellipse p(dx, dy) >= pm around its centre, p = A' dx^2 + B' dx dy + C' dy^2
// with the pre-scaled conic (A', C' < 0) and pm = kPMin widened by a margin
// that keeps every decision below conservative against FP32 rounding.  For a
// fixed dy, dx ranges over s dy +- sqrt((m - k dy^2) / a) with a = -A',
// s = B' / 2a, k = -C' - B'^2 / 4a > 0 and m = -pm; the ellipse spans
// |dy| <= sqrt(m / k), and its right-most point has
// dy* = sign(s) sqrt(m s^2 a / (k (k + s^2 a))) (the left-most point is its
// mirror image).  The x-extent of the ellipse within a horizontal band
// [Y0, Y1] is therefore [xL(dyL), xR(dyR)] with dyR, dyL = +-dy* clamped to the
// band, which makes both the tile span of a tile row and the warp blocks a
// Gaussian reaches exact (up to the margin).  Every operation is rounded
// explicitly so the count and emission passes take identical decisions.
struct SupportEllipse {
  float ia, s, k, m, dym, dys;  // ia = 1 / a
};

// Square root from the hardware approximation: a deterministic function of
// its input (so count and emission agree); its error is covered by the slack
// in band_extent.
__device__ __forceinline__ float sqrt_hw(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ SupportEllipse support_of(float4 cn) {
  SupportEllipse e;
  e.ia = __frcp_rn(-cn.x);
  e.s = __fmul_rn(__fmul_rn(cn.y, 0.5f), e.ia);
  e.k = __fsub_rn(-cn.z, __fmul_rn(__fmul_rn(__fmul_rn(cn.y, cn.y), 0.25f), e.ia));
  e.m = -(kPMin * 1.001f - 1e-3f);
  if (!(e.k > 0.f)) {  // not an ellipse (cannot happen for a valid conic): reach nothing
    e.k = 0.f;
    e.dym = -1.f;
    e.dys = 0.f;
    return e;
  }
  e.dym = sqrt_hw(__fmul_rn(e.m, __frcp_rn(e.k)));
  const float t = __fmul_rn(__fmul_rn(e.s, e.s), __frcp_rn(e.ia));
  e.dys = copysignf(sqrt_hw(__fmul_rn(__fmul_rn(e.m, t), __frcp_rn(__fmul_rn(e.k, __fadd_rn(e.k, t))))), e.s);
  return e;
}

// x-extent [*xl, *xr] (relative to the centre) of the ellipse within the band
// dy in [Y0, Y1] (relative to the centre); false if the band misses it.
__device__ __forceinline__ bool band_extent(const SupportEllipse& e, float Y0, float Y1, float* xl, float* xr) {
  const float lo = fmaxf(Y0, -e.dym), hi = fminf(Y1, e.dym);
  if (!(lo <= __fadd_rn(hi, 1e-3f))) return false;
  const float yr = fminf(fmaxf(e.dys, lo), hi), yl = fminf(fmaxf(-e.dys, lo), hi);
  const float hr = sqrt_hw(fmaxf(__fmul_rn(__fsub_rn(e.m, __fmul_rn(__fmul_rn(e.k, yr), yr)), e.ia), 0.f));
  const float hl = sqrt_hw(fmaxf(__fmul_rn(__fsub_rn(e.m, __fmul_rn(__fmul_rn(e.k, yl), yl)), e.ia), 0.f));
  // slack: 1e-3 px plus a relative 1e-5 for the approximate square roots
  *xr = __fadd_rn(__fmaf_rn(hr, 1.00001f, __fmul_rn(e.s, yr)), 1e-3f);
  *xl = __fsub_rn(__fmaf_rn(hl, -1.00001f, __fmul_rn(e.s, yl)), 1e-3f);
  return true;
}

// Instance keys: bits [0, 28) pair index, [28, 48) global tile, [48, 64) the
// half blocks of the tile that the Gaussian reaches (bit 2 b + h: the left
// (h = 0) or right (h = 1) 4 x WY half of the 8 x WY warp block b of
// TileLayout, blocks row-major).  Only the tile bits are sorted.
constexpr int kPairBits = 28;
constexpr u64 kPairMask = (1ull << kPairBits) - 1ull;
constexpr int kTileShift = 28;
constexpr unsigned kTileMask = (1u << 20) - 1u;
constexpr int kMaskShift = 48;
// Rectangles of more tiles than this are emitted whole (every tile).
constexpr int kTightMax = 1024;

__device__ __forceinline__ unsigned half_bits(u64 key, int b) { return (unsigned)(key >> (kMaskShift + 2 * b)) & 3u; }
__device__ __forceinline__ bool block_bit(u64 key, int b) { return half_bits(key, b) != 0u; }
__device__ __forceinline__ unsigned pair_of_inst(u64 key) { return (unsigned)(key & kPairMask); }

// Tiles [*j0, *j1] (offsets from the rectangle's first column) of tile row
// ty of rectangle r that the ellipse reaches; false if none.  Whole
// rectangles (more than kTightMax tiles) keep every tile.
// r0 = (u_hi, v_hi, u_lo, v_lo).
__device__ __forceinline__ bool row_span(const SupportEllipse& e, float4 r0, short4 r, int ty, int tw, int th,
                                         bool whole, int* j0, int* j1) {
  if (whole) {
    *j0 = 0;
    *j1 = r.z - r.x;
    return true;
  }
  const float vl = df_sub_round(r0.y, r0.w, (float)(ty * th));
  float xl, xr;
  if (!band_extent(e, -vl, __fsub_rn((float)(th - 1), vl), &xl, &xr)) return false;
  const float ux = df_sub_round(r0.x, r0.z, (float)(r.x * tw));  // centre relative to the rectangle's left edge
  const float itw = __int_as_float((127 - (__ffs(tw) - 1)) << 23);  // 1 / tw (a power of two): exact
  const float a0 = ceilf(__fmul_rn(__fsub_rn(__fadd_rn(ux, xl), (float)(tw - 1)), itw));
  const float a1 = floorf(__fmul_rn(__fadd_rn(ux, xr), itw));
  *j0 = (int)fminf(fmaxf(a0, 0.f), 32767.f);
  *j1 = (int)fmaxf(fminf(a1, (float)(r.z - r.x)), -1.f);
  return *j0 <= *j1;
}

// Tiles of the rectangle r that the Gaussian reaches (the emission pass
// emits exactly these).
__device__ __forceinline__ uint32_t tight_count(float4 r0, float4 cn, short4 r, int tw, int th) {
  const bool whole = (r.z - r.x + 1) * (r.w - r.y + 1) > kTightMax;
  const SupportEllipse e = support_of(cn);
  uint32_t k = 0;
  for (int ty = r.y; ty <= r.w; ++ty) {
    int j0, j1;
    if (row_span(e, r0, r, ty, tw, th, whole, &j0, &j1)) k += (uint32_t)(j1 - j0 + 1);
  }
  return k;
}

// x-extents of the ellipse in the nbr bands of warp blocks (wy pixel rows
// each) of a tile row; vl is the centre relative to the row's top.  Returns
// the bitmask of bands the ellipse reaches.
__device__ __forceinline__ unsigned block_bands(const SupportEllipse& e, float vl, int wy, int nbr, float* bl,
                                                float* br) {
  unsigned bands = 0;
  for (int rb = 0; rb < nbr; ++rb) {
    const float y0 = __fsub_rn((float)(rb * wy), vl);
    if (band_extent(e, y0, __fadd_rn(y0, (float)(wy - 1)), &bl[rb], &br[rb])) bands |= 1u << rb;
  }
  return bands;
}

// Half blocks (4 columns each, 2 wpr per row) of one tile of that row that
// the ellipse reaches; ul is the centre relative to the tile's left edge.
// Bit 2 (rb wpr + c / 2) + (c & 1) for half column c of band rb: the half
// columns [ceil((ul + bl - 3) / 4), floor((ul + br) / 4)] of each band (the
// extents carry 1e-3 px of slack, more than the rounding here).
__device__ __forceinline__ unsigned tile_block_mask(unsigned bands, const float* bl, const float* br, float ul,
                                                    int wpr, int nbr) {
  unsigned mask = 0;
  const float cmax = (float)(2 * wpr - 1);
  for (int rb = 0; rb < nbr; ++rb) {
    if (!((bands >> rb) & 1u)) continue;
    const float c0 = fmaxf(ceilf((ul + bl[rb] - 3.f) * 0.25f), 0.f);
    const float c1 = fminf(floorf((ul + br[rb]) * 0.25f), cmax);
    if (c0 <= c1) {
      const unsigned run = (2u << (int)c1) - (1u << (int)c0);  // bits c0..c1
      mask |= run << (2 * rb * wpr);
    }
  }
  return mask;
}

// FP32 camera depth in the fixed order ((R20 mx + R21 my) + R22 mz) + t2.
__device__ __forceinline__ float cam_depth(const DevCam& c, float mx, float my, float mz) {
  return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.R[6], mx), __fmul_rn(c.R[7], my)), __fmul_rn(c.R[8], mz)), c.t[2]);
}

// Rotation of the normalised quaternion (w, x, y, z).
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float* R) {
  R[0] = 1.f - 2.f * (y * y + z * z);
  R[1] = 2.f * (x * y - w * z);
  R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);
  R[4] = 1.f - 2.f * (x * x + z * z);
  R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);
  R[7] = 2.f * (y * z + w * x);
  R[8] = 1.f - 2.f * (x * x + y * y);
}

// ============================================================================
// 1. preprocess
// ============================================================================
template <int DEG>
__global__ void __launch_bounds__(256, 4) k_preprocess_fwd(RasterArgs a) {
  const long long n = a.n;
  constexpr int D = (DEG + 1) * (DEG + 1);
  // this thread's SH coefficients, loaded once at its first visible view:
  // element k at shc[k * blockDim.x] (3 D x blockDim.x floats of dynamic shared memory)
  extern __shared__ float s_dyn[];
  float* const shc = s_dyn + threadIdx.x;
  const int bd = blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float* g = a.g;
    const long long S = a.stride;
    bool have_sh = false;
    const float mx = g[0 * S + i], my = g[1 * S + i], mz = g[2 * S + i];
    // 3D covariance Sigma = M M^T, M = R(q) diag(exp(log s))
    const float s0 = __expf(g[3 * S + i]), s1 = __expf(g[4 * S + i]), s2 = __expf(g[5 * S + i]);
    float qw = g[6 * S + i], qx = g[7 * S + i], qy = g[8 * S + i], qz = g[9 * S + i];
    const float qinv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= qinv; qx *= qinv; qy *= qinv; qz *= qinv;
    float R[9];
    quat_rot(qw, qx, qy, qz, R);
    const float M[9] = {R[0] * s0, R[1] * s1, R[2] * s2, R[3] * s0, R[4] * s1, R[5] * s2, R[6] * s0, R[7] * s1, R[8] * s2};
    const float S00 = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    const float S01 = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    const float S02 = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    const float S11 = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    const float S12 = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    const float S22 = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    const float opac = 1.f / (1.f + __expf(-g[10 * S + i]));
    if (dcg_oob((u64)a.V * (u64)n, (u64)a.cap_pairs + 1ull, a.errword)) return;
    for (int v = 0; v < a.V; ++v) {
      const long long vi = (long long)v * n + i;
      const DevCam& c = a.cams[v];
      const float z = cam_depth(c, mx, my, mz);
      a.depth[vi] = z;
      if (!(z > c.znear)) {
        a.touched[vi] = 0;
        a.rect[vi] = make_short4(0, 0, -1, -1);
        continue;
      }
      // projected centre in double-float
      const DF txd = df_affine(c.R[0], c.R[1], c.R[2], mx, my, mz, c.t[0]);
      const DF tyd = df_affine(c.R[3], c.R[4], c.R[5], mx, my, mz, c.t[1]);
      const DF tzd = df_affine(c.R[6], c.R[7], c.R[8], mx, my, mz, c.t[2]);
      const DF ud = df_scale_add(c.fx, df_div(txd, tzd), c.cx);
      const DF vd = df_scale_add(c.fy, df_div(tyd, tzd), c.cy);
      // Jacobian of the perspective map with x/z, y/z clamped
      const float iz = 1.f / z;
      const float rx = fminf(fmaxf(txd.hi * iz, c.xlo), c.xhi);
      const float ry = fminf(fmaxf(tyd.hi * iz, c.ylo), c.yhi);
      const float jx = c.fx * iz, jy = c.fy * iz;
      // Tm = J W: rows (fx/z)(W0 - rx W2), (fy/z)(W1 - ry W2)
      const float T0x = jx * (c.R[0] - rx * c.R[6]), T0y = jx * (c.R[1] - rx * c.R[7]), T0z = jx * (c.R[2] - rx * c.R[8]);
      const float T1x = jy * (c.R[3] - ry * c.R[6]), T1y = jy * (c.R[4] - ry * c.R[7]), T1z = jy * (c.R[5] - ry * c.R[8]);
      const float u0 = S00 * T0x + S01 * T0y + S02 * T0z;
      const float u1 = S01 * T0x + S11 * T0y + S12 * T0z;
      const float u2 = S02 * T0x + S12 * T0y + S22 * T0z;
      const float ca = T0x * u0 + T0y * u1 + T0z * u2 + kDilate;
      const float cb = T1x * u0 + T1y * u1 + T1z * u2;
      const float w0 = S00 * T1x + S01 * T1y + S02 * T1z;
      const float w1 = S01 * T1x + S11 * T1y + S12 * T1z;
      const float w2 = S02 * T1x + S12 * T1y + S22 * T1z;
      const float cc = T1x * w0 + T1y * w1 + T1z * w2 + kDilate;
      const float det = ca * cc - cb * cb;
      // exact bounding box of q <= 9, rounded outwards to whole pixels
      const float ex = 3.f * sqrtf(ca), ey = 3.f * sqrtf(cc);
      const float px0 = fmaxf(floorf(__fsub_rn(ud.hi, ex)), 0.f);
      const float px1 = fminf(ceilf(__fadd_rn(ud.hi, ex)), (float)(c.W - 1));
      const float py0 = fmaxf(floorf(__fsub_rn(vd.hi, ey)), 0.f);
      const float py1 = fminf(ceilf(__fadd_rn(vd.hi, ey)), (float)(c.H - 1));
      if (!(det > 0.f) || !(px0 <= px1) || !(py0 <= py1)) {
        a.touched[vi] = 0;
        a.rect[vi] = make_short4(0, 0, -1, -1);
        continue;
      }
      // tile sizes are powers of two and the pixel bounds are >= 0: shifts
      const int sw = __ffs(a.tile_w) - 1, sh = __ffs(a.tile_h) - 1;
      const int tx0 = (int)px0 >> sw, tx1 = (int)px1 >> sw;
      const int ty0 = (int)py0 >> sh, ty1 = (int)py1 >> sh;
      const short4 rc = make_short4((short)tx0, (short)ty0, (short)tx1, (short)ty1);
      a.rect[vi] = rc;
      const float idet = 1.f / det;
      const float A = cc * idet, B = -cb * idet, Cn = ca * idet;
      const float4 r0 = make_float4(ud.hi, vd.hi, ud.lo, vd.lo);
      const float4 cn = make_float4(-0.5f * kLog2e * A, -kLog2e * B, -0.5f * kLog2e * Cn, opac);
      // tiles of the rectangle that the support ellipse reaches, from the
      // binning record the emission reads back (the centre's leading parts
      // only: the support margin of 1e-3 px covers the rest, < 1e-4 px)
      const float4 b0 = make_float4(ud.hi, vd.hi, cn.x, cn.y);
      const float4 b1 = make_float4(cn.z, __int_as_float((tx0 & 0xffff) | (ty0 << 16)),
                                    __int_as_float((tx1 & 0xffff) | (ty1 << 16)), 0.f);
      a.bin[2 * vi + 0] = b0;
      a.bin[2 * vi + 1] = b1;
      a.touched[vi] = tight_count(make_float4(b0.x, b0.y, 0.f, 0.f), make_float4(b0.z, b0.w, b1.x, 0.f), rc,
                                  a.tile_w, a.tile_h);
      // colour: SH of the direction from the camera centre
      float dx = mx - c.C[0], dy = my - c.C[1], dz = mz - c.C[2];
      const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
      dx *= il; dy *= il; dz *= il;
      float Y[16];
      sh_basis(DEG, dx, dy, dz, Y);
      if (!have_sh) {
#pragma unroll
        for (int k = 0; k < 3 * D; ++k) shc[k * bd] = g[(11 + k) * S + i];
        have_sh = true;
      }
      float col[3];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) acc += shc[(3 * k + ch) * bd] * Y[k];
        col[ch] = fmaxf(acc + 0.5f, 0.f);
      }
      a.rec[3 * vi + 0] = r0;
      a.rec[3 * vi + 1] = cn;
      a.rec[3 * vi + 2] = make_float4(col[0], col[1], col[2], z);
    }
  }
}

// ============================================================================
// 2-6. binning
// ============================================================================
// Depth keys: [count | view | depth bits | index].  The bits above the view
// carry min(tiles touched, cmax) when the key has room (cmax > 0), so that
// the instance-offset scan reads the key alone; cmax itself means "look the
// count up".  Only the depth bits are sorted; the rest rides along.
struct DepthKey {
  int ib;       // index bits
  int vb;       // view bits
  int cs;       // shift of the count field
  unsigned cmax;
  __device__ u64 pair(u64 key, long long n) const {
    const u64 v = (key >> (31 + ib)) & ((1ull << vb) - 1ull);
    const u64 i = key & ((1ull << ib) - 1);
    return v * (u64)n + i;
  }
  __device__ int view(u64 key) const { return (int)((key >> (31 + ib)) & ((1ull << vb) - 1ull)); }
};
// Unsigned 32-bit division by an invariant divisor d >= 1 with one
// multiply-high, after Granlund and Montgomery, "Division by Invariant
// Integers using Multiplication" (PLDI 1994), Fig. 4.1: with l = ceil(log2 d)
// and m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((k - t) >> min(l, 1))) >>
// max(l - 1, 0), t = the high word of m k; exact for every 32-bit k.
struct DivU32 {
  unsigned m;
  int s1, s2;
  static DivU32 make(unsigned d) {
    int l = 0;
    while ((1ull << l) < (unsigned long long)d) ++l;
    DivU32 r;
    r.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1ull);
    r.s1 = l < 1 ? l : 1;
    r.s2 = l > 1 ? l - 1 : 0;
    return r;
  }
  __device__ __forceinline__ unsigned div(unsigned k) const {
    const unsigned t = __umulhi(m, k);
    return (t + ((k - t) >> s1)) >> s2;
  }
};

// Key source of the depth sort's first pass: pair k = v n + i (every pair
// of the views, in order) yields the depth key of a visible pair (one that
// touches a tile); the pass keeps the visible pairs in pair order, so the
// compaction and the first digit's scatter are one pass.
struct PairKeySrc {
  const float* depth;  // written for every pair by the preprocess
  const uint32_t* touched;
  unsigned n;          // pair indices fit in 28 bits
  DivU32 dn;           // division by n
  DepthKey dk;
  __device__ __forceinline__ bool operator()(u64 k, u64* key) const {
    const uint32_t t = touched[k];
    const float z = depth[k];
    const unsigned kk = (unsigned)k, v = dn.div(kk), i = kk - v * n;
    u64 x = ((u64)v << (31 + dk.ib)) | ((u64)__float_as_uint(z) << dk.ib) | (u64)i;
    if (dk.cmax) x |= (u64)min(t, dk.cmax) << dk.cs;
    *key = x;
    return t != 0u;
  }
};
struct InstCount {
  const u64* list;
  const uint32_t* touched;
  long long n;
  DepthKey dk;
  __device__ u64 of_key(u64 key) const {
    if (dk.cmax) {
      const unsigned c = (unsigned)(key >> dk.cs);
      if (c < dk.cmax) return c;
    }
    return touched[dk.pair(key, n)];
  }
  __device__ u64 operator()(u64 s) const { return of_key(list[s]); }
};

// Instance offsets: the exclusive scan, in depth order, of the tiles each
// visible pair reaches (an ordered partitioned scan as part_scan_emit, with
// partitions of a multiple of 4 pairs so that a thread reads 4 consecutive
// keys and writes 4 offsets with 16-byte accesses).
__device__ __forceinline__ void partition4_of(u64 n, u64* beg, u64* end) {
  const u64 P = gridDim.x;
  const u64 len = (((n + P - 1) / P) + 3) & ~3ull;
  const u64 b = (u64)blockIdx.x * len, e = b + len;
  *beg = b < n ? b : n;
  *end = e < n ? e : n;
}

// 4 counts of the group of pairs [k0, k0 + 4) (0 past end)
__device__ __forceinline__ void inst_counts4(const InstCount& f, u64 k0, u64 end, u64 c[4]) {
  if (k0 + 4 <= end) {
    const ulonglong2 a = reinterpret_cast<const ulonglong2*>(f.list + k0)[0];
    const ulonglong2 b = reinterpret_cast<const ulonglong2*>(f.list + k0)[1];
    c[0] = f.of_key(a.x);
    c[1] = f.of_key(a.y);
    c[2] = f.of_key(b.x);
    c[3] = f.of_key(b.y);
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r) c[r] = k0 + r < end ? f(k0 + r) : 0ull;
  }
}

__global__ void __launch_bounds__(256) k_inst_reduce(const u64* n_ptr, InstCount f, u64* part) {
  const u64 n = *n_ptr;
  u64 beg, end;
  partition4_of(n, &beg, &end);
  u64 acc = 0;
  for (u64 k0 = beg + 4ull * threadIdx.x; k0 < end; k0 += 4ull * blockDim.x) {
    u64 c[4];
    inst_counts4(f, k0, end, c);
    acc += c[0] + c[1] + c[2] + c[3];
  }
  __shared__ u64 red[32];
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane_id() == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    u64 s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(256) k_inst_offsets(const u64* n_ptr, InstCount f, const u64* part, u64* offs) {
  const u64 n = *n_ptr;
  u64 beg, end;
  partition4_of(n, &beg, &end);
  u64 base = part[blockIdx.x];
  for (u64 c0 = beg; c0 < end; c0 += 4ull * blockDim.x) {
    const u64 k0 = c0 + 4ull * threadIdx.x;
    u64 c[4];
    inst_counts4(f, k0, end, c);
    u64 tot;
    const u64 o0 = base + block_excl_scan<u64>(c[0] + c[1] + c[2] + c[3], &tot);
    const u64 o1 = o0 + c[0], o2 = o1 + c[1], o3 = o2 + c[2];
    if (k0 + 4 <= end) {
      reinterpret_cast<ulonglong2*>(offs + k0)[0] = make_ulonglong2(o0, o1);
      reinterpret_cast<ulonglong2*>(offs + k0)[1] = make_ulonglong2(o2, o3);
    } else {
      const u64 o[4] = {o0, o1, o2, o3};
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (k0 + r < end) offs[k0 + r] = o[r];
    }
    base += tot;
  }
}

// One thread per visible pair (in depth order) writes its instances: the
// tiles of its rectangle that the support ellipse reaches (row spans, the
// same as the count in k_preprocess_fwd), each with the mask of the tile's
// half blocks the ellipse reaches (band extents once per tile row).
struct InstEmit {
  const u64* list;
  const float4* bin;
  const DevCam* cams;
  long long n;
  DepthKey dk;
  int tw, th;
  u64* inst;
  u64 cap;
  u64 cap_pairs;     // bounds-check build: pair and tile indices against their buffers
  unsigned n_tiles;
  unsigned* errword;
  // The instances of the pair of depth key `key` from offset `off` on, from
  // its 32-byte binning record (b0, b1: centre (leading parts), conic, tile
  // rectangle); the caller has checked the pair index.
  __device__ void emit(u64 key, u64 off, float4 b0, float4 b1) const {
    const u64 vi = dk.pair(key, n);
    const int v = dk.view(key);
    const int p0 = __float_as_int(b1.y), p1 = __float_as_int(b1.z);
    const short4 r = make_short4((short)(p0 & 0xffff), (short)(p0 >> 16), (short)(p1 & 0xffff), (short)(p1 >> 16));
    const float4 r0 = make_float4(b0.x, b0.y, 0.f, 0.f), cn = make_float4(b0.z, b0.w, b1.x, 0.f);
    const bool whole = (r.z - r.x + 1) * (r.w - r.y + 1) > kTightMax;
    const SupportEllipse e = support_of(cn);
    const u64 base = (u64)cams[v].tile_base;
    const int ntx = cams[v].ntx;
    const int wy = tw * th / 64, wpr = tw / 8, nbr = 64 >> (__ffs(tw) - 1);  // th / wy = 64 / tw (a power of two)
    u64 o = off;
    for (int ty = r.y; ty <= r.w; ++ty) {
      int j0, j1;
      if (!row_span(e, r0, r, ty, tw, th, whole, &j0, &j1)) continue;
      float bl[4], br[4];
      const unsigned bands = block_bands(e, df_sub_round(r0.y, r0.w, (float)(ty * th)), wy, nbr, bl, br);
      const u64 row = base + (u64)ty * ntx + (u64)r.x;
      for (int j = j0; j <= j1; ++j, ++o) {
        const float ul = df_sub_round(r0.x, r0.z, (float)((r.x + j) * tw));
        const u64 m = tile_block_mask(bands, bl, br, ul, wpr, nbr);
        if (dcg_oob(row + (u64)j, n_tiles, errword)) continue;
        if (o < cap) inst[o] = (m << kMaskShift) | ((row + (u64)j) << kTileShift) | vi;
      }
    }
  }
};

// The emission, one thread per visible pair in depth order (grid-stride),
// software-pipelined through shared memory by cp.async: while a thread emits
// pair s, the binning record of its next pair and the key and offset of the
// pair after that are on their way (double-buffered per thread; a slot is
// refilled only after the thread has used what it held).
__global__ void __launch_bounds__(256) k_emit_inst(const u64* n_ptr, const u64* __restrict__ offs, InstEmit e) {
  __shared__ u64 s_key[2][256], s_off[2][256];
  __shared__ float4 s_bin[2][2][256];
  const int t = threadIdx.x;
  const u64 n = *n_ptr;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  u64 s = blockIdx.x * (u64)blockDim.x + t;
  if (s >= n) return;
  // the first pair's key and offset, then its record; the next pair's key and offset
  cp_async8(&s_key[0][t], e.list + s);
  cp_async8(&s_off[0][t], offs + s);
  cp_async_commit();
  cp_async_wait<0>();
  bool ok = true;
  {
    const u64 vi = e.dk.pair(s_key[0][t], e.n);
    ok = !dcg_oob(vi, e.cap_pairs, e.errword);
    if (ok) {
      cp_async16(&s_bin[0][0][t], e.bin + 2 * vi + 0);
      cp_async16(&s_bin[0][1][t], e.bin + 2 * vi + 1);
    }
  }
  if (s + stride < n) {
    cp_async8(&s_key[1][t], e.list + s + stride);
    cp_async8(&s_off[1][t], offs + s + stride);
  }
  cp_async_commit();
  for (int c = 0; s < n; s += stride, c ^= 1) {
    cp_async_wait<0>();  // this pair's record, the next pair's key and offset
    const u64 key = s_key[c][t], off = s_off[c][t];
    const float4 b0 = s_bin[c][0][t], b1 = s_bin[c][1][t];
    const bool ok_here = ok;
    ok = true;
    if (s + stride < n) {
      const u64 vi = e.dk.pair(s_key[c ^ 1][t], e.n);
      ok = !dcg_oob(vi, e.cap_pairs, e.errword);
      if (ok) {
        cp_async16(&s_bin[c ^ 1][0][t], e.bin + 2 * vi + 0);
        cp_async16(&s_bin[c ^ 1][1][t], e.bin + 2 * vi + 1);
      }
    }
    if (ok_here) e.emit(key, off, b0, b1);  // uses this slot's key, offset and record
    if (s + 2 * stride < n) {
      cp_async8(&s_key[c][t], e.list + s + 2 * stride);
      cp_async8(&s_off[c][t], offs + s + 2 * stride);
    }
    cp_async_commit();
  }
}

__global__ void k_clamp_inst(DevCounters* c, u64 cap, unsigned* errword) {
  const u64 k = c->n_inst;
  c->n_inst_c = k < cap ? k : cap;
  if (k > cap) atomicOr(errword, ERRW_CAPACITY_BIT);
}

// Per-tile ranges [start, end) of the sorted instances.  A thread takes 4
// consecutive instances (two 16-byte loads where all 4 exist) and compares
// their tiles with each other and with the instances either side.
__device__ __forceinline__ unsigned tile_of_inst(u64 key) { return (unsigned)(key >> kTileShift) & kTileMask; }

__global__ void k_ranges(const u64* __restrict__ inst, const u64* n_ptr, uint2* __restrict__ ranges, unsigned n_tiles,
                         unsigned* errword) {
  const u64 K = *n_ptr;
  const u64 G = (K + 3) / 4;
  for (u64 gi = blockIdx.x * (u64)blockDim.x + threadIdx.x; gi < G; gi += (u64)gridDim.x * blockDim.x) {
    const u64 k0 = 4 * gi;
    unsigned t[6];  // t[0]: the instance before, t[1..4]: the group, t[5]: the instance after
    if (k0 + 4 <= K) {
      const ulonglong2 a = reinterpret_cast<const ulonglong2*>(inst)[2 * gi];
      const ulonglong2 b = reinterpret_cast<const ulonglong2*>(inst)[2 * gi + 1];
      t[1] = tile_of_inst(a.x);
      t[2] = tile_of_inst(a.y);
      t[3] = tile_of_inst(b.x);
      t[4] = tile_of_inst(b.y);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) t[1 + j] = k0 + j < K ? tile_of_inst(inst[k0 + j]) : 0xffffffffu;
    }
    t[0] = k0 > 0 ? tile_of_inst(inst[k0 - 1]) : 0xffffffffu;
    t[5] = k0 + 4 < K ? tile_of_inst(inst[k0 + 4]) : 0xffffffffu;
#pragma unroll
    for (int j = 1; j <= 4; ++j) {
      const u64 k = k0 + j - 1;
      if (k >= K) break;
      if (dcg_oob(t[j], n_tiles, errword)) continue;
      if (t[j - 1] != t[j]) ranges[t[j]].x = (unsigned)k;
      if (t[j + 1] != t[j]) ranges[t[j]].y = (unsigned)(k + 1);
    }
  }
}

// ============================================================================
// 7. forward blend
// ============================================================================
__device__ __forceinline__ int view_of_tile(const DevCam* cams, int V, unsigned gt) {
  int v = 0;
  while (v + 1 < V && (int)gt >= cams[v + 1].tile_base) ++v;
  return v;
}

// Pixel layout of a tile: 8 warps, each owning an 8 x (4 PPT) block of pixels
// (lane -> 8 columns x 4 rows, each thread PPT rows spaced by 4), so that a
// warp can skip a staged Gaussian whose 3-sigma box misses its block.
template <int TW, int TH>
struct TileLayout {
  static constexpr int PPT = TW * TH / 256;
  static constexpr int WY = 4 * PPT;     // rows of a warp block
  static constexpr int WPR = TW / 8;     // warp blocks per tile row
  static_assert(WPR * (TH / WY) == 8, "eight warp blocks per tile");
};

// Forward blend.  One block per tile (taken from a device queue); each of
// its 8 warps owns an 8 x WY pixel block and walks the tile's depth-sorted
// list on its own: 32 instances per step, one per lane, are tested against
// the warp block (either half bit), survivors are compacted in order into a per-warp shared
// buffer and blended by all lanes.  A warp stops when its pixels are done;
// there is no block barrier inside a tile.
template <int TW, int TH, int STAGE>
__global__ void __launch_bounds__(256) k_blend_fwd(RasterArgs a, const u64* __restrict__ inst, float* __restrict__ rgb,
                                                   float* __restrict__ dout) {
  using L = TileLayout<TW, TH>;
  constexpr int PPT = L::PPT;
  __shared__ float2 s_xy[8][32];
  __shared__ float4 s_con[8][32];
  __shared__ float4 s_col[8][32];
  __shared__ unsigned s_rel[8][32];
  __shared__ unsigned s_tile;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int bx0 = (w % L::WPR) * 8, by0 = (w / L::WPR) * L::WY;
  const int lx = bx0 + (lane & 7);
  const int ly = by0 + (lane >> 3);
  const unsigned lt = lanemask_lt();
  for (;;) {
    __syncthreads();
    if (tid == 0) s_tile = atomicAdd(&a.counters->tile_queue, 1u);
    __syncthreads();
    const unsigned gt = s_tile;
    if (gt >= (unsigned)a.n_tiles) break;
    const int v = view_of_tile(a.cams, a.V, gt);
    const DevCam& c = a.cams[v];
    const int W = c.W, H = c.H;
    const int local = (int)gt - c.tile_base;
    const int ty = local / c.ntx, tx = local - ty * c.ntx;
    const int x0 = tx * TW, y0 = ty * TH;
    const float x0f = (float)x0, y0f = (float)y0;
    float T[PPT], Tf[PPT], Cr[PPT], Cg[PPT], Cb[PPT], Dz[PPT];
    uint32_t last[PPT];
    unsigned ev = 0, nb = 0;  // evaluations of (live pixel, Gaussian) pairs by this thread
    const int px = x0 + lx;
    int alive = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int py = y0 + ly + 4 * k;
      T[k] = (px < W && py < H) ? 1.f : 0.f;
      Tf[k] = T[k];
      Cr[k] = Cg[k] = Cb[k] = Dz[k] = 0.f;
      last[k] = 0;
      alive |= T[k] > 0.f;
    }
    const uint2 rg = a.ranges[gt];
    for (unsigned b0 = rg.x; b0 < rg.y && __any_sync(0xffffffffu, alive); b0 += 32) {
      const unsigned idx = b0 + lane;
      bool pass = false;
      unsigned vi = 0;
      if (idx < rg.y) {
        const u64 key = inst[idx];
        vi = pair_of_inst(key);
        pass = block_bit(key, w);
      }
      const unsigned m = __ballot_sync(0xffffffffu, pass);
      if (pass) {
        const float4 r0 = a.rec[3ull * vi + 0];
        const int slot = __popc(m & lt);
        s_xy[w][slot] = make_float2(df_sub_round(r0.x, r0.z, x0f), df_sub_round(r0.y, r0.w, y0f));
        s_con[w][slot] = a.rec[3ull * vi + 1];
        s_col[w][slot] = a.rec[3ull * vi + 2];
        s_rel[w][slot] = idx - rg.x;
      }
      __syncwarp();
      const int cnt = __popc(m);
      for (int j = 0; j < cnt; ++j) {
        const float2 xy = s_xy[w][j];
        const float4 cq = s_con[w][j];
        const float dx = __fsub_rn((float)lx, xy.x);
        const float sx = __fmul_rn(dx, __fmul_rn(cq.x, dx));
        const float bx = __fmul_rn(cq.y, dx);
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          if (T[k] > 0.f) {
            ++ev;
            const float dy = __fsub_rn((float)(ly + 4 * k), xy.y);
            const float p = blend_power(sx, bx, cq.z, dy);
            if (p >= kPMin) {
              const float al = fminf(kAlphaMax, __fmul_rn(cq.w, ex2_approx(p)));
              if (al >= kAlphaMin) {
                const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, al));
                if (Tn < kTMin) {
                  Tf[k] = T[k];
                  T[k] = 0.f;
                } else {
                  const float4 cl = s_col[w][j];
                  const float wgt = al * T[k];
                  Cr[k] += wgt * cl.x;
                  Cg[k] += wgt * cl.y;
                  Cb[k] += wgt * cl.z;
                  Dz[k] += wgt * cl.w;
                  T[k] = Tn;
                  last[k] = s_rel[w][j] + 1;
                  ++nb;
                }
              }
            }
          }
        }
      }
      __syncwarp();
      alive = 0;
#pragma unroll
      for (int k = 0; k < PPT; ++k) alive |= T[k] > 0.f;
    }
    {
      const unsigned wev = __reduce_add_sync(0xffffffffu, ev), wnb = __reduce_add_sync(0xffffffffu, nb);
      if (lane == 0 && wev) atomicAdd(&a.counters->n_eval, (unsigned long long)wev);
      if (lane == 0 && wnb) atomicAdd(&a.counters->n_blend, (unsigned long long)wnb);
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int py = y0 + ly + 4 * k;
      if (px < W && py < H) {
        const long long P = (long long)W * H;
        const long long pix = (long long)py * W + px;
        rgb[3 * c.pix_off + pix] = Cr[k];
        rgb[3 * c.pix_off + P + pix] = Cg[k];
        rgb[3 * c.pix_off + 2 * P + pix] = Cb[k];
        dout[c.pix_off + pix] = Dz[k];
        a.T_final[c.pix_off + pix] = T[k] > 0.f ? T[k] : Tf[k];
        a.n_contrib[c.pix_off + pix] = last[k];
      }
    }
  }
}

// ============================================================================
// 8. backward blend
// ============================================================================
// Sum over the 32 lanes of N values with a transposed butterfly: each step
// halves the number of values a lane carries, so N = 10 costs 12 shuffles
// instead of 50.  Afterwards lane l holds the total of component *comp; *has
// is true for exactly one lane per component.  FIRST = 8 sums within each
// half-warp separately (lanes 0-15 and 16-31, 11 shuffles for N = 10).
template <int N, int FIRST = 16>
__device__ __forceinline__ float warp_sum_transpose(float (&v)[N], int* comp, bool* has) {
  const unsigned lane = threadIdx.x & 31u;
  int base = 0, cnt = N;
  int n = N;
  unsigned shared_bits = 0;  // lane bits over which the final value is replicated
#pragma unroll
  for (int o = FIRST; o >= 1; o >>= 1) {
    const bool bit = (lane & (unsigned)o) != 0u;
    if (n > 1) {
      const int half = (n + 1) / 2;
#pragma unroll
      for (int k = 0; k < (N + 1) / 2; ++k) {
        if (k < half) {
          const float hi = (k + half < n) ? v[k + half] : 0.f;
          const float send = bit ? v[k] : hi;
          const float keep = bit ? hi : v[k];
          v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      if (bit) {
        base += half;
        cnt = cnt > half ? cnt - half : 0;
      } else {
        cnt = cnt < half ? cnt : half;
      }
      n = half;
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
      shared_bits |= (unsigned)o;
    }
  }
  *comp = base;
  *has = cnt > 0 && (lane & shared_bits) == 0u;
  return v[0];
}

// Backward blend.  One block per tile; the tile's list is cut into segments
// of STAGE Gaussians taken from the end (last contributor) backwards.  Within
// a segment every warp walks it on its own, 32 instances per step in reverse
// order (filtered by the warp block and the warp's last contributor,
// compacted with a ballot), recomputes transmittance by division and adds the
// warp-reduced 2D gradients of each Gaussian into a block-shared accumulator;
// at the end of the segment the accumulators go to global memory with one
// set of vector atomics per Gaussian.
template <int TW, int TH, int STAGE>
__global__ void __launch_bounds__(256) k_blend_bwd(RasterArgs a, const u64* __restrict__ inst,
                                                   const float* __restrict__ dL_drgb,
                                                   const float* __restrict__ dL_ddepth) {
  using L = TileLayout<TW, TH>;
  constexpr int PPT = L::PPT;
  __shared__ float2 s_xy[8][32];
  __shared__ float4 s_con[8][32];
  __shared__ float4 s_col[8][32];
  __shared__ unsigned s_rel[8][32];
  __shared__ float s_acc[STAGE][10];
  __shared__ unsigned s_tile;
  __shared__ unsigned s_maxlast;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int bx0 = (w % L::WPR) * 8, by0 = (w / L::WPR) * L::WY;
  const int lx = bx0 + (lane & 7);
  const int ly = by0 + (lane >> 3);
  const unsigned lt = lanemask_lt();
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      s_tile = atomicAdd(&a.counters->tile_queue_bwd, 1u);
      s_maxlast = 0;
    }
    __syncthreads();
    const unsigned gt = s_tile;
    if (gt >= (unsigned)a.n_tiles) break;
    const int v = view_of_tile(a.cams, a.V, gt);
    const DevCam& c = a.cams[v];
    const int W = c.W, H = c.H;
    const int local = (int)gt - c.tile_base;
    const int ty = local / c.ntx, tx = local - ty * c.ntx;
    const int x0 = tx * TW, y0 = ty * TH;
    const float x0f = (float)x0, y0f = (float)y0;
    const long long P = (long long)W * H;
    float T[PPT], gr[PPT], gg[PPT], gb[PPT], gd[PPT], Dg[PPT];
    uint32_t last[PPT];
    const int px = x0 + lx;
    uint32_t mylast = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int py = y0 + ly + 4 * k;
      last[k] = 0;
      T[k] = 0.f;
      gr[k] = gg[k] = gb[k] = gd[k] = 0.f;
      if (px < W && py < H) {
        const long long pix = (long long)py * W + px;
        T[k] = a.T_final[c.pix_off + pix];
        last[k] = a.n_contrib[c.pix_off + pix];
        gr[k] = dL_drgb[3 * c.pix_off + pix];
        gg[k] = dL_drgb[3 * c.pix_off + P + pix];
        gb[k] = dL_drgb[3 * c.pix_off + 2 * P + pix];
        gd[k] = dL_ddepth[c.pix_off + pix];
      }
      Dg[k] = 0.f;
      mylast = max(mylast, last[k]);
    }
    const int warplast = (int)__reduce_max_sync(0xffffffffu, mylast);
    if (lane == 0) atomicMax(&s_maxlast, (unsigned)warplast);
    __syncthreads();
    const int maxlast = (int)s_maxlast;
    const uint2 rg = a.ranges[gt];
    for (int send = maxlast; send > 0; send -= STAGE) {
      const int sbeg = max(0, send - STAGE);
      for (int e = tid; e < (send - sbeg) * 10; e += 256) (&s_acc[0][0])[e] = 0.f;
      __syncthreads();
      // this warp's part of the segment: relative indices [sbeg, min(send, warplast))
      for (int hi = min(send, warplast); hi > sbeg; hi -= 32) {
        const int rel = hi - 1 - lane;  // lane 0 takes the largest index: compaction keeps reverse order
        bool pass = false;
        unsigned vi = 0;
        if (rel >= sbeg) {
          const u64 key = inst[rg.x + rel];
          vi = pair_of_inst(key);
          pass = block_bit(key, w);
        }
        const unsigned m = __ballot_sync(0xffffffffu, pass);
        if (pass) {
          const float4 r0 = a.rec[3ull * vi + 0];
          const int slot = __popc(m & lt);
          s_xy[w][slot] = make_float2(df_sub_round(r0.x, r0.z, x0f), df_sub_round(r0.y, r0.w, y0f));
          s_con[w][slot] = a.rec[3ull * vi + 1];
          s_col[w][slot] = a.rec[3ull * vi + 2];
          s_rel[w][slot] = (unsigned)rel;
        }
        __syncwarp();
        const int cnt = __popc(m);
        for (int j = 0; j < cnt; ++j) {
          const int r = (int)s_rel[w][j];
          const float2 xy = s_xy[w][j];
          const float4 cq = s_con[w][j];
          const float dx = __fsub_rn((float)lx, xy.x);
          const float sx = __fmul_rn(dx, __fmul_rn(cq.x, dx));
          const float bx = __fmul_rn(cq.y, dx);
          float acc[10];
#pragma unroll
          for (int q = 0; q < 10; ++q) acc[q] = 0.f;
          bool any = false;
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            if (r < (int)last[k]) {
              const float dy = __fsub_rn((float)(ly + 4 * k), xy.y);
              const float p = blend_power(sx, bx, cq.z, dy);
              if (p >= kPMin) {
                const float G = ex2_approx(p);
                const float araw = __fmul_rn(cq.w, G);
                const float al = fminf(kAlphaMax, araw);
                if (al >= kAlphaMin) {
                  any = true;
                  const float4 cl = s_col[w][j];
                  T[k] = __fdividef(T[k], 1.f - al);
                  const float wgt = al * T[k];
                  acc[6] += wgt * gr[k];
                  acc[7] += wgt * gg[k];
                  acc[8] += wgt * gb[k];
                  acc[9] += wgt * gd[k];
                  // dL/dalpha = T (c . g - D) with D = sum over channels of g times the
                  // colour (and depth) composited behind this Gaussian; D follows the
                  // same over-recursion as the colours themselves
                  const float cg = cl.x * gr[k] + cl.y * gg[k] + cl.z * gb[k] + cl.w * gd[k];
                  const float dal = T[k] * (cg - Dg[k]);
                  Dg[k] = al * cg + (1.f - al) * Dg[k];
                  if (araw < kAlphaMax) {
                    // moments of dL/dalpha * G; the conic and opacity factors are applied per
                    // Gaussian in k_preprocess_bwd
                    const float gG = dal * G;
                    const float gx = gG * dx, gy = gG * dy;
                    acc[5] += gG;
                    acc[0] += gx;
                    acc[1] += gy;
                    acc[2] += gx * dx;
                    acc[3] += gx * dy;
                    acc[4] += gy * dy;
                  }
                }
              }
            }
          }
          if (__any_sync(0xffffffffu, any)) {
            int comp;
            bool has;
            const float tot = warp_sum_transpose<10>(acc, &comp, &has);
            if (has) atomicAdd(&s_acc[r - sbeg][comp], tot);
          }
        }
        __syncwarp();
      }
      __syncthreads();
      for (int j = tid; j < send - sbeg; j += 256) {
        const float* q = s_acc[j];
        const float4 g0 = make_float4(q[0], q[1], q[2], q[3]);
        const float4 g1 = make_float4(q[4], q[5], q[6], q[7]);
        const bool n0 = g0.x != 0.f || g0.y != 0.f || g0.z != 0.f || g0.w != 0.f;
        const bool n1 = g1.x != 0.f || g1.y != 0.f || g1.z != 0.f || g1.w != 0.f;
        const bool n2 = q[8] != 0.f || q[9] != 0.f;
        if (n0 || n1 || n2) {
          float4* gp = a.grad2d + 3ull * pair_of_inst(inst[rg.x + sbeg + j]);
          if (n0) atomicAdd(gp + 0, g0);
          if (n1) atomicAdd(gp + 1, g1);
          if (n2) atomicAdd(reinterpret_cast<float2*>(gp + 2), make_float2(q[8], q[9]));
        }
      }
      __syncthreads();
    }
  }
}

// ============================================================================
// Warp-per-block blends.  The per-warp work is that of the block-per-tile
// kernels (one 8 x WY pixel block of a tile, its own walk of the tile's
// list), but every warp takes its (tile, block) items from a device queue on
// its own, so there is no block barrier anywhere: a warp whose pixels finish
// early moves on at once.  Items are numbered tile-major (8 per tile), so the
// warps of one SM tend to share a tile's list in L1.  The backward has no
// tile-shared accumulator: after the warp reduction each of the 10 lanes that
// hold a component of a Gaussian's 2D gradient adds it to global memory
// (one red instruction per Gaussian and warp).  Per-pixel arithmetic is that
// of the block-per-tile kernels, so images are identical.
template <int TW, int TH>
__global__ void __launch_bounds__(256) k_blend_fwd_q(RasterArgs a, const u64* __restrict__ inst,
                                                     float* __restrict__ rgb, float* __restrict__ dout) {
  using L = TileLayout<TW, TH>;
  constexpr int PPT = L::PPT;
  __shared__ float2 s_xy[8][32];
  __shared__ float4 s_con[8][32];
  __shared__ float4 s_col[8][32];
  __shared__ unsigned s_rel[8][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const unsigned n_items = 8u * (unsigned)a.n_tiles;
  for (;;) {
    unsigned item = 0;
    if (lane == 0) item = atomicAdd(&a.counters->tile_queue, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    const unsigned gt = item >> 3, wb = item & 7u;
    const int bx0 = (int)(wb % L::WPR) * 8, by0 = (int)(wb / L::WPR) * L::WY;
    const int lx = bx0 + (lane & 7);
    const int ly = by0 + (lane >> 3);
    const int v = view_of_tile(a.cams, a.V, gt);
    const DevCam& c = a.cams[v];
    const int W = c.W, H = c.H;
    const int local = (int)gt - c.tile_base;
    const int ty = local / c.ntx, tx = local - ty * c.ntx;
    const int x0 = tx * TW, y0 = ty * TH;
    const float x0f = (float)x0, y0f = (float)y0;
    float T[PPT], Tf[PPT], Cr[PPT], Cg[PPT], Cb[PPT], Dz[PPT];
    uint32_t last[PPT];
    unsigned ev = 0, nb = 0;
    const int px = x0 + lx;
    int alive = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int py = y0 + ly + 4 * k;
      T[k] = (px < W && py < H) ? 1.f : 0.f;
      Tf[k] = T[k];
      Cr[k] = Cg[k] = Cb[k] = Dz[k] = 0.f;
      last[k] = 0;
      alive |= T[k] > 0.f;
    }
    const uint2 rg = a.ranges[gt];
    for (unsigned b0 = rg.x; b0 < rg.y && __any_sync(0xffffffffu, alive); b0 += 32) {
      const unsigned idx = b0 + lane;
      bool pass = false;
      unsigned vi = 0;
      if (idx < rg.y) {
        const u64 key = inst[idx];
        vi = pair_of_inst(key);
        pass = block_bit(key, wb);
      }
      const unsigned m = __ballot_sync(0xffffffffu, pass);
      if (pass) {
        const float4 r0 = a.rec[3ull * vi + 0];
        const int slot = __popc(m & lt);
        s_xy[w][slot] = make_float2(df_sub_round(r0.x, r0.z, x0f), df_sub_round(r0.y, r0.w, y0f));
        s_con[w][slot] = a.rec[3ull * vi + 1];
        s_col[w][slot] = a.rec[3ull * vi + 2];
        s_rel[w][slot] = idx - rg.x;
      }
      __syncwarp();
      const int cnt = __popc(m);
      for (int j = 0; j < cnt; ++j) {
        const float2 xy = s_xy[w][j];
        const float4 cq = s_con[w][j];
        const float dx = __fsub_rn((float)lx, xy.x);
        const float sx = __fmul_rn(dx, __fmul_rn(cq.x, dx));
        const float bx = __fmul_rn(cq.y, dx);
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          if (T[k] > 0.f) {
            ++ev;
            const float dy = __fsub_rn((float)(ly + 4 * k), xy.y);
            const float p = blend_power(sx, bx, cq.z, dy);
            if (p >= kPMin) {
              const float al = fminf(kAlphaMax, __fmul_rn(cq.w, ex2_approx(p)));
              if (al >= kAlphaMin) {
                const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, al));
                if (Tn < kTMin) {
                  Tf[k] = T[k];
                  T[k] = 0.f;
                } else {
                  const float4 cl = s_col[w][j];
                  const float wgt = al * T[k];
                  Cr[k] += wgt * cl.x;
                  Cg[k] += wgt * cl.y;
                  Cb[k] += wgt * cl.z;
                  Dz[k] += wgt * cl.w;
                  T[k] = Tn;
                  last[k] = s_rel[w][j] + 1;
                  ++nb;
                }
              }
            }
          }
        }
      }
      __syncwarp();
      alive = 0;
#pragma unroll
      for (int k = 0; k < PPT; ++k) alive |= T[k] > 0.f;
    }
    {
      const unsigned wev = __reduce_add_sync(0xffffffffu, ev), wnb = __reduce_add_sync(0xffffffffu, nb);
      if (lane == 0 && wev) atomicAdd(&a.counters->n_eval, (unsigned long long)wev);
      if (lane == 0 && wnb) atomicAdd(&a.counters->n_blend, (unsigned long long)wnb);
    }
    const long long P = (long long)W * H;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int py = y0 + ly + 4 * k;
      if (px < W && py < H && !dcg_oob((u64)(c.pix_off + (long long)py * W + px), (u64)a.n_pix, a.errword)) {
        const long long pix = (long long)py * W + px;
        rgb[3 * c.pix_off + pix] = Cr[k];
        rgb[3 * c.pix_off + P + pix] = Cg[k];
        rgb[3 * c.pix_off + 2 * P + pix] = Cb[k];
        dout[c.pix_off + pix] = Dz[k];
        a.T_final[c.pix_off + pix] = T[k] > 0.f ? T[k] : Tf[k];
        a.n_contrib[c.pix_off + pix] = last[k];
      }
    }
  }
}

template <int TW, int TH>
__global__ void __launch_bounds__(256) k_blend_bwd_q(RasterArgs a, const u64* __restrict__ inst,
                                                     const float* __restrict__ dL_drgb,
                                                     const float* __restrict__ dL_ddepth) {
  using L = TileLayout<TW, TH>;
  constexpr int PPT = L::PPT;
  __shared__ float2 s_xy[8][32];
  __shared__ float4 s_con[8][32];
  __shared__ float4 s_col[8][32];
  __shared__ unsigned s_rel[8][32];
  __shared__ unsigned s_vi[8][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const unsigned n_items = 8u * (unsigned)a.n_tiles;
  float* const g2 = reinterpret_cast<float*>(a.grad2d);
  for (;;) {
    unsigned item = 0;
    if (lane == 0) item = atomicAdd(&a.counters->tile_queue_bwd, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    const unsigned gt = item >> 3, wb = item & 7u;
    const int bx0 = (int)(wb % L::WPR) * 8, by0 = (int)(wb / L::WPR) * L::WY;
    const int lx = bx0 + (lane & 7);
    const int ly = by0 + (lane >> 3);
    const int v = view_of_tile(a.cams, a.V, gt);
    const DevCam& c = a.cams[v];
    const int W = c.W, H = c.H;
    const int local = (int)gt - c.tile_base;
    const int ty = local / c.ntx, tx = local - ty * c.ntx;
    const int x0 = tx * TW, y0 = ty * TH;
    const float x0f = (float)x0, y0f = (float)y0;
    const long long P = (long long)W * H;
    float T[PPT], gr[PPT], gg[PPT], gb[PPT], gd[PPT], Dg[PPT];
    uint32_t last[PPT];
    const int px = x0 + lx;
    uint32_t mylast = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int py = y0 + ly + 4 * k;
      last[k] = 0;
      T[k] = 0.f;
      gr[k] = gg[k] = gb[k] = gd[k] = 0.f;
      if (px < W && py < H) {
        const long long pix = (long long)py * W + px;
        T[k] = a.T_final[c.pix_off + pix];
        last[k] = a.n_contrib[c.pix_off + pix];
        gr[k] = dL_drgb[3 * c.pix_off + pix];
        gg[k] = dL_drgb[3 * c.pix_off + P + pix];
        gb[k] = dL_drgb[3 * c.pix_off + 2 * P + pix];
        gd[k] = dL_ddepth[c.pix_off + pix];
      }
      Dg[k] = 0.f;
      mylast = max(mylast, last[k]);
    }
    const int warplast = (int)__reduce_max_sync(0xffffffffu, mylast);
    const uint2 rg = a.ranges[gt];
    for (int hi = warplast; hi > 0; hi -= 32) {
      const int rel = hi - 1 - lane;  // lane 0 takes the largest index: compaction keeps reverse order
      bool pass = false;
      unsigned vi = 0;
      if (rel >= 0) {
        const u64 key = inst[rg.x + rel];
        vi = pair_of_inst(key);
        pass = block_bit(key, wb);
      }
      const unsigned m = __ballot_sync(0xffffffffu, pass);
      if (pass) {
        const float4 r0 = a.rec[3ull * vi + 0];
        const int slot = __popc(m & lt);
        s_xy[w][slot] = make_float2(df_sub_round(r0.x, r0.z, x0f), df_sub_round(r0.y, r0.w, y0f));
        s_con[w][slot] = a.rec[3ull * vi + 1];
        s_col[w][slot] = a.rec[3ull * vi + 2];
        s_rel[w][slot] = (unsigned)rel;
        s_vi[w][slot] = vi;
      }
      __syncwarp();
      const int cnt = __popc(m);
      for (int j = 0; j < cnt; ++j) {
        const int r = (int)s_rel[w][j];
        const float2 xy = s_xy[w][j];
        const float4 cq = s_con[w][j];
        const float dx = __fsub_rn((float)lx, xy.x);
        const float sx = __fmul_rn(dx, __fmul_rn(cq.x, dx));
        const float bx = __fmul_rn(cq.y, dx);
        float acc[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) acc[q] = 0.f;
        bool any = false;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          if (r < (int)last[k]) {
            const float dy = __fsub_rn((float)(ly + 4 * k), xy.y);
            const float p = blend_power(sx, bx, cq.z, dy);
            if (p >= kPMin) {
              const float G = ex2_approx(p);
              const float araw = __fmul_rn(cq.w, G);
              const float al = fminf(kAlphaMax, araw);
              if (al >= kAlphaMin) {
                any = true;
                const float4 cl = s_col[w][j];
                T[k] = __fdividef(T[k], 1.f - al);
                const float wgt = al * T[k];
                acc[6] += wgt * gr[k];
                acc[7] += wgt * gg[k];
                acc[8] += wgt * gb[k];
                acc[9] += wgt * gd[k];
                // dL/dalpha = T (c . g - D) with D = sum over channels of g times the
                // colour (and depth) composited behind this Gaussian; D follows the
                // same over-recursion as the colours themselves
                const float cg = cl.x * gr[k] + cl.y * gg[k] + cl.z * gb[k] + cl.w * gd[k];
                const float dal = T[k] * (cg - Dg[k]);
                Dg[k] = al * cg + (1.f - al) * Dg[k];
                if (araw < kAlphaMax) {
                  // moments of dL/dalpha * G; the conic and opacity factors are applied per
                  // Gaussian in k_preprocess_bwd
                  const float gG = dal * G;
                  const float gx = gG * dx, gy = gG * dy;
                  acc[5] += gG;
                  acc[0] += gx;
                  acc[1] += gy;
                  acc[2] += gx * dx;
                  acc[3] += gx * dy;
                  acc[4] += gy * dy;
                }
              }
            }
          }
        }
        if (__any_sync(0xffffffffu, any)) {
          int comp;
          bool has;
          const float tot = warp_sum_transpose<10>(acc, &comp, &has);
          if (has && tot != 0.f) atomicAdd(g2 + 12ull * s_vi[w][j] + comp, tot);
        }
      }
      __syncwarp();
    }
  }
}

// ============================================================================
// Half-warp blends.  As the warp-per-block kernels, but the two halves of a
// warp own the two 4 x WY halves of its 8 x WY block (lane l: half l / 16,
// column l % 4, row (l / 4) % 4) and each half walks its own list: an
// instance enters the list of each half whose pixels its support ellipse may
// reach (two bits of the instance mask).  A small Gaussian that reaches one
// half occupies 16 lanes instead of 32, and the other half takes the next
// Gaussian of its own list in the same step.  The forward compacts each
// batch of 32 tile instances into two lists and pads the shorter one with
// transparent entries.  The backward keeps a ring buffer of R entries per
// half in shared memory, refilled 32 tile instances at a time while a half
// holds fewer than 32, so that a half can run ahead of the other across scan
// batches; a half with nothing to do steps through a neutral entry (slot R).
// A half whose pixels are all done (forward) or whose instances lie behind
// all of its pixels' last contributors (backward) takes no more instances.
// The backward reduces each half's Gaussian over its 16 lanes (one
// transposed butterfly serves both halves).  Per-pixel arithmetic and order
// are those of the other kernels, so images are identical.
constexpr int kRingB = 60;  // ring entries per half (static shared memory under 48 KB)

// Steps the halves run before the next refill: together while both hold
// entries; otherwise the one that holds entries runs until a refill fits
// (nothing is left to scan, or its count is down to R - 32).
__device__ __forceinline__ int ring_steps(int pL, int pR, bool more, int R) {
  if (pL > 0 && pR > 0) return min(pL, pR);
  const int p = max(pL, pR);
  return more ? p - (R - 32) : p;
}

template <int TW, int TH>
__global__ void __launch_bounds__(256, TW * TH == 256 ? 4 : 0) k_blend_fwd_h(RasterArgs a, const u64* __restrict__ inst,
                                                     float* __restrict__ rgb, float* __restrict__ dout) {
  using L = TileLayout<TW, TH>;
  constexpr int PPT = L::PPT;
  // per warp and half: the compacted list of this batch
  __shared__ float2 s_xy[8][2][32];
  __shared__ float4 s_con[8][2][32];
  __shared__ float4 s_col[8][2][32];
  __shared__ unsigned s_rel[8][2][32];
  // per warp and lane: the next batch's pair record and the key after it,
  // staged by cp.async while the current batch blends
  __shared__ float4 s_srec[8][3][32];
  __shared__ u64 s_skey[8][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4;
  const unsigned lt = lanemask_lt();
  const unsigned n_items = 8u * (unsigned)a.n_tiles;
  for (;;) {
    unsigned item = 0;
    if (lane == 0) item = atomicAdd(&a.counters->tile_queue, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    const unsigned gt = item >> 3, wb = item & 7u;
    const int bx0 = (int)(wb % L::WPR) * 8, by0 = (int)(wb / L::WPR) * L::WY;
    const int lx = bx0 + 4 * h + (lane & 3);
    const int ly = by0 + ((lane >> 2) & 3);
    const int v = view_of_tile(a.cams, a.V, gt);
    const DevCam& c = a.cams[v];
    const int W = c.W, H = c.H;
    const int local = (int)gt - c.tile_base;
    const int ty = local / c.ntx, tx = local - ty * c.ntx;
    const int x0 = tx * TW, y0 = ty * TH;
    const float x0f = (float)x0, y0f = (float)y0;
    float T[PPT], Tf[PPT], Cr[PPT], Cg[PPT], Cb[PPT], Dz[PPT];
    uint32_t last[PPT];
    unsigned ev = 0, nb = 0;
    const int px = x0 + lx;
    int alive = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int py = y0 + ly + 4 * k;
      T[k] = (px < W && py < H) ? 1.f : 0.f;
      Tf[k] = T[k];
      Cr[k] = Cg[k] = Cb[k] = Dz[k] = 0.f;
      last[k] = 0;
      alive |= T[k] > 0.f;
    }
    uint2 rg = a.ranges[gt];
    if (dcg_oob(rg.y, (u64)a.cap_inst + 1ull, a.errword)) rg.y = rg.x;
    // software pipeline over the batches, staged in shared memory by
    // cp.async (no registers hold loads in flight): while a batch blends, the
    // records of the next batch's instances that reach this warp block and
    // the keys of the batch after it are on their way.  A lane overwrites its
    // staging slots only after it has used what they held.
    unsigned hbn = 0;
    if (rg.x + lane < rg.y) cp_async8(&s_skey[w][lane], inst + rg.x + lane);
    cp_async_commit();
    cp_async_wait<0>();
    if (rg.x + lane < rg.y) {
      const u64 k0 = s_skey[w][lane];
      const unsigned vi0 = pair_of_inst(k0);
      hbn = half_bits(k0, wb);
      if (hbn && dcg_oob(vi0, (u64)a.cap_pairs, a.errword)) hbn = 0u;
      if (hbn) {
        cp_async16(&s_srec[w][0][lane], a.rec + 3ull * vi0 + 0);
        cp_async16(&s_srec[w][1][lane], a.rec + 3ull * vi0 + 1);
        cp_async16(&s_srec[w][2][lane], a.rec + 3ull * vi0 + 2);
      }
    }
    if (rg.x + 32 + lane < rg.y) cp_async8(&s_skey[w][lane], inst + rg.x + 32 + lane);
    cp_async_commit();
    for (unsigned b0 = rg.x; b0 < rg.y; b0 += 32) {
      const unsigned am = __ballot_sync(0xffffffffu, alive);
      if (am == 0u) break;
      const unsigned idx = b0 + lane;
      unsigned hb = hbn;
      cp_async_wait<0>();  // this batch's records, the next batch's keys
      float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), cn = r0, cl = r0;
      if (hb) {
        r0 = s_srec[w][0][lane];
        cn = s_srec[w][1][lane];
        cl = s_srec[w][2][lane];
      }
      unsigned vin = 0;
      hbn = 0;
      if (idx + 32 < rg.y) {
        const u64 k1 = s_skey[w][lane];
        vin = pair_of_inst(k1);
        hbn = half_bits(k1, wb);
        if (hbn && dcg_oob(vin, (u64)a.cap_pairs, a.errword)) hbn = 0u;
      }
      if ((am & 0xffffu) == 0u) hb &= 2u;
      if ((am >> 16) == 0u) hb &= 1u;
      const unsigned mL = __ballot_sync(0xffffffffu, hb & 1u), mR = __ballot_sync(0xffffffffu, hb & 2u);
      if (hb) {
        const float2 xy = make_float2(df_sub_round(r0.x, r0.z, x0f), df_sub_round(r0.y, r0.w, y0f));
        const unsigned rel = idx - rg.x + 1;  // the instance's rank in the tile list + 1: its "last" value
        if (hb & 1u) {
          const int sl = __popc(mL & lt);
          s_xy[w][0][sl] = xy;
          s_con[w][0][sl] = cn;
          s_col[w][0][sl] = cl;
          s_rel[w][0][sl] = rel;
        }
        if (hb & 2u) {
          const int sl = __popc(mR & lt);
          s_xy[w][1][sl] = xy;
          s_con[w][1][sl] = cn;
          s_col[w][1][sl] = cl;
          s_rel[w][1][sl] = rel;
        }
      }
      // the shorter list is padded to the longer one with transparent
      // entries (opacity 0: alpha 0 < 1/255), so both halves step together
      // without a branch
      const int cL = __popc(mL), cR = __popc(mR), cmax = max(cL, cR);
      const int cmine = h ? cR : cL;
      if (lane >= cL && lane < cmax) {
        s_xy[w][0][lane] = make_float2(0.f, 0.f);
        s_con[w][0][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (lane >= cR && lane < cmax) {
        s_xy[w][1][lane] = make_float2(0.f, 0.f);
        s_con[w][1][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      // the next batch's records and the keys after it (this lane's staged
      // record and key were used above)
      if (hbn) {
        cp_async16(&s_srec[w][0][lane], a.rec + 3ull * vin + 0);
        cp_async16(&s_srec[w][1][lane], a.rec + 3ull * vin + 1);
        cp_async16(&s_srec[w][2][lane], a.rec + 3ull * vin + 2);
      }
      if (idx + 64 < rg.y) cp_async8(&s_skey[w][lane], inst + idx + 64);
      cp_async_commit();
      __syncwarp();
      // evaluations counted per batch: a pixel live at its start is evaluated
      // by every real step until it terminates
      unsigned nev[PPT];
#pragma unroll
      for (int k = 0; k < PPT; ++k) nev[k] = T[k] > 0.f ? (unsigned)cmine : 0u;
      for (int j = 0; j < cmax; ++j) {
        const float2 xy = s_xy[w][h][j];
        const float4 cq = s_con[w][h][j];
        const float dx = __fsub_rn((float)lx, xy.x);
        const float sx = __fmul_rn(dx, __fmul_rn(cq.x, dx));
        const float bx = __fmul_rn(cq.y, dx);
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          // the support, alpha and termination tests as predicates (one
          // branch, for the compositing itself)
          const float dy = __fsub_rn((float)(ly + 4 * k), xy.y);
          const float p = blend_power(sx, bx, cq.z, dy);
          const float al = fminf(kAlphaMax, __fmul_rn(cq.w, ex2_approx(p)));
          const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, al));
          const bool live = T[k] > 0.f;
          const bool hit = live && p >= kPMin && al >= kAlphaMin;
          const bool stop = hit && Tn < kTMin;
          if (stop) {
            Tf[k] = T[k];
            T[k] = 0.f;
            nev[k] = (unsigned)j + 1u;
          } else if (hit) {
            const float4 cl = s_col[w][h][j];
            const float wgt = al * T[k];
            Cr[k] += wgt * cl.x;
            Cg[k] += wgt * cl.y;
            Cb[k] += wgt * cl.z;
            Dz[k] += wgt * cl.w;
            T[k] = Tn;
            last[k] = s_rel[w][h][j];
            ++nb;
          }
        }
      }
      __syncwarp();
      alive = 0;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        alive |= T[k] > 0.f;
        ev += nev[k];
      }
    }
    cp_async_wait<0>();  // nothing of this item left in flight (a batch loop that stops early)
    {
      const unsigned wev = __reduce_add_sync(0xffffffffu, ev), wnb = __reduce_add_sync(0xffffffffu, nb);
      if (lane == 0 && wev) atomicAdd(&a.counters->n_eval, (unsigned long long)wev);
      if (lane == 0 && wnb) atomicAdd(&a.counters->n_blend, (unsigned long long)wnb);
    }
    const long long P = (long long)W * H;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int py = y0 + ly + 4 * k;
      if (px < W && py < H && !dcg_oob((u64)(c.pix_off + (long long)py * W + px), (u64)a.n_pix, a.errword)) {
        const long long pix = (long long)py * W + px;
        rgb[3 * c.pix_off + pix] = Cr[k];
        rgb[3 * c.pix_off + P + pix] = Cg[k];
        rgb[3 * c.pix_off + 2 * P + pix] = Cb[k];
        dout[c.pix_off + pix] = Dz[k];
        a.T_final[c.pix_off + pix] = T[k] > 0.f ? T[k] : Tf[k];
        a.n_contrib[c.pix_off + pix] = last[k];
      }
    }
  }
}

template <int TW, int TH>
__global__ void __launch_bounds__(256) k_blend_bwd_h(RasterArgs a, const u64* __restrict__ inst,
                                                     const float* __restrict__ dL_drgb,
                                                     const float* __restrict__ dL_ddepth) {
  using L = TileLayout<TW, TH>;
  constexpr int PPT = L::PPT;
  constexpr int R = kRingB;
  __shared__ float2 s_xy[8][2][R + 1];
  __shared__ float4 s_con[8][2][R + 1];
  __shared__ float4 s_col[8][2][R + 1];
  __shared__ unsigned s_rel[8][2][R + 1];
  __shared__ unsigned s_vi[8][2][R + 1];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4;
  const unsigned lt = lanemask_lt();
  const unsigned n_items = 8u * (unsigned)a.n_tiles;
  float* const g2 = reinterpret_cast<float*>(a.grad2d);
  if (lane < 2) s_rel[w][lane][R] = 0x7fffffffu;  // the neutral entry: behind every pixel's last contributor
  for (;;) {
    unsigned item = 0;
    if (lane == 0) item = atomicAdd(&a.counters->tile_queue_bwd, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    const unsigned gt = item >> 3, wb = item & 7u;
    const int bx0 = (int)(wb % L::WPR) * 8, by0 = (int)(wb / L::WPR) * L::WY;
    const int lx = bx0 + 4 * h + (lane & 3);
    const int ly = by0 + ((lane >> 2) & 3);
    const int v = view_of_tile(a.cams, a.V, gt);
    const DevCam& c = a.cams[v];
    const int W = c.W, H = c.H;
    const int local = (int)gt - c.tile_base;
    const int ty = local / c.ntx, tx = local - ty * c.ntx;
    const int x0 = tx * TW, y0 = ty * TH;
    const float x0f = (float)x0, y0f = (float)y0;
    const long long P = (long long)W * H;
    float T[PPT], gr[PPT], gg[PPT], gb[PPT], gd[PPT], Dg[PPT];
    uint32_t last[PPT];
    const int px = x0 + lx;
    uint32_t mylast = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int py = y0 + ly + 4 * k;
      last[k] = 0;
      T[k] = 0.f;
      gr[k] = gg[k] = gb[k] = gd[k] = 0.f;
      if (px < W && py < H) {
        const long long pix = (long long)py * W + px;
        T[k] = a.T_final[c.pix_off + pix];
        last[k] = a.n_contrib[c.pix_off + pix];
        gr[k] = dL_drgb[3 * c.pix_off + pix];
        gg[k] = dL_drgb[3 * c.pix_off + P + pix];
        gb[k] = dL_drgb[3 * c.pix_off + 2 * P + pix];
        gd[k] = dL_ddepth[c.pix_off + pix];
      }
      Dg[k] = 0.f;
      mylast = max(mylast, last[k]);
    }
    // per half: the largest contributor count of its pixels
    const unsigned lastL = __reduce_max_sync(0xffffffffu, h ? 0u : mylast);
    const unsigned lastR = __reduce_max_sync(0xffffffffu, h ? mylast : 0u);
    const uint2 rg = a.ranges[gt];
    int hi = (int)max(lastL, lastR);  // instances [0, hi) are still to scan, from the end
    int hL = 0, hR = 0, pL = 0, pR = 0;
    __syncwarp();
    for (;;) {
      while (hi > 0 && (pL < 32 || pR < 32) && pL <= R - 32 && pR <= R - 32) {
        const int rel = hi - 1 - lane;  // lane 0 takes the largest index: rings keep reverse order
        unsigned hb = 0, vi = 0;
        if (rel >= 0) {
          const u64 key = inst[rg.x + rel];
          vi = pair_of_inst(key);
          hb = half_bits(key, wb);
          if ((unsigned)rel >= lastL) hb &= 2u;
          if ((unsigned)rel >= lastR) hb &= 1u;
        }
        const unsigned mL = __ballot_sync(0xffffffffu, hb & 1u), mR = __ballot_sync(0xffffffffu, hb & 2u);
        if (hb) {
          const float4 r0 = a.rec[3ull * vi + 0];
          const float2 xy = make_float2(df_sub_round(r0.x, r0.z, x0f), df_sub_round(r0.y, r0.w, y0f));
          const float4 cn = a.rec[3ull * vi + 1], cl = a.rec[3ull * vi + 2];
          if (hb & 1u) {
            int sl = hL + pL + __popc(mL & lt);
            sl -= sl >= R ? R : 0;
            sl -= sl >= R ? R : 0;
            s_xy[w][0][sl] = xy;
            s_con[w][0][sl] = cn;
            s_col[w][0][sl] = cl;
            s_rel[w][0][sl] = (unsigned)rel;
            s_vi[w][0][sl] = vi;
          }
          if (hb & 2u) {
            int sl = hR + pR + __popc(mR & lt);
            sl -= sl >= R ? R : 0;
            sl -= sl >= R ? R : 0;
            s_xy[w][1][sl] = xy;
            s_con[w][1][sl] = cn;
            s_col[w][1][sl] = cl;
            s_rel[w][1][sl] = (unsigned)rel;
            s_vi[w][1][sl] = vi;
          }
        }
        pL += __popc(mL);
        pR += __popc(mR);
        hi -= 32;
      }
      __syncwarp();
      if (pL == 0 && pR == 0) break;
      const int n = ring_steps(pL, pR, hi > 0, R);
      const int pm = h ? pR : pL, hm = h ? hR : hL;
      for (int s = 0; s < n; ++s) {
        int e = hm + s;
        e -= e >= R ? R : 0;
        e = s < pm ? e : R;
        float acc[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) acc[q] = 0.f;
        bool any = false;
        const int r = (int)s_rel[w][h][e];
        const float2 xy = s_xy[w][h][e];
        const float4 cq = s_con[w][h][e];
        const float dx = __fsub_rn((float)lx, xy.x);
        const float sx = __fmul_rn(dx, __fmul_rn(cq.x, dx));
        const float bx = __fmul_rn(cq.y, dx);
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          // the support and alpha tests as predicates (one branch)
          const float dy = __fsub_rn((float)(ly + 4 * k), xy.y);
          const float p = blend_power(sx, bx, cq.z, dy);
          const float G = ex2_approx(p);
          const float araw = __fmul_rn(cq.w, G);
          const float al = fminf(kAlphaMax, araw);
          if (r < (int)last[k] && p >= kPMin && al >= kAlphaMin) {
            any = true;
            const float4 cl = s_col[w][h][e];
            T[k] = __fdividef(T[k], 1.f - al);
            const float wgt = al * T[k];
            acc[6] += wgt * gr[k];
            acc[7] += wgt * gg[k];
            acc[8] += wgt * gb[k];
            acc[9] += wgt * gd[k];
            // dL/dalpha = T (c . g - D) with D = sum over channels of g times the
            // colour (and depth) composited behind this Gaussian; D follows the
            // same over-recursion as the colours themselves
            const float cg = cl.x * gr[k] + cl.y * gg[k] + cl.z * gb[k] + cl.w * gd[k];
            const float dal = T[k] * (cg - Dg[k]);
            Dg[k] = al * cg + (1.f - al) * Dg[k];
            // moments of dL/dalpha G (none through a clamped alpha); the
            // conic and opacity factors are applied per Gaussian in
            // k_preprocess_bwd
            if (araw < kAlphaMax) {
              const float gG = dal * G;
              const float gx = gG * dx, gy = gG * dy;
              acc[5] += gG;
              acc[0] += gx;
              acc[1] += gy;
              acc[2] += gx * dx;
              acc[3] += gx * dy;
              acc[4] += gy * dy;
            }
          }
        }
        if (__any_sync(0xffffffffu, any)) {
          int comp;
          bool has;
          const float tot = warp_sum_transpose<10, 8>(acc, &comp, &has);
          if (has && tot != 0.f) atomicAdd(g2 + 12ull * s_vi[w][h][e] + comp, tot);
        }
      }
      const int nL = min(n, pL), nR = min(n, pR);
      hL += nL;
      hL -= hL >= R ? R : 0;
      hR += nR;
      hR -= hR >= R ? R : 0;
      pL -= nL;
      pR -= nR;
      __syncwarp();
    }
  }
}

// Backward blend with Gaussians on the lanes.  One warp per (tile, half
// block): the half's 4 x WY pixels and the Gaussians of the tile's list that
// reach the half (its half-block bit), taken 16 at a time from the end, the
// deepest first.  Both half-warps hold the same 16 Gaussians (lane l and
// l + 16 hold Gaussian l & 15) and take two pixels of the half block at a
// time, one each: the lanes evaluate their Gaussians at their half's pixel,
// and one warp scan in lane order (deep to front) over the affine maps
//   (T, Q) -> (r T, Q + r alpha (c . g) T),   r = 1 / (1 - alpha)
// (the reverse traversal of one pixel past one Gaussian; identity where the
// Gaussian does not composite) gives every lane what the traversal gives one
// Gaussian at a time: the transmittance in front of it, T_j = T_behind A_j,
// and the loss-weighted colour composited behind it,
// Q_j = Q_behind + T_behind B_j - T_j alpha_j (c_j . g), with
// dL/dalpha_j = T_j (c_j . g) - Q_j / (1 - alpha_j).  The pixel's
// (T_behind, Q_behind) then move past the chunk.  Every lane accumulates its
// Gaussian's 2D-gradient moments over its half's pixels, so no reduction
// over Gaussians is needed: after the pixels the two half-warps' sums are
// added and each Gaussian's ten sums go to its gradient slot with vector
// atomics.
constexpr int kRingG = 64;  // staged Gaussians per warp
constexpr int kChunkG = 16;  // Gaussians per chunk (lanes of a half-warp)

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}
__device__ __forceinline__ void red_add_v2(float* p, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

template <int TW, int TH>
__global__ void __launch_bounds__(256, 4) k_blend_bwd_g(RasterArgs a, const u64* __restrict__ inst,
                                                     const float* __restrict__ dL_drgb,
                                                     const float* __restrict__ dL_ddepth) {
  using L = TileLayout<TW, TH>;
  constexpr int WY = L::WY;
  constexpr int NP = 4 * WY;  // pixels of a half block
  constexpr int R = kRingG;
  constexpr int CH = kChunkG;
  __shared__ float4 s_r0[8][R];   // the ring: pair records as stored (centre, conic, colour)
  __shared__ float4 s_con[8][R];
  __shared__ float4 s_col[8][R];
  __shared__ int s_rel[8][R];
  __shared__ unsigned s_vi[8][R];
  __shared__ u64 s_key[8][32];    // the next refill's instance keys
  __shared__ float4 s_g[8][NP];   // dL/d(r, g, b, depth) of each pixel of the half
  __shared__ float4 s_st[8][NP];  // (T behind, Q behind, last contributor (int bits), unused)
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, hl = lane >> 4, gl = lane & 15;
  const unsigned lt = lanemask_lt();
  const unsigned n_items = 16u * (unsigned)a.n_tiles;
  float* const g2 = reinterpret_cast<float*>(a.grad2d);
  for (;;) {
    unsigned item = 0;
    if (lane == 0) item = atomicAdd(&a.counters->tile_queue_bwd, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    const unsigned gt = item >> 4, wb = (item >> 1) & 7u, h = item & 1u;
    const int bx0 = (int)(wb % L::WPR) * 8 + 4 * (int)h, by0 = (int)(wb / L::WPR) * WY;
    const int v = view_of_tile(a.cams, a.V, gt);
    const DevCam& c = a.cams[v];
    const int W = c.W, H = c.H;
    const int local = (int)gt - c.tile_base;
    const int ty = local / c.ntx, tx = local - ty * c.ntx;
    const int x0 = tx * TW, y0 = ty * TH;
    const float x0f = (float)x0, y0f = (float)y0;
    const long long P = (long long)W * H;
    // the half's pixels: loss gradients and the forward's end state
    unsigned mylast = 0;
    for (int p = lane; p < NP; p += 32) {
      const int px = x0 + bx0 + (p & 3), py = y0 + by0 + (p >> 2);
      float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
      float Tf = 0.f;
      unsigned last = 0;
      if (px < W && py < H && !dcg_oob((u64)(c.pix_off + (long long)py * W + px), (u64)a.n_pix, a.errword)) {
        const long long pix = (long long)py * W + px;
        Tf = a.T_final[c.pix_off + pix];
        last = a.n_contrib[c.pix_off + pix];
        g = make_float4(dL_drgb[3 * c.pix_off + pix], dL_drgb[3 * c.pix_off + P + pix],
                        dL_drgb[3 * c.pix_off + 2 * P + pix], dL_ddepth[c.pix_off + pix]);
      }
      s_g[w][p] = g;
      s_st[w][p] = make_float4(Tf, 0.f, __int_as_float((int)last), 0.f);
      mylast = max(mylast, last);
    }
    int hi = (int)__reduce_max_sync(0xffffffffu, mylast);  // instances [0, hi) are still to scan
    const uint2 rg = a.ranges[gt];
    if (dcg_oob((u64)rg.x + (u64)hi, (u64)a.cap_inst + 1ull, a.errword)) hi = 0;
    // The ring is refilled while it holds fewer than two chunks, so the
    // records of the next chunk are in flight (cp.async) while this one is
    // blended; the keys of the next refill are staged one refill ahead.
    // Commit groups: one per refill (its records and the next keys); old =
    // ring entries from the head whose records lie in older groups.
    int hd = 0, pc = 0, old = 0;  // ring head, count, entries of older groups
    if (hi > 0 && hi - 1 - lane >= 0) cp_async8(&s_key[w][lane], inst + rg.x + (hi - 1 - lane));
    cp_async_commit();
    __syncwarp();
    for (;;) {
      while (hi > 0 && pc < 2 * CH) {
        cp_async_wait<0>();  // this refill's keys, and every record asked for so far
        __syncwarp();
        old = pc;
        const int rel = hi - 1 - lane;  // lane 0 takes the largest index: the ring keeps reverse order
        bool take = false;
        unsigned vi = 0;
        if (rel >= 0) {
          const u64 key = s_key[w][lane];
          vi = pair_of_inst(key);
          take = (half_bits(key, (int)wb) >> h) & 1u;
          if (take && dcg_oob(vi, (u64)a.cap_pairs, a.errword)) take = false;
        }
        const unsigned m = __ballot_sync(0xffffffffu, take);  // also: every lane has read its key
        if (take) {
          int sl = hd + pc + __popc(m & lt);
          sl -= sl >= R ? R : 0;
          sl -= sl >= R ? R : 0;
          cp_async16(&s_r0[w][sl], a.rec + 3ull * vi + 0);
          cp_async16(&s_con[w][sl], a.rec + 3ull * vi + 1);
          cp_async16(&s_col[w][sl], a.rec + 3ull * vi + 2);
          s_rel[w][sl] = rel;
          s_vi[w][sl] = vi;
        }
        pc += __popc(m);
        hi -= 32;
        if (hi > 0 && hi - 1 - lane >= 0) cp_async8(&s_key[w][lane], inst + rg.x + (hi - 1 - lane));
        cp_async_commit();
      }
      if (pc == 0) break;
      const int cnt = min(pc, CH);
      // the chunk's records: in older groups, or also in the newest one
      if (cnt <= old)
        cp_async_wait<1>();
      else
        cp_async_wait<0>();
      __syncwarp();
      int e = hd + gl;
      e -= e >= R ? R : 0;
      const bool mine = gl < cnt;
      float2 xy = make_float2(0.f, 0.f);
      if (mine) {
        const float4 r0 = s_r0[w][e];
        xy = make_float2(df_sub_round(r0.x, r0.z, x0f), df_sub_round(r0.y, r0.w, y0f));
      }
      const float4 cq = mine ? s_con[w][e] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 cl = mine ? s_col[w][e] : make_float4(0.f, 0.f, 0.f, 0.f);
      const int rl = mine ? s_rel[w][e] : 0x7fffffff;
      const unsigned vi = mine ? s_vi[w][e] : 0u;
      const int minrel = __shfl_sync(0xffffffffu, rl, cnt - 1);  // the chunk's front-most instance
      float acc[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) acc[q] = 0.f;
      // this half-warp's two pixel columns of the half block: hl and hl + 2
      float dxc[2], sxc[2], bxc[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        dxc[q] = __fsub_rn((float)(bx0 + 2 * q + hl), xy.x);
        sxc[q] = __fmul_rn(dxc[q], __fmul_rn(cq.x, dxc[q]));
        bxc[q] = __fmul_rn(cq.y, dxc[q]);
      }
      for (int rr = 0; rr < WY; ++rr) {
        const float dy = __fsub_rn((float)(by0 + rr), xy.y);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int p = 4 * rr + 2 * q + hl;  // this half-warp's pixel
          const float4 st = s_st[w][p];
          const int lastp = __float_as_int(st.z);
          // pixels whose last contributor lies in front of the whole chunk take no part
          if (!__any_sync(0xffffffffu, minrel < lastp)) continue;
          // the same decisions, bit for bit, as the forward blend
          const float pw = blend_power(sxc[q], bxc[q], cq.z, dy);
          const float G = ex2_approx(pw);
          const float araw = __fmul_rn(cq.w, G);
          const float al = fminf(kAlphaMax, araw);
          const bool valid = rl < lastp && pw >= kPMin && al >= kAlphaMin;
          if (!__any_sync(0xffffffffu, valid)) continue;  // nothing composites: the states are unchanged
          const float4 g = s_g[w][p];
          const float r = valid ? rcp_approx(__fsub_rn(1.f, al)) : 1.f;
          const float cg = cl.x * g.x + cl.y * g.y + cl.z * g.z + cl.w * g.w;
          float A = r, B = valid ? r * al * cg : 0.f;
#pragma unroll
          for (int o = 1; o < CH; o <<= 1) {
            const float Au = __shfl_up_sync(0xffffffffu, A, o, CH);
            const float Bu = __shfl_up_sync(0xffffffffu, B, o, CH);
            if (gl >= o) {
              B = fmaf(Au, B, Bu);
              A = Au * A;
            }
          }
          const float Tj = st.x * A;
          if (valid) {
            const float wgt = al * Tj;
            acc[6] += wgt * g.x;
            acc[7] += wgt * g.y;
            acc[8] += wgt * g.z;
            acc[9] += wgt * g.w;
            // moments of dL/dalpha G (none through a clamped alpha); the conic
            // and opacity factors are applied per Gaussian in k_preprocess_bwd
            if (araw < kAlphaMax) {
              const float Q = fmaf(st.x, B, st.y) - wgt * cg;
              const float dal = Tj * cg - Q * r;
              const float gG = dal * G;
              const float gx = gG * dxc[q], gy = gG * dy;
              acc[5] += gG;
              acc[0] += gx;
              acc[1] += gy;
              acc[2] += gx * dxc[q];
              acc[3] += gx * dy;
              acc[4] += gy * dy;
            }
          }
          // the half's last lane holds the whole chunk's map: the pixel moves past it
          if (gl == CH - 1) {
            s_st[w][p].x = st.x * A;
            s_st[w][p].y = fmaf(st.x, B, st.y);
          }
        }
      }
      // the two half-warps hold partial sums of the same Gaussians
      bool any = false;
#pragma unroll
      for (int q = 0; q < 10; ++q) {
        acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], 16);
        any |= acc[q] != 0.f;
      }
      if (hl == 0 && mine && any) {
        float* s = g2 + 12ull * vi;
        red_add_v4(s, acc[0], acc[1], acc[2], acc[3]);
        red_add_v4(s + 4, acc[4], acc[5], acc[6], acc[7]);
        red_add_v2(s + 8, acc[8], acc[9]);
      }
      hd += cnt;
      hd -= hd >= R ? R : 0;
      pc -= cnt;
      old = old > cnt ? old - cnt : 0;
      __syncwarp();
    }
    cp_async_wait<0>();  // nothing of this item left in flight
    __syncwarp();
  }
}

// Backward variant without per-Gaussian warp reductions: every lane adds its
// own contribution to a private slot of a block-shared accumulator
// [segment Gaussian][component][lane] (shared-memory atomics, since warps of
// the block may touch the same Gaussian); at the end of each segment of
// kSlotSeg Gaussians the block sums the 32 slots (rotated to avoid bank
// conflicts), zeroes them, and issues the global vector atomics.
constexpr int kSlotSeg = 64;
constexpr size_t kSlotSmem = sizeof(float) * kSlotSeg * 10 * 32;

template <int TW, int TH>
__global__ void __launch_bounds__(256) k_blend_bwd_slots(RasterArgs a, const u64* __restrict__ inst,
                                                         const float* __restrict__ dL_drgb,
                                                         const float* __restrict__ dL_ddepth) {
  using L = TileLayout<TW, TH>;
  constexpr int PPT = L::PPT;
  extern __shared__ float s_slot[];  // [kSlotSeg][10][32]
  __shared__ float2 s_xy[8][32];
  __shared__ float4 s_con[8][32];
  __shared__ float4 s_col[8][32];
  __shared__ unsigned s_rel[8][32];
  __shared__ float s_sum[kSlotSeg][10];
  __shared__ unsigned s_tile;
  __shared__ unsigned s_maxlast;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int bx0 = (w % L::WPR) * 8, by0 = (w / L::WPR) * L::WY;
  const int lx = bx0 + (lane & 7);
  const int ly = by0 + (lane >> 3);
  const unsigned lt = lanemask_lt();
  for (int e = tid; e < kSlotSeg * 10 * 32; e += 256) s_slot[e] = 0.f;
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      s_tile = atomicAdd(&a.counters->tile_queue_bwd, 1u);
      s_maxlast = 0;
    }
    __syncthreads();
    const unsigned gt = s_tile;
    if (gt >= (unsigned)a.n_tiles) break;
    const int v = view_of_tile(a.cams, a.V, gt);
    const DevCam& c = a.cams[v];
    const int W = c.W, H = c.H;
    const int local = (int)gt - c.tile_base;
    const int ty = local / c.ntx, tx = local - ty * c.ntx;
    const int x0 = tx * TW, y0 = ty * TH;
    const float x0f = (float)x0, y0f = (float)y0;
    const long long P = (long long)W * H;
    float T[PPT], gr[PPT], gg[PPT], gb[PPT], gd[PPT], Dg[PPT];
    uint32_t last[PPT];
    const int px = x0 + lx;
    uint32_t mylast = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int py = y0 + ly + 4 * k;
      last[k] = 0;
      T[k] = 0.f;
      gr[k] = gg[k] = gb[k] = gd[k] = 0.f;
      if (px < W && py < H) {
        const long long pix = (long long)py * W + px;
        T[k] = a.T_final[c.pix_off + pix];
        last[k] = a.n_contrib[c.pix_off + pix];
        gr[k] = dL_drgb[3 * c.pix_off + pix];
        gg[k] = dL_drgb[3 * c.pix_off + P + pix];
        gb[k] = dL_drgb[3 * c.pix_off + 2 * P + pix];
        gd[k] = dL_ddepth[c.pix_off + pix];
      }
      Dg[k] = 0.f;
      mylast = max(mylast, last[k]);
    }
    const int warplast = (int)__reduce_max_sync(0xffffffffu, mylast);
    if (lane == 0) atomicMax(&s_maxlast, (unsigned)warplast);
    __syncthreads();
    const int maxlast = (int)s_maxlast;
    const uint2 rg = a.ranges[gt];
    for (int send = maxlast; send > 0; send -= kSlotSeg) {
      const int sbeg = max(0, send - kSlotSeg);
      for (int hi = min(send, warplast); hi > sbeg; hi -= 32) {
        const int rel = hi - 1 - lane;
        bool pass = false;
        unsigned vi = 0;
        if (rel >= sbeg) {
          const u64 key = inst[rg.x + rel];
          vi = pair_of_inst(key);
          pass = block_bit(key, w);
        }
        const unsigned m = __ballot_sync(0xffffffffu, pass);
        if (pass) {
          const float4 r0 = a.rec[3ull * vi + 0];
          const int slot = __popc(m & lt);
          s_xy[w][slot] = make_float2(df_sub_round(r0.x, r0.z, x0f), df_sub_round(r0.y, r0.w, y0f));
          s_con[w][slot] = a.rec[3ull * vi + 1];
          s_col[w][slot] = a.rec[3ull * vi + 2];
          s_rel[w][slot] = (unsigned)rel;
        }
        __syncwarp();
        const int cnt = __popc(m);
        for (int j = 0; j < cnt; ++j) {
          const int r = (int)s_rel[w][j];
          const float2 xy = s_xy[w][j];
          const float4 cq = s_con[w][j];
          const float dx = __fsub_rn((float)lx, xy.x);
          const float sx = __fmul_rn(dx, __fmul_rn(cq.x, dx));
          const float bx = __fmul_rn(cq.y, dx);
          float acc[10];
#pragma unroll
          for (int q = 0; q < 10; ++q) acc[q] = 0.f;
          bool any = false;
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            if (r < (int)last[k]) {
              const float dy = __fsub_rn((float)(ly + 4 * k), xy.y);
              const float p = blend_power(sx, bx, cq.z, dy);
              if (p >= kPMin) {
                const float G = ex2_approx(p);
                const float araw = __fmul_rn(cq.w, G);
                const float al = fminf(kAlphaMax, araw);
                if (al >= kAlphaMin) {
                  any = true;
                  const float4 cl = s_col[w][j];
                  T[k] = __fdividef(T[k], 1.f - al);
                  const float wgt = al * T[k];
                  acc[6] += wgt * gr[k];
                  acc[7] += wgt * gg[k];
                  acc[8] += wgt * gb[k];
                  acc[9] += wgt * gd[k];
                  // dL/dalpha = T (c . g - D) with D = sum over channels of g times the
                  // colour (and depth) composited behind this Gaussian; D follows the
                  // same over-recursion as the colours themselves
                  const float cg = cl.x * gr[k] + cl.y * gg[k] + cl.z * gb[k] + cl.w * gd[k];
                  const float dal = T[k] * (cg - Dg[k]);
                  Dg[k] = al * cg + (1.f - al) * Dg[k];
                  if (araw < kAlphaMax) {
                    // moments of dL/dalpha * G; the conic and opacity factors are applied per
                    // Gaussian in k_preprocess_bwd
                    const float gG = dal * G;
                    const float gx = gG * dx, gy = gG * dy;
                    acc[5] += gG;
                    acc[0] += gx;
                    acc[1] += gy;
                    acc[2] += gx * dx;
                    acc[3] += gx * dy;
                    acc[4] += gy * dy;
                  }
                }
              }
            }
          }
          if (any) {
            float* sl = s_slot + (size_t)(r - sbeg) * 320 + lane;
#pragma unroll
            for (int q = 0; q < 10; ++q) atomicAdd(sl + 32 * q, acc[q]);
          }
        }
        __syncwarp();
      }
      __syncthreads();
      const int cnt_seg = send - sbeg;
      for (int e = tid; e < cnt_seg * 10; e += 256) {
        float* sl = s_slot + (size_t)e * 32;
        float acc = 0.f;
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
          const int kk = (k + tid) & 31;
          acc += sl[kk];
          sl[kk] = 0.f;
        }
        (&s_sum[0][0])[e] = acc;
      }
      __syncthreads();
      for (int j = tid; j < cnt_seg; j += 256) {
        const float* q = s_sum[j];
        const float4 g0 = make_float4(q[0], q[1], q[2], q[3]);
        const float4 g1 = make_float4(q[4], q[5], q[6], q[7]);
        const bool n0 = g0.x != 0.f || g0.y != 0.f || g0.z != 0.f || g0.w != 0.f;
        const bool n1 = g1.x != 0.f || g1.y != 0.f || g1.z != 0.f || g1.w != 0.f;
        const bool n2 = q[8] != 0.f || q[9] != 0.f;
        if (n0 || n1 || n2) {
          float4* gp = a.grad2d + 3ull * pair_of_inst(inst[rg.x + sbeg + j]);
          if (n0) atomicAdd(gp + 0, g0);
          if (n1) atomicAdd(gp + 1, g1);
          if (n2) atomicAdd(reinterpret_cast<float2*>(gp + 2), make_float2(q[8], q[9]));
        }
      }
      __syncthreads();
    }
  }
}

// ============================================================================
// 9. preprocess backward
// ============================================================================
// 128 threads per block; the SH-coefficient gradients (3 (DEG+1)^2 per
// Gaussian, summed over views) are accumulated in the thread's own column of
// shared memory instead of registers.
constexpr int kPreBwdThreads = 128;
template <int DEG>
__global__ void __launch_bounds__(kPreBwdThreads, 4) k_preprocess_bwd(RasterArgs a, float* __restrict__ out,
                                                                   long long ostride, float* __restrict__ dpose) {
  const long long n = a.n;
  constexpr int D = (DEG + 1) * (DEG + 1);
  constexpr int T = kPreBwdThreads;
  // dynamic shared memory, one column per thread: its SH coefficients
  // (element k at shc[k T]), the colour gradient of each contributing view
  // (channel ch of view v at gcv[(3 v + ch) T]), from which the SH gradients
  // are summed after the view loop, and two slots for the 2D gradients of
  // the views it reaches (slot s, component c at gsl[(3 s + c) T]).  The
  // coefficients and each next reached view's gradients arrive by cp.async
  // while the current view is worked on.
  extern __shared__ float s_dyn[];
  float* const shc = s_dyn + threadIdx.x;
  float* const gcv = s_dyn + 3 * D * T + threadIdx.x;
  float4* const gsl = reinterpret_cast<float4*>(s_dyn + (3 * D + 3 * a.V) * T) + threadIdx.x;
  const long long S = a.stride;
  // one pass over all threads of the grid; lanes past n still join the warp reductions
  const long long n_round = ((n + 31) / 32) * 32;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_round; i += (long long)gridDim.x * blockDim.x) {
    const bool live = i < n;
    const float* g = a.g;
    unsigned vact = 0;  // views with a colour gradient
    float gm[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, go = 0.f;
    float mx = 0, my = 0, mz = 0, sc[3] = {1, 1, 1}, qn[4] = {1, 0, 0, 0}, qlen = 1.f, R[9], M[9], opac = 0.5f;
    float S00 = 0, S01 = 0, S02 = 0, S11 = 0, S12 = 0, S22 = 0;
    if (live) {
      mx = g[0 * S + i]; my = g[1 * S + i]; mz = g[2 * S + i];
      sc[0] = __expf(g[3 * S + i]); sc[1] = __expf(g[4 * S + i]); sc[2] = __expf(g[5 * S + i]);
      const float q0 = g[6 * S + i], q1 = g[7 * S + i], q2 = g[8 * S + i], q3 = g[9 * S + i];
      qlen = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
      const float iq = 1.f / qlen;
      qn[0] = q0 * iq; qn[1] = q1 * iq; qn[2] = q2 * iq; qn[3] = q3 * iq;
      opac = 1.f / (1.f + __expf(-g[10 * S + i]));
    }
    quat_rot(qn[0], qn[1], qn[2], qn[3], R);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) M[3 * r + k] = R[3 * r + k] * sc[k];
    S00 = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    S01 = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    S02 = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    S11 = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    S12 = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    S22 = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    float dSig[6] = {0, 0, 0, 0, 0, 0};  // dS + dS^T accumulated over views: entries 00 01 02 11 12 22
    // the views this Gaussian reaches, all loads in flight together
    unsigned tmask = 0;
    const bool in_cap = !dcg_oob((u64)a.V * (u64)n, (u64)a.cap_pairs + 1ull, a.errword);
#pragma unroll
    for (int v = 0; v < kMaxViewsApi; ++v)
      if (live && in_cap && v < a.V && a.touched[(long long)v * n + i] != 0u) tmask |= 1u << v;
    // the SH coefficients of a Gaussian that reaches a view, then the 2D
    // gradients of its first reached view (commit groups in that order)
    if (tmask) {
#pragma unroll
      for (int k = 0; k < 3 * D; ++k) cp_async4(shc + k * T, g + (11 + k) * S + i);
    }
    cp_async_commit();
    if (tmask) {
      const long long vi0 = (long long)(__ffs(tmask) - 1) * n + i;
#pragma unroll
      for (int c = 0; c < 3; ++c) cp_async16(gsl + c * T, a.grad2d + 3 * vi0 + c);
    }
    cp_async_commit();
    int slot = 0;
    for (int v = 0; v < a.V; ++v) {
      float pose[6] = {0, 0, 0, 0, 0, 0};
      const long long vi = (long long)v * n + i;
      bool act = (tmask >> v) & 1u;
      float4 g0 = make_float4(0, 0, 0, 0), g1 = g0, g2 = g0;
      if (act) {
        // the next reached view's gradients into the other slot (read, and
        // used, at the previous reached view), then this view's
        const unsigned rest = tmask & ~((2u << v) - 1u);
        if (rest) {
          const long long vn = (long long)(__ffs(rest) - 1) * n + i;
#pragma unroll
          for (int c = 0; c < 3; ++c) cp_async16(gsl + (3 * (slot ^ 1) + c) * T, a.grad2d + 3 * vn + c);
        }
        cp_async_commit();
        cp_async_wait<1>();
        g0 = gsl[(3 * slot + 0) * T];
        g1 = gsl[(3 * slot + 1) * T];
        g2 = gsl[(3 * slot + 2) * T];
        slot ^= 1;
        act = (g0.x != 0.f) | (g0.y != 0.f) | (g0.z != 0.f) | (g0.w != 0.f) | (g1.x != 0.f) | (g1.y != 0.f) |
              (g1.z != 0.f) | (g1.w != 0.f) | (g2.x != 0.f) | (g2.y != 0.f);
        if (act) {  // consumed: the slot is zero again for the next backward
          const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
          a.grad2d[3 * vi + 0] = z4;
          a.grad2d[3 * vi + 1] = z4;
          a.grad2d[3 * vi + 2] = z4;
        }
      }
      if (act) {
        const DevCam& c = a.cams[v];
        const float tx = c.R[0] * mx + c.R[1] * my + c.R[2] * mz + c.t[0];
        const float ty = c.R[3] * mx + c.R[4] * my + c.R[5] * mz + c.t[1];
        const float tz = cam_depth(c, mx, my, mz);
        const float iz = 1.f / tz, iz2 = iz * iz;
        const float rxu = tx * iz, ryu = ty * iz;
        const bool clx = rxu < c.xlo || rxu > c.xhi, cly = ryu < c.ylo || ryu > c.yhi;
        const float rx = fminf(fmaxf(rxu, c.xlo), c.xhi), ry = fminf(fmaxf(ryu, c.ylo), c.yhi);
        const float J00 = c.fx * iz, J02 = -c.fx * rx * iz, J11 = c.fy * iz, J12 = -c.fy * ry * iz;
        const float T0[3] = {J00 * c.R[0] + J02 * c.R[6], J00 * c.R[1] + J02 * c.R[7], J00 * c.R[2] + J02 * c.R[8]};
        const float T1[3] = {J11 * c.R[3] + J12 * c.R[6], J11 * c.R[4] + J12 * c.R[7], J11 * c.R[5] + J12 * c.R[8]};
        const float ST0[3] = {S00 * T0[0] + S01 * T0[1] + S02 * T0[2], S01 * T0[0] + S11 * T0[1] + S12 * T0[2],
                              S02 * T0[0] + S12 * T0[1] + S22 * T0[2]};
        const float ST1[3] = {S00 * T1[0] + S01 * T1[1] + S02 * T1[2], S01 * T1[0] + S11 * T1[1] + S12 * T1[2],
                              S02 * T1[0] + S12 * T1[1] + S22 * T1[2]};
        const float ca = T0[0] * ST0[0] + T0[1] * ST0[1] + T0[2] * ST0[2] + kDilate;
        const float cb = T1[0] * ST0[0] + T1[1] * ST0[1] + T1[2] * ST0[2];
        const float cc = T1[0] * ST1[0] + T1[1] * ST1[1] + T1[2] * ST1[2] + kDilate;
        const float det = ca * cc - cb * cb;
        const float id = 1.f / det, id2 = id * id;
        // The blends accumulate, over the pixels, moments of g = dL/dalpha * G:
        // (sum g dx, sum g dy, sum g dx^2, sum g dx dy, sum g dy^2, sum g), with
        // dx = x - u, and the colour and depth sums.  Since alpha = o 2^p and
        // p = A' dx^2 + B' dx dy + C' dy^2, dL/dp = o ln2 g per pixel.
        const float fo = opac * kLn2;
        const float Ap = -0.5f * kLog2e * cc * id, Bp = kLog2e * cb * id, Cp = -0.5f * kLog2e * ca * id;
        const float du = -fo * (2.f * Ap * g0.x + Bp * g0.y), dv = -fo * (Bp * g0.x + 2.f * Cp * g0.y);
        // gradients of the unscaled conic entries (A' = -A log2(e) / 2, B' = -B log2(e), C' = -C log2(e) / 2)
        const float dA = fo * g0.z * (-0.5f * kLog2e), dB = fo * g0.w * (-kLog2e), dC = fo * g1.x * (-0.5f * kLog2e);
        const float dop = g1.y;
        const float dcol[3] = {g1.z, g1.w, g2.x};
        const float dzz = g2.y;
        // conic = inverse of [[a, b], [b, c]]
        const float da = dA * (-cc * cc * id2) + dB * (cb * cc * id2) + dC * (id - ca * cc * id2);
        const float db = dA * (2.f * cb * cc * id2) + dB * (-id - 2.f * cb * cb * id2) + dC * (2.f * ca * cb * id2);
        const float dc = dA * (id - cc * ca * id2) + dB * (cb * ca * id2) + dC * (-ca * ca * id2);
        // Sigma gradient (symmetrised: G = dS + dS^T)
        dSig[0] += 2.f * (da * T0[0] * T0[0] + db * T0[0] * T1[0] + dc * T1[0] * T1[0]);
        dSig[1] += 2.f * da * T0[0] * T0[1] + db * (T0[0] * T1[1] + T1[0] * T0[1]) + 2.f * dc * T1[0] * T1[1];
        dSig[2] += 2.f * da * T0[0] * T0[2] + db * (T0[0] * T1[2] + T1[0] * T0[2]) + 2.f * dc * T1[0] * T1[2];
        dSig[3] += 2.f * (da * T0[1] * T0[1] + db * T0[1] * T1[1] + dc * T1[1] * T1[1]);
        dSig[4] += 2.f * da * T0[1] * T0[2] + db * (T0[1] * T1[2] + T1[1] * T0[2]) + 2.f * dc * T1[1] * T1[2];
        dSig[5] += 2.f * (da * T0[2] * T0[2] + db * T0[2] * T1[2] + dc * T1[2] * T1[2]);
        // Tm gradient
        float dT0[3], dT1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          dT0[k] = 2.f * da * ST0[k] + db * ST1[k];
          dT1[k] = db * ST0[k] + 2.f * dc * ST1[k];
        }
        // Tm = J W -> dJ = dTm W^T ; dW = J^T dTm
        const float dJ00 = dT0[0] * c.R[0] + dT0[1] * c.R[1] + dT0[2] * c.R[2];
        const float dJ02 = dT0[0] * c.R[6] + dT0[1] * c.R[7] + dT0[2] * c.R[8];
        const float dJ11 = dT1[0] * c.R[3] + dT1[1] * c.R[4] + dT1[2] * c.R[5];
        const float dJ12 = dT1[0] * c.R[6] + dT1[1] * c.R[7] + dT1[2] * c.R[8];
        float dt[3];
        dt[0] = du * c.fx * iz;
        dt[1] = dv * c.fy * iz;
        dt[2] = -(du * c.fx * tx + dv * c.fy * ty) * iz2 + dzz;
        dt[2] += -(dJ00 * c.fx + dJ11 * c.fy) * iz2;
        if (!clx) {
          dt[0] += -dJ02 * c.fx * iz2;
          dt[2] += 2.f * dJ02 * c.fx * tx * iz2 * iz;
        } else {
          dt[2] += dJ02 * c.fx * rx * iz2;
        }
        if (!cly) {
          dt[1] += -dJ12 * c.fy * iz2;
          dt[2] += 2.f * dJ12 * c.fy * ty * iz2 * iz;
        } else {
          dt[2] += dJ12 * c.fy * ry * iz2;
        }
        // dW (rows k, cols j) = J[0][k] dT0[j] + J[1][k] dT1[j]; J = [[J00,0,J02],[0,J11,J12]]
        float dW[9];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          dW[0 + j] = J00 * dT0[j];
          dW[3 + j] = J11 * dT1[j];
          dW[6 + j] = J02 * dT0[j] + J12 * dT1[j];
        }
        // opacity
        go += dop * opac * (1.f - opac);
        // colour
        float dx = mx - c.C[0], dy = my - c.C[1], dz = mz - c.C[2];
        const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
        const float il = 1.f / dist;
        dx *= il; dy *= il; dz *= il;
        float Y[16];
        sh_basis(DEG, dx, dy, dz, Y);
        float wsum[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) wsum[k] = 0.f;
        vact |= 1u << v;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          float sh[D];
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            sh[k] = shc[(3 * k + ch) * T];
            acc += sh[k] * Y[k];
          }
          const float gc = (acc + 0.5f < 0.f) ? 0.f : dcol[ch];  // no gradient through a clamped channel
          gcv[(3 * v + ch) * T] = gc;
#pragma unroll
          for (int k = 0; k < D; ++k) wsum[k] += gc * sh[k];
        }
        float gdir[3] = {0, 0, 0};
        sh_grad_acc(DEG, dx, dy, dz, wsum, gdir);
        const float dd = gdir[0] * dx + gdir[1] * dy + gdir[2] * dz;
        const float gmu_sh[3] = {(gdir[0] - dx * dd) * il, (gdir[1] - dy * dd) * il, (gdir[2] - dz * dd) * il};
        // mean: t = W mu + t_cw
#pragma unroll
        for (int k = 0; k < 3; ++k) gm[k] += c.R[k] * dt[0] + c.R[3 + k] * dt[1] + c.R[6 + k] * dt[2] + gmu_sh[k];
        // pose twist (v, w)
        pose[0] = dt[0] + c.R[0] * gmu_sh[0] + c.R[1] * gmu_sh[1] + c.R[2] * gmu_sh[2];
        pose[1] = dt[1] + c.R[3] * gmu_sh[0] + c.R[4] * gmu_sh[1] + c.R[5] * gmu_sh[2];
        pose[2] = dt[2] + c.R[6] * gmu_sh[0] + c.R[7] * gmu_sh[1] + c.R[8] * gmu_sh[2];
        pose[3] = ty * dt[2] - tz * dt[1];
        pose[4] = tz * dt[0] - tx * dt[2];
        pose[5] = tx * dt[1] - ty * dt[0];
        // rotation inside Tm: Mr = W dW^T, dw = (Mr12 - Mr21, Mr20 - Mr02, Mr01 - Mr10)
        float Mr[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int q = 0; q < 3; ++q)
            Mr[3 * r + q] = c.R[3 * r + 0] * dW[3 * q + 0] + c.R[3 * r + 1] * dW[3 * q + 1] + c.R[3 * r + 2] * dW[3 * q + 2];
        pose[3] += Mr[5] - Mr[7];
        pose[4] += Mr[6] - Mr[2];
        pose[5] += Mr[1] - Mr[3];
      }
      if (dpose && __any_sync(0xffffffffu, act)) {
        int comp;
        bool has;
        const float tot = warp_sum_transpose<6>(pose, &comp, &has);
        if (has) atomicAdd(&dpose[v * 6 + comp], tot);
      }
    }
    if (!live) continue;
    // Sigma = M M^T -> dM = G M with G the symmetrised gradient
    const float G[9] = {dSig[0], dSig[1], dSig[2], dSig[1], dSig[3], dSig[4], dSig[2], dSig[4], dSig[5]};
    float dRm[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float dMrk = G[3 * r + 0] * M[0 + k] + G[3 * r + 1] * M[3 + k] + G[3 * r + 2] * M[6 + k];
        dRm[3 * r + k] = dMrk * sc[k];
        gs[k] += dMrk * R[3 * r + k];
      }
    const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    float dq[4];
    dq[0] = 2.f * (-dRm[1] * z + dRm[2] * y + dRm[3] * z - dRm[5] * x - dRm[6] * y + dRm[7] * x);
    dq[1] = 2.f * (dRm[1] * y + dRm[2] * z + dRm[3] * y - 2.f * dRm[4] * x - dRm[5] * w + dRm[6] * z + dRm[7] * w -
                   2.f * dRm[8] * x);
    dq[2] = 2.f * (-2.f * dRm[0] * y + dRm[1] * x + dRm[2] * w + dRm[3] * x + dRm[5] * z - dRm[6] * w + dRm[7] * z -
                   2.f * dRm[8] * y);
    dq[3] = 2.f * (-2.f * dRm[0] * z - dRm[1] * w + dRm[2] * x + dRm[3] * w - 2.f * dRm[4] * z + dRm[5] * y +
                   dRm[6] * x + dRm[7] * y);
    const float qd = dq[0] * w + dq[1] * x + dq[2] * y + dq[3] * z;
    const float iq = 1.f / qlen;
#pragma unroll
    for (int k = 0; k < 4; ++k) gq[k] = (dq[k] - qn[k] * qd) * iq;
    out[0 * ostride + i] = gm[0];
    out[1 * ostride + i] = gm[1];
    out[2 * ostride + i] = gm[2];
    out[3 * ostride + i] = gs[0] * sc[0];
    out[4 * ostride + i] = gs[1] * sc[1];
    out[5 * ostride + i] = gs[2] * sc[2];
    out[6 * ostride + i] = gq[0];
    out[7 * ostride + i] = gq[1];
    out[8 * ostride + i] = gq[2];
    out[9 * ostride + i] = gq[3];
    out[10 * ostride + i] = go;
    // SH gradients: sum over the contributing views (ascending) of gc Y(dir)
    float gsh[3 * D];
#pragma unroll
    for (int k = 0; k < 3 * D; ++k) gsh[k] = 0.f;
    for (unsigned m = vact; m != 0u; m &= m - 1u) {
      const int v = __ffs(m) - 1;
      const DevCam& c = a.cams[v];
      float dx = mx - c.C[0], dy = my - c.C[1], dz = mz - c.C[2];
      const float il = 1.f / sqrtf(dx * dx + dy * dy + dz * dz);
      dx *= il; dy *= il; dz *= il;
      float Y[16];
      sh_basis(DEG, dx, dy, dz, Y);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float gc = gcv[(3 * v + ch) * T];
#pragma unroll
        for (int k = 0; k < D; ++k) gsh[3 * k + ch] += gc * Y[k];
      }
    }
#pragma unroll
    for (int k = 0; k < 3 * D; ++k) out[(11 + k) * ostride + i] = gsh[k];
  }
}

// ============================================================================
// host orchestration
// ============================================================================
template <int TW, int TH, int STAGE>
static void blend_fwd_launch(RasterArgs& a, const u64* inst, float* rgb, float* dout, cudaStream_t st) {
  static int occ = -1;
  if (occ < 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_blend_fwd<TW, TH, STAGE>, 256, 0);
  const int grid = max(1, min(a.n_tiles, a.num_sms * max(occ, 1)));
  k_blend_fwd<TW, TH, STAGE><<<grid, 256, 0, st>>>(a, inst, rgb, dout);
}
template <int TW, int TH, int STAGE>
static void blend_bwd_launch(RasterArgs& a, const u64* inst, const float* dr, const float* dd, cudaStream_t st) {
  static int occ = -1;
  if (occ < 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_blend_bwd<TW, TH, STAGE>, 256, 0);
  const int grid = max(1, min(a.n_tiles, a.num_sms * max(occ, 1)));
  k_blend_bwd<TW, TH, STAGE><<<grid, 256, 0, st>>>(a, inst, dr, dd);
}

template <int TW, int TH>
static void blend_bwd_slots_launch(RasterArgs& a, const u64* inst, const float* dr, const float* dd, cudaStream_t st) {
  static int occ = -1;
  if (occ < 0) {
    cudaFuncSetAttribute(k_blend_bwd_slots<TW, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlotSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_blend_bwd_slots<TW, TH>, 256, kSlotSmem);
  }
  const int grid = max(1, min(a.n_tiles, a.num_sms * max(occ, 1)));
  k_blend_bwd_slots<TW, TH><<<grid, 256, kSlotSmem, st>>>(a, inst, dr, dd);
}

template <int TW, int TH>
static void blend_q_launch(bool fwd, RasterArgs& a, const u64* inst, float* rgb, float* dout, const float* dr,
                           const float* dd, cudaStream_t st) {
  static int occ_f = -1, occ_b = -1;
  if (occ_f < 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, k_blend_fwd_q<TW, TH>, 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, k_blend_bwd_q<TW, TH>, 256, 0);
  }
  const int occ = fwd ? occ_f : occ_b;
  const int grid = max(1, min(a.n_tiles, a.num_sms * max(occ, 1)));
  if (fwd)
    k_blend_fwd_q<TW, TH><<<grid, 256, 0, st>>>(a, inst, rgb, dout);
  else
    k_blend_bwd_q<TW, TH><<<grid, 256, 0, st>>>(a, inst, dr, dd);
}

template <int TW, int TH>
static void blend_h_launch(bool fwd, RasterArgs& a, const u64* inst, float* rgb, float* dout, const float* dr,
                           const float* dd, cudaStream_t st) {
  static int occ_f = -1, occ_b = -1;
  if (occ_f < 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, k_blend_fwd_h<TW, TH>, 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, k_blend_bwd_h<TW, TH>, 256, 0);
  }
  static int occ_g = -1;
  if (occ_g < 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_g, k_blend_bwd_g<TW, TH>, 256, 0);
  if (!fwd && !a.bwd_pix) {  // Gaussians on the lanes: items are (tile, half block)
    const int grid = max(1, min(2 * a.n_tiles, a.num_sms * max(occ_g, 1)));
    k_blend_bwd_g<TW, TH><<<grid, 256, 0, st>>>(a, inst, dr, dd);
    return;
  }
  const int occ = fwd ? occ_f : occ_b;
  const int grid = max(1, min(a.n_tiles, a.num_sms * max(occ, 1)));
  if (fwd)
    k_blend_fwd_h<TW, TH><<<grid, 256, 0, st>>>(a, inst, rgb, dout);
  else
    k_blend_bwd_h<TW, TH><<<grid, 256, 0, st>>>(a, inst, dr, dd);
}

static void blend_h_dispatch(bool fwd, RasterArgs& a, const u64* inst, float* rgb, float* dout, const float* dr,
                             const float* dd, cudaStream_t st) {
  if (a.tile_w == 32 && a.tile_h == 32) blend_h_launch<32, 32>(fwd, a, inst, rgb, dout, dr, dd, st);
  else if (a.tile_w == 32 && a.tile_h == 16) blend_h_launch<32, 16>(fwd, a, inst, rgb, dout, dr, dd, st);
  else blend_h_launch<16, 16>(fwd, a, inst, rgb, dout, dr, dd, st);
}

static void blend_q_dispatch(bool fwd, RasterArgs& a, const u64* inst, float* rgb, float* dout, const float* dr,
                             const float* dd, cudaStream_t st) {
  if (a.tile_w == 32 && a.tile_h == 32) blend_q_launch<32, 32>(fwd, a, inst, rgb, dout, dr, dd, st);
  else if (a.tile_w == 32 && a.tile_h == 16) blend_q_launch<32, 16>(fwd, a, inst, rgb, dout, dr, dd, st);
  else blend_q_launch<16, 16>(fwd, a, inst, rgb, dout, dr, dd, st);
}

#define DCG_STAGES(TW, TH, CALL)                  \
  switch (a.stage) {                              \
    case 64: CALL(TW, TH, 64); break;             \
    case 96: CALL(TW, TH, 96); break;             \
    case 192: CALL(TW, TH, 192); break;           \
    case 256: CALL(TW, TH, 256); break;           \
    default: CALL(TW, TH, 128); break;            \
  }
#define DCG_TILES(CALL)                                                   \
  if (a.tile_w == 32 && a.tile_h == 32) { DCG_STAGES(32, 32, CALL) }      \
  else if (a.tile_w == 32 && a.tile_h == 16) { DCG_STAGES(32, 16, CALL) } \
  else { DCG_STAGES(16, 16, CALL) }

// Dynamic shared memory of the preprocess kernels: the SH coefficients of
// every thread of the block (3 (deg + 1)^2 floats each).
static size_t sh_smem(int deg, int threads) { return sizeof(float) * 3 * (deg + 1) * (deg + 1) * threads; }
// ... and, in the backward, the colour gradient of every view (3 floats each)
// SH coefficients, per-view colour gradients, and two staging slots of a
// view's 2D gradients (3 float4) per thread
static size_t sh_smem_bwd(int deg, int V) {
  return sh_smem(deg, kPreBwdThreads) + sizeof(float) * 3 * V * kPreBwdThreads + sizeof(float4) * 6 * kPreBwdThreads;
}

static void preprocess_smem_init() {
  static bool done = false;
  if (done) return;
  done = true;
  cudaFuncSetAttribute(k_preprocess_fwd<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_smem(0, 256));
  cudaFuncSetAttribute(k_preprocess_fwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_smem(1, 256));
  cudaFuncSetAttribute(k_preprocess_fwd<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_smem(2, 256));
  cudaFuncSetAttribute(k_preprocess_fwd<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_smem(3, 256));
  cudaFuncSetAttribute(k_preprocess_bwd<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_smem_bwd(0, kMaxViewsApi));
  cudaFuncSetAttribute(k_preprocess_bwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_smem_bwd(1, kMaxViewsApi));
  cudaFuncSetAttribute(k_preprocess_bwd<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_smem_bwd(2, kMaxViewsApi));
  cudaFuncSetAttribute(k_preprocess_bwd<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_smem_bwd(3, kMaxViewsApi));
}

static int grid_for(long long n, int num_sms) {
  long long b = (n + 255) / 256;
  long long cap = (long long)num_sms * 8;
  return (int)max(1ll, min(b, cap));
}

void raster_forward(RasterArgs& a, float* rgb, float* dout, u64** list_sorted, u64** inst_sorted, cudaStream_t st) {
  preprocess_smem_init();
  cudaMemsetAsync(a.counters, 0, sizeof(DevCounters), st);
  const long long pairs = (long long)a.V * a.n;
  a.prof(PH_PRE_FWD, true, st);
  if (a.n > 0) {
    const int gr = grid_for(a.n, a.num_sms);
    switch (a.deg) {
      case 0: k_preprocess_fwd<0><<<gr, 256, sh_smem(0, 256), st>>>(a); break;
      case 1: k_preprocess_fwd<1><<<gr, 256, sh_smem(1, 256), st>>>(a); break;
      case 2: k_preprocess_fwd<2><<<gr, 256, sh_smem(2, 256), st>>>(a); break;
      default: k_preprocess_fwd<3><<<gr, 256, sh_smem(3, 256), st>>>(a); break;
    }
    count_launch();
  }
  a.prof(PH_PRE_FWD, false, st);
  a.prof(PH_BINNING, true, st);
  // Partitions of the scans and sorts: about one 2048-key scatter chunk each,
  // from the host's bound on the item count (visible pairs <= V n; instances
  // taken as <= 4 V n, a bound for speed only: any count is sorted correctly),
  // at most the 8 per SM the scratch is sized for.  Small views then run a
  // few hundred partitions instead of 1184 nearly empty ones.
  auto parts = [&](long long bound) {
    return (int)std::max(1ll, std::min<long long>((bound + 2047) / 2048, (long long)a.P));
  };
  const int Pp = parts(pairs);
  const int Pi = parts(std::min<long long>(a.cap_inst, 4 * pairs));
  // compaction into depth keys
  DepthKey dk;
  dk.ib = a.idx_bits;
  dk.vb = 0;
  while ((1 << dk.vb) < a.V) ++dk.vb;
  dk.cs = 31 + dk.ib + dk.vb;
  const int cbits = 64 - dk.cs;
  dk.cmax = cbits >= 4 ? (1u << (cbits < 20 ? cbits : 20)) - 1u : 0u;
  // Only the 31 depth bits are sorted: the view bits above them ride along,
  // since the stable tile sort below separates the views anyway.  The first
  // pass reads the pairs themselves and keeps the visible ones (the
  // compaction), counting them into n_vis; the other passes sort the list.
  const int lbits = 31;
  const PairKeySrc psrc{a.depth, a.touched, (unsigned)a.n, DivU32::make((unsigned)std::max<long long>(a.n, 1)), dk};
  radix_pass(psrc, nullptr, (u64)pairs, a.list_b, a.idx_bits, 8, a.hist, Pp, &a.counters->n_vis, st);
  u64* ls = radix_sort(a.list_b, a.list_a, &a.counters->n_vis, a.idx_bits + 8, a.idx_bits + lbits, a.hist, Pp, st);
  // instance offsets by an ordered scan (the free list buffer holds them),
  // then the emission itself, one thread per visible pair with no barriers
  u64* offs = ls == a.list_a ? a.list_b : a.list_a;
  {
    const InstCount ic{ls, a.touched, a.n, dk};
    k_inst_reduce<<<Pp, 256, 0, st>>>(&a.counters->n_vis, ic, a.part);
    k_part_scan<<<1, 1024, 0, st>>>(a.part, Pp, &a.counters->n_inst);
    k_inst_offsets<<<Pp, 256, 0, st>>>(&a.counters->n_vis, ic, a.part, offs);
  }
  k_emit_inst<<<a.num_sms * 8, 256, 0, st>>>(
      &a.counters->n_vis, offs,
      InstEmit{ls, a.bin, a.cams, a.n, dk, a.tile_w, a.tile_h, a.inst_a, (u64)a.cap_inst, (u64)a.cap_pairs,
               (unsigned)a.n_tiles, a.errword});
  k_clamp_inst<<<1, 1, 0, st>>>(a.counters, (u64)a.cap_inst, a.errword);
  int tb = 1;
  while ((1ll << tb) < (long long)a.n_tiles) ++tb;
  u64* is = radix_sort(a.inst_a, a.inst_b, &a.counters->n_inst_c, kTileShift, kTileShift + tb, a.hist, Pi, st);
  cudaMemsetAsync(a.ranges, 0, sizeof(uint2) * (size_t)max(a.n_tiles, 1), st);
  k_ranges<<<a.num_sms * 8, 256, 0, st>>>(is, &a.counters->n_inst_c, a.ranges, (unsigned)a.n_tiles, a.errword);
  count_launch(4 + 3 * ((lbits + 7) / 8) + 3 * ((tb + 7) / 8) + 2);
  a.prof(PH_BINNING, false, st);
  a.prof(PH_BLEND_FWD, true, st);
  if (a.stage == 32) {
    blend_q_dispatch(true, a, is, rgb, dout, nullptr, nullptr, st);
  } else if (a.stage == 16) {
    blend_h_dispatch(true, a, is, rgb, dout, nullptr, nullptr, st);
  } else {
#define FWD_CALL(TW, TH, SG) blend_fwd_launch<TW, TH, SG>(a, is, rgb, dout, st)
    DCG_TILES(FWD_CALL)
#undef FWD_CALL
  }
  count_launch();
  a.prof(PH_BLEND_FWD, false, st);
  *list_sorted = ls;
  *inst_sorted = is;
}

void raster_backward(RasterArgs& a, const u64* inst_sorted, const float* dL_drgb, const float* dL_ddepth, float* grads,
                     long long g_stride, float* dL_dpose, cudaStream_t st) {
  preprocess_smem_init();
  cudaMemsetAsync(&a.counters->tile_queue_bwd, 0, sizeof(unsigned), st);
  if (dL_dpose) cudaMemsetAsync(dL_dpose, 0, sizeof(float) * 6 * a.V, st);
  a.prof(PH_BLEND_BWD, true, st);
  if (a.stage == 32) {
    blend_q_dispatch(false, a, inst_sorted, nullptr, nullptr, dL_drgb, dL_ddepth, st);
  } else if (a.stage == 16) {
    blend_h_dispatch(false, a, inst_sorted, nullptr, nullptr, dL_drgb, dL_ddepth, st);
  } else if (a.bwd_slots) {
    if (a.tile_w == 32 && a.tile_h == 32) blend_bwd_slots_launch<32, 32>(a, inst_sorted, dL_drgb, dL_ddepth, st);
    else if (a.tile_w == 32 && a.tile_h == 16) blend_bwd_slots_launch<32, 16>(a, inst_sorted, dL_drgb, dL_ddepth, st);
    else blend_bwd_slots_launch<16, 16>(a, inst_sorted, dL_drgb, dL_ddepth, st);
  } else {
#define BWD_CALL(TW, TH, SG) blend_bwd_launch<TW, TH, SG>(a, inst_sorted, dL_drgb, dL_ddepth, st)
    DCG_TILES(BWD_CALL)
#undef BWD_CALL
  }
  count_launch();
  a.prof(PH_BLEND_BWD, false, st);
  a.prof(PH_PRE_BWD, true, st);
  if (a.n > 0) {
    const int gr = (int)std::min<long long>((a.n + kPreBwdThreads - 1) / kPreBwdThreads, (long long)a.num_sms * 16);
    switch (a.deg) {
      case 0: k_preprocess_bwd<0><<<gr, kPreBwdThreads, sh_smem_bwd(0, a.V), st>>>(a, grads, g_stride, dL_dpose); break;
      case 1: k_preprocess_bwd<1><<<gr, kPreBwdThreads, sh_smem_bwd(1, a.V), st>>>(a, grads, g_stride, dL_dpose); break;
      case 2: k_preprocess_bwd<2><<<gr, kPreBwdThreads, sh_smem_bwd(2, a.V), st>>>(a, grads, g_stride, dL_dpose); break;
      default: k_preprocess_bwd<3><<<gr, kPreBwdThreads, sh_smem_bwd(3, a.V), st>>>(a, grads, g_stride, dL_dpose); break;
    }
    count_launch();
  }
  a.prof(PH_PRE_BWD, false, st);
}

// ============================================================================
// L1 parts of Eq. 2-4 (image L1 with weight wimg = 1 - lambda_s, depth L1
// with weight lambda_depth), per view means
// ============================================================================
__global__ void k_loss_l1(const float* __restrict__ rgb, const float* __restrict__ depth,
                          const float* __restrict__ trgb, const float* __restrict__ tdepth, const DevCam* cams, int V,
                          long long n_pix, float wimg, float lam, float* __restrict__ dr, float* __restrict__ dd,
                          float* __restrict__ part) {
  float acc = 0.f;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n_pix; p += (long long)gridDim.x * blockDim.x) {
    int v = 0;
    while (v + 1 < V && p >= cams[v + 1].pix_off) ++v;
    const long long off = cams[v].pix_off;
    const long long P = (long long)cams[v].W * cams[v].H;
    const long long l = p - off;
    const float i3 = wimg / (3.f * (float)P), i1 = lam / (float)P;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const long long k = 3 * off + ch * P + l;
      const float d = rgb[k] - trgb[k];
      dr[k] = d > 0.f ? i3 : (d < 0.f ? -i3 : 0.f);
      acc += fabsf(d) * i3;
    }
    const float e = depth[p] - tdepth[p];
    dd[p] = e > 0.f ? i1 : (e < 0.f ? -i1 : 0.f);
    acc += fabsf(e) * i1;
  }
  // deterministic: fixed-order block reduction, one partial per block
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float s2 = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s2;
  }
}

// Sums the per-block partials in a fixed order and adds the total to *loss.
__global__ void k_loss_final(const float* __restrict__ part, int nb, float* loss) {
  __shared__ float red[32];
  float acc = 0.f;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[b];
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float s2 = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (threadIdx.x == 0) *loss += s2;
  }
}

int loss_partials(int num_sms) { return num_sms * 8; }

void launch_loss_l1(const float* rgb, const float* depth, const float* trgb, const float* tdepth, const DevCam* cams,
                    int V, long long n_pix, float wimg, float lam, float* dr, float* dd, float* loss, float* part,
                    int num_sms, cudaStream_t st) {
  if (n_pix <= 0) return;
  const int nb = grid_for(n_pix, num_sms);  // <= loss_partials(num_sms)
  k_loss_l1<<<nb, 256, 0, st>>>(rgb, depth, trgb, tdepth, cams, V, n_pix, wimg, lam, dr, dd, part);
  k_loss_final<<<1, 256, 0, st>>>(part, nb, loss);
  count_launch(2);
}

}  // namespace dcg
