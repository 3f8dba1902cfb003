// Plain, slow FP64 CPU oracle for the chunked Gaussian-splatting mapper hot path.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library may link, call or
// include this file; only the tests, the smoke check and the benchmark's CPU
// baseline leg use it.  It shares no code, header or constant with the CUDA
// path: every quantity below is written out from its definition.
//
// What it computes, and where each definition comes from:
//   * chunk coordinate and 63-bit chunk id        -- Sec. III-D, Eq. 5 and Eq. 6
//   * frustum planes from the view-projection
//     matrix, flat and hierarchical chunk cull,
//     distance filter                              -- Sec. III-D "Frustum Culling"
//   * Gaussian projection, SH colour, per-pixel
//     front-to-back blending of RGB and depth      -- Sec. III-E (rasterise RGB and depth of
//                                                     the visible subset) with the 3DGS
//                                                     representation of Sec. I / II (SH degree 3)
//   * analytic gradient of a loss seed through the
//     renderer to every Gaussian parameter and to
//     the camera pose                              -- Sec. III-C, Eq. 2-4 (losses are optimised
//                                                     through differentiable rendering)
// The paper does not print the rasteriser; the readings taken here (3-sigma
// support of the dilated 2D Gaussian, alpha clamp 0.99, cut-offs 1/255 and
// 1e-4, 0.3 px dilation, real SH with Condon-Shortley phase, un-normalised
// depth, sample point of pixel (x,y) at (x,y)) are listed with the design notes.
//
// Precision: FP64 everywhere, except the chunk key, which is a definition
// evaluated in FP32 (the precision the kernel decides it in), and
// orc_depth_f32, the FP32 depth used as the sort key.
// Build: g++ -O2 -fPIC -shared -fopenmp -ffp-contract=off (no FMA contraction).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

// Camera: pinhole intrinsics, image size, world->camera rigid transform
// (row-major 4x4), near and far distance.
struct OrcCam {
  double fx, fy, cx, cy;
  int32_t W, H;
  int32_t pad0, pad1;
  double Tcw[16];
  double znear, zfar;
};

// ---------------------------------------------------------------------------
// Eq. 5 / Eq. 6: chunk coordinate floor((p + s/2)/s) per axis, then
// EncodedID = (cx+2^20)*2^42 + (cy+2^20)*2^21 + (cz+2^20).
// Evaluated in FP32 with one rounding per operation (add, divide) and floor.
// A coordinate outside [-2^20, 2^20-1] (the paper's +-1M chunk range) or a
// non-finite position sets bad[i]=1 and yields key 0.
// ---------------------------------------------------------------------------
int orc_chunk_keys(const float* means, int64_t n, float s, int32_t* coords, uint64_t* keys,
                   uint8_t* bad) {
  const float half = 0.5f * s;  // exact: scaling by a power of two
  for (int64_t i = 0; i < n; ++i) {
    int ok = 1;
    int32_t c[3];
    for (int a = 0; a < 3; ++a) {
      volatile float t = means[3 * i + a] + half;
      volatile float q = t / s;
      float f = std::floor((float)q);
      if (!(f >= -1048576.0f && f <= 1048575.0f)) {
        ok = 0;
        c[a] = 0;
      } else {
        c[a] = (int32_t)f;
      }
    }
    coords[3 * i + 0] = c[0];
    coords[3 * i + 1] = c[1];
    coords[3 * i + 2] = c[2];
    bad[i] = (uint8_t)(!ok);
    if (ok) {
      const uint64_t off = 1ull << 20;
      keys[i] = ((uint64_t)((int64_t)c[0] + (int64_t)off) << 42) |
                ((uint64_t)((int64_t)c[1] + (int64_t)off) << 21) |
                (uint64_t)((int64_t)c[2] + (int64_t)off);
    } else {
      keys[i] = 0;
    }
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Frustum cull (Sec. III-D): planes are extracted from the view-projection
// matrix VP = P * Tcw (Gribb-Hartmann: row4 +- row_i).  P maps a camera-frame
// point (X,Y,Z) to clip space so that x/w in [-1,1] <=> u in [0,W],
// y/w in [-1,1] <=> v in [0,H] and z/w in [-1,1] <=> Z in [znear, zfar].
// A box is kept iff, for all six planes (a,b,c,d), the box vertex furthest
// along (a,b,c) satisfies ((a*x + b*y) + c*z) + d >= 0, and the distance from
// the camera centre to the box is <= dfar (distance-based filtering).
// Evaluation order is fixed as written (no FMA), in FP64.
// ---------------------------------------------------------------------------
static void orc_planes(const OrcCam* cam, double planes[6][4], double C[3]) {
  const double W = cam->W, H = cam->H, zn = cam->znear, zf = cam->zfar;
  double P[16] = {0};
  P[0] = 2.0 * cam->fx / W;
  P[2] = (2.0 * cam->cx - W) / W;
  P[5] = 2.0 * cam->fy / H;
  P[6] = (2.0 * cam->cy - H) / H;
  P[10] = (zf + zn) / (zf - zn);
  P[11] = -2.0 * zf * zn / (zf - zn);
  P[14] = 1.0;
  double VP[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 4; ++k) acc = acc + P[4 * i + k] * cam->Tcw[4 * k + j];
      VP[4 * i + j] = acc;
    }
  for (int j = 0; j < 4; ++j) {
    planes[0][j] = VP[12 + j] + VP[0 + j];  // u >= 0
    planes[1][j] = VP[12 + j] - VP[0 + j];  // u <= W
    planes[2][j] = VP[12 + j] + VP[4 + j];  // v >= 0
    planes[3][j] = VP[12 + j] - VP[4 + j];  // v <= H
    planes[4][j] = VP[12 + j] + VP[8 + j];  // Z >= znear
    planes[5][j] = VP[12 + j] - VP[8 + j];  // Z <= zfar
  }
  // camera centre C = -R^T t
  for (int j = 0; j < 3; ++j) {
    double acc = cam->Tcw[0 + j] * cam->Tcw[3];
    acc = acc + cam->Tcw[4 + j] * cam->Tcw[7];
    acc = acc + cam->Tcw[8 + j] * cam->Tcw[11];
    C[j] = -acc;
  }
}

static int orc_box_visible(const double planes[6][4], const double C[3], double dfar,
                           const double lo[3], const double hi[3]) {
  for (int p = 0; p < 6; ++p) {
    const double* pl = planes[p];
    double vx = pl[0] >= 0.0 ? hi[0] : lo[0];
    double vy = pl[1] >= 0.0 ? hi[1] : lo[1];
    double vz = pl[2] >= 0.0 ? hi[2] : lo[2];
    double val = ((pl[0] * vx + pl[1] * vy) + pl[2] * vz) + pl[3];
    if (val < 0.0) return 0;
  }
  double d2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    double e = 0.0;
    if (C[a] < lo[a]) e = lo[a] - C[a];
    else if (C[a] > hi[a]) e = C[a] - hi[a];
    d2 = d2 + e * e;
  }
  return d2 <= dfar * dfar;
}

// Chunk c (integer coords) covers [c*s - s/2, c*s + s/2) on each axis.
static void orc_chunk_box(const int32_t lo_c[3], const int32_t hi_c[3], double s, double lo[3],
                          double hi[3]) {
  for (int a = 0; a < 3; ++a) {
    lo[a] = (double)lo_c[a] * s - 0.5 * s;
    hi[a] = (double)hi_c[a] * s + 0.5 * s;
  }
}

// Recursive region test: reject the whole region if its box fails, otherwise
// split it along its longest axis until single chunks are reached.
static void orc_cull_region(const double planes[6][4], const double C[3], double dfar, double s,
                            const int32_t* coords, std::vector<int64_t>& idx, int32_t lo_c[3],
                            int32_t hi_c[3], uint8_t* mask) {
  if (idx.empty()) return;
  double lo[3], hi[3];
  orc_chunk_box(lo_c, hi_c, s, lo, hi);
  if (!orc_box_visible(planes, C, dfar, lo, hi)) return;
  int ax = 0;
  int64_t ext = -1;
  for (int a = 0; a < 3; ++a) {
    int64_t e = (int64_t)hi_c[a] - lo_c[a];
    if (e > ext) { ext = e; ax = a; }
  }
  if (ext == 0) {
    for (int64_t k : idx) mask[k] = 1;  // a single chunk cell: the test above was the chunk test
    return;
  }
  int32_t mid = (int32_t)(((int64_t)lo_c[ax] + (int64_t)hi_c[ax]) >> 1);
  std::vector<int64_t> a_idx, b_idx;
  for (int64_t k : idx) (coords[3 * k + ax] <= mid ? a_idx : b_idx).push_back(k);
  int32_t lo_b[3] = {lo_c[0], lo_c[1], lo_c[2]}, hi_a[3] = {hi_c[0], hi_c[1], hi_c[2]};
  hi_a[ax] = mid;
  lo_b[ax] = mid + 1;
  orc_cull_region(planes, C, dfar, s, coords, a_idx, lo_c, hi_a, mask);
  orc_cull_region(planes, C, dfar, s, coords, b_idx, lo_b, hi_c, mask);
}

// mask[k] = 1 iff chunk k (integer coords[3k..3k+2]) is visible.
// hierarchical = 0: every chunk tested on its own; 1: recursive region subdivision.
int orc_cull(const int32_t* coords, int64_t n_chunks, double s, const OrcCam* cam, double dfar,
             int hierarchical, uint8_t* mask) {
  double planes[6][4], C[3];
  orc_planes(cam, planes, C);
  std::memset(mask, 0, (size_t)n_chunks);
  if (!hierarchical) {
    for (int64_t k = 0; k < n_chunks; ++k) {
      double lo[3], hi[3];
      orc_chunk_box(&coords[3 * k], &coords[3 * k], s, lo, hi);
      mask[k] = (uint8_t)orc_box_visible(planes, C, dfar, lo, hi);
    }
    return 0;
  }
  if (n_chunks == 0) return 0;
  int32_t lo_c[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi_c[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
  std::vector<int64_t> idx((size_t)n_chunks);
  for (int64_t k = 0; k < n_chunks; ++k) {
    idx[(size_t)k] = k;
    for (int a = 0; a < 3; ++a) {
      lo_c[a] = std::min(lo_c[a], coords[3 * k + a]);
      hi_c[a] = std::max(hi_c[a], coords[3 * k + a]);
    }
  }
  orc_cull_region(planes, C, dfar, s, coords, idx, lo_c, hi_c, mask);
  return 0;
}

// Returns the six planes (a,b,c,d) and the camera centre, for tests.
int orc_frustum_planes(const OrcCam* cam, double* planes24, double* C3) {
  double planes[6][4];
  orc_planes(cam, planes, C3);
  std::memcpy(planes24, planes, sizeof(planes));
  return 0;
}

// ---------------------------------------------------------------------------
// Real spherical harmonics with Condon-Shortley phase, any degree l <= 3 used
// here.  On the unit sphere (x,y,z) = (sin t cos p, sin t sin p, cos t):
//   Y_l0  = K_l^0 P_l(z)
//   Y_lm  = sqrt2 K_l^m (-1)^m P_l^(m)(z) Re((x+iy)^m)      m > 0
//   Y_l-m = sqrt2 K_l^m (-1)^m P_l^(m)(z) Im((x+iy)^m)      m > 0
// with K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), P_l^(m) the m-th derivative
// of the Legendre polynomial, and (1-z^2)^(m/2) e^{imp} = (x+iy)^m.
// This polynomial form also gives the gradient in R^3; its tangential part is
// what the chain rule through the normalised direction keeps.
// Index k = l*l + l + m.
// ---------------------------------------------------------------------------
static double orc_fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= (double)i;
  return f;
}
static double orc_binom(int n, int k) { return orc_fact(n) / (orc_fact(k) * orc_fact(n - k)); }

// d^m/dz^m of the Legendre polynomial P_l at z.
static double orc_legendre_deriv(int l, int m, double z) {
  // P_l(z) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k,l) z^(l-2k)
  double acc = 0.0;
  for (int k = 0; 2 * k <= l; ++k) {
    int p = l - 2 * k;
    if (p < m) continue;
    double coef = ((k & 1) ? -1.0 : 1.0) * orc_binom(l, k) * orc_binom(2 * l - 2 * k, l);
    double dcoef = 1.0;
    for (int j = 0; j < m; ++j) dcoef *= (double)(p - j);
    acc += coef * dcoef * std::pow(z, (double)(p - m));
  }
  return acc / std::pow(2.0, (double)l);
}

static void orc_cpow(double x, double y, int m, double* re, double* im) {
  double r = 1.0, i = 0.0;
  for (int k = 0; k < m; ++k) {
    double nr = r * x - i * y, ni = r * y + i * x;
    r = nr;
    i = ni;
  }
  *re = r;
  *im = i;
}

static void orc_sh(int l, int m, const double d[3], double* val, double grad[3]) {
  const double PI = 3.14159265358979323846;
  int am = m < 0 ? -m : m;
  double K = std::sqrt((2.0 * l + 1.0) / (4.0 * PI) * orc_fact(l - am) / orc_fact(l + am));
  double sgn = (am & 1) ? -1.0 : 1.0;
  double Pm = sgn * orc_legendre_deriv(l, am, d[2]);
  double dPm = sgn * orc_legendre_deriv(l, am + 1, d[2]);
  double A, dAx, dAy;
  if (am == 0) {
    A = 1.0;
    dAx = 0.0;
    dAy = 0.0;
  } else {
    double re, im, re1, im1;
    orc_cpow(d[0], d[1], am, &re, &im);
    orc_cpow(d[0], d[1], am - 1, &re1, &im1);
    if (m > 0) {
      A = re;
      dAx = am * re1;
      dAy = -am * im1;
    } else {
      A = im;
      dAx = am * im1;
      dAy = am * re1;
    }
  }
  double N = (m == 0) ? K : std::sqrt(2.0) * K;
  *val = N * Pm * A;
  if (grad) {
    grad[0] = N * Pm * dAx;
    grad[1] = N * Pm * dAy;
    grad[2] = N * dPm * A;
  }
}

// out[i*16 + k] = Y_k(dirs[i]) for k < (deg+1)^2 (rest zero).
int orc_sh_basis(int deg, const double* dirs, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < 16; ++k) out[16 * i + k] = 0.0;
    for (int l = 0; l <= deg; ++l)
      for (int m = -l; m <= l; ++m) {
        double v;
        orc_sh(l, m, &dirs[3 * i], &v, nullptr);
        out[16 * i + l * l + l + m] = v;
      }
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Projection of one Gaussian into one camera (FP64).
// Parameter record (AoS, F = 11 + 3*(deg+1)^2 doubles):
//   [0..2] mean, [3..5] log-scale, [6..9] quaternion (w,x,y,z, unnormalised),
//   [10] opacity logit, [11 + 3k + ch] SH coefficient k, colour channel ch.
// ---------------------------------------------------------------------------
struct OrcProj {
  int vis;
  float z32;          // FP32 depth: the blend-order key and the near-plane decision
  double t[3];
  double u, v, z;
  double tx_c, ty_c;  // clamped camera-plane coordinates used by the Jacobian
  int clamp_x, clamp_y;
  double J[6];        // 2x3
  double Tm[6];       // J * W (2x3)
  double S3[9];       // 3D covariance
  double M[9], R[9], s[3], qn[4], qlen;
  double a, b, c, det, A, B, Cc;  // 2D covariance (dilated) and its inverse
  double ex, ey;
  double dir[3], dist;
  double Y[16], Yg[16][3];
  double raw[3], rgb[3];
  double o;
};

static inline int orc_nsh(int deg) { return (deg + 1) * (deg + 1); }

static void orc_project(const double* p, int deg, const OrcCam* cam, OrcProj* g) {
  const double* T = cam->Tcw;
  const double Wm[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
  for (int r = 0; r < 3; ++r)
    g->t[r] = Wm[3 * r + 0] * p[0] + Wm[3 * r + 1] * p[1] + Wm[3 * r + 2] * p[2] + T[4 * r + 3];
  g->z = g->t[2];
  // The order of blending and the near-plane test are discrete decisions; they
  // are taken on the FP32 depth ((W20*mx + W21*my) + W22*mz) + t2 (one
  // rounding per operation), the precision the kernel decides them in.
  {
    volatile float a = (float)T[8] * (float)p[0];
    volatile float b = (float)T[9] * (float)p[1];
    volatile float ab = a + b;
    volatile float c = (float)T[10] * (float)p[2];
    volatile float abc = ab + c;
    volatile float r = abc + (float)T[11];
    g->z32 = r;
  }
  g->vis = g->z32 > (float)cam->znear;
  if (!g->vis) return;
  const double tx = g->t[0], ty = g->t[1], tz = g->t[2];
  g->u = cam->fx * tx / tz + cam->cx;
  g->v = cam->fy * ty / tz + cam->cy;
  // Jacobian of the perspective map, with x/z and y/z clamped to the image
  // plane extended by 15% of the image size on each side.
  const double xlo = (-0.15 * cam->W - cam->cx) / cam->fx, xhi = (1.15 * cam->W - cam->cx) / cam->fx;
  const double ylo = (-0.15 * cam->H - cam->cy) / cam->fy, yhi = (1.15 * cam->H - cam->cy) / cam->fy;
  double rx = tx / tz, ry = ty / tz;
  g->clamp_x = (rx < xlo || rx > xhi);
  g->clamp_y = (ry < ylo || ry > yhi);
  rx = std::min(std::max(rx, xlo), xhi);
  ry = std::min(std::max(ry, ylo), yhi);
  g->tx_c = rx * tz;
  g->ty_c = ry * tz;
  g->J[0] = cam->fx / tz; g->J[1] = 0.0; g->J[2] = -cam->fx * g->tx_c / (tz * tz);
  g->J[3] = 0.0; g->J[4] = cam->fy / tz; g->J[5] = -cam->fy * g->ty_c / (tz * tz);
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c)
      g->Tm[3 * r + c] = g->J[3 * r + 0] * Wm[0 + c] + g->J[3 * r + 1] * Wm[3 + c] + g->J[3 * r + 2] * Wm[6 + c];
  // 3D covariance  Sigma = R S S^T R^T
  for (int a = 0; a < 3; ++a) g->s[a] = std::exp(p[3 + a]);
  g->qlen = std::sqrt(p[6] * p[6] + p[7] * p[7] + p[8] * p[8] + p[9] * p[9]);
  for (int a = 0; a < 4; ++a) g->qn[a] = p[6 + a] / g->qlen;
  const double w = g->qn[0], x = g->qn[1], y = g->qn[2], z = g->qn[3];
  double* R = g->R;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) g->M[3 * r + c] = R[3 * r + c] * g->s[c];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += g->M[3 * r + k] * g->M[3 * c + k];
      g->S3[3 * r + c] = acc;
    }
  // 2D covariance  Tm Sigma Tm^T + 0.3 I
  double cov[2][2];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      double acc = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) acc += g->Tm[3 * r + i] * g->S3[3 * i + j] * g->Tm[3 * c + j];
      cov[r][c] = acc;
    }
  g->a = cov[0][0] + 0.3;
  g->b = cov[0][1];
  g->c = cov[1][1] + 0.3;
  g->det = g->a * g->c - g->b * g->b;
  if (!(g->det > 0.0)) { g->vis = 0; return; }
  g->A = g->c / g->det;
  g->B = -g->b / g->det;
  g->Cc = g->a / g->det;
  // exact bounding box of the 3-sigma ellipse q <= 9
  g->ex = 3.0 * std::sqrt(g->a);
  g->ey = 3.0 * std::sqrt(g->c);
  // colour from SH, evaluated along the viewing direction (mean - camera centre)
  double Cw[3];
  for (int j = 0; j < 3; ++j) Cw[j] = -(T[0 + j] * T[3] + T[4 + j] * T[7] + T[8 + j] * T[11]);
  double d[3] = {p[0] - Cw[0], p[1] - Cw[1], p[2] - Cw[2]};
  g->dist = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int a = 0; a < 3; ++a) g->dir[a] = d[a] / g->dist;
  const int D = orc_nsh(deg);
  for (int l = 0; l <= deg; ++l)
    for (int m = -l; m <= l; ++m) {
      int k = l * l + l + m;
      orc_sh(l, m, g->dir, &g->Y[k], g->Yg[k]);
    }
  for (int ch = 0; ch < 3; ++ch) {
    double acc = 0.0;
    for (int k = 0; k < D; ++k) acc += p[11 + 3 * k + ch] * g->Y[k];
    g->raw[ch] = acc + 0.5;
    g->rgb[ch] = g->raw[ch] < 0.0 ? 0.0 : g->raw[ch];
  }
  g->o = 1.0 / (1.0 + std::exp(-p[10]));
}

// Per-Gaussian projection outputs for tests: per Gaussian 16 doubles
// [vis, u, v, z, A, B, C, o, r, g, b, ex, ey, a, b2d, c2d].
int orc_project_all(const double* params, int64_t n, int deg, const OrcCam* cam, double* out) {
  const int F = 11 + 3 * orc_nsh(deg);
  for (int64_t i = 0; i < n; ++i) {
    OrcProj g;
    orc_project(&params[F * i], deg, cam, &g);
    double* o = &out[16 * i];
    for (int k = 0; k < 16; ++k) o[k] = 0.0;
    o[0] = g.vis;
    o[3] = g.z;
    if (!g.vis) continue;
    o[1] = g.u; o[2] = g.v; o[4] = g.A; o[5] = g.B; o[6] = g.Cc; o[7] = g.o;
    o[8] = g.rgb[0]; o[9] = g.rgb[1]; o[10] = g.rgb[2];
    o[11] = g.ex; o[12] = g.ey; o[13] = g.a; o[14] = g.b; o[15] = g.c;
  }
  return 0;
}

// Which Gaussians take the clamped branch of the perspective Jacobian:
// out[i] = clamp_x | clamp_y << 1 (0 for Gaussians culled by the near plane).
int orc_clamp_flags(const double* params, int64_t n, int deg, const OrcCam* cam, int32_t* out) {
  const int F = 11 + 3 * orc_nsh(deg);
  for (int64_t i = 0; i < n; ++i) {
    OrcProj g;
    orc_project(&params[F * i], deg, cam, &g);
    out[i] = g.vis ? (g.clamp_x | (g.clamp_y << 1)) : 0;
  }
  return 0;
}

// FP32 camera depth, the sort key of the kernels: ((W20*mx + W21*my) + W22*mz) + t2,
// one rounding per operation.
int orc_depth_f32(const float* means, int64_t n, const float* Tcw, float* z) {
  for (int64_t i = 0; i < n; ++i) {
    volatile float a = Tcw[8] * means[3 * i + 0];
    volatile float b = Tcw[9] * means[3 * i + 1];
    volatile float ab = a + b;
    volatile float c = Tcw[10] * means[3 * i + 2];
    volatile float abc = ab + c;
    volatile float r = abc + Tcw[11];
    z[i] = r;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Per-pixel blending (the definition).  For pixel (x, y), sample point (x, y):
//   candidates: visible Gaussians with q = d^T Sigma'^-1 d <= 9, d = (x-u, y-v),
//               and alpha = min(0.99, o exp(-q/2)) >= 1/255;
//   order: ascending (depth, index);
//   front to back: stop before any Gaussian with T (1-alpha) < 1e-4;
//   otherwise C += T alpha c, D += T alpha z, T *= (1 - alpha).  Background 0.
// Order: ascending (FP32 depth key, index), see orc_project.
// flags (for comparing with an FP32 implementation): bit0 a Gaussian whose q
// lies within the band of 9 that would pass the alpha test, bit1 alpha within
// its band of the 1/255 cut-off, bit2 T(1-alpha) within its band of the 1e-4
// cut-off.  Each band is a constant relative floor (eps_q, eps_a, eps_t) plus
// k times a first-order bound of the error with which an FP32 evaluation
// (unit roundoff u = 2^-24) reaches the same quantity:
//   q:     e_q = u (6 S + 3 q kappa_det + 2 (|g_x| (|dx| + 32) + |g_y| (|dy| + 32)))
//          S = |A| dx^2 + 2 |B dx dy| + |C| dy^2 (the terms of q before they
//          cancel), kappa_det = (|a c| + b^2) / (a c - b^2) (the relative error
//          of the covariance's determinant, which scales every conic
//          coefficient), g = conic d (an offset d held with an absolute error of
//          u (|d| + 32) px moves q by 2 g . delta);
//   alpha: relative e_a = e_q / 2 + 16 u (alpha = o exp(-q/2); 16 u covers the
//          opacity, the exponential and the product);
//   T:     relative e_T after n Gaussians = sum_j (alpha_j / (1 - alpha_j)) e_a,j
//          + 2 u per factor (each (1 - alpha) inherits alpha's error scaled by
//          alpha / (1 - alpha), and the product rounds once per factor).
// ---------------------------------------------------------------------------
struct OrcCand {
  float z;
  int64_t i;
  double alpha, G, q;
  double ea;  // relative FP32 error bound of alpha (flags only)
};

struct OrcScene {
  int deg, F;
  std::vector<OrcProj> proj;
  std::vector<int64_t> vis;
};

static void orc_scene(const double* params, int64_t n, int deg, const OrcCam* cam, OrcScene* sc) {
  sc->deg = deg;
  sc->F = 11 + 3 * orc_nsh(deg);
  sc->proj.resize((size_t)n);
  sc->vis.clear();
  // every Gaussian is projected independently
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) orc_project(&params[sc->F * i], deg, cam, &sc->proj[(size_t)i]);
  for (int64_t i = 0; i < n; ++i)
    if (sc->proj[(size_t)i].vis) sc->vis.push_back(i);
}

struct OrcEps {
  double q, a, t, k;  // constant relative floors of the three bands, factor on the derived bounds
};

static const double kOrcU32 = 1.0 / 16777216.0;  // 2^-24, FP32 unit roundoff

// First-order bound of the FP32 error of q at offset (dx, dy), see above.
static double orc_q_error(const OrcProj& g, double dx, double dy, double q) {
  const double S = std::fabs(g.A) * dx * dx + 2.0 * std::fabs(g.B * dx * dy) + std::fabs(g.Cc) * dy * dy;
  const double kdet = (std::fabs(g.a * g.c) + g.b * g.b) / g.det;
  const double gx = g.A * dx + g.B * dy, gy = g.B * dx + g.Cc * dy;
  const double cen = 2.0 * (std::fabs(gx) * (std::fabs(dx) + 32.0) + std::fabs(gy) * (std::fabs(dy) + 32.0));
  return kOrcU32 * (6.0 * S + 3.0 * std::fabs(q) * kdet + cen);
}

static int orc_collect(const OrcScene& sc, const OrcCam* cam, double x, double y,
                       std::vector<OrcCand>& cand, const OrcEps* eps, int* flags) {
  cand.clear();
  int fl = 0;
  const double a_cut = 1.0 / 255.0;
  for (int64_t i : sc.vis) {
    const OrcProj& g = sc.proj[(size_t)i];
    double dx = x - g.u, dy = y - g.v;
    double q = g.A * dx * dx + 2.0 * g.B * dx * dy + g.Cc * dy * dy;
    double ea = 0.0;
    if (eps) {
      const double eq = eps->k * orc_q_error(g, dx, dy, q);
      ea = eq / 2.0 + eps->k * 16.0 * kOrcU32;
      if (std::fabs(q - 9.0) <= eps->q * 9.0 + eq && g.o * std::exp(-4.5) >= a_cut * (1.0 - eps->a - ea)) fl |= 1;
    }
    if (q > 9.0) continue;
    double G = std::exp(-0.5 * q);
    double araw = g.o * G;
    if (eps && std::fabs(araw - a_cut) <= (eps->a + ea) * a_cut) fl |= 2;
    double alpha = araw < 0.99 ? araw : 0.99;
    if (alpha < a_cut) continue;
    cand.push_back({g.z32, i, alpha, G, q, ea});
  }
  std::sort(cand.begin(), cand.end(), [](const OrcCand& l, const OrcCand& r) {
    return l.z < r.z || (l.z == r.z && l.i < r.i);
  });
  if (flags) *flags = fl;
  return 0;
}

// Number of Gaussians blended (the prefix before the termination point).
static size_t orc_blend_prefix(const std::vector<OrcCand>& cand, const OrcEps* eps, int* flags,
                               double* T_out) {
  double T = 1.0, eT = 0.0;
  size_t n = 0;
  int fl = flags ? *flags : 0;
  for (; n < cand.size(); ++n) {
    const double a = cand[n].alpha;
    double Tn = T * (1.0 - a);
    if (eps) {
      eT += a / (1.0 - a) * cand[n].ea + eps->k * 2.0 * kOrcU32;
      if (std::fabs(Tn - 1e-4) <= eps->t * 1e-4 + eT * Tn) fl |= 4;
    }
    if (Tn < 1e-4) break;
    T = Tn;
  }
  if (flags) *flags = fl;
  if (T_out) *T_out = T;
  return n;
}

static int orc_threads(int nt) {
#ifdef _OPENMP
  return nt > 0 ? nt : omp_get_max_threads();
#else
  (void)nt;
  return 1;
#endif
}

// Render the m listed pixels (pix[2k] = x, pix[2k+1] = y).
int orc_render(const double* params, int64_t n, int deg, const OrcCam* cam, const int32_t* pix,
               int64_t m, const double* eps4, int n_threads, double* rgb, double* depth,
               double* T_final, int32_t* n_contrib, int32_t* flags) {
  OrcScene sc;
  orc_scene(params, n, deg, cam, &sc);
  OrcEps eps = {eps4[0], eps4[1], eps4[2], eps4[3]};
  const int nt = orc_threads(n_threads);
#pragma omp parallel num_threads(nt)
  {
    std::vector<OrcCand> cand;
#pragma omp for schedule(dynamic, 16)
    for (int64_t k = 0; k < m; ++k) {
      int fl = 0;
      orc_collect(sc, cam, (double)pix[2 * k], (double)pix[2 * k + 1], cand, &eps, &fl);
      size_t nb = orc_blend_prefix(cand, &eps, &fl, nullptr);
      double T = 1.0, C[3] = {0, 0, 0}, D = 0.0;
      for (size_t j = 0; j < nb; ++j) {
        const OrcProj& g = sc.proj[(size_t)cand[j].i];
        double w = T * cand[j].alpha;
        for (int ch = 0; ch < 3; ++ch) C[ch] += w * g.rgb[ch];
        D += w * g.z;
        T = T * (1.0 - cand[j].alpha);
      }
      for (int ch = 0; ch < 3; ++ch) rgb[3 * k + ch] = C[ch];
      depth[k] = D;
      T_final[k] = T;
      n_contrib[k] = (int32_t)nb;
      flags[k] = fl;
    }
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Analytic backward.  Input: dL/dC (m x 3) and dL/dD (m) for the listed pixels.
// Output: dL/dparams (n x F, accumulated into grad, which the caller zeroes)
// and dL/dxi (6, accumulated) for the pose perturbation Tcw <- exp(xi^) Tcw,
// xi = (v, w): a camera-frame point moves by v + w x t.
//
// Per pixel, with contributors i = 0..n-1 in blend order, T_i the
// transmittance before i and S_i the colour/depth blended behind i divided by
// T_{i+1}:  dL/dc_i = T_i a_i g,  dL/da_i = T_i ((c_i - S_i).g + (z_i - Sd_i) gd).
// alpha = min(0.99, o G): no gradient when clamped; G = exp(-q/2).
// Per Gaussian the chain then goes through the conic inverse, the 2D
// covariance T Sigma T^T (T = J W), the perspective Jacobian J(t), the 3D
// covariance R S S^T R^T, the quaternion normalisation, exp of the
// log-scale, the sigmoid, the SH basis and the normalised viewing direction.
// ---------------------------------------------------------------------------
int orc_render_bwd(const double* params, int64_t n, int deg, const OrcCam* cam, const int32_t* pix,
                   int64_t m, const double* dL_drgb, const double* dL_ddepth, int n_threads,
                   double* grad, double* grad_pose) {
  OrcScene sc;
  orc_scene(params, n, deg, cam, &sc);
  const int F = sc.F;
  const int nt = orc_threads(n_threads);
  // 2D gradient per Gaussian: du, dv, dA, dB, dC, do, dr, dg, db, dz
  std::vector<std::vector<double>> g2_t((size_t)nt);
#pragma omp parallel num_threads(nt)
  {
#ifdef _OPENMP
    const int tid = omp_get_thread_num();
#else
    const int tid = 0;
#endif
    std::vector<double>& g2 = g2_t[(size_t)tid];
    g2.assign((size_t)n * 10, 0.0);
    std::vector<OrcCand> cand;
    std::vector<double> Tpre;
#pragma omp for schedule(dynamic, 16)
    for (int64_t k = 0; k < m; ++k) {
      const double x = (double)pix[2 * k], y = (double)pix[2 * k + 1];
      orc_collect(sc, cam, x, y, cand, nullptr, nullptr);
      size_t nb = orc_blend_prefix(cand, nullptr, nullptr, nullptr);
      Tpre.resize(nb);
      double T = 1.0;
      for (size_t j = 0; j < nb; ++j) {
        Tpre[j] = T;
        T = T * (1.0 - cand[j].alpha);
      }
      const double* gC = &dL_drgb[3 * k];
      const double gD = dL_ddepth[k];
      double S[3] = {0, 0, 0}, Sd = 0.0;
      for (size_t jj = nb; jj-- > 0;) {
        const OrcCand& cd = cand[jj];
        const OrcProj& g = sc.proj[(size_t)cd.i];
        const double Ti = Tpre[jj], al = cd.alpha;
        double* out = &g2[(size_t)cd.i * 10];
        double dal = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
          out[6 + ch] += Ti * al * gC[ch];
          dal += (g.rgb[ch] - S[ch]) * gC[ch];
        }
        out[9] += Ti * al * gD;
        dal += (g.z - Sd) * gD;
        dal *= Ti;
        for (int ch = 0; ch < 3; ++ch) S[ch] = al * g.rgb[ch] + (1.0 - al) * S[ch];
        Sd = al * g.z + (1.0 - al) * Sd;
        if (g.o * cd.G >= 0.99) continue;  // clamped alpha
        out[5] += dal * cd.G;
        double dG = dal * g.o;
        double dq = -0.5 * cd.G * dG;
        double dx = x - g.u, dy = y - g.v;
        out[2] += dq * dx * dx;
        out[3] += dq * 2.0 * dx * dy;
        out[4] += dq * dy * dy;
        out[0] += -dq * 2.0 * (g.A * dx + g.B * dy);
        out[1] += -dq * 2.0 * (g.B * dx + g.Cc * dy);
      }
    }
  }
  std::vector<double> g2((size_t)n * 10, 0.0);
  for (int t = 0; t < nt; ++t)
    for (size_t j = 0; j < g2.size(); ++j) g2[j] += g2_t[(size_t)t][j];

  const double* T = cam->Tcw;
  const double Wm[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
  double pose[6] = {0, 0, 0, 0, 0, 0};
  const int D = orc_nsh(deg);
  for (int64_t i = 0; i < n; ++i) {
    const OrcProj& g = sc.proj[(size_t)i];
    if (!g.vis) continue;
    const double* d2 = &g2[(size_t)i * 10];
    bool any = false;
    for (int j = 0; j < 10; ++j) any |= (d2[j] != 0.0);
    if (!any) continue;
    const double* p = &params[F * i];
    double* gp = &grad[F * i];
    double dt[3] = {0, 0, 0};  // dL/dt (camera-frame mean)
    // u = fx tx/tz + cx, v = fy ty/tz + cy, depth = tz
    const double tx = g.t[0], ty = g.t[1], tz = g.t[2];
    dt[0] += d2[0] * cam->fx / tz;
    dt[1] += d2[1] * cam->fy / tz;
    dt[2] += -d2[0] * cam->fx * tx / (tz * tz) - d2[1] * cam->fy * ty / (tz * tz) + d2[9];
    // conic (A,B,C) = inverse of [[a,b],[b,c]]
    const double a = g.a, b = g.b, c = g.c, det = g.det, det2 = det * det;
    const double dA = d2[2], dB = d2[3], dC = d2[4];
    double da = dA * (-c * c / det2) + dB * (b * c / det2) + dC * (1.0 / det - a * c / det2);
    double db = dA * (2.0 * b * c / det2) + dB * (-1.0 / det - 2.0 * b * b / det2) + dC * (2.0 * a * b / det2);
    double dc = dA * (1.0 / det - c * a / det2) + dB * (b * a / det2) + dC * (-a * a / det2);
    // a = T0 S T0^T + 0.3, b = T0 S T1^T, c = T1 S T1^T + 0.3
    const double* Tm = g.Tm;
    double dSig[9];
    for (int r = 0; r < 3; ++r)
      for (int s2 = 0; s2 < 3; ++s2)
        dSig[3 * r + s2] = da * Tm[r] * Tm[s2] + db * Tm[r] * Tm[3 + s2] + dc * Tm[3 + r] * Tm[3 + s2];
    double ST0[3], ST1[3];
    for (int r = 0; r < 3; ++r) {
      ST0[r] = g.S3[3 * r + 0] * Tm[0] + g.S3[3 * r + 1] * Tm[1] + g.S3[3 * r + 2] * Tm[2];
      ST1[r] = g.S3[3 * r + 0] * Tm[3] + g.S3[3 * r + 1] * Tm[4] + g.S3[3 * r + 2] * Tm[5];
    }
    double dTm[6];
    for (int j = 0; j < 3; ++j) {
      dTm[j] = 2.0 * da * ST0[j] + db * ST1[j];
      dTm[3 + j] = db * ST0[j] + 2.0 * dc * ST1[j];
    }
    // Tm = J W  ->  dJ = dTm W^T, dW = J^T dTm
    double dJ[6], dW[9];
    for (int r = 0; r < 2; ++r)
      for (int k = 0; k < 3; ++k)
        dJ[3 * r + k] = dTm[3 * r + 0] * Wm[3 * k + 0] + dTm[3 * r + 1] * Wm[3 * k + 1] + dTm[3 * r + 2] * Wm[3 * k + 2];
    for (int k = 0; k < 3; ++k)
      for (int c2 = 0; c2 < 3; ++c2) dW[3 * k + c2] = g.J[k] * dTm[c2] + g.J[3 + k] * dTm[3 + c2];
    // J(t): J00 = fx/tz, J02 = -fx tx'/tz^2 (tx' = tx unless clamped, then tx' = L tz)
    dt[2] += dJ[0] * (-cam->fx / (tz * tz)) + dJ[4] * (-cam->fy / (tz * tz));
    if (!g.clamp_x) {
      dt[0] += dJ[2] * (-cam->fx / (tz * tz));
      dt[2] += dJ[2] * (2.0 * cam->fx * tx / (tz * tz * tz));
    } else {
      dt[2] += dJ[2] * (cam->fx * (g.tx_c / tz) / (tz * tz));
    }
    if (!g.clamp_y) {
      dt[1] += dJ[5] * (-cam->fy / (tz * tz));
      dt[2] += dJ[5] * (2.0 * cam->fy * ty / (tz * tz * tz));
    } else {
      dt[2] += dJ[5] * (cam->fy * (g.ty_c / tz) / (tz * tz));
    }
    // Sigma = M M^T, M = R diag(s)
    double dM[9];
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 3; ++k) {
        double acc = 0.0;
        for (int j = 0; j < 3; ++j) acc += (dSig[3 * r + j] + dSig[3 * j + r]) * g.M[3 * j + k];
        dM[3 * r + k] = acc;
      }
    double dR[9], ds[3] = {0, 0, 0};
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 3; ++k) {
        dR[3 * r + k] = dM[3 * r + k] * g.s[k];
        ds[k] += dM[3 * r + k] * g.R[3 * r + k];
      }
    for (int k = 0; k < 3; ++k) gp[3 + k] += ds[k] * g.s[k];
    // R(q) for unit q = (w,x,y,z)
    const double w = g.qn[0], x = g.qn[1], y = g.qn[2], z = g.qn[3];
    double dq[4];
    dq[0] = dR[1] * (-2 * z) + dR[2] * (2 * y) + dR[3] * (2 * z) + dR[5] * (-2 * x) + dR[6] * (-2 * y) + dR[7] * (2 * x);
    dq[1] = dR[1] * (2 * y) + dR[2] * (2 * z) + dR[3] * (2 * y) + dR[4] * (-4 * x) + dR[5] * (-2 * w) +
            dR[6] * (2 * z) + dR[7] * (2 * w) + dR[8] * (-4 * x);
    dq[2] = dR[0] * (-4 * y) + dR[1] * (2 * x) + dR[2] * (2 * w) + dR[3] * (2 * x) + dR[5] * (2 * z) +
            dR[6] * (-2 * w) + dR[7] * (2 * z) + dR[8] * (-4 * y);
    dq[3] = dR[0] * (-4 * z) + dR[1] * (-2 * w) + dR[2] * (2 * x) + dR[3] * (2 * w) + dR[4] * (-4 * z) +
            dR[5] * (2 * y) + dR[6] * (2 * x) + dR[7] * (2 * y);
    double qd = dq[0] * g.qn[0] + dq[1] * g.qn[1] + dq[2] * g.qn[2] + dq[3] * g.qn[3];
    for (int k = 0; k < 4; ++k) gp[6 + k] += (dq[k] - g.qn[k] * qd) / g.qlen;
    // opacity
    gp[10] += d2[5] * g.o * (1.0 - g.o);
    // colour: SH coefficients and viewing direction
    double ddir[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ++ch) {
      if (g.raw[ch] < 0.0) continue;
      const double gc = d2[6 + ch];
      for (int k2 = 0; k2 < D; ++k2) {
        gp[11 + 3 * k2 + ch] += gc * g.Y[k2];
        for (int a2 = 0; a2 < 3; ++a2) ddir[a2] += gc * p[11 + 3 * k2 + ch] * g.Yg[k2][a2];
      }
    }
    double dd = ddir[0] * g.dir[0] + ddir[1] * g.dir[1] + ddir[2] * g.dir[2];
    double dmu_sh[3];
    for (int a2 = 0; a2 < 3; ++a2) dmu_sh[a2] = (ddir[a2] - g.dir[a2] * dd) / g.dist;
    // t = W mu + t_cw
    for (int a2 = 0; a2 < 3; ++a2) {
      gp[a2] += Wm[0 + a2] * dt[0] + Wm[3 + a2] * dt[1] + Wm[6 + a2] * dt[2] + dmu_sh[a2];
    }
    // pose: dt -> v and w x t; W inside Tm -> w; camera centre moves by -W^T v
    pose[0] += dt[0];
    pose[1] += dt[1];
    pose[2] += dt[2];
    pose[3] += ty * dt[2] - tz * dt[1];
    pose[4] += tz * dt[0] - tx * dt[2];
    pose[5] += tx * dt[1] - ty * dt[0];
    // Mrot = W dW^T; dL/dw = (M12 - M21, M20 - M02, M01 - M10)
    double Mr[9];
    for (int r = 0; r < 3; ++r)
      for (int c2 = 0; c2 < 3; ++c2)
        Mr[3 * r + c2] = Wm[3 * r + 0] * dW[3 * c2 + 0] + Wm[3 * r + 1] * dW[3 * c2 + 1] + Wm[3 * r + 2] * dW[3 * c2 + 2];
    pose[3] += Mr[5] - Mr[7];
    pose[4] += Mr[6] - Mr[2];
    pose[5] += Mr[1] - Mr[3];
    // dL/dCam = -dmu_sh, dCam = -W^T v  ->  dL/dv += W dmu_sh
    for (int r = 0; r < 3; ++r) pose[r] += Wm[3 * r + 0] * dmu_sh[0] + Wm[3 * r + 1] * dmu_sh[1] + Wm[3 * r + 2] * dmu_sh[2];
  }
  for (int k = 0; k < 6; ++k) grad_pose[k] += pose[k];
  return 0;
}

}  // extern "C"
