// Chunk kernels: Eq. 5 / Eq. 6 ids, frustum cull of chunk cubes, visible-list
// compaction, and page gather/scatter between the device page pool and the
// active buffer (Sec. III-D, III-E).
#include "kernels.cuh"
#include "device_scan.cuh"

namespace dcg {

unsigned long long g_launches = 0;

// ----------------------------------------------------------------------------
// Eq. 5 / Eq. 6 in FP32: c = floor((p + s/2) / s) with one rounding per
// operation (no contraction), key = (cx+2^20)<<42 | (cy+2^20)<<21 | (cz+2^20).
__device__ __forceinline__ bool chunk_coord(float p, float s, int* c) {
  const float q = __fdiv_rn(__fadd_rn(p, 0.5f * s), s);
  const float f = floorf(q);
  const bool ok = (f >= -1048576.0f) && (f <= 1048575.0f);  // false for NaN
  *c = ok ? (int)f : 0;
  return ok;
}

__device__ __forceinline__ u64 encode_id(int cx, int cy, int cz) {
  return ((u64)(unsigned)(cx + (1 << 20)) << 42) | ((u64)(unsigned)(cy + (1 << 20)) << 21) |
         (u64)(unsigned)(cz + (1 << 20));
}

// means: component m of Gaussian i at means[i * row + m * col]
__global__ void k_chunk_keys(const float* __restrict__ means, long long row, long long col, long long n, float s,
                             u64* __restrict__ keys, unsigned* errword) {
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int c[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) ok &= chunk_coord(means[i * row + a * col], s, &c[a]);
    keys[i] = ok ? encode_id(c[0], c[1], c[2]) : 0ull;
    bad |= !ok;
  }
  if (__any_sync(0xffffffffu, bad) && lane_id() == 0) atomicOr(errword, ERRW_KEY_RANGE_BIT);
}

void launch_chunk_keys(const float* means, long long row, long long col, long long n, float s, u64* keys,
                       unsigned* errword, int num_sms, cudaStream_t st) {
  if (n <= 0) return;
  long long blocks = (n + 255) / 256;
  int g = (int)(blocks < (long long)num_sms * 8 ? blocks : (long long)num_sms * 8);
  k_chunk_keys<<<g, 256, 0, st>>>(means, row, col, n, s, keys, errword);
  count_launch();
}

// ----------------------------------------------------------------------------
// Frustum cull in FP64 with a fixed evaluation order (every product rounded,
// sums left to right): planes from VP = P * Tcw (Gribb-Hartmann), p-vertex
// test per plane, then squared distance from the camera centre to the cube.
__device__ void cull_planes(const dcg_camera& cam, double pl[6][4], double C[3]) {
  const double W = (double)cam.W, H = (double)cam.H, zn = (double)cam.znear, zf = (double)cam.zfar;
  const double fx = cam.fx, fy = cam.fy, cx = cam.cx, cy = cam.cy;
  double P[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) P[k] = 0.0;
  P[0] = __ddiv_rn(__dmul_rn(2.0, fx), W);
  P[2] = __ddiv_rn(__dsub_rn(__dmul_rn(2.0, cx), W), W);
  P[5] = __ddiv_rn(__dmul_rn(2.0, fy), H);
  P[6] = __ddiv_rn(__dsub_rn(__dmul_rn(2.0, cy), H), H);
  P[10] = __ddiv_rn(__dadd_rn(zf, zn), __dsub_rn(zf, zn));
  P[11] = __ddiv_rn(__dmul_rn(__dmul_rn(-2.0, zf), zn), __dsub_rn(zf, zn));
  P[14] = 1.0;
  double T[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) T[k] = (double)cam.Tcw[k];
  double VP[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 4; ++k) acc = __dadd_rn(acc, __dmul_rn(P[4 * i + k], T[4 * k + j]));
      VP[4 * i + j] = acc;
    }
  for (int j = 0; j < 4; ++j) {
    pl[0][j] = __dadd_rn(VP[12 + j], VP[0 + j]);
    pl[1][j] = __dsub_rn(VP[12 + j], VP[0 + j]);
    pl[2][j] = __dadd_rn(VP[12 + j], VP[4 + j]);
    pl[3][j] = __dsub_rn(VP[12 + j], VP[4 + j]);
    pl[4][j] = __dadd_rn(VP[12 + j], VP[8 + j]);
    pl[5][j] = __dsub_rn(VP[12 + j], VP[8 + j]);
  }
  for (int j = 0; j < 3; ++j) {
    double acc = __dmul_rn(T[0 + j], T[3]);
    acc = __dadd_rn(acc, __dmul_rn(T[4 + j], T[7]));
    acc = __dadd_rn(acc, __dmul_rn(T[8 + j], T[11]));
    C[j] = -acc;
  }
}

__device__ bool cull_box(const double pl[6][4], const double C[3], double dfar, const double lo[3],
                         const double hi[3]) {
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const double vx = pl[p][0] >= 0.0 ? hi[0] : lo[0];
    const double vy = pl[p][1] >= 0.0 ? hi[1] : lo[1];
    const double vz = pl[p][2] >= 0.0 ? hi[2] : lo[2];
    double val = __dadd_rn(__dmul_rn(pl[p][0], vx), __dmul_rn(pl[p][1], vy));
    val = __dadd_rn(val, __dmul_rn(pl[p][2], vz));
    val = __dadd_rn(val, pl[p][3]);
    if (val < 0.0) return false;
  }
  double d2 = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double e = 0.0;
    if (C[a] < lo[a]) e = __dsub_rn(lo[a], C[a]);
    else if (C[a] > hi[a]) e = __dsub_rn(C[a], hi[a]);
    d2 = __dadd_rn(d2, __dmul_rn(e, e));
  }
  return d2 <= __dmul_rn(dfar, dfar);
}

// One block row of the cull: view v = blockIdx.y against chunks strided over
// blockIdx.x; mask [V][C] (may be null), vis [C] OR-union.
__device__ __forceinline__ void cull_view(const dcg_camera& cam, const int32_t* __restrict__ coords, int C, float s,
                                          float dfar, uint8_t* __restrict__ mask, uint8_t* __restrict__ vis) {
  __shared__ double pl[6][4];
  __shared__ double Cc[3];
  const int v = blockIdx.y;
  if (threadIdx.x == 0) cull_planes(cam, pl, Cc);
  __syncthreads();
  const double sd = (double)s;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < C; k += gridDim.x * blockDim.x) {
    double lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double cs = __dmul_rn((double)coords[3 * k + a], sd);
      lo[a] = __dsub_rn(cs, __dmul_rn(0.5, sd));
      hi[a] = __dadd_rn(cs, __dmul_rn(0.5, sd));
    }
    const bool ok = cull_box(pl, Cc, (double)dfar, lo, hi);
    if (mask) mask[(long long)v * C + k] = ok ? 1 : 0;
    if (ok) vis[k] = 1;
  }
}

// cameras in device memory
__global__ void k_cull(const int32_t* __restrict__ coords, int C, const dcg_camera* __restrict__ cams, float s,
                       float dfar, uint8_t* __restrict__ mask, uint8_t* __restrict__ vis) {
  cull_view(cams[blockIdx.y], coords, C, s, dfar, mask, vis);
}

// cameras passed by value in the kernel's parameters
__global__ void k_cull_tab(const int32_t* __restrict__ coords, int C, const CullCams cams, float s, float dfar,
                           uint8_t* __restrict__ mask, uint8_t* __restrict__ vis) {
  cull_view(cams.c[blockIdx.y], coords, C, s, dfar, mask, vis);
}

// Single block: ordered compaction of vis[0..C) into list, count into *n.
__global__ void k_compact_list(const uint8_t* __restrict__ vis, int C, int32_t* __restrict__ list, int32_t* n) {
  int base = 0;
  for (int c0 = 0; c0 < C; c0 += blockDim.x) {
    const int k = c0 + threadIdx.x;
    const int f = (k < C && vis[k]) ? 1 : 0;
    int tot;
    const int off = block_excl_scan<int>(f, &tot);
    if (f) list[base + off] = k;
    base += tot;
  }
  if (threadIdx.x == 0) *n = base;
}

cudaError_t launch_cull(const int32_t* coords, int C, const dcg_camera* cams, const CullCams* tab, int V, float s,
                        float dfar, uint8_t* mask, uint8_t* vis, int32_t* list, int32_t* n, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(vis, 0, (size_t)(C > 0 ? C : 1), st);
  if (e != cudaSuccess) return e;
  if (C > 0) {
    dim3 grid((C + 255) / 256, V);
    if (tab)
      k_cull_tab<<<grid, 256, 0, st>>>(coords, C, *tab, s, dfar, mask, vis);
    else
      k_cull<<<grid, 256, 0, st>>>(coords, C, cams, s, dfar, mask, vis);
  }
  k_compact_list<<<1, 1024, 0, st>>>(vis, C, list, n);
  count_launch(C > 0 ? 2 : 1);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Page copies.  A page holds page_g Gaussians component-major with Fp
// components: component c of slot j at page[c * page_g + j].
// desc[3d .. 3d+2] = (page index, count, offset in the active buffer).
// Components [c0, c0 + nc) of each page map to rows 0 .. nc-1 of `active`.
// cnt floats from s to t, coalesced, four loads in flight per thread
__device__ __forceinline__ void copy_run(const float* __restrict__ s, float* __restrict__ t, long long cnt) {
  const long long B = blockDim.x;
  long long j = threadIdx.x;
  for (; j + 3 * B < cnt; j += 4 * B) {
    const float a0 = s[j], a1 = s[j + B], a2 = s[j + 2 * B], a3 = s[j + 3 * B];
    t[j] = a0;
    t[j + B] = a1;
    t[j + 2 * B] = a2;
    t[j + 3 * B] = a3;
  }
  for (; j < cnt; j += B) t[j] = s[j];
}

__global__ void k_gather_pages(const float* __restrict__ pool, long long page_g, int Fp, int c0, int nc,
                               const long long* __restrict__ desc, float* __restrict__ active, long long stride) {
  const long long d = blockIdx.x;
  const long long page = desc[3 * d], cnt = desc[3 * d + 1], off = desc[3 * d + 2];
  const float* src = pool + page * page_g * Fp + (long long)c0 * page_g;
  for (int c = blockIdx.y; c < nc; c += gridDim.y)
    copy_run(src + (long long)c * page_g, active + (long long)c * stride + off, cnt);
}

__global__ void k_scatter_pages(float* __restrict__ pool, long long page_g, int Fp, int c0, int nc,
                                const long long* __restrict__ desc, const float* __restrict__ active,
                                long long stride) {
  const long long d = blockIdx.x;
  const long long page = desc[3 * d], cnt = desc[3 * d + 1], off = desc[3 * d + 2];
  float* dst = pool + page * page_g * Fp + (long long)c0 * page_g;
  for (int c = blockIdx.y; c < nc; c += gridDim.y)
    copy_run(active + (long long)c * stride + off, dst + (long long)c * page_g, cnt);
}

// Load verification: checksum of a chunk's pages, the sum over its used
// words w of w * (2 i + 1) mod 2^64, i the word's index in the chunk's page
// sequence ((page * Fp + component) * page_g + row).  One launch per page:
// `page` is page number p of the chunk, holding `cnt` rows; the sum is added
// to *out (order-independent, so the result is deterministic).
__global__ void k_page_checksum(const float* __restrict__ page, long long p, long long page_g, int Fp, long long cnt,
                                unsigned long long* __restrict__ out) {
  const unsigned* src = reinterpret_cast<const unsigned*>(page);
  unsigned long long acc = 0ull;
  for (int c = blockIdx.y; c < Fp; c += gridDim.y) {
    const unsigned long long base = ((unsigned long long)p * Fp + c) * (unsigned long long)page_g;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < cnt; j += (long long)gridDim.x * blockDim.x)
      acc += (unsigned long long)src[(long long)c * page_g + j] * (2ull * (base + (unsigned long long)j) + 1ull);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

void launch_page_checksum(const float* page, long long p, long long page_g, int Fp, long long cnt,
                          unsigned long long* out, cudaStream_t st) {
  if (cnt <= 0) return;
  const long long bx = (cnt + 255) / 256;
  dim3 grid((unsigned)(bx < 8 ? bx : 8), Fp < 32 ? Fp : 32);
  k_page_checksum<<<grid, 256, 0, st>>>(page, p, page_g, Fp, cnt, out);
  count_launch();
}

// Chunk index and row within the chunk of every active row: the last
// gathered chunk whose first active row is at or before it (off ascending).
__global__ void k_active_map(const long long* __restrict__ off, const int32_t* __restrict__ chunk, int nl, long long n,
                             int32_t* __restrict__ chunk_out, int32_t* __restrict__ row_out) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= j) lo = mid; else hi = mid - 1;
    }
    if (chunk_out) chunk_out[j] = chunk[lo];
    if (row_out) row_out[j] = (int32_t)(j - off[lo]);
  }
}

void launch_active_map(const long long* off, const int32_t* chunk, int nl, long long n, int32_t* chunk_out,
                       int32_t* row_out, int num_sms, cudaStream_t st) {
  if (n <= 0 || nl <= 0) return;
  const long long blocks = (n + 255) / 256;
  k_active_map<<<(int)(blocks < num_sms * 8ll ? blocks : num_sms * 8ll), 256, 0, st>>>(off, chunk, nl, n, chunk_out,
                                                                                     row_out);
  count_launch();
}

void launch_page_copy(bool gather, float* pool, long long page_g, int Fp, int c0, int nc, const long long* desc, int nd,
                      float* active, long long stride, cudaStream_t st) {
  if (nd <= 0 || nc <= 0) return;
  dim3 grid(nd, nc < 16 ? nc : 16);
  if (gather)
    k_gather_pages<<<grid, 256, 0, st>>>(pool, page_g, Fp, c0, nc, desc, active, stride);
  else
    k_scatter_pages<<<grid, 256, 0, st>>>(pool, page_g, Fp, c0, nc, desc, active, stride);
  count_launch();
}

// Planar source rows [src_off, src_off + cnt) of component c -> page slots.
__global__ void k_rows_to_page(const float* __restrict__ src, long long stride, long long src_off, long long cnt,
                               int F, float* __restrict__ page, long long page_g) {
  for (int c = blockIdx.y; c < F; c += gridDim.y)
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < cnt; j += (long long)gridDim.x * blockDim.x)
      page[(long long)c * page_g + j] = src[(long long)c * stride + src_off + j];
}

}  // namespace dcg
