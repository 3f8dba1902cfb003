// Loop-closure correction of the gathered chunks (Sec. III-F "Cross-Chunk
// Transformation"): each Gaussian of a chunk that an affected keyframe's
// frustum cull keeps, and whose centre projects into that keyframe's image
// (pose before the correction), moves rigidly with the keyframe,
//   x' = R_k x + t_k,   q' = q_k (x) q   (Hamilton product),
// where (R_k, t_k) is the keyframe's correction and q_k its rotation as a unit
// quaternion.  A Gaussian seen by several keyframes moves with the first of
// them only (the global transformation mask).  The camera transform, the
// projection and the corrected position are evaluated in FP32 with one
// rounding per operation in a fixed order, so that the visibility decision
// and the chunk ids recomputed from the result (Eq. 5/6) are reproducible.
#include <algorithm>

#include "device_scan.cuh"
#include "kernels.cuh"

namespace dcg {

__device__ __forceinline__ float dot3_rn(const float* r, float x, float y, float z, float t) {
  return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r[0], x), __fmul_rn(r[1], y)), __fmul_rn(r[2], z)), t);
}

// skip_done: flags[i] != 0 on entry marks a Gaussian that an earlier keyframe
// has already moved (the global transformation mask carried across loads of
// the keyframe-by-keyframe order); it is left alone and its flag cleared.
__global__ void k_loop_transform(float* __restrict__ act, long long stride, long long n,
                                 const long long* __restrict__ seg_off, const int* __restrict__ seg_chunk, int nseg,
                                 const uint8_t* __restrict__ mask, int C, const LcView* __restrict__ kf, int K,
                                 uint32_t* __restrict__ flags, int skip_done) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (skip_done && flags[i] != 0u) {
      flags[i] = 0u;
      continue;
    }
    // chunk of active Gaussian i: the last segment starting at or before i
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (seg_off[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    const int c = seg_chunk[lo];
    const float x = act[0 * stride + i], y = act[1 * stride + i], z = act[2 * stride + i];
    uint32_t f = 0;
    for (int k = 0; k < K; ++k) {
      if (!mask[(long long)k * C + c]) continue;
      const LcView& v = kf[k];
      const float tx = dot3_rn(v.R + 0, x, y, z, v.t[0]);
      const float ty = dot3_rn(v.R + 3, x, y, z, v.t[1]);
      const float tz = dot3_rn(v.R + 6, x, y, z, v.t[2]);
      if (!(tz > v.znear && tz <= v.zfar)) continue;
      const float u = __fadd_rn(__fmul_rn(v.fx, __fdiv_rn(tx, tz)), v.cx);
      const float w = __fadd_rn(__fmul_rn(v.fy, __fdiv_rn(ty, tz)), v.cy);
      if (!(u >= 0.f && u < (float)v.W && w >= 0.f && w < (float)v.H)) continue;
      act[0 * stride + i] = dot3_rn(v.C + 0, x, y, z, v.C[3]);
      act[1 * stride + i] = dot3_rn(v.C + 4, x, y, z, v.C[7]);
      act[2 * stride + i] = dot3_rn(v.C + 8, x, y, z, v.C[11]);
      const float a0 = v.q[0], a1 = v.q[1], a2 = v.q[2], a3 = v.q[3];
      const float b0 = act[6 * stride + i], b1 = act[7 * stride + i], b2 = act[8 * stride + i], b3 = act[9 * stride + i];
      act[6 * stride + i] = a0 * b0 - a1 * b1 - a2 * b2 - a3 * b3;
      act[7 * stride + i] = a0 * b1 + a1 * b0 + a2 * b3 - a3 * b2;
      act[8 * stride + i] = a0 * b2 - a1 * b3 + a2 * b0 + a3 * b1;
      act[9 * stride + i] = a0 * b3 + a1 * b2 - a2 * b1 + a3 * b0;
      f = (uint32_t)k + 1u;
      break;
    }
    flags[i] = f;
  }
}

// dst[c][j] = src[c][perm[j]] for c < rows, j < n (planar rows).
__global__ void k_permute_rows(const float* __restrict__ src, long long sstride, float* __restrict__ dst,
                               long long dstride, const long long* __restrict__ perm, long long n, int rows) {
  for (int c = blockIdx.y; c < rows; c += gridDim.y)
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
      dst[(long long)c * dstride + j] = src[(long long)c * sstride + perm[j]];
}

// Opacity reset of Sec. III-F: logit <- min(logit, cap) for rows [0, n).
__global__ void k_cap_rows(float* __restrict__ row, long long n, float cap) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
    row[j] = fminf(row[j], cap);
}

// Redistribution on the device.  The gathered rows form nseg segments (chunk
// k owns rows [seg_off[k], seg_off[k + 1])); a row moves if its recomputed
// chunk id differs from its segment's.  k_lc_moved turns the transformed
// flag of each row into its moved flag and counts the transformed rows;
// the moved rows (ascending) are then compacted by the ordered scan.  A row
// the call did not transform keeps its position and therefore its chunk.
__device__ __forceinline__ int lc_seg_of(const long long* __restrict__ seg_off, int nseg, long long i) {
  int lo = 0, hi = nseg - 1;  // last k with seg_off[k] <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (seg_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_lc_moved(uint32_t* __restrict__ flags, const u64* __restrict__ keys, long long n,
                           const long long* __restrict__ seg_off, const u64* __restrict__ seg_key, int nseg,
                           unsigned long long* n_transformed) {
  unsigned long long cnt = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    // only a Gaussian transformed by this call can have left its chunk
    const bool t = flags[i] != 0u;
    cnt += t;
    flags[i] = t && keys[i] != seg_key[lc_seg_of(seg_off, nseg, i)] ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(n_transformed, cnt);
}

struct LcMovedCount {
  const uint32_t* f;
  __device__ u64 operator()(u64 i) const { return f[i]; }
};
struct LcMovedEmit {
  long long* idx;
  u64* key_out;
  const u64* keys;
  __device__ void operator()(u64 i, u64 off, u64) const {
    idx[off] = (long long)i;
    key_out[off] = keys[i];
  }
};

// Destination of every row in the redistributed order: a moved row is the
// j-th moved row, j = the number of moved rows before it, and goes to
// mdest[j]; a staying row of segment k keeps its rank among the segment's
// stays: dest = i - (moved rows before i) + seg_base[k].  perm[dest] = i.
__global__ void k_lc_dest(const uint32_t* __restrict__ moved, long long n, const long long* __restrict__ seg_off,
                          const long long* __restrict__ seg_base, int nseg, const long long* __restrict__ midx,
                          const long long* __restrict__ mdest, long long nm, long long* __restrict__ perm) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    long long lo = 0, hi = nm;  // moved rows with index < i
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (midx[mid] < i) lo = mid + 1; else hi = mid;
    }
    const long long d = moved[i] ? mdest[lo] : i - lo + seg_base[lc_seg_of(seg_off, nseg, i)];
    perm[d] = i;
  }
}

void launch_lc_moved(uint32_t* flags, const u64* keys, long long n, const long long* seg_off, const u64* seg_key,
                     int nseg, unsigned long long* n_transformed, long long* midx, u64* mkey, u64* part, int P,
                     u64* n_moved, int num_sms, cudaStream_t st) {
  if (n <= 0) return;
  const long long blocks = (n + 255) / 256;
  k_lc_moved<<<(int)std::min<long long>(blocks, (long long)num_sms * 8), 256, 0, st>>>(flags, keys, n, seg_off,
                                                                                     seg_key, nseg, n_transformed);
  part_scan_emit(nullptr, (u64)n, LcMovedCount{flags}, LcMovedEmit{midx, mkey, keys}, part, P, n_moved, st);
  count_launch(4);
}

void launch_lc_dest(const uint32_t* moved, long long n, const long long* seg_off, const long long* seg_base, int nseg,
                    const long long* midx, const long long* mdest, long long nm, long long* perm, int num_sms,
                    cudaStream_t st) {
  if (n <= 0) return;
  const long long blocks = (n + 255) / 256;
  k_lc_dest<<<(int)std::min<long long>(blocks, (long long)num_sms * 8), 256, 0, st>>>(moved, n, seg_off, seg_base,
                                                                                    nseg, midx, mdest, nm, perm);
  count_launch();
}

void launch_loop_transform(float* act, long long stride, long long n, const long long* seg_off, const int* seg_chunk,
                           int nseg, const uint8_t* mask, int C, const LcView* kf, int K, uint32_t* flags, int skip_done,
                           int num_sms, cudaStream_t st) {
  if (n <= 0) return;
  const long long blocks = (n + 255) / 256;
  k_loop_transform<<<(int)std::min<long long>(blocks, (long long)num_sms * 8), 256, 0, st>>>(
      act, stride, n, seg_off, seg_chunk, nseg, mask, C, kf, K, flags, skip_done);
  count_launch();
}

void launch_permute_rows(const float* src, long long sstride, float* dst, long long dstride, const long long* perm,
                         long long n, int rows, int num_sms, cudaStream_t st) {
  if (n <= 0 || rows <= 0) return;
  const long long blocks = (n + 255) / 256;
  dim3 grid((unsigned)std::min<long long>(blocks, (long long)num_sms * 4), (unsigned)std::min(rows, 16));
  k_permute_rows<<<grid, 256, 0, st>>>(src, sstride, dst, dstride, perm, n, rows);
  count_launch();
}

void launch_cap_rows(float* row, long long n, float cap, int num_sms, cudaStream_t st) {
  if (n <= 0) return;
  const long long blocks = (n + 255) / 256;
  k_cap_rows<<<(int)std::min<long long>(blocks, (long long)num_sms * 8), 256, 0, st>>>(row, n, cap);
  count_launch();
}

}  // namespace dcg
