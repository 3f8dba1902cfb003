// Device scan top level and the stable LSD radix sort (hand-written; no library sort).
#include "device_scan.cuh"

namespace dcg {

__global__ void k_part_scan(u64* part, int P, u64* total_out) {
  // one block of 1024 threads; each thread scans a contiguous run of part[]
  const int T = blockDim.x;
  const int per = (P + T - 1) / T;
  const int b = threadIdx.x * per;
  const int e = min(P, b + per);
  u64 s = 0;
  for (int i = b; i < e; ++i) s += part[i];
  u64 tot;
  u64 ex = block_excl_scan<u64>(s, &tot);
  for (int i = b; i < e; ++i) {
    u64 v = part[i];
    part[i] = ex;
    ex += v;
  }
  if (threadIdx.x == 0) {
    part[P] = tot;
    if (total_out) *total_out = tot;
  }
}

// Peer mask of a lane's digit within the warp, from one ballot per digit bit
// (stable ranking without match_any); lanes with !valid never match a valid lane.
template <int NB>
__device__ __forceinline__ unsigned digit_peers(unsigned d, bool valid) {
  const unsigned vb = __ballot_sync(0xffffffffu, valid);
  unsigned peers = valid ? vb : ~vb;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const bool bit = (d >> b) & 1u;
    const unsigned bb = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? bb : ~bb;
  }
  return peers;
}

// Per-block digit histogram of the block's partition.  Each thread loads
// kHistUnroll keys (strided by the block size) before counting them, so that
// several loads are in flight per thread; counts go to one shared-memory
// histogram per warp (native shared atomics; the order of equal digits does
// not matter for a count), summed at the end.
constexpr int kHistUnroll = 4;

__global__ void __launch_bounds__(256) k_radix_hist(const u64* keys, const u64* n_ptr, int shift, int nbits,
                                                    uint32_t* hist) {
  __shared__ uint32_t h[8][256];  // one histogram per warp, summed at the end
  const u64 n = *n_ptr;
  u64 beg, end;
  partition_of(n, &beg, &end);
#pragma unroll
  for (int w = 0; w < 8; ++w) h[w][threadIdx.x] = 0;
  __syncthreads();
  const u64 mask = (1ull << nbits) - 1;
  uint32_t* const hw = h[threadIdx.x >> 5];
  for (u64 c0 = beg; c0 < end; c0 += (u64)kHistUnroll * blockDim.x) {
    u64 k[kHistUnroll];
#pragma unroll
    for (int r = 0; r < kHistUnroll; ++r) {
      const u64 i = c0 + (u64)r * blockDim.x + threadIdx.x;
      k[r] = i < end ? keys[i] : 0ull;
    }
#pragma unroll
    for (int r = 0; r < kHistUnroll; ++r) {
      const u64 i = c0 + (u64)r * blockDim.x + threadIdx.x;
      if (i < end) atomicAdd(&hw[(unsigned)((k[r] >> shift) & mask)], 1u);
    }
  }
  __syncthreads();
  uint32_t t = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) t += h[w][threadIdx.x];
  hist[threadIdx.x * gridDim.x + blockIdx.x] = t;
}

// One block per digit: exclusive scan of hist[d][0..P) in place; the digit's
// total goes to totals[d].
__global__ void k_radix_scan(uint32_t* hist, int P, uint32_t* totals) {
  uint32_t* row = hist + (size_t)blockIdx.x * P;
  uint32_t carry = 0;
  for (int b0 = 0; b0 < P; b0 += blockDim.x) {
    const int b = b0 + threadIdx.x;
    const uint32_t v = b < P ? row[b] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan<uint32_t>(v, &tot);
    if (b < P) row[b] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// Stable scatter.  The block walks its partition in chunks of 8 warps x 256
// items; warp w owns the chunk's w-th run of 256 consecutive items and ranks
// them round by round (32 lanes per round) with per-warp digit counters, so
// that the rank order equals the input order.  The chunk is then reordered by
// digit in shared memory and written out as contiguous runs per digit
// (coalesced stores).  The digit bases (exclusive scan of the 256 digit
// totals) are computed by every block.
constexpr int kSortWarps = 8;
constexpr int kSortRounds = 8;
constexpr int kSortChunk = kSortWarps * 32 * kSortRounds;

template <int NB>
__global__ void __launch_bounds__(256) k_radix_scatter(const u64* in, u64* out, const u64* n_ptr, int shift,
                                                       const uint32_t* hist, const uint32_t* totals) {
  constexpr int nbits = NB;
  __shared__ uint32_t wcnt[kSortWarps][256];
  __shared__ uint32_t run[256];
  __shared__ uint32_t cstart[256];
  __shared__ u64 stage[kSortChunk];
  const u64 n = *n_ptr;
  u64 beg, end;
  partition_of(n, &beg, &end);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const u64 mask = (1ull << nbits) - 1;
  {
    uint32_t tot;
    const uint32_t base = block_excl_scan<uint32_t>(totals[tid], &tot);
    run[tid] = base + hist[tid * gridDim.x + blockIdx.x];
  }
  for (u64 c0 = beg; c0 < end; c0 += kSortChunk) {
#pragma unroll
    for (int k = 0; k < kSortWarps; ++k) wcnt[k][tid] = 0;
    __syncthreads();
    u64 key[kSortRounds];
    uint32_t pos[kSortRounds];
    unsigned dig[kSortRounds];
    const unsigned lt = lanemask_lt();
    // all loads of the chunk first (several in flight per thread), then the ranking
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
      const u64 i = c0 + (u64)w * 256 + (u64)r * 32 + lane;
      key[r] = i < end ? in[i] : 0ull;
    }
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
      const u64 i = c0 + (u64)w * 256 + (u64)r * 32 + lane;
      const bool valid = i < end;
      const unsigned d = valid ? (unsigned)((key[r] >> shift) & mask) : 0u;
      dig[r] = valid ? d : 256u;
      const unsigned peers = digit_peers<NB>(d, valid);
      const unsigned rank = __popc(peers & lt);
      const unsigned base = valid ? wcnt[w][d] : 0u;
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = base + __popc(peers);
      __syncwarp();
      pos[r] = base + rank;
    }
    __syncthreads();
    // exclusive scan across warps for digit `tid`, then over digits for the chunk
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kSortWarps; ++k) {
      const uint32_t t = wcnt[k][tid];
      wcnt[k][tid] = acc;
      acc += t;
    }
    {
      uint32_t tot;
      cstart[tid] = block_excl_scan<uint32_t>(acc, &tot);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
      const unsigned d = dig[r];
      if (d < 256u) stage[cstart[d] + wcnt[w][d] + pos[r]] = key[r];
    }
    __syncthreads();
    const int cnt = (int)min((u64)kSortChunk, end - c0);
    for (int p = tid; p < cnt; p += 256) {
      const u64 k = stage[p];
      const unsigned d = (unsigned)((k >> shift) & mask);
      out[run[d] + (uint32_t)p - cstart[d]] = k;
    }
    __syncthreads();
    run[tid] += acc;
    __syncthreads();
  }
}

u64* radix_sort(u64* a, u64* b, const u64* n_ptr, int lo, int hi, uint32_t* hist, int P, cudaStream_t s) {
  u64* src = a;
  u64* dst = b;
  uint32_t* totals = hist + 256 * (size_t)P;
  for (int sh = lo; sh < hi; sh += 8) {
    const int nb = min(8, hi - sh);
    k_radix_hist<<<P, 256, 0, s>>>(src, n_ptr, sh, nb, hist);
    k_radix_scan<<<256, 256, 0, s>>>(hist, P, totals);
    switch (nb) {  // the digit width as a compile-time constant (unrolled ranking)
      case 1: k_radix_scatter<1><<<P, 256, 0, s>>>(src, dst, n_ptr, sh, hist, totals); break;
      case 2: k_radix_scatter<2><<<P, 256, 0, s>>>(src, dst, n_ptr, sh, hist, totals); break;
      case 3: k_radix_scatter<3><<<P, 256, 0, s>>>(src, dst, n_ptr, sh, hist, totals); break;
      case 4: k_radix_scatter<4><<<P, 256, 0, s>>>(src, dst, n_ptr, sh, hist, totals); break;
      case 5: k_radix_scatter<5><<<P, 256, 0, s>>>(src, dst, n_ptr, sh, hist, totals); break;
      case 6: k_radix_scatter<6><<<P, 256, 0, s>>>(src, dst, n_ptr, sh, hist, totals); break;
      case 7: k_radix_scatter<7><<<P, 256, 0, s>>>(src, dst, n_ptr, sh, hist, totals); break;
      default: k_radix_scatter<8><<<P, 256, 0, s>>>(src, dst, n_ptr, sh, hist, totals); break;
    }
    u64* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

}  // namespace dcg
