// Stable LSD radix sort passes over u64 keys, templated on where a pass
// reads its keys from (hand-written; no library sort).
//
// A key source is a functor  bool operator()(u64 i, u64* key) const  that
// yields the key of item i, or false when item i holds no key.  KeySrc reads
// a key array; a source that forms keys on the fly lets the first pass of a
// sort read the raw items directly, so that a compaction (items without a
// key dropped, the rest kept in item order) and the first digit's stable
// scatter are one pass.  Every kernel runs on a fixed grid of P blocks over
// contiguous partitions of the items (partition_of), which keeps the sort
// stable.
#pragma once

#include "device_scan.cuh"

namespace dcg {

struct KeySrc {
  const u64* keys;
  __device__ __forceinline__ bool operator()(u64 i, u64* key) const {
    *key = keys[i];
    return true;
  }
};

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

template <class Src>
__global__ void __launch_bounds__(256) k_radix_hist(Src src, const u64* n_ptr, u64 n_host, int shift, int nbits,
                                                    uint32_t* hist) {
  __shared__ uint32_t h[8][256];  // one histogram per warp, summed at the end
  const u64 n = n_ptr ? *n_ptr : n_host;
  u64 beg, end;
  partition_of(n, &beg, &end);
#pragma unroll
  for (int w = 0; w < 8; ++w) h[w][threadIdx.x] = 0;
  __syncthreads();
  const u64 mask = (1ull << nbits) - 1;
  uint32_t* const hw = h[threadIdx.x >> 5];
  for (u64 c0 = beg; c0 < end; c0 += (u64)kHistUnroll * blockDim.x) {
    u64 k[kHistUnroll];
    bool ok[kHistUnroll];
#pragma unroll
    for (int r = 0; r < kHistUnroll; ++r) {
      const u64 i = c0 + (u64)r * blockDim.x + threadIdx.x;
      ok[r] = i < end && src(i, &k[r]);
    }
#pragma unroll
    for (int r = 0; r < kHistUnroll; ++r)
      if (ok[r]) atomicAdd(&hw[(unsigned)((k[r] >> shift) & mask)], 1u);
  }
  __syncthreads();
  uint32_t t = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) t += h[w][threadIdx.x];
  hist[threadIdx.x * gridDim.x + blockIdx.x] = t;
}

// One block per digit: exclusive scan of hist[d][0..P) in place; the digit's
// total goes to totals[d] (sort_scan.cu).
__global__ void k_radix_scan(uint32_t* hist, int P, uint32_t* totals);

// Stable scatter.  The block walks its partition in chunks of 8 warps x 256
// items; warp w owns the chunk's w-th run of 256 consecutive items and ranks
// the keys among them round by round (32 lanes per round) with per-warp
// digit counters, so that the rank order equals the item order.  The chunk's
// keys are then reordered by digit in shared memory and written out as
// contiguous runs per digit (coalesced stores).  The digit bases (exclusive
// scan of the 256 digit totals) are computed by every block; their sum, the
// number of keys, goes to *count_out (block 0) when count_out is given.
constexpr int kSortWarps = 8;
constexpr int kSortRounds = 8;
constexpr int kSortChunk = kSortWarps * 32 * kSortRounds;

template <int NB, class Src>
__global__ void __launch_bounds__(256) k_radix_scatter(Src src, const u64* n_ptr, u64 n_host, u64* out, int shift,
                                                       const uint32_t* hist, const uint32_t* totals,
                                                       u64* count_out) {
  constexpr int nbits = NB;
  __shared__ uint32_t wcnt[kSortWarps][256];
  __shared__ uint32_t run[256];
  __shared__ uint32_t cstart[256];
  __shared__ u64 stage[kSortChunk];
  const u64 n = n_ptr ? *n_ptr : n_host;
  u64 beg, end;
  partition_of(n, &beg, &end);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const u64 mask = (1ull << nbits) - 1;
  {
    uint32_t tot;
    const uint32_t base = block_excl_scan<uint32_t>(totals[tid], &tot);
    run[tid] = base + hist[tid * gridDim.x + blockIdx.x];
    if (count_out && blockIdx.x == 0 && tid == 0) *count_out = tot;
  }
  for (u64 c0 = beg; c0 < end; c0 += kSortChunk) {
#pragma unroll
    for (int k = 0; k < kSortWarps; ++k) wcnt[k][tid] = 0;
    __syncthreads();
    u64 key[kSortRounds];
    uint32_t pos[kSortRounds];
    unsigned dig[kSortRounds];
    bool ok[kSortRounds];
    const unsigned lt = lanemask_lt();
    // all loads of the chunk first (several in flight per thread), then the ranking
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
      const u64 i = c0 + (u64)w * 256 + (u64)r * 32 + lane;
      ok[r] = i < end && src(i, &key[r]);
    }
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
      const bool valid = ok[r];
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
    uint32_t cnt;  // keys in the chunk
    cstart[tid] = block_excl_scan<uint32_t>(acc, &cnt);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
      const unsigned d = dig[r];
      if (d < 256u) stage[cstart[d] + wcnt[w][d] + pos[r]] = key[r];
    }
    __syncthreads();
    for (int p = tid; p < (int)cnt; p += 256) {
      const u64 k = stage[p];
      const unsigned d = (unsigned)((k >> shift) & mask);
      out[run[d] + (uint32_t)p - cstart[d]] = k;
    }
    __syncthreads();
    run[tid] += acc;
    __syncthreads();
  }
}

// One pass on digit [shift, shift + nb), nb <= 8: histogram, scan, stable
// scatter of the keys of src (items [0, *n_ptr), or [0, n_host) when n_ptr is
// null) into dst.  `hist` holds 256 * (P + 1) entries; the number of keys
// goes to *count_out when given.
template <class Src>
void radix_pass(Src src, const u64* n_ptr, u64 n_host, u64* dst, int shift, int nb, uint32_t* hist, int P,
                u64* count_out, cudaStream_t s) {
  uint32_t* totals = hist + 256 * (size_t)P;
  k_radix_hist<Src><<<P, 256, 0, s>>>(src, n_ptr, n_host, shift, nb, hist);
  k_radix_scan<<<256, 256, 0, s>>>(hist, P, totals);
  switch (nb) {  // the digit width as a compile-time constant (unrolled ranking)
#define DCG_SCATTER(B)                                                                                      \
  case B:                                                                                                   \
    k_radix_scatter<B, Src><<<P, 256, 0, s>>>(src, n_ptr, n_host, dst, shift, hist, totals, count_out);   \
    break;
    DCG_SCATTER(1)
    DCG_SCATTER(2)
    DCG_SCATTER(3)
    DCG_SCATTER(4)
    DCG_SCATTER(5)
    DCG_SCATTER(6)
    DCG_SCATTER(7)
    default:
      k_radix_scatter<8, Src><<<P, 256, 0, s>>>(src, n_ptr, n_host, dst, shift, hist, totals, count_out);
      break;
#undef DCG_SCATTER
  }
}

}  // namespace dcg
