// Partitioned device scan and LSD radix sort whose item counts are read from
// device memory, so that a whole render call can be captured in a CUDA graph.
//
// Every kernel here runs on a fixed grid of P blocks; block b owns the
// contiguous partition [b*len, min(n, (b+1)*len)) with len = ceil(n/P) and
// walks it in order, which makes the scan ordered and the sort stable.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace dcg {

typedef unsigned long long u64;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Asynchronous global -> shared copies (no registers hold the data in
// flight); a thread's copies complete in commit-group order.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void partition_of(u64 n, u64* beg, u64* end) {
  const u64 P = gridDim.x;
  const u64 len = (n + P - 1) / P;
  u64 b = (u64)blockIdx.x * len;
  u64 e = b + len;
  *beg = b < n ? b : n;
  *end = e < n ? e : n;
}

// Inclusive warp scan.
template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, o);
    if ((int)lane_id() >= o) v += t;
  }
  return v;
}

// Exclusive block scan of one value per thread (blockDim.x <= 1024, multiple of 32).
// Returns the exclusive prefix and writes the block total to *total.
template <class T>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
  __shared__ T warp_sums[32];
  __shared__ T total_s;
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane_id() == 31) warp_sums[w] = inc;
  __syncthreads();
  if (w == 0) {
    T s = (int)lane_id() < nw ? warp_sums[lane_id()] : T(0);
    T si = warp_incl_scan(s);
    if ((int)lane_id() < nw) warp_sums[lane_id()] = si - s;
    if (lane_id() == 31) total_s = si;  // lanes >= nw add 0: lane 31 holds the total
  }
  __syncthreads();
  T ex = warp_sums[w] + inc - v;
  *total = total_s;
  __syncthreads();
  return ex;
}

// ----------------------------------------------------------------------------
// Ordered partitioned scan with a fused consumer.
//   CountF: u64 operator()(u64 i) const   -- items item i produces
//   EmitF : void operator()(u64 i, u64 offset, u64 count) const
// part[0..P) partial sums, part[P] total.
// Items per thread per step of the partition walks (several loads in flight).
constexpr int kScanItems = 4;

template <class CountF>
__global__ void k_part_reduce(const u64* n_ptr, u64 n_host, CountF f, u64* part) {
  const u64 n = n_ptr ? *n_ptr : n_host;
  u64 beg, end;
  partition_of(n, &beg, &end);
  u64 acc = 0;
  for (u64 c0 = beg; c0 < end; c0 += (u64)kScanItems * blockDim.x) {
    u64 v[kScanItems];
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
      const u64 i = c0 + (u64)r * blockDim.x + threadIdx.x;
      v[r] = i < end ? f(i) : 0;
    }
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) acc += v[r];
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

// Single block: exclusive scan of part[0..P) in place, total to part[P] and *total_out.
__global__ void k_part_scan(u64* part, int P, u64* total_out);

// Emission in item order: each step covers kScanItems * blockDim items, thread
// t the consecutive items [c0 + kScanItems t, c0 + kScanItems (t + 1)).
template <class CountF, class EmitF>
__global__ void k_part_emit(const u64* n_ptr, u64 n_host, CountF f, EmitF e, const u64* part) {
  const u64 n = n_ptr ? *n_ptr : n_host;
  u64 beg, end;
  partition_of(n, &beg, &end);
  u64 base = part[blockIdx.x];
  for (u64 c0 = beg; c0 < end; c0 += (u64)kScanItems * blockDim.x) {
    const u64 i0 = c0 + (u64)kScanItems * threadIdx.x;
    u64 cnt[kScanItems];
    u64 sum = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
      cnt[r] = i0 + r < end ? f(i0 + r) : 0;
      sum += cnt[r];
    }
    u64 tot;
    u64 off = base + block_excl_scan<u64>(sum, &tot);
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
      if (cnt[r]) e(i0 + r, off, cnt[r]);
      off += cnt[r];
    }
    base += tot;
  }
}

// ----------------------------------------------------------------------------
// LSD radix sort passes over u64 keys on digits [shift, shift+nbits),
// nbits <= 8 (kernels in radix.cuh).  hist layout: [256][P] digit-major
// (per-block counts, then per-digit exclusive prefixes over blocks),
// followed by the 256 digit totals.

// Host driver: stable sort of keys[0..*n_ptr) on bits [lo, hi), ping-pong
// between a and b; returns the buffer holding the result.  `hist` holds
// 256 * (P + 1) entries.
u64* radix_sort(u64* a, u64* b, const u64* n_ptr, int lo, int hi, uint32_t* hist, int P, cudaStream_t s);

// Host driver for the scan: P blocks, `part` holds P + 1 u64.
template <class CountF, class EmitF>
inline void part_scan_emit(const u64* n_ptr, u64 n_host, CountF f, EmitF e, u64* part, int P, u64* total_out,
                           cudaStream_t s) {
  k_part_reduce<CountF><<<P, 256, 0, s>>>(n_ptr, n_host, f, part);
  k_part_scan<<<1, 1024, 0, s>>>(part, P, total_out);
  k_part_emit<CountF, EmitF><<<P, 256, 0, s>>>(n_ptr, n_host, f, e, part);
}

}  // namespace dcg
