// Device scan top level and the stable LSD radix sort (hand-written; no library sort).
#include "radix.cuh"

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

u64* radix_sort(u64* a, u64* b, const u64* n_ptr, int lo, int hi, uint32_t* hist, int P, cudaStream_t s) {
  u64* src = a;
  u64* dst = b;
  for (int sh = lo; sh < hi; sh += 8) {
    radix_pass(KeySrc{src}, n_ptr, 0, dst, sh, min(8, hi - sh), hist, P, nullptr, s);
    u64* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

}  // namespace dcg
