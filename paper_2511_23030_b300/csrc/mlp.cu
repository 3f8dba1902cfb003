// Learned chunk-prefetch proposal: a small MLP 128 (99 used) -> 256 -> 256 ->
// 256 -> 1 with GELU (erf form) and a sigmoid output, trained with binary
// cross-entropy and Adam.  GEMMs run on the tensor cores in BF16 with FP32
// accumulation: by default with tcgen05.mma into tensor memory, operands
// staged by TMA (k_gemm_tc), or with mma.sync m16n8k16 (k_gemm_bf16, the
// pre-Blackwell path, kept selectable); weights are kept in FP32 (master
// copy) and converted to BF16 for every step.  Nothing here changes what is
// rendered: the exact frustum cull decides the active set, the MLP only
// proposes chunks whose copy can start early.
#include <cuda.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "kernels.cuh"

namespace dcg {

constexpr int kIn = 128, kHid = 256;
// flat parameter layout: W1[128][256] b1[256] W2[256][256] b2 W3[256][256] b3 w4[256] b4[1]
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kIn * kHid, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kHid, kOffW4 = kOffB3 + kHid, kOffB4 = kOffW4 + kHid,
              kNParams = kOffB4 + 1;

__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float(((unsigned)h) << 16); }
// float -> bf16, round to nearest even (finite inputs)
__device__ __forceinline__ uint16_t f2bf(float f) {
  unsigned u = __float_as_uint(f);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

// ----------------------------------------------------------------------------
// C[M,N] = A[M,K] B[K,N] with general element strides, BF16 in, FP32
// accumulate.  Tiles of 64x64x32 staged in shared memory in canonical layout
// (A as [m][k], B as [n][k], rows padded by 8 elements), 4 warps each
// computing 32x32 with mma.sync.m16n8k16.  M, N multiples of 64, K of 32.
enum Epi { EPI_F32 = 0, EPI_BIAS_GELU = 1, EPI_DGELU = 2 };

struct GemmArgs {
  const uint16_t* A;
  long long a_m, a_k;
  const uint16_t* B;
  long long b_n, b_k;
  int M, N, K;
  int epi;
  float* C;          // EPI_F32: C[m*N+n] = acc (+= if accumulate)
  int accumulate;
  const float* bias; // EPI_BIAS_GELU: z = acc + bias[n]
  float* Z;          //   z stored FP32 [M,N]
  uint16_t* H;       //   gelu(z) stored BF16 [M,N]
  const float* Zin;  // EPI_DGELU: out = acc * gelu'(Zin[m,n]) stored BF16 in H
};

constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;

__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g) {
  __shared__ __align__(16) uint16_t As[BM][BK + PAD];
  __shared__ __align__(16) uint16_t Bs[BN][BK + PAD];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gq = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 128) {
      const int m = e / BK, k = e % BK;
      As[m][k] = g.A[(long long)(m0 + m) * g.a_m + (long long)(k0 + k) * g.a_k];
    }
    for (int e = tid; e < BN * BK; e += 128) {
      const int n = e / BK, k = e % BK;
      Bs[n][k] = g.B[(long long)(n0 + n) * g.b_n + (long long)(k0 + k) * g.b_k];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + 16 * i + gq;
        a[i][0] = *reinterpret_cast<const unsigned*>(&As[r][kk + 2 * tq]);
        a[i][1] = *reinterpret_cast<const unsigned*>(&As[r + 8][kk + 2 * tq]);
        a[i][2] = *reinterpret_cast<const unsigned*>(&As[r][kk + 2 * tq + 8]);
        a[i][3] = *reinterpret_cast<const unsigned*>(&As[r + 8][kk + 2 * tq + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + 8 * j + gq;
        b[j][0] = *reinterpret_cast<const unsigned*>(&Bs[c][kk + 2 * tq]);
        b[j][1] = *reinterpret_cast<const unsigned*>(&Bs[c][kk + 2 * tq + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b[j][0]), "r"(b[j][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm + 16 * i + gq + (r >= 2 ? 8 : 0);
        const int n = n0 + wn + 8 * j + 2 * tq + (r & 1);
        const long long o = (long long)m * g.N + n;
        const float v = acc[i][j][r];
        if (g.epi == EPI_F32) {
          g.C[o] = g.accumulate ? g.C[o] + v : v;
        } else if (g.epi == EPI_BIAS_GELU) {
          const float z = v + g.bias[n];
          g.Z[o] = z;
          g.H[o] = f2bf(gelu(z));
        } else {
          g.H[o] = f2bf(v * gelu_grad(g.Zin[o]));
        }
      }
}

static void gemm(const GemmArgs& g, cudaStream_t s) {
  dim3 grid(g.N / BN, g.M / BM);
  k_gemm_bf16<<<grid, 128, 0, s>>>(g);
  count_launch();
}

// ----------------------------------------------------------------------------
// The same GEMMs on Blackwell's tensor cores: C[M,N] = A[M,K] B[N,K]^T with
// both operands K-major (row-major with K contiguous), BF16, FP32
// accumulation in tensor memory.  One CTA of 8 warps computes a 128 x 64 tile
// of C: K is walked in steps of 64 through a 4-stage ring of shared memory
// that TMA fills (128-byte swizzle, one mbarrier per stage counting the bytes
// that arrive); one thread of warp 1 issues tcgen05.mma (M 128, N 64, K 16;
// four per stage) into a 64-column TMEM accumulator and commits each stage
// back to the TMA thread (warp 0) when its MMAs have read it; after the last
// stage every warp reads 32 TMEM lanes (rows of C) x 32 columns with
// tcgen05.ld (warps w and w + 4 share the lanes of w's quarter, one column
// half each) and runs the same epilogues as the mma.sync kernel, with 16-byte
// stores.  Every mbarrier wait is bounded in time: on expiry the kernel sets
// the MLP's error word, stops issuing, waits (bounded) for the copies it
// started, frees its TMEM and returns.
namespace tc {

constexpr int BM = 128, BN = 64, BK = 64, STAGES = 4, THREADS = 256;
constexpr int A_BYTES = BM * BK * 2;            // 16 KB
constexpr int B_BYTES = BN * BK * 2;            // 8 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;  // 24 KB, a multiple of the 1024-byte swizzle atom
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 128;  // + alignment slack + barriers
constexpr long long kWaitCycles = 4000000000ll;  // about 2 s at the maximum SM clock

// instruction descriptor of tcgen05.mma kind::f16: D F32 (bits 4-5 = 1), A and
// B BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit
// 17, M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}
// wait for the phase of parity `parity` to complete, at most kWaitCycles
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned* err) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) {
      atomicOr(err, 1u);
      return false;
    }
  }
  return true;
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1 (bit 46),
// swizzle mode 2 (bits 61-63); the start address advances by 32 bytes per
// K step of 16 inside a swizzle row
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

struct Epilogue {
  int M, N;            // rows of C (valid), columns of C (row pitch)
  int epi;
  float* C;            // EPI_F32
  int accumulate;
  const float* bias;   // EPI_BIAS_GELU
  float* Z;
  uint16_t* H;
  const float* Zin;    // EPI_DGELU
  unsigned* err;       // bounded waits that gave up
};

__global__ void __launch_bounds__(THREADS) k_gemm_tc(const __grid_constant__ CUtensorMap ta,
                                                     const __grid_constant__ CUtensorMap tb, int K, Epilogue e) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);  // full[4], empty[4], done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int KT = K / BK;
  const uint32_t full0 = su32(bars), empty0 = su32(bars + STAGES), done = su32(bars + 2 * STAGES);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * s));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * s));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done));
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&ta) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tb) : "memory");
  }
  if (warp == 0) {  // the accumulator: BN columns of 128 lanes x 32 bits
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)), "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  int issued = 0;  // stages the TMA thread filled
  if (warp == 0 && lane == 0) {
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % STAGES;
      if (kt >= STAGES && !mbar_wait(empty0 + 8 * s, (uint32_t)((kt / STAGES - 1) & 1), e.err)) *abort_flag = 1;
      if (*abort_flag) break;
      const uint32_t sa = su32(smem + s * STAGE_BYTES), sb = sa + A_BYTES, fb = full0 + 8 * s;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(STAGE_BYTES) : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(sa),
          "l"(&ta), "r"(kt * BK), "r"(m0), "r"(fb)
          : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(sb),
          "l"(&tb), "r"(kt * BK), "r"(n0), "r"(fb)
          : "memory");
      issued = kt + 1;
    }
  } else if (warp == 1 && lane == 0) {
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % STAGES;
      if (!mbar_wait(full0 + 8 * s, (uint32_t)((kt / STAGES) & 1), e.err)) *abort_flag = 1;
      if (*abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = su32(smem + s * STAGE_BYTES), sb = sa + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t da = sdesc(sa + 32 * kk), db = sdesc(sb + 32 * kk);
        const uint32_t acc = (kt | kk) != 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      // the stage is free again once these MMAs have read it
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty0 + 8 * s)
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done) : "memory");
  }
  __syncwarp();
  // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of the tile),
  // columns 32 (w / 4) .. + 31 (warp-uniform: tcgen05.ld is .sync.aligned)
  const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0u, e.err) && !*abort_flag);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int q = warp & 3, c = 32 * (warp >> 2);
    const int m = m0 + 32 * q + lane;
    uint32_t v[32];
    const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (m < e.M) {
      const int nb = n0 + c;                       // first of this thread's 32 columns
      const long long o = (long long)m * e.N + nb;  // 32-element aligned: 16-byte vector accesses
      if (e.epi == EPI_F32) {
        float4* dst = reinterpret_cast<float4*>(e.C + o);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float4 a = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]), __uint_as_float(v[4 * j + 2]),
                                 __uint_as_float(v[4 * j + 3]));
          if (e.accumulate) {
            const float4 b = dst[j];
            a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
          }
          dst[j] = a;
        }
      } else {
        uint32_t hb[16];
        if (e.epi == EPI_BIAS_GELU) {
          float4* zd = reinterpret_cast<float4*>(e.Z + o);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float z[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) z[t] = __uint_as_float(v[4 * j + t]) + e.bias[nb + 4 * j + t];
            zd[j] = make_float4(z[0], z[1], z[2], z[3]);
            hb[2 * j] = (uint32_t)f2bf(gelu(z[0])) | ((uint32_t)f2bf(gelu(z[1])) << 16);
            hb[2 * j + 1] = (uint32_t)f2bf(gelu(z[2])) | ((uint32_t)f2bf(gelu(z[3])) << 16);
          }
        } else {
          const float4* zi = reinterpret_cast<const float4*>(e.Zin + o);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float4 zz = zi[j];
            const float g0 = __uint_as_float(v[4 * j]) * gelu_grad(zz.x), g1 = __uint_as_float(v[4 * j + 1]) * gelu_grad(zz.y);
            const float g2 = __uint_as_float(v[4 * j + 2]) * gelu_grad(zz.z), g3 = __uint_as_float(v[4 * j + 3]) * gelu_grad(zz.w);
            hb[2 * j] = (uint32_t)f2bf(g0) | ((uint32_t)f2bf(g1) << 16);
            hb[2 * j + 1] = (uint32_t)f2bf(g2) | ((uint32_t)f2bf(g3) << 16);
          }
        }
        uint4* hd = reinterpret_cast<uint4*>(e.H + o);
#pragma unroll
        for (int j = 0; j < 4; ++j) hd[j] = make_uint4(hb[4 * j], hb[4 * j + 1], hb[4 * j + 2], hb[4 * j + 3]);
      }
    }
  }
  // copies this CTA started and nobody consumed (only after a wait gave up)
  if (warp == 0 && lane == 0)
    for (int kt = issued > STAGES ? issued - STAGES : 0; kt < issued; ++kt)
      mbar_wait(full0 + 8 * (kt % STAGES), (uint32_t)((kt / STAGES) & 1), e.err);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

}  // namespace tc

// host side of the tensor-core path: 2D tensor maps over K-major BF16
// matrices (rows x K, row pitch `pitch` elements), boxes of 64 x box_rows
// with the 128-byte swizzle the MMA descriptors expect; the encoder comes
// from the driver through the runtime (no link-time driver dependency)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

static bool kmajor_map(CUtensorMap* m, const uint16_t* base, long long rows, long long K, long long pitch,
                       int box_rows) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc || (reinterpret_cast<uintptr_t>(base) & 15u) || (pitch * 2) % 16 || K % tc::BK) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(pitch * 2)};
  const cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C[M,N] = A[M,K] B[N,K]^T on tcgen05, A and B K-major with row pitches lda, ldb
static cudaError_t gemm_tc(const uint16_t* A, long long lda, const uint16_t* B, long long ldb, int M, int N, int K,
                           const tc::Epilogue& e, cudaStream_t s) {
  CUtensorMap ma, mb;
  if (N % tc::BN || !kmajor_map(&ma, A, M, K, lda, tc::BM) || !kmajor_map(&mb, B, N, K, ldb, tc::BN))
    return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t r = cudaFuncSetAttribute(tc::k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
    if (r != cudaSuccess) return r;
    attr = true;
  }
  dim3 grid((M + tc::BM - 1) / tc::BM, N / tc::BN);
  tc::k_gemm_tc<<<grid, tc::THREADS, tc::SMEM_BYTES, s>>>(ma, mb, K, e);
  count_launch();
  return cudaGetLastError();
}

// dst[c * ld_dst + r] = src[r * ld_src + c] for r < R, c < C (BF16), 32 x 32 tiles
__global__ void k_transpose_bf16(const uint16_t* __restrict__ src, int R, int C, int ld_src, uint16_t* __restrict__ dst,
                                 int ld_dst) {
  __shared__ uint16_t t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = r0 + y, c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (r < R && c < C) ? src[(long long)r * ld_src + c] : (uint16_t)0;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y, r = r0 + threadIdx.x;
    if (r < R && c < C) dst[(long long)c * ld_dst + r] = t[threadIdx.x][y];
  }
}

static void transpose_bf16(const uint16_t* src, int R, int C, int ld_src, uint16_t* dst, int ld_dst, cudaStream_t s) {
  dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
  k_transpose_bf16<<<grid, block, 0, s>>>(src, R, C, ld_src, dst, ld_dst);
  count_launch();
}

// ----------------------------------------------------------------------------
// small kernels
__global__ void k_to_bf16(const float* __restrict__ src, uint16_t* __restrict__ dst, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = f2bf(src[i]);
}

// logits[m] = sum_k H3[m,k] w4[k] + b4; one warp per row
__global__ void k_head_fwd(const uint16_t* __restrict__ H3, const float* __restrict__ P, int B, float* __restrict__ logit,
                           float* __restrict__ prob) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= B) return;
  float acc = 0.f;
  for (int k = lane; k < kHid; k += 32) acc += bf2f(H3[(long long)warp * kHid + k]) * bf2f(f2bf(P[kOffW4 + k]));
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    const float z = acc + P[kOffB4];
    logit[warp] = z;
    if (prob) prob[warp] = 1.f / (1.f + __expf(-z));
  }
}

// BCE with logits, mean over the batch: L = mean(max(z,0) - z y + log(1 + exp(-|z|))),
// dL/dz = (sigmoid(z) - y) / B.  Also dH3 = dz w4 -> dZ3 = dH3 gelu'(Z3) (BF16),
// dw4 += H3^T dz and db4 += sum dz (block partials + atomics), loss += L.
__global__ void k_head_bwd(const float* __restrict__ logit, const float* __restrict__ y, const uint16_t* __restrict__ H3,
                           const float* __restrict__ Z3, const float* __restrict__ P, int B, uint16_t* __restrict__ dZ3,
                           float* __restrict__ G, float* __restrict__ loss) {
  const int m = blockIdx.x;  // one block of 256 threads per sample row
  const int k = threadIdx.x;
  const float z = logit[m];
  const float sg = 1.f / (1.f + __expf(-z));
  const float dz = (sg - y[m]) / (float)B;
  const long long o = (long long)m * kHid + k;
  const float w4 = bf2f(f2bf(P[kOffW4 + k]));
  dZ3[o] = f2bf(dz * w4 * gelu_grad(Z3[o]));
  atomicAdd(&G[kOffW4 + k], bf2f(H3[o]) * dz);
  if (k == 0) {
    atomicAdd(&G[kOffB4], dz);
    const float l = fmaxf(z, 0.f) - z * y[m] + log1pf(__expf(-fabsf(z)));
    atomicAdd(loss, l / (float)B);
  }
}

// db[n] += sum_m dZ[m,n]
__global__ void k_colsum(const uint16_t* __restrict__ dZ, int M, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float acc = 0.f;
  for (int m = 0; m < M; ++m) acc += bf2f(dZ[(long long)m * N + n]);
  db[n] += acc;
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m1, float* __restrict__ m2,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float g = G[i];
    const float a = b1 * m1[i] + (1.f - b1) * g;
    const float b = b2 * m2[i] + (1.f - b2) * g * g;
    m1[i] = a;
    m2[i] = b;
    P[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

// ----------------------------------------------------------------------------
// Features of one frame: the SE(3) logarithm xi_k = log(T_t^-1 T_{t-k}) of the
// pose of each of the last 16 keyframes relative to the current one
// (k = 0..15; T = camera-to-world), translation scaled by 1/16 m and
// rotation in radians, then for each candidate chunk its centre in the
// current camera frame scaled by 1/60 m; zero padding to 128 columns.
struct PoseHist {
  float Tcw[16][12];  // world->camera 3x4 of frames t, t-1, ..., t-15
};

__device__ void se3_log_rel(const float* A, const float* Bm, float* xi) {
  // relative transform Rel = Tcw_A * Twc_B (pose of camera B in camera A's frame)
  float Rb_t[9], tb[3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Rb_t[3 * r + c] = Bm[4 * c + r];  // R_B^T
  for (int r = 0; r < 3; ++r) tb[r] = -(Rb_t[3 * r + 0] * Bm[3] + Rb_t[3 * r + 1] * Bm[7] + Rb_t[3 * r + 2] * Bm[11]);
  float R[9], t[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) R[3 * r + c] = A[4 * r + 0] * Rb_t[c] + A[4 * r + 1] * Rb_t[3 + c] + A[4 * r + 2] * Rb_t[6 + c];
    t[r] = A[4 * r + 0] * tb[0] + A[4 * r + 1] * tb[1] + A[4 * r + 2] * tb[2] + A[4 * r + 3];
  }
  const float tr = R[0] + R[4] + R[8];
  const float ct = fminf(1.f, fmaxf(-1.f, 0.5f * (tr - 1.f)));
  const float th = acosf(ct);
  const float st = sinf(th);
  // rotation vector w = th / (2 sin th) (R - R^T)^vee, with the small-angle limit 1/2
  const float f = th < 1e-4f ? 0.5f + th * th / 12.f : th / (2.f * st);
  const float w[3] = {f * (R[7] - R[5]), f * (R[2] - R[6]), f * (R[3] - R[1])};
  // u = V^-1 t, V^-1 = I - 1/2 [w]x + (1/th^2)(1 - th sin th / (2 (1 - cos th))) [w]x^2
  const float g = th < 1e-3f ? 1.f / 12.f : (1.f - th * st / (2.f * (1.f - ct))) / (th * th);
  float wx_t[3] = {w[1] * t[2] - w[2] * t[1], w[2] * t[0] - w[0] * t[2], w[0] * t[1] - w[1] * t[0]};
  float wx2_t[3] = {w[1] * wx_t[2] - w[2] * wx_t[1], w[2] * wx_t[0] - w[0] * wx_t[2], w[0] * wx_t[1] - w[1] * wx_t[0]};
  for (int r = 0; r < 3; ++r) xi[r] = (t[r] - 0.5f * wx_t[r] + g * wx2_t[r]) * (1.f / 16.f);
  for (int r = 0; r < 3; ++r) xi[3 + r] = w[r];
}

__global__ void k_mlp_features(PoseHist ph, const int32_t* __restrict__ coords, float s, const int32_t* __restrict__ cand,
                               int n_cand, int n_rows, uint16_t* __restrict__ x) {
  __shared__ float tw[96];
  if (threadIdx.x < 16) se3_log_rel(ph.Tcw[0], ph.Tcw[threadIdx.x], &tw[6 * threadIdx.x]);
  __syncthreads();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rows; r += gridDim.x * blockDim.x) {
    uint16_t* row = x + (long long)r * kIn;
    if (r >= n_cand) {
      for (int k = 0; k < kIn; ++k) row[k] = 0;
      continue;
    }
    for (int k = 0; k < 96; ++k) row[k] = f2bf(tw[k]);
    const int c = cand[r];
    const float p[3] = {coords[3 * c] * s, coords[3 * c + 1] * s, coords[3 * c + 2] * s};
    const float* T = ph.Tcw[0];
    for (int a = 0; a < 3; ++a)
      row[96 + a] = f2bf((T[4 * a + 0] * p[0] + T[4 * a + 1] * p[1] + T[4 * a + 2] * p[2] + T[4 * a + 3]) * (1.f / 60.f));
    for (int k = 99; k < kIn; ++k) row[k] = 0;
  }
}

// dst row r = src row perm[r] (rows of `cols` BF16 values); also y
__global__ void k_gather_rows(const uint16_t* __restrict__ src, const float* __restrict__ ysrc,
                              const int32_t* __restrict__ perm, int n, int cols, uint16_t* __restrict__ dst,
                              float* __restrict__ ydst) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * cols;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / cols, k = e - r * cols;
    dst[e] = src[(long long)perm[r] * cols + k];
    if (k == 0) ydst[r] = ysrc[perm[r]];
  }
}

}  // namespace dcg

using namespace dcg;

struct dcg_mlp {
  int max_batch = 0;
  float* P = nullptr;  // FP32 master parameters (flat)
  float* G = nullptr;  // gradients (flat)
  float* m1 = nullptr;
  float* m2 = nullptr;
  uint16_t* Pb = nullptr;  // BF16 copy of P
  float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr;
  uint16_t *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *dZ = nullptr, *dZ2 = nullptr;
  float* logit = nullptr;
  long long t = 0;
  // tensor-core path: K-major operands (transposed weights W^T [256][K],
  // transposed layer input and dZ [256][batch] for the weight gradients)
  int gemm = DCG_MLP_GEMM_TCGEN05;
  uint16_t* WT = nullptr;  // W1^T [256][128], W2^T [256][256], W3^T [256][256]
  uint16_t *Ta = nullptr, *Tb = nullptr;
  unsigned* err = nullptr;  // a bounded wait of k_gemm_tc gave up
  cudaError_t launch_err = cudaSuccess;  // first failure to set up or launch a tensor-core GEMM
};

namespace {

template <class T>
cudaError_t mal(T** p, size_t n) {
  return cudaMalloc((void**)p, sizeof(T) * (n > 0 ? n : 1));
}

constexpr int kOffWT1 = 0, kOffWT2 = kHid * kIn, kOffWT3 = kOffWT2 + kHid * kHid, kNWT = kOffWT3 + kHid * kHid;

void tc_run(dcg_mlp* m, cudaError_t r) {
  if (r != cudaSuccess && m->launch_err == cudaSuccess) m->launch_err = r;
}

tc::Epilogue tc_epi(dcg_mlp* m, int M, const GemmArgs& g) {
  tc::Epilogue e{};
  e.M = M;
  e.N = g.N;
  e.epi = g.epi;
  e.C = g.C;
  e.accumulate = g.accumulate;
  e.bias = g.bias;
  e.Z = g.Z;
  e.H = g.H;
  e.Zin = g.Zin;
  e.err = m->err;
  return e;
}

// forward through the three hidden layers; returns logits in m->logit
void mlp_forward(dcg_mlp* m, const uint16_t* x, int B, float* prob, cudaStream_t s) {
  k_to_bf16<<<64, 256, 0, s>>>(m->P, m->Pb, kNParams);
  count_launch();
  const uint16_t* Pb = m->Pb;
  if (m->gemm == DCG_MLP_GEMM_TCGEN05) {
    // W^T (K-major B operands) of the three hidden layers
    transpose_bf16(Pb + kOffW1, kIn, kHid, kHid, m->WT + kOffWT1, kIn, s);
    transpose_bf16(Pb + kOffW2, kHid, kHid, kHid, m->WT + kOffWT2, kHid, s);
    transpose_bf16(Pb + kOffW3, kHid, kHid, kHid, m->WT + kOffWT3, kHid, s);
    GemmArgs g{};
    g.epi = EPI_BIAS_GELU;
    g.N = kHid;
    g.bias = m->P + kOffB1; g.Z = m->Z1; g.H = m->H1;
    tc_run(m, gemm_tc(x, kIn, m->WT + kOffWT1, kIn, B, kHid, kIn, tc_epi(m, B, g), s));
    g.bias = m->P + kOffB2; g.Z = m->Z2; g.H = m->H2;
    tc_run(m, gemm_tc(m->H1, kHid, m->WT + kOffWT2, kHid, B, kHid, kHid, tc_epi(m, B, g), s));
    g.bias = m->P + kOffB3; g.Z = m->Z3; g.H = m->H3;
    tc_run(m, gemm_tc(m->H2, kHid, m->WT + kOffWT3, kHid, B, kHid, kHid, tc_epi(m, B, g), s));
    k_head_fwd<<<(B * 32 + 255) / 256, 256, 0, s>>>(m->H3, m->P, B, m->logit, prob);
    count_launch();
    return;
  }
  GemmArgs g{};
  g.epi = EPI_BIAS_GELU;
  g.M = B;
  g.N = kHid;
  // layer 1: X[B,128] W1[128,256]
  g.A = x; g.a_m = kIn; g.a_k = 1; g.K = kIn;
  g.B = Pb + kOffW1; g.b_n = 1; g.b_k = kHid;
  g.bias = m->P + kOffB1; g.Z = m->Z1; g.H = m->H1;
  gemm(g, s);
  // layer 2
  g.A = m->H1; g.a_m = kHid; g.a_k = 1; g.K = kHid;
  g.B = Pb + kOffW2; g.bias = m->P + kOffB2; g.Z = m->Z2; g.H = m->H2;
  gemm(g, s);
  // layer 3
  g.A = m->H2; g.B = Pb + kOffW3; g.bias = m->P + kOffB3; g.Z = m->Z3; g.H = m->H3;
  gemm(g, s);
  k_head_fwd<<<(B * 32 + 255) / 256, 256, 0, s>>>(m->H3, m->P, B, m->logit, prob);
  count_launch();
}

// gradients of the mean BCE into m->G (overwritten), loss added to *loss
void mlp_backward(dcg_mlp* m, const uint16_t* x, const float* y, int B, float* loss, cudaStream_t s) {
  cudaMemsetAsync(m->G, 0, sizeof(float) * kNParams, s);
  k_head_bwd<<<B, kHid, 0, s>>>(m->logit, y, m->H3, m->Z3, m->P, B, m->dZ, m->G, loss);
  count_launch();
  const uint16_t* Pb = m->Pb;
  struct L {
    const uint16_t* in;  // layer input activations [B, K]
    int K;
    int offW, offB;
    const float* Zprev;  // pre-activation of the layer below (null for the first layer)
  } layers[3] = {{x, kIn, kOffW1, kOffB1, nullptr}, {m->H1, kHid, kOffW2, kOffB2, m->Z1}, {m->H2, kHid, kOffW3, kOffB3, m->Z2}};
  uint16_t* dcur = m->dZ;   // dZ of the current layer [B, 256]
  uint16_t* dnext = m->dZ2;
  const bool tcg = m->gemm == DCG_MLP_GEMM_TCGEN05;
  for (int l = 2; l >= 0; --l) {
    const L& ly = layers[l];
    // dW[K,256] = in^T dZ : M' = K, N' = 256, K' = B
    GemmArgs gw{};
    gw.epi = EPI_F32;
    gw.M = ly.K; gw.N = kHid; gw.K = B;
    gw.A = ly.in; gw.a_m = 1; gw.a_k = ly.K;
    gw.B = dcur; gw.b_n = 1; gw.b_k = kHid;
    gw.C = m->G + ly.offW;
    if (tcg) {  // both operands K-major along the batch: in^T [K][B], dZ^T [256][B]
      transpose_bf16(ly.in, B, ly.K, ly.K, m->Ta, B, s);
      transpose_bf16(dcur, B, kHid, kHid, m->Tb, B, s);
      tc_run(m, gemm_tc(m->Ta, B, m->Tb, B, ly.K, kHid, B, tc_epi(m, ly.K, gw), s));
    } else {
      gemm(gw, s);
    }
    k_colsum<<<(kHid + 127) / 128, 128, 0, s>>>(dcur, B, kHid, m->G + ly.offB);
    count_launch();
    if (l > 0) {
      // dH_prev[B,256] = dZ W^T, then dZ_prev = dH_prev gelu'(Z_prev)
      GemmArgs gx{};
      gx.epi = EPI_DGELU;
      gx.M = B; gx.N = kHid; gx.K = kHid;
      gx.A = dcur; gx.a_m = kHid; gx.a_k = 1;
      gx.B = Pb + ly.offW; gx.b_n = kHid; gx.b_k = 1;
      gx.Zin = ly.Zprev;
      gx.H = dnext;
      if (tcg)  // W [K_in][256] is already K-major along the output index
        tc_run(m, gemm_tc(dcur, kHid, Pb + ly.offW, kHid, B, kHid, kHid, tc_epi(m, B, gx), s));
      else
        gemm(gx, s);
      uint16_t* t = dcur;
      dcur = dnext;
      dnext = t;
    }
  }
}

}  // namespace

extern "C" {

dcg_status dcg_mlp_create(int32_t max_batch, dcg_mlp** out) {
  if (!out || max_batch <= 0 || max_batch % 64) return DCG_ERR_ARG;
  dcg_mlp* m = new dcg_mlp();
  m->max_batch = max_batch;
  const size_t BH = (size_t)max_batch * kHid;
  bool ok = mal(&m->P, kNParams) == cudaSuccess && mal(&m->G, kNParams) == cudaSuccess &&
            mal(&m->m1, kNParams) == cudaSuccess && mal(&m->m2, kNParams) == cudaSuccess &&
            mal(&m->Pb, kNParams) == cudaSuccess && mal(&m->Z1, BH) == cudaSuccess && mal(&m->Z2, BH) == cudaSuccess &&
            mal(&m->Z3, BH) == cudaSuccess && mal(&m->H1, BH) == cudaSuccess && mal(&m->H2, BH) == cudaSuccess &&
            mal(&m->H3, BH) == cudaSuccess && mal(&m->dZ, BH) == cudaSuccess && mal(&m->dZ2, BH) == cudaSuccess &&
            mal(&m->logit, (size_t)max_batch) == cudaSuccess && mal(&m->WT, (size_t)kNWT) == cudaSuccess &&
            mal(&m->Ta, BH) == cudaSuccess && mal(&m->Tb, BH) == cudaSuccess && mal(&m->err, 1) == cudaSuccess;
  if (!ok) {
    dcg_mlp_destroy(m);
    return DCG_ERR_OOM;
  }
  cudaMemset(m->P, 0, sizeof(float) * kNParams);
  cudaMemset(m->m1, 0, sizeof(float) * kNParams);
  cudaMemset(m->m2, 0, sizeof(float) * kNParams);
  cudaMemset(m->err, 0, sizeof(unsigned));
  int dev = 0, major = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  m->gemm = major >= 10 ? DCG_MLP_GEMM_TCGEN05 : DCG_MLP_GEMM_MMA_SYNC;
  *out = m;
  return DCG_OK;
}

dcg_status dcg_mlp_set_gemm(dcg_mlp* m, int32_t kind) {
  if (!m || (kind != DCG_MLP_GEMM_TCGEN05 && kind != DCG_MLP_GEMM_MMA_SYNC)) return DCG_ERR_ARG;
  m->gemm = kind;
  return DCG_OK;
}

dcg_status dcg_mlp_destroy(dcg_mlp* m) {
  if (!m) return DCG_ERR_ARG;
  cudaFree(m->P); cudaFree(m->G); cudaFree(m->m1); cudaFree(m->m2); cudaFree(m->Pb);
  cudaFree(m->Z1); cudaFree(m->Z2); cudaFree(m->Z3); cudaFree(m->H1); cudaFree(m->H2); cudaFree(m->H3);
  cudaFree(m->dZ); cudaFree(m->dZ2); cudaFree(m->logit);
  cudaFree(m->WT); cudaFree(m->Ta); cudaFree(m->Tb); cudaFree(m->err);
  delete m;
  return DCG_OK;
}

int32_t dcg_mlp_num_params(void) { return kNParams; }

dcg_status dcg_mlp_set_params(dcg_mlp* m, const float* host_params) {
  if (!m || !host_params) return DCG_ERR_ARG;
  if (cudaMemcpy(m->P, host_params, sizeof(float) * kNParams, cudaMemcpyHostToDevice) != cudaSuccess) return DCG_ERR_CUDA;
  cudaMemset(m->m1, 0, sizeof(float) * kNParams);
  cudaMemset(m->m2, 0, sizeof(float) * kNParams);
  m->t = 0;
  return DCG_OK;
}

dcg_status dcg_mlp_get_params(dcg_mlp* m, float* host_params) {
  if (!m || !host_params) return DCG_ERR_ARG;
  if (cudaMemcpy(host_params, m->P, sizeof(float) * kNParams, cudaMemcpyDeviceToHost) != cudaSuccess) return DCG_ERR_CUDA;
  unsigned err = 0;
  if (cudaMemcpy(&err, m->err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return DCG_ERR_CUDA;
  if (err) {  // reported once
    cudaMemset(m->err, 0, sizeof(unsigned));
    return DCG_ERR_TIMEOUT;
  }
  return DCG_OK;
}

// the first tensor-core GEMM that could not be set up or launched since the last call
static dcg_status take_launch_err(dcg_mlp* m) {
  const cudaError_t r = m->launch_err;
  m->launch_err = cudaSuccess;
  return r == cudaSuccess ? DCG_OK : (r == cudaErrorInvalidValue ? DCG_ERR_ARG : DCG_ERR_CUDA);
}

dcg_status dcg_mlp_forward(dcg_mlp* m, const uint16_t* x, int32_t B, float* prob, void* stream) {
  if (!m || !x || !prob || B <= 0 || B > m->max_batch || B % 64) return DCG_ERR_ARG;
  mlp_forward(m, x, B, prob, (cudaStream_t)stream);
  const dcg_status ls = take_launch_err(m);
  if (ls != DCG_OK) return ls;
  return cudaGetLastError() == cudaSuccess ? DCG_OK : DCG_ERR_CUDA;
}

dcg_status dcg_mlp_grads(dcg_mlp* m, const uint16_t* x, const float* y, int32_t B, float* grads, float* loss,
                         void* stream) {
  if (!m || !x || !y || !loss || B <= 0 || B > m->max_batch || B % 64) return DCG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  mlp_forward(m, x, B, nullptr, s);
  mlp_backward(m, x, y, B, loss, s);
  if (grads) cudaMemcpyAsync(grads, m->G, sizeof(float) * kNParams, cudaMemcpyDeviceToDevice, s);
  const dcg_status ls = take_launch_err(m);
  if (ls != DCG_OK) return ls;
  return cudaGetLastError() == cudaSuccess ? DCG_OK : DCG_ERR_CUDA;
}

dcg_status dcg_mlp_features(const float* pose_hist, const int32_t* coords, float chunk_size, const int32_t* cand,
                            int32_t n_cand, int32_t n_rows, uint16_t* x, void* stream) {
  if (!pose_hist || n_cand < 0 || n_rows < n_cand || (n_cand > 0 && (!coords || !cand)) || !x) return DCG_ERR_ARG;
  PoseHist ph;
  for (int k = 0; k < 16; ++k)
    for (int e = 0; e < 12; ++e) ph.Tcw[k][e] = pose_hist[16 * k + e];
  if (n_rows > 0) {
    k_mlp_features<<<(n_rows + 255) / 256, 256, 0, (cudaStream_t)stream>>>(ph, coords, chunk_size, cand, n_cand, n_rows, x);
    count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? DCG_OK : DCG_ERR_CUDA;
}

dcg_status dcg_mlp_gather_rows(const uint16_t* x, const float* y, const int32_t* perm, int32_t n, uint16_t* x_out,
                               float* y_out, void* stream) {
  if (!x || !y || !perm || n < 0 || !x_out || !y_out) return DCG_ERR_ARG;
  if (n > 0) {
    k_gather_rows<<<592, 256, 0, (cudaStream_t)stream>>>(x, y, perm, n, kIn, x_out, y_out);
    count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? DCG_OK : DCG_ERR_CUDA;
}

dcg_status dcg_mlp_train_step(dcg_mlp* m, const uint16_t* x, const float* y, int32_t B, float lr, float* loss,
                              void* stream) {
  dcg_status st = dcg_mlp_grads(m, x, y, B, nullptr, loss, stream);
  if (st != DCG_OK) return st;
  m->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - (float)std::pow(b1, (double)m->t), c2 = 1.f - (float)std::pow(b2, (double)m->t);
  k_adam<<<128, 256, 0, (cudaStream_t)stream>>>(m->P, m->G, m->m1, m->m2, kNParams, lr, b1, b2, 1e-8f, c1, c2);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? DCG_OK : DCG_ERR_CUDA;
}

}  // extern "C"
