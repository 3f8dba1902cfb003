// Adam over the active set, with the first and second moments stored per
// Gaussian beside its parameters (they travel with the chunk through the
// device pool and the host tier).  The paper optimises the Gaussian
// parameters of the active chunks against the loss of Eq. 2-4 (Sec. III-E
// "Optimization") with per-Gaussian optimizer state (Sec. III-F resets it
// for the merged regions after a loop closure); the update is Adam
// (Kingma & Ba) with bias correction:
//   m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
//   p <- p - (lr_c / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps).
// Planar rows: component c of Gaussian i at row c; one grid row per
// component (its learning rate), float4 accesses where rows are aligned.
#include <algorithm>

#include "kernels.cuh"

namespace dcg {

__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, float a, const AdamArgs& aa) {
  m = aa.beta1 * m + (1.f - aa.beta1) * g;
  v = aa.beta2 * v + (1.f - aa.beta2) * (g * g);
  p = p - a * (m / (sqrtf(v) * aa.isb2 + aa.eps));
}

template <bool VEC>
__global__ void __launch_bounds__(256) k_adam(float* __restrict__ p, long long ps, const float* __restrict__ g,
                                              long long gs, float* __restrict__ m, float* __restrict__ v,
                                              long long ms, long long n, AdamArgs aa) {
  const int c = blockIdx.y;
  const float a = aa.step[c];
  float* pr = p + (long long)c * ps;
  const float* gr = g + (long long)c * gs;
  float* mr = m + (long long)c * ms;
  float* vr = v + (long long)c * ms;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, dt = (long long)gridDim.x * blockDim.x;
  if (VEC) {
    const long long n4 = n / 4;
    for (long long i = t0; i < n4; i += dt) {
      float4 P = reinterpret_cast<float4*>(pr)[i];
      const float4 G = reinterpret_cast<const float4*>(gr)[i];
      float4 M = reinterpret_cast<float4*>(mr)[i];
      float4 Vv = reinterpret_cast<float4*>(vr)[i];
      adam1(P.x, G.x, M.x, Vv.x, a, aa);
      adam1(P.y, G.y, M.y, Vv.y, a, aa);
      adam1(P.z, G.z, M.z, Vv.z, a, aa);
      adam1(P.w, G.w, M.w, Vv.w, a, aa);
      reinterpret_cast<float4*>(pr)[i] = P;
      reinterpret_cast<float4*>(mr)[i] = M;
      reinterpret_cast<float4*>(vr)[i] = Vv;
    }
    for (long long i = 4 * n4 + t0; i < n; i += dt) adam1(pr[i], gr[i], mr[i], vr[i], a, aa);
  } else {
    for (long long i = t0; i < n; i += dt) adam1(pr[i], gr[i], mr[i], vr[i], a, aa);
  }
}

void launch_adam(float* p, long long ps, const float* g, long long gs, float* m, float* v, long long ms, long long n,
                 int F, const AdamArgs& aa, int num_sms, cudaStream_t st) {
  if (n <= 0) return;
  auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
  const bool vec = al16(p) && al16(g) && al16(m) && al16(v) && ps % 4 == 0 && gs % 4 == 0 && ms % 4 == 0;
  const long long items = vec ? (n + 3) / 4 : n;
  // about 4 waves of 256-thread blocks over all components
  const long long per_row = std::max(1ll, std::min((items + 255) / 256, (long long)num_sms * 32 / std::max(F, 1) + 1));
  dim3 grid((unsigned)per_row, (unsigned)F);
  if (vec)
    k_adam<true><<<grid, 256, 0, st>>>(p, ps, g, gs, m, v, ms, n, aa);
  else
    k_adam<false><<<grid, 256, 0, st>>>(p, ps, g, gs, m, v, ms, n, aa);
  count_launch();
}

}  // namespace dcg
