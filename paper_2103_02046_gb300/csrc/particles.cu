// Per-particle kernels: bounding box, leapfrog kick/drift, emittance reductions, and small
// helpers. All particle state here is FP64 [n][3] in caller memory.
#include <algorithm>

#include "p3m_internal.cuh"

namespace p3m {
namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(int64_t n, int t = kThreads) {
  return static_cast<unsigned>((n + t - 1) / t);
}

// order-preserving map of finite doubles to unsigned 64-bit keys
__device__ __forceinline__ unsigned long long ordered_key(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_bbox(const double* __restrict__ x, int64_t n, unsigned long long* __restrict__ mn,
                       unsigned long long* __restrict__ mx, int* __restrict__ bad) {
  unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
  int b = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    for (int d = 0; d < 3; ++d) {
      const double v = x[3 * i + d];
      if (!isfinite(v)) {
        b = 1;
        continue;
      }
      const unsigned long long k = ordered_key(v);
      lo[d] = min(lo[d], k);
      hi[d] = max(hi[d], k);
    }
  }
  for (int d = 0; d < 3; ++d) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
  }
  b = __any_sync(0xffffffffu, b);
  if ((threadIdx.x & 31) == 0) {
    for (int d = 0; d < 3; ++d) {
      atomicMin(mn + d, lo[d]);
      atomicMax(mx + d, hi[d]);
    }
    if (b) atomicOr(bad, 1);
  }
}

__global__ void k_kick_drift(double* __restrict__ x, double* __restrict__ p,
                             const double* __restrict__ f, int64_t n3, double kick, double drift) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= n3) return;
  const double pn = p[t] + kick * f[t];
  p[t] = pn;
  if (drift != 0.0) x[t] += drift * pn;
}

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, int64_t n3, double a) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t < n3) y[t] += a * x[t];
}

__global__ void k_scale(double* __restrict__ y, const double* __restrict__ x, int64_t n3, double a) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t < n3) y[t] = a * x[t];
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sums of K values per particle over the particles, in a fixed order: block b adds a fixed
// stride of particles and reduces them in a fixed tree into part[b][0..K); k_part_combine then
// adds the kEmitBlocks parts in order. No atomics: the emittance is reproducible run to run.
template <int K, typename F>
__device__ void block_sums(F get, int64_t n, double* __restrict__ part) {
  double s[K];
  for (int k = 0; k < K; ++k) s[k] = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    get(i, s);
  __shared__ double ws[K][kThreads / 32];
  for (int k = 0; k < K; ++k) {
    const double v = warp_sum(s[k]);
    if ((threadIdx.x & 31) == 0) ws[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) v += ws[threadIdx.x][w];
    part[blockIdx.x * 16 + threadIdx.x] = v;
  }
}

// red[k0 + k] = sum over blocks of part[b][k0 + k], k < K, in block order
__global__ void k_part_combine(const double* __restrict__ part, int nb, int k0, int K,
                               double* __restrict__ red) {
  const int k = threadIdx.x;
  if (k >= K) return;
  double v = 0.0;
  for (int b = 0; b < nb; ++b) v += part[b * 16 + k0 + k];
  red[k0 + k] = v;
}

__global__ void k_mom_first(const double* __restrict__ x, const double* __restrict__ p, int64_t n,
                            double* __restrict__ part) {
  block_sums<6>(
      [&](int64_t i, double* s) {
        for (int d = 0; d < 3; ++d) {
          s[d] += x[3 * i + d];
          s[3 + d] += p[3 * i + d];
        }
      },
      n, part);
}

// centred second moments <du^2>, <dp^2>, <du dp> per axis into part[b][6..15)
__global__ void k_mom_second(const double* __restrict__ x, const double* __restrict__ p, int64_t n,
                             const double* __restrict__ red, double* __restrict__ part) {
  const double inv = 1.0 / static_cast<double>(n);
  const double mx[3] = {red[0] * inv, red[1] * inv, red[2] * inv};
  const double mp[3] = {red[3] * inv, red[4] * inv, red[5] * inv};
  block_sums<9>(
      [&](int64_t i, double* s) {
        for (int d = 0; d < 3; ++d) {
          const double du = x[3 * i + d] - mx[d], dp = p[3 * i + d] - mp[d];
          s[3 * d] += du * du;
          s[3 * d + 1] += dp * dp;
          s[3 * d + 2] += du * dp;
        }
      },
      n, part + 6);
}

__global__ void k_emit_finish(const double* __restrict__ red, int64_t n, double mc,
                              double* __restrict__ eps3) {
  const int d = threadIdx.x;
  if (d >= 3) return;
  const double inv = 1.0 / static_cast<double>(n);
  const double a = red[6 + 3 * d] * inv, b = red[7 + 3 * d] * inv, c = red[8 + 3 * d] * inv;
  eps3[d] = sqrt(fmax(a * b - c * c, 0.0)) / mc;
}

// gradient of sum_u eps_u: (du <dp^2> - dp <du dp>) / (N (M c)^2 eps) and the p counterpart
__global__ void k_emit_grad(const double* __restrict__ x, const double* __restrict__ p, int64_t n,
                            const double* __restrict__ red, double mc, double* __restrict__ gx,
                            double* __restrict__ gp) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= 3 * n) return;
  const int d = static_cast<int>(t % 3);
  const double inv = 1.0 / static_cast<double>(n);
  const double a = red[6 + 3 * d] * inv, b = red[7 + 3 * d] * inv, c = red[8 + 3 * d] * inv;
  const double eps = sqrt(fmax(a * b - c * c, 0.0)) / mc;
  const double den = static_cast<double>(n) * mc * mc * eps;
  const double du = x[t] - red[d] * inv, dp = p[t] - red[3 + d] * inv;
  if (gx) gx[t] = den > 0.0 ? (du * b - dp * c) / den : 0.0;
  if (gp) gp[t] = den > 0.0 ? (dp * a - du * c) / den : 0.0;
}

__global__ void k_energy_out(const double* __restrict__ acc, double pp_scale, double pm_scale,
                             double* __restrict__ energy) {
  if (threadIdx.x == 0) {
    energy[0] = pp_scale * acc[0];
    energy[1] = pm_scale * acc[1];
  }
}

// FP32 throughput probe: every thread runs 8 independent chains of fused multiply-adds
// a <- a b + c (packed: two lanes of a float2 per instruction). Nothing depends on memory, so the
// launch measures the FMA pipe alone. The chains' sum is written only in a case that cannot
// occur (|a| stays below 2 for b < 1, c small), which keeps the compiler from dropping them.
__device__ float g_probe_sink;

template <bool kPacked>
__global__ void __launch_bounds__(256) k_fma_probe(int iters) {
  const float b = 0.9999f, c = 1e-4f;
  float s = 0.f;
  if constexpr (kPacked) {
    float2 a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = make_float2(1e-3f * u, 2e-3f * threadIdx.x);
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll 4
    for (int k = 0; k < iters; ++k)
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = __ffma2_rn(a[u], b2, c2);
#pragma unroll
    for (int u = 0; u < 8; ++u) s += a[u].x + a[u].y;
  } else {
    float a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = 1e-3f * u + 2e-3f * threadIdx.x;
#pragma unroll 4
    for (int k = 0; k < iters; ++k)
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = fmaf(a[u], b, c);
#pragma unroll
    for (int u = 0; u < 8; ++u) s += a[u];
  }
  if (s == 1234567.f) g_probe_sink = s;
}

}  // namespace

void launch_bbox(const double* x, int64_t n, double* red, cudaStream_t s) {
  auto* mn = reinterpret_cast<unsigned long long*>(red);
  auto* mx = mn + 3;
  int* bad = reinterpret_cast<int*>(red + 6);
  cudaMemsetAsync(mn, 0xff, 3 * sizeof(unsigned long long), s);
  cudaMemsetAsync(mx, 0x00, 3 * sizeof(unsigned long long), s);
  cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (n > 0)
    k_bbox<<<static_cast<unsigned>(std::min<int64_t>(blocks_for(n), 1216)), kThreads, 0, s>>>(
        x, n, mn, mx, bad);
}

void launch_kick_drift(double* x, double* p, const double* f, int64_t n, double kick, double drift,
                       cudaStream_t s) {
  if (n > 0) k_kick_drift<<<blocks_for(3 * n), kThreads, 0, s>>>(x, p, f, 3 * n, kick, drift);
}

void launch_axpy(double* y, const double* x, int64_t n3, double a, cudaStream_t s) {
  if (n3 > 0) k_axpy<<<blocks_for(n3), kThreads, 0, s>>>(y, x, n3, a);
}

void launch_scale(double* y, const double* x, int64_t n3, double a, cudaStream_t s) {
  if (n3 > 0) k_scale<<<blocks_for(n3), kThreads, 0, s>>>(y, x, n3, a);
}

void launch_emittance(const double* x, const double* p, int64_t n, double mc, double* eps3,
                      double* gx, double* gp, double* part, double* red, cudaStream_t s) {
  const int blocks = static_cast<int>(std::min<int64_t>(blocks_for(n), kEmitBlocks));
  k_mom_first<<<blocks, kThreads, 0, s>>>(x, p, n, part);
  k_part_combine<<<1, 32, 0, s>>>(part, blocks, 0, 6, red);
  k_mom_second<<<blocks, kThreads, 0, s>>>(x, p, n, red, part);
  k_part_combine<<<1, 32, 0, s>>>(part, blocks, 6, 9, red);
  if (eps3) k_emit_finish<<<1, 32, 0, s>>>(red, n, mc, eps3);
  if (gx || gp) k_emit_grad<<<blocks_for(3 * n), kThreads, 0, s>>>(x, p, n, red, mc, gx, gp);
}

void launch_energy_out(const p3m_ctx* c, double* energy) {
  // short range: (1/2) q sum_i phi^S_i with phi^S in units k_e q / r_c;
  // long range: (1/2) q sum_m W[m] phi[m] (W = assignment weights, phi in volts)
  const double pp_scale = 0.5 * c->g.ke * c->g.q * c->g.q / c->g.rc;
  const double pm_scale = 0.5 * c->g.q;
  k_energy_out<<<1, 32, 0, c->work>>>(c->energy_acc, pp_scale, pm_scale, energy);
}

}  // namespace p3m

extern "C" p3m_status p3m_fp32_probe(int32_t packed, int32_t iters, double* flops, void* stream) {
  if (!flops || iters < 1) return P3M_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return P3M_ECUDA;
  const unsigned blocks = static_cast<unsigned>(sms) * 8u;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (packed)
    p3m::k_fma_probe<true><<<blocks, 256, 0, st>>>(iters);
  else
    p3m::k_fma_probe<false><<<blocks, 256, 0, st>>>(iters);
  // 8 chains per thread, one FMA (2 flops) per chain and step, two lanes when packed
  *flops = static_cast<double>(blocks) * 256.0 * iters * 8.0 * 2.0 * (packed ? 2.0 : 1.0);
  return cudaGetLastError() == cudaSuccess ? P3M_OK : P3M_ECUDA;
}
