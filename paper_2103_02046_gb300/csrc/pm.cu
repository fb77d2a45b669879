// Long-range (particle-mesh) half of P3M: charge assignment, Green's-function convolution on the
// doubled mesh (free space plus the planar-cathode image term), and interpolation of the force.
//
//  * assignment (eq. (rho_L), W = W^L): TSC (one order above the paper's cloud-in-cell
//    example, eq. (interpolation_splines_b0)) or CIC, accumulated with atomics;
//  * solve (eq. (phi_L) with eq. (GreenFunc_planar_cathode)):
//      phi = k_e [ K_f (*) Q  -  K_i (*) Q_rev ],  Q_rev[., ., j] = Q[., ., n_z - 1 - j],
//    where K_i samples G^L at the image offsets (x_g - S(x_g')); in Fourier space the reversed
//    charge is a phase times the spectrum at -k_z, so both terms share one forward transform;
//  * force (eq. (eom_p3m_coord), first term) with the analytic derivative of W.
//
// FP32 path: the mesh potential of a bunch is a few hundred times larger than its differences
// between neighbouring nodes, so differencing an FP32 potential would lose ~1e-5 of the force.
// The FP32 path therefore convolves Q with the three forward-difference kernels
// K(m + e_d) - K(m) (a factor e^{2 pi i k_d / M_d} - 1 in Fourier space) and assembles the
// analytic-derivative force from the difference fields D_d = phi(g + e_d) - phi(g) by
// summation by parts:
//   sum_a phi_a dw(a) = (1/2 - u) D_{c-1} + (1/2 + u) D_c   (TSC),   = D_c   (CIC).
// This is the same discrete force; only the rounding moves from phi to its differences.
#include <cmath>
#include <type_traits>

#include "p3m_internal.cuh"

namespace p3m {
namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(uint64_t n, int t = kThreads) {
  return static_cast<unsigned>((n + t - 1) / t);
}


// ---------------------------------------------------------------------------------------------
// Green's-function spectra (built once per geometry, in FP64)
// ---------------------------------------------------------------------------------------------
__global__ void k_sample_kernel(Geom g, double* __restrict__ out, int image) {
  const size_t total = static_cast<size_t>(g.M[0]) * g.M[1] * g.M[2];
  const size_t idx = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (idx >= total) return;
  const int ix = static_cast<int>(idx % g.M[0]);
  const int iy = static_cast<int>((idx / g.M[0]) % g.M[1]);
  const int iz = static_cast<int>(idx / (static_cast<size_t>(g.M[0]) * g.M[1]));
  if (ix == g.n[0] || iy == g.n[1] || iz == g.n[2]) {  // the one offset never used
    out[idx] = 0.0;
    return;
  }
  const int mx = ix < g.n[0] ? ix : ix - g.M[0];
  const int my = iy < g.n[1] ? iy : iy - g.M[1];
  const int mz = iz < g.n[2] ? iz : iz - g.M[2];
  const double X = mx * g.h[0], Y = my * g.h[1];
  double Z;
  if (image) {
    const double d = g.lo[2] - g.zc;
    Z = 2.0 * d + static_cast<double>(mz + g.n[2] - 1) * g.h[2];
  } else {
    Z = mz * g.h[2];
  }
  const double r = sqrt(X * X + Y * Y + Z * Z);
  out[idx] = r > 0.0 ? erf(g.alpha * r) / r : 2.0 * g.alpha * 0.56418958354775628695;  // 1/sqrt(pi)
}

__device__ double infl_factor(const Geom& g, int kx, int ky, int kz) {
  // 1 / U(k)^2 with U = prod_d sinc(pi kappa_d / M_d)^(order + 1)
  const int kk[3] = {kx, ky < g.M[1] / 2 + 1 ? ky : ky - g.M[1], kz < g.M[2] / 2 + 1 ? kz : kz - g.M[2]};
  double U = 1.0;
  for (int d = 0; d < 3; ++d) {
    const double t = static_cast<double>(kk[d]) / g.M[d];
    const double s = (kk[d] == 0) ? 1.0 : sinpi(t) / (3.14159265358979323846 * t);
    double p = 1.0;
    for (int o = 0; o <= g.order; ++o) p *= s;
    U *= p;
  }
  return 1.0 / (U * U);
}

// Optimal influence function of eq. (Ghfinal) with its alias sums, as a factor on the sampled
// kernel spectra: sum_m U^2(k_m) R(k_m) / [R(k) (sum_m U^2(k_m))^2], k_m = k + 2 pi m / h,
// |m_d| <= 2, U = prod_d sinc(k_d h_d / 2)^(order + 1), R(k) = e^{-k^2 / (4 alpha^2)} / k^2;
// 1 at k = 0. Computed once per context, in FP64.
constexpr int kAlias = 2;
__device__ double alias_factor(const Geom& g, int kx, int ky, int kz) {
  const int kk[3] = {kx, ky < g.M[1] / 2 + 1 ? ky : ky - g.M[1],
                     kz < g.M[2] / 2 + 1 ? kz : kz - g.M[2]};
  if (kk[0] == 0 && kk[1] == 0 && kk[2] == 0) return 1.0;
  const double pi = 3.14159265358979323846;
  const double inv4a2 = 1.0 / (4.0 * g.alpha * g.alpha);
  double a[3][2 * kAlias + 1], q2[3][2 * kAlias + 1], den = 1.0;
  for (int d = 0; d < 3; ++d) {
    double su = 0.0;
    for (int m = -kAlias; m <= kAlias; ++m) {
      const double t = static_cast<double>(kk[d]) / g.M[d] + m;
      const double sc = (t == 0.0) ? 1.0 : sinpi(t) / (pi * t);
      double u2 = 1.0;
      for (int o = 0; o <= g.order; ++o) u2 *= sc * sc;
      const double q = 2.0 * pi * t / g.h[d];
      q2[d][m + kAlias] = q * q;
      a[d][m + kAlias] = u2 * exp(-q * q * inv4a2);
      su += u2;
    }
    den *= su;
  }
  double num = 0.0;
  for (int mz = 0; mz <= 2 * kAlias; ++mz)
    for (int my = 0; my <= 2 * kAlias; ++my)
      for (int mx = 0; mx <= 2 * kAlias; ++mx) {
        const double qq = q2[0][mx] + q2[1][my] + q2[2][mz];  // > 0 since k != 0
        num += a[0][mx] * a[1][my] * a[2][mz] / qq;
      }
  const double qk = q2[0][kAlias] + q2[1][kAlias] + q2[2][kAlias];
  return num * qk / (exp(-qk * inv4a2) * den * den);
}

template <typename T>
__global__ void k_finish_kernels(Geom g, const double2* __restrict__ Sf,
                                 const double2* __restrict__ Si, T* __restrict__ kf,
                                 typename std::conditional<sizeof(T) == 4, float2, double2>::type* __restrict__ ki,
                                 double scale, int influence) {
  const int Hx = g.M[0] / 2 + 1;
  const size_t total = static_cast<size_t>(Hx) * g.M[1] * g.M[2];
  const size_t idx = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (idx >= total) return;
  const int kx = static_cast<int>(idx % Hx);
  const int ky = static_cast<int>((idx / Hx) % g.M[1]);
  const int kz = static_cast<int>(idx / (static_cast<size_t>(Hx) * g.M[1]));
  double sc = scale;
  if (influence == 1) sc *= infl_factor(g, kx, ky, kz);
  if (influence == 2) sc *= alias_factor(g, kx, ky, kz);
  kf[idx] = static_cast<T>(Sf[idx].x * sc);  // the free kernel is even in every axis: real spectrum
  if (Si) {
    // fold the phase of the z-reversal: Qrev^(k) = e^{-2 pi i kz (nz - 1)/Mz} Q^(kx, ky, -kz)
    const long long t = (2LL * kz * (g.n[2] - 1)) % (2LL * g.M[2]);
    double sn, cs;
    sincospi(-static_cast<double>(t) / g.M[2], &sn, &cs);
    const double2 a = Si[idx];
    ki[idx].x = static_cast<T>((a.x * cs - a.y * sn) * sc);
    ki[idx].y = static_cast<T>((a.x * sn + a.y * cs) * sc);
  }
}

// ---------------------------------------------------------------------------------------------
// Charge assignment
// ---------------------------------------------------------------------------------------------
template <typename T>
struct Axis {
  int c;     // first node of the weight support
  T w[3];    // weights on nodes c .. c+S-1
  T dw[3];   // d/ds of the weights
  T gl, gr;  // coefficients of D_{c0-1} and D_{c0} in sum_a phi_a dw(a) (TSC: c0 = c+1)
};

template <typename T>
__device__ __forceinline__ Axis<T> axis_weights(int order, int c, T f) {
  // c: TSC nearest node (f = s - c in [-1/2, 1/2]) or CIC lower node (f in [0, 1))
  Axis<T> a;
  if (order == 2) {
    a.c = c - 1;
    const T l = T(0.5) - f, r = T(0.5) + f;
    a.w[0] = T(0.5) * l * l;
    a.w[1] = T(0.75) - f * f;
    a.w[2] = T(0.5) * r * r;
    a.dw[0] = -l;
    a.dw[1] = T(-2) * f;
    a.dw[2] = r;
    a.gl = l;
    a.gr = r;
  } else {
    a.c = c;
    a.w[0] = T(1) - f;
    a.w[1] = f;
    a.w[2] = T(0);
    a.dw[0] = T(-1);
    a.dw[1] = T(1);
    a.dw[2] = T(0);
    a.gl = T(0);
    a.gr = T(1);
  }
  return a;
}

// FP32 path: the assignment node and offset per axis, recomputed from the 32-byte position
// record (hi + lo in cutoff units) in double-float arithmetic exactly as the sort did, plus the
// sort's correction near knots (see kRowBits).
__device__ __forceinline__ void particle_axes(const Geom& g, const float4* __restrict__ recp,
                                              uint32_t i, Axis<float> ax[3]) {
  float4 h, l;
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(h.x), "=f"(h.y), "=f"(h.z), "=f"(h.w), "=f"(l.x), "=f"(l.y), "=f"(l.z), "=f"(l.w)
      : "l"(recp + 2 * static_cast<size_t>(i)));
  const uint32_t code = __float_as_uint(l.w) >> kRowBits;
  const float hs[3] = {h.x, h.y, h.z}, ls[3] = {l.x, l.y, l.z};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const DF sm = df_mul(DF{hs[d], ls[d]}, g.rch_df[d]);
    const float cf = (g.order == 2) ? floorf(sm.hi + 0.5f) : floorf(sm.hi);
    const float c = cf + static_cast<float>(static_cast<int>((code >> (2 * d)) & 3u) - 1);
    const float u = __fadd_rn(__fsub_rn(sm.hi, c), sm.lo);  // sm.hi - c is exact
    ax[d] = axis_weights<float>(g.order, static_cast<int>(c), u);
  }
}

// FP64 path: offsets and packed node from the assignment record.
__device__ __forceinline__ void particle_axes(const Geom& g, const Rec64* __restrict__ recm,
                                              uint32_t i, Axis<double> ax[3]) {
  const Rec64 r = recm[i];
  const uint32_t node = static_cast<uint32_t>(r.idx);
  ax[0] = axis_weights<double>(g.order, static_cast<int>(node & 1023u), r.u[0]);
  ax[1] = axis_weights<double>(g.order, static_cast<int>((node >> 10) & 1023u), r.u[1]);
  ax[2] = axis_weights<double>(g.order, static_cast<int>(node >> 20), r.u[2]);
}

__device__ __forceinline__ long long orig_index(const float4* recp, uint32_t i) {
  return __float_as_int(recp[2 * i].w);  // FP32 records: hi at 2i carries the index
}
__device__ __forceinline__ long long orig_index(const Rec64* recp, uint32_t i) {
  return recp[i].idx;
}

// ---------------------------------------------------------------------------------------------
// Charge assignment with a shared-memory tile: a block takes kDepPerBlock consecutive sorted
// particles (one stretch of an x-row of cells, so their supports overlap heavily), sums their
// weights into a tile of the mesh covering the block's bounding box, then adds the non-zero tile
// entries to the mesh with one global atomic each. Blocks whose box does not fit the tile fall
// back to global atomics per weight.
// ---------------------------------------------------------------------------------------------
constexpr int kDepThreads = 256;
constexpr int kDepItems = 4;
constexpr int kDepPerBlock = kDepThreads * kDepItems;
constexpr int kTileBytes = 32768;

template <typename T, bool kDipole>
__global__ void __launch_bounds__(kDepThreads)
    k_deposit_tiled(Geom g, const uint32_t* __restrict__ total,
                    const typename RecT<T>::type* __restrict__ recm,
                    const typename RecT<T>::type* __restrict__ recp,
                    const double* __restrict__ w, T* __restrict__ qpad) {
  // FP32 charge deposit: the tile accumulates in unsigned 32-bit fixed point, because integer
  // shared-memory atomics are native while float ones are compare-and-swap loops. A tile node
  // receives at most one weight from each of the block's 1024 particles: at most 27/64 with TSC
  // (2^23 per unit of weight keeps the sum below 1024 * 27/64 * 2^23 < 2^32) and at most 1 with
  // CIC (2^21 per unit: below 2^31). Sums inside a tile are then exact and independent of the
  // order of the particles.
  constexpr bool kFixed = (sizeof(T) == 4) && !kDipole;
  using Slot = typename std::conditional<kFixed, unsigned int, T>::type;
  constexpr int kTile = kTileBytes / sizeof(Slot);
  __shared__ Slot tile[kTile];
  __shared__ int bmin[3], bmax[3];
  const uint32_t N = *total;
  const uint32_t b0 = blockIdx.x * kDepPerBlock;
  if (b0 >= N) return;
  const int S = g.order == 2 ? 3 : 2;
  const float fix_scale = g.order == 2 ? 8388608.0f : 2097152.0f;
  const float fix_inv = 1.0f / fix_scale;
  if (threadIdx.x < 3) {
    bmin[threadIdx.x] = 1 << 30;
    bmax[threadIdx.x] = -1;
  }
  __syncthreads();
  int lmin[3] = {1 << 30, 1 << 30, 1 << 30}, lmax[3] = {-1, -1, -1};
#pragma unroll
  for (int k = 0; k < kDepItems; ++k) {
    const uint32_t i = b0 + k * kDepThreads + threadIdx.x;
    if (i < N) {
      Axis<T> ax[3];
      particle_axes(g, recm, i, ax);
      for (int d = 0; d < 3; ++d) {
        lmin[d] = min(lmin[d], ax[d].c);
        lmax[d] = max(lmax[d], ax[d].c + S - 1);
      }
    }
  }
  for (int d = 0; d < 3; ++d) {
    int a = lmin[d], b = lmax[d];
    for (int o = 16; o > 0; o >>= 1) {
      a = min(a, __shfl_xor_sync(0xffffffffu, a, o));
      b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&bmin[d], a);
      atomicMax(&bmax[d], b);
    }
  }
  __syncthreads();
  const int ex = bmax[0] - bmin[0] + 1, ey = bmax[1] - bmin[1] + 1, ez = bmax[2] - bmin[2] + 1;
  const bool use_tile = static_cast<long long>(ex) * ey * ez <= kTile;
  if (use_tile)
    for (int t = threadIdx.x; t < ex * ey * ez; t += kDepThreads) tile[t] = Slot(0);
  __syncthreads();
  for (int k = 0; k < kDepItems; ++k) {
    const uint32_t i = b0 + k * kDepThreads + threadIdx.x;
    if (i >= N) continue;
    Axis<T> A[3];
    particle_axes(g, recm, i, A);
    T wv[3] = {T(0), T(0), T(0)};
    if (kDipole) {
      const long long idx = orig_index(recp, i);
      for (int d = 0; d < 3; ++d) wv[d] = static_cast<T>(w[3 * idx + d] * g.inv_h[d]);
    }
    for (int c = 0; c < S; ++c)
      for (int b = 0; b < S; ++b)
        for (int a = 0; a < S; ++a) {
          T v;
          if (kDipole)
            v = wv[0] * A[0].dw[a] * A[1].w[b] * A[2].w[c] +
                wv[1] * A[0].w[a] * A[1].dw[b] * A[2].w[c] +
                wv[2] * A[0].w[a] * A[1].w[b] * A[2].dw[c];
          else
            v = A[0].w[a] * A[1].w[b] * A[2].w[c];
          const int gx = A[0].c + a, gy = A[1].c + b, gz = A[2].c + c;
          if (use_tile) {
            Slot* slot = &tile[((gz - bmin[2]) * ey + (gy - bmin[1])) * ex + (gx - bmin[0])];
            if constexpr (kFixed)
              atomicAdd(slot, __float2uint_rn(static_cast<float>(v) * fix_scale));
            else
              atomicAdd(slot, v);
          } else
            atomicAdd(qpad + real_index(g, gx, gy, gz), v);
        }
  }
  if (!use_tile) return;
  __syncthreads();
  for (int t = threadIdx.x; t < ex * ey * ez; t += kDepThreads) {
    T v;
    if constexpr (kFixed)
      v = static_cast<T>(static_cast<float>(tile[t]) * fix_inv);
    else
      v = tile[t];
    if (v != T(0)) {
      const int gx = bmin[0] + t % ex, gy = bmin[1] + (t / ex) % ey, gz = bmin[2] + t / (ex * ey);
      atomicAdd(qpad + real_index(g, gx, gy, gz), v);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Deterministic charge assignment (deterministic = 1, FP64 path): every weight is added to its
// node as a 128-bit fixed-point integer (two 64-bit words, the carry taken from the low word's
// returned old value), so the node sums are exact and independent of the order of the adds.
// The charge weights lie in [0, 1] and use 62 fractional bits; the dipole deposit of the adjoint
// scales by 2^(61 - e), with 2^e above the largest |w_i|_1 / h of this call, found first by a
// max reduction (an order-free operation). A node sum of up to 2^31 weights stays below 2^93.
// ---------------------------------------------------------------------------------------------
constexpr int kDetBlocks = 1024;  // fixed grid of the deterministic reductions

__device__ __forceinline__ void add128(unsigned long long* acc, long long v) {
  const unsigned long long lo = static_cast<unsigned long long>(v);
  const unsigned long long old = atomicAdd(acc, lo);
  const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  atomicAdd(acc + 1, (v < 0 ? ~0ull : 0ull) + carry);
}

// largest sum_d |w_d| / h_d over the particles (non-negative doubles order as their bits)
__global__ void k_dipole_bound(Geom g, const uint32_t* __restrict__ total,
                               const Rec64* __restrict__ recp, const double* __restrict__ w,
                               unsigned long long* __restrict__ bound) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  double b = 0.0;
  if (i < *total) {
    const long long idx = recp[i].idx;
    for (int d = 0; d < 3; ++d) b += fabs(w[3 * idx + d]) * g.inv_h[d];
  }
  for (int o = 16; o > 0; o >>= 1) b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  if ((threadIdx.x & 31) == 0 && b > 0.0)
    atomicMax(bound, static_cast<unsigned long long>(__double_as_longlong(b)));
}

__device__ __forceinline__ double det_scale(bool dipole, const unsigned long long* bound) {
  if (!dipole) return 4611686018427387904.0;  // 2^62
  const double b = __longlong_as_double(static_cast<long long>(*bound));
  if (!(b > 0.0)) return 1.0;
  return ldexp(1.0, 61 - (ilogb(b) + 1));
}

template <bool kDipole>
__global__ void k_deposit_det(Geom g, const uint32_t* __restrict__ total,
                              const Rec64* __restrict__ recm, const Rec64* __restrict__ recp,
                              const double* __restrict__ w,
                              const unsigned long long* __restrict__ bound,
                              unsigned long long* __restrict__ q128) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *total) return;
  const int S = g.order == 2 ? 3 : 2;
  const double scale = det_scale(kDipole, bound);
  Axis<double> A[3];
  particle_axes(g, recm, i, A);
  double wv[3] = {0.0, 0.0, 0.0};
  if (kDipole) {
    const long long idx = recp[i].idx;
    for (int d = 0; d < 3; ++d) wv[d] = w[3 * idx + d] * g.inv_h[d];
  }
  for (int c = 0; c < S; ++c)
    for (int b = 0; b < S; ++b)
      for (int a = 0; a < S; ++a) {
        double v;
        if (kDipole)
          v = wv[0] * A[0].dw[a] * A[1].w[b] * A[2].w[c] +
              wv[1] * A[0].w[a] * A[1].dw[b] * A[2].w[c] +
              wv[2] * A[0].w[a] * A[1].w[b] * A[2].dw[c];
        else
          v = A[0].w[a] * A[1].w[b] * A[2].w[c];
        const size_t node = (static_cast<size_t>(A[2].c + c) * g.n[1] + (A[1].c + b)) * g.n[0] +
                            (A[0].c + a);
        add128(q128 + 2 * node, __double2ll_rn(v * scale));
      }
}

// the exact 128-bit node sums, rounded to FP64, into the doubled mesh's n^3 block
template <bool kDipole>
__global__ void k_q128_to_mesh(Geom g, const unsigned long long* __restrict__ q128,
                               const unsigned long long* __restrict__ bound,
                               double* __restrict__ qpad) {
  const size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  const size_t nn = static_cast<size_t>(g.n[0]) * g.n[1] * g.n[2];
  if (t >= nn) return;
  const unsigned long long lo = q128[2 * t];
  const long long hi = static_cast<long long>(q128[2 * t + 1]);
  const double v = static_cast<double>(hi) * 18446744073709551616.0 + static_cast<double>(lo);
  const int gx = static_cast<int>(t % g.n[0]);
  const int gy = static_cast<int>((t / g.n[0]) % g.n[1]);
  const int gz = static_cast<int>(t / (static_cast<size_t>(g.n[0]) * g.n[1]));
  qpad[real_index(g, gx, gy, gz)] = v / det_scale(kDipole, bound);
}

// Fixed-order sums for the deterministic energies: each block adds a fixed stride of the terms
// and reduces them in a fixed tree into part[block]; one block then adds the parts in order.
__device__ __forceinline__ double block_tree_sum(double v) {
  __shared__ double ws[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < kThreads / 32; ++k) r += ws[k];
  __syncthreads();
  return r;
}

__global__ void k_det_part_pp(const uint32_t* __restrict__ total, const D4* __restrict__ fpp,
                              double* __restrict__ part) {
  const uint32_t N = *total;
  double s = 0.0;
  for (uint32_t i = blockIdx.x * kThreads + threadIdx.x; i < N; i += kDetBlocks * kThreads)
    s += fpp[i].w;
  const double r = block_tree_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

__global__ void k_det_part_mesh(Geom g, const double* __restrict__ qpad,
                                const double* __restrict__ phi, double* __restrict__ part) {
  const size_t nn = static_cast<size_t>(g.n[0]) * g.n[1] * g.n[2];
  double s = 0.0;
  for (size_t t = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; t < nn;
       t += static_cast<size_t>(kDetBlocks) * kThreads) {
    const int gx = static_cast<int>(t % g.n[0]);
    const int gy = static_cast<int>((t / g.n[0]) % g.n[1]);
    const int gz = static_cast<int>(t / (static_cast<size_t>(g.n[0]) * g.n[1]));
    const size_t r = real_index(g, gx, gy, gz);
    s += qpad[r] * phi[r];
  }
  const double r = block_tree_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

__global__ void k_det_combine(const double* __restrict__ part, double* __restrict__ out) {
  double s = 0.0;
  for (int k = threadIdx.x; k < kDetBlocks; k += kThreads) s += part[k];
  const double r = block_tree_sum(s);
  if (threadIdx.x == 0) *out = r;
}

// ---------------------------------------------------------------------------------------------
// Spectral multiply: base(k) = Kf(k) Q(k) - Ki(k) Q(kx, ky, -kz); outputs the potential
// spectrum and/or the three difference spectra; accumulates sum_m W[m] phi[m] by Parseval.
// ---------------------------------------------------------------------------------------------
template <typename T>
using C2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;

template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  C2<T> r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

template <typename T>
__global__ void k_green_multiply(Geom g, const C2<T>* __restrict__ qhat, const T* __restrict__ kf,
                                 const C2<T>* __restrict__ ki, const float2* __restrict__ dfac,
                                 C2<T>* __restrict__ dhat, C2<T>* __restrict__ phihat,
                                 double* __restrict__ energy, size_t ncplx) {
  const int Hx = g.M[0] / 2 + 1;
  const int Mz = g.M[2];
  // grid: x covers the (kx, ky) plane with 32-bit indices, y is kz in [0, Mz/2]
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool inside = t < static_cast<uint32_t>(Hx) * static_cast<uint32_t>(g.M[1]);
  double e = 0.0;
  if (inside) {
    const int kx = static_cast<int>(t % static_cast<uint32_t>(Hx));
    const int ky = static_cast<int>(t / static_cast<uint32_t>(Hx));
    const int kz = blockIdx.y;
    const int kz2 = (Mz - kz) % Mz;
    const size_t ia = (static_cast<size_t>(kz) * g.M[1] + ky) * Hx + kx;
    const size_t ib = (static_cast<size_t>(kz2) * g.M[1] + ky) * Hx + kx;
    const C2<T> a = qhat[ia], b = qhat[ib];
    C2<T> ba, bb;
    ba.x = kf[ia] * a.x;
    ba.y = kf[ia] * a.y;
    bb.x = kf[ib] * b.x;
    bb.y = kf[ib] * b.y;
    if (ki) {
      const C2<T> ta = cmul<T>(ki[ia], b), tb = cmul<T>(ki[ib], a);
      ba.x -= ta.x;
      ba.y -= ta.y;
      bb.x -= tb.x;
      bb.y -= tb.y;
    }
    if (energy) {
      const T wx = (kx == 0 || 2 * kx == g.M[0]) ? T(1) : T(2);
      T ee = wx * (a.x * ba.x + a.y * ba.y);
      if (kz2 != kz) ee += wx * (b.x * bb.x + b.y * bb.y);
      e = static_cast<double>(ee);
    }
    if (phihat) {
      phihat[ia] = ba;
      if (kz2 != kz) phihat[ib] = bb;
    }
    if (dhat) {
      const float2* fx = dfac;
      const float2* fy = dfac + Hx;
      const float2* fz = dfac + Hx + g.M[1];
      C2<T> f;
      f.x = fx[kx].x; f.y = fx[kx].y;
      dhat[ia] = cmul<T>(ba, f);
      f.x = fy[ky].x; f.y = fy[ky].y;
      dhat[ncplx + ia] = cmul<T>(ba, f);
      f.x = fz[kz].x; f.y = fz[kz].y;
      dhat[2 * ncplx + ia] = cmul<T>(ba, f);
      if (kz2 != kz) {
        f.x = fx[kx].x; f.y = fx[kx].y;
        dhat[ib] = cmul<T>(bb, f);
        f.x = fy[ky].x; f.y = fy[ky].y;
        dhat[ncplx + ib] = cmul<T>(bb, f);
        f.x = fz[kz2].x; f.y = fz[kz2].y;
        dhat[2 * ncplx + ib] = cmul<T>(bb, f);
      }
    }
  }
  if (energy) {
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    __shared__ double ws[kThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x < 32) {
      double v = threadIdx.x < kThreads / 32 ? ws[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (threadIdx.x == 0) atomicAdd(energy, v);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Interpolation of the long-range force and combination with the short-range force
// ---------------------------------------------------------------------------------------------
// FP32: from the forward-difference fields D_d (volts).
__device__ __forceinline__ void grad_from_diff(const Geom& g, const float* __restrict__ D,
                                               size_t nreal, const Axis<float> ax[3], float G[3]) {
  const int S = g.order == 2 ? 3 : 2;
  const int off = g.order == 2 ? 0 : 1;  // TSC: D nodes c, c+1 (= c0-1, c0); CIC: node c only
  // x derivative
  {
    const float* Dx = D;
    float acc = 0.f;
    for (int c = 0; c < S; ++c)
      for (int b = 0; b < S; ++b) {
        const float wyz = ax[1].w[b] * ax[2].w[c];
        const size_t r = real_index(g, ax[0].c, ax[1].c + b, ax[2].c + c);
        acc += wyz * (ax[0].gl * Dx[r] * (1 - off) + ax[0].gr * Dx[r + 1 - off]);
      }
    G[0] = acc;
  }
  {
    const float* Dy = D + nreal;
    float acc = 0.f;
    for (int c = 0; c < S; ++c)
      for (int a = 0; a < S; ++a) {
        const float wxz = ax[0].w[a] * ax[2].w[c];
        const float lo = off ? 0.f : Dy[real_index(g, ax[0].c + a, ax[1].c, ax[2].c + c)];
        const float hi = Dy[real_index(g, ax[0].c + a, ax[1].c + 1 - off, ax[2].c + c)];
        acc += wxz * (ax[1].gl * lo + ax[1].gr * hi);
      }
    G[1] = acc;
  }
  {
    const float* Dz = D + 2 * nreal;
    float acc = 0.f;
    for (int b = 0; b < S; ++b)
      for (int a = 0; a < S; ++a) {
        const float wxy = ax[0].w[a] * ax[1].w[b];
        const float lo = off ? 0.f : Dz[real_index(g, ax[0].c + a, ax[1].c + b, ax[2].c)];
        const float hi = Dz[real_index(g, ax[0].c + a, ax[1].c + b, ax[2].c + 1 - off)];
        acc += wxy * (ax[2].gl * lo + ax[2].gr * hi);
      }
    G[2] = acc;
  }
}

// FP64: from the potential phi (volts), analytic derivative of W.
__device__ __forceinline__ void grad_from_phi(const Geom& g, const double* __restrict__ phi,
                                              const Axis<double> ax[3], double G[3]) {
  // G_x = sum_c w_c sum_b w_b sum_a phi dw_a, and likewise for y and z, summed axis by axis
  // (sums along x per row, then along y per plane, then along z): about 90 FP64 operations per
  // particle instead of 243 for the node-by-node triple products (FP64 units are scarce here)
  const int S = g.order == 2 ? 3 : 2;
  G[0] = G[1] = G[2] = 0.0;
  for (int c = 0; c < S; ++c) {
    double ty = 0.0, tdy = 0.0, tdx = 0.0;  // sum_b of w_b sx, dw_b sx, w_b sdx
    for (int b = 0; b < S; ++b) {
      const double* row = phi + real_index(g, ax[0].c, ax[1].c + b, ax[2].c + c);
      double sx = 0.0, sdx = 0.0;  // sum_a of phi w_a, phi dw_a
      for (int a = 0; a < S; ++a) {
        const double p = row[a];
        sx = fma(p, ax[0].w[a], sx);
        sdx = fma(p, ax[0].dw[a], sdx);
      }
      ty = fma(ax[1].w[b], sx, ty);
      tdy = fma(ax[1].dw[b], sx, tdy);
      tdx = fma(ax[1].w[b], sdx, tdx);
    }
    G[0] = fma(ax[2].w[c], tdx, G[0]);
    G[1] = fma(ax[2].w[c], tdy, G[1]);
    G[2] = fma(ax[2].dw[c], ty, G[2]);
  }
}

// Central-difference field, interpolated with W (force_diff = 1): G_d = sum_g W (phi_{g+e_d} -
// phi_{g-e_d}) / 2 in mesh units (F = -q G / h as for the analytic derivative). FP32 from the
// forward differences D_d(g) = phi_{g+e_d} - phi_g, FP64 from phi.
__device__ __forceinline__ void grad_central_diff(const Geom& g, const float* __restrict__ D,
                                                  size_t nreal, const Axis<float> ax[3],
                                                  float G[3]) {
  const int S = g.order == 2 ? 3 : 2;
  const size_t stride[3] = {1, static_cast<size_t>(g.M[0]),
                            static_cast<size_t>(g.M[0]) * g.M[1]};
  G[0] = G[1] = G[2] = 0.f;
  for (int c = 0; c < S; ++c)
    for (int b = 0; b < S; ++b)
      for (int a = 0; a < S; ++a) {
        const float W = ax[0].w[a] * ax[1].w[b] * ax[2].w[c];
        const size_t r = real_index(g, ax[0].c + a, ax[1].c + b, ax[2].c + c);
        for (int d = 0; d < 3; ++d) G[d] += W * (D[d * nreal + r] + D[d * nreal + r - stride[d]]);
      }
  for (int d = 0; d < 3; ++d) G[d] *= 0.5f;
}

__device__ __forceinline__ void grad_central_phi(const Geom& g, const double* __restrict__ phi,
                                                 const Axis<double> ax[3], double G[3]) {
  const int S = g.order == 2 ? 3 : 2;
  const size_t stride[3] = {1, static_cast<size_t>(g.M[0]),
                            static_cast<size_t>(g.M[0]) * g.M[1]};
  G[0] = G[1] = G[2] = 0.0;
  for (int c = 0; c < S; ++c)
    for (int b = 0; b < S; ++b)
      for (int a = 0; a < S; ++a) {
        const double W = ax[0].w[a] * ax[1].w[b] * ax[2].w[c];
        const size_t r = real_index(g, ax[0].c + a, ax[1].c + b, ax[2].c + c);
        for (int d = 0; d < 3; ++d) G[d] += W * (phi[r + stride[d]] - phi[r - stride[d]]);
      }
  for (int d = 0; d < 3; ++d) G[d] *= 0.5;
}

template <typename T>
__global__ void k_interp(Geom g, const uint32_t* __restrict__ total,
                         const typename RecT<T>::type* __restrict__ recm,
                         const T* __restrict__ field, size_t nreal, void* __restrict__ fpp,
                         const float4* __restrict__ fplo, const float4* __restrict__ fbig,
                         int parts, float pp_scale_f, double pp_scale) {
  // F = F^L + F^S for sorted particle i, written over its short-range entry (sorted order, so
  // the writes are coalesced); k_unpermute then puts the forces in the caller's order
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *total) return;
  Axis<T> ax[3];
  particle_axes(g, recm, i, ax);
  if constexpr (sizeof(T) == 4) {
    // FP32 path: long and short range combined in FP32
    float F[3] = {0.f, 0.f, 0.f};
    if (parts & 2) {
      float G[3];
      if (g.force_diff)
        grad_central_diff(g, field, nreal, ax, G);
      else
        grad_from_diff(g, field, nreal, ax, G);
      for (int d = 0; d < 3; ++d) F[d] = g.fscale_f[d] * G[d];
    }
    float4* out = reinterpret_cast<float4*>(fpp) + i;
    if (parts & 1) {
      // the short range: coarse x, y, z with the fine z part (float4), fine x and y (float2),
      // big terms (float4)
      const float4 s = *out, b = fbig[i];
      const float2 l = reinterpret_cast<const float2*>(fplo)[i];
      F[0] = fmaf(pp_scale_f, (s.x + l.x) + b.x, F[0]);
      F[1] = fmaf(pp_scale_f, (s.y + l.y) + b.y, F[1]);
      F[2] = fmaf(pp_scale_f, (s.z + s.w) + b.z, F[2]);
    }
    *out = make_float4(F[0], F[1], F[2], 0.f);
  } else {
    double F[3] = {0.0, 0.0, 0.0};
    if (parts & 2) {
      T G[3];
      if (g.force_diff)
        grad_central_phi(g, field, ax, G);
      else
        grad_from_phi(g, field, ax, G);
      for (int d = 0; d < 3; ++d) F[d] = g.fscale[d] * static_cast<double>(G[d]);
    }
    D4* out = reinterpret_cast<D4*>(fpp) + i;
    if (parts & 1) {
      const D4 s = *out;
      F[0] += pp_scale * s.x;
      F[1] += pp_scale * s.y;
      F[2] += pp_scale * s.z;
    }
    *out = D4{F[0], F[1], F[2], 0.0};
  }
}

// f[i] = the force of input particle i, gathered from sorted order through its sorted position
// (keys[i] after the scatter); particles left out of the sort (outside the mesh) get zero.
template <typename T>
__global__ void k_unpermute(const uint32_t* __restrict__ pos, int64_t n,
                            const void* __restrict__ fsorted, double* __restrict__ f) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = pos[i];
  double F[3] = {0.0, 0.0, 0.0};
  if (k != kInvalidKey) {
    if constexpr (sizeof(T) == 4) {
      const float4 s = reinterpret_cast<const float4*>(fsorted)[k];
      F[0] = float_to_double_exact(s.x);
      F[1] = float_to_double_exact(s.y);
      F[2] = float_to_double_exact(s.z);
    } else {
      const D4 s = reinterpret_cast<const D4*>(fsorted)[k];
      F[0] = s.x;
      F[1] = s.y;
      F[2] = s.z;
    }
  }
  f[3 * i] = F[0];
  f[3 * i + 1] = F[1];
  f[3 * i + 2] = F[2];
}

// ---------------------------------------------------------------------------------------------
// Adjoint gather. pass 0: acc += -q (grad grad sum_g phi_g W) w_k   (phi of the charges)
//                 pass 1: out_k = acc - q sum_g chi_g grad W          (chi of the dipoles),
// where chi carries the factor q of the stored kernel, so -q^2 sum chi_true grad W appears as
// -q sum chi grad W.
// ---------------------------------------------------------------------------------------------
// Hessian sum_g phi_g d2W/dxi_d dxi_e in mesh units (no 1/h factors) from the difference fields.
__device__ void hess_from_diff(const Geom& g, const float* __restrict__ D, size_t nreal,
                               const Axis<float> ax[3], float H[3][3]) {
  const int S = g.order == 2 ? 3 : 2;
  const bool tsc = g.order == 2;
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < 3; ++e) H[d][e] = 0.f;
  for (int d = 0; d < 3; ++d) {
    const float* Dd = D + d * nreal;
    const int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
    // values of the d-derivative sum along the other axes' nodes
    for (int j2 = 0; j2 < S; ++j2)
      for (int j1 = 0; j1 < S; ++j1) {
        int node[3];
        node[o1] = ax[o1].c + j1;
        node[o2] = ax[o2].c + j2;
        node[d] = ax[d].c;  // TSC: c0 - 1; CIC: c
        const float D0 = Dd[real_index(g, node[0], node[1], node[2])];
        node[d] = ax[d].c + 1;
        const float D1 = tsc ? Dd[real_index(g, node[0], node[1], node[2])] : 0.f;
        const float grad = tsc ? ax[d].gl * D0 + ax[d].gr * D1 : D0;
        const float secd = tsc ? D1 - D0 : 0.f;  // phi_{c-1} - 2 phi_c + phi_{c+1}
        const float w1 = ax[o1].w[j1], w2 = ax[o2].w[j2];
        H[d][d] += secd * w1 * w2;
        H[d][o1] += grad * ax[o1].dw[j1] * w2;
        H[d][o2] += grad * w1 * ax[o2].dw[j2];
      }
  }
  // symmetrise the mixed terms (each was accumulated from both axes' difference fields)
  for (int d = 0; d < 3; ++d)
    for (int e = d + 1; e < 3; ++e) {
      const float m = 0.5f * (H[d][e] + H[e][d]);
      H[d][e] = H[e][d] = m;
    }
}

__device__ void hess_from_phi(const Geom& g, const double* __restrict__ phi,
                              const Axis<double> ax[3], double H[3][3]) {
  const int S = g.order == 2 ? 3 : 2;
  // second derivative of the 1D weights: TSC {1, -2, 1}, CIC 0
  const double d2[3] = {1.0, -2.0, 1.0};
  const bool tsc = g.order == 2;
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < 3; ++e) H[d][e] = 0.0;
  for (int c = 0; c < S; ++c)
    for (int b = 0; b < S; ++b) {
      const double* row = phi + real_index(g, ax[0].c, ax[1].c + b, ax[2].c + c);
      for (int a = 0; a < S; ++a) {
        const double p = row[a];
        if (tsc) {
          H[0][0] += p * d2[a] * ax[1].w[b] * ax[2].w[c];
          H[1][1] += p * ax[0].w[a] * d2[b] * ax[2].w[c];
          H[2][2] += p * ax[0].w[a] * ax[1].w[b] * d2[c];
        }
        H[0][1] += p * ax[0].dw[a] * ax[1].dw[b] * ax[2].w[c];
        H[0][2] += p * ax[0].dw[a] * ax[1].w[b] * ax[2].dw[c];
        H[1][2] += p * ax[0].w[a] * ax[1].dw[b] * ax[2].dw[c];
      }
    }
  H[1][0] = H[0][1];
  H[2][0] = H[0][2];
  H[2][1] = H[1][2];
}

template <typename T>
__global__ void k_vjp_gather(Geom g, const uint32_t* __restrict__ total,
                             const typename RecT<T>::type* __restrict__ recm,
                             const typename RecT<T>::type* __restrict__ recp,
                             const T* __restrict__ field, size_t nreal,
                             const double* __restrict__ w, double* __restrict__ acc,
                             double* __restrict__ out, int pass,
                             const float4* __restrict__ pp_vjp, double pp_scale) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *total) return;
  Axis<T> ax[3];
  particle_axes(g, recm, i, ax);
  const long long idx = orig_index(recp, i);
  if (pass == 0) {
    T H[3][3];
    if constexpr (sizeof(T) == 4)
      hess_from_diff(g, field, nreal, ax, H);
    else
      hess_from_phi(g, field, ax, H);
    const double wv[3] = {w[3 * idx], w[3 * idx + 1], w[3 * idx + 2]};
    // short-range part: already in acc (FP64 path) or, FP32 path, in pp_vjp (cutoff units)
    double sr[3] = {0.0, 0.0, 0.0};
    if (pp_vjp) {
      const float4 v = pp_vjp[i];
      sr[0] = pp_scale * v.x;
      sr[1] = pp_scale * v.y;
      sr[2] = pp_scale * v.z;
    } else {
      for (int d = 0; d < 3; ++d) sr[d] = acc[3 * i + d];
    }
    for (int d = 0; d < 3; ++d) {
      double hw = 0.0;
      for (int e = 0; e < 3; ++e) hw += static_cast<double>(H[d][e]) * (g.inv_h[d] * g.inv_h[e]) * wv[e];
      acc[3 * i + d] = sr[d] - g.q * hw;
    }
  } else {
    T G[3];
    if constexpr (sizeof(T) == 4)
      grad_from_diff(g, field, nreal, ax, G);
    else
      grad_from_phi(g, field, ax, G);
    for (int d = 0; d < 3; ++d)
      out[3 * idx + d] = acc[3 * i + d] + g.fscale[d] * static_cast<double>(G[d]);
  }
}

template <typename T>
__global__ void k_get_mesh(Geom g, const T* __restrict__ src, double scale,
                           double* __restrict__ out) {
  const size_t total = static_cast<size_t>(g.n[0]) * g.n[1] * g.n[2];
  const size_t idx = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (idx >= total) return;
  const int x = static_cast<int>(idx % g.n[0]);
  const int y = static_cast<int>((idx / g.n[0]) % g.n[1]);
  const int z = static_cast<int>(idx / (static_cast<size_t>(g.n[0]) * g.n[1]));
  out[idx] = scale * static_cast<double>(src[real_index(g, x, y, z)]);
}

}  // namespace

// ---------------------------------------------------------------------------------------------
cudaError_t build_green(p3m_ctx* c) {
  const Geom& g = c->g;
  const size_t nreal = c->n_real, ncplx = c->n_cplx;
  double* samp = nullptr;
  double2* sf = nullptr;
  double2* si = nullptr;
  cufftHandle plan = 0;
  bool have_plan = false;
  cudaError_t err = cudaSuccess;
  auto fail = [&](cudaError_t e) {
    if (have_plan) cufftDestroy(plan);
    cudaFree(samp);
    cudaFree(sf);
    cudaFree(si);
    return e;
  };
  if ((err = cudaMalloc(&samp, sizeof(double) * nreal)) != cudaSuccess) return fail(err);
  if ((err = cudaMalloc(&sf, sizeof(double2) * ncplx)) != cudaSuccess) return fail(err);
  if (g.pm_bc == 1 && (err = cudaMalloc(&si, sizeof(double2) * ncplx)) != cudaSuccess) return fail(err);
  if (cufftPlan3d(&plan, g.M[2], g.M[1], g.M[0], CUFFT_D2Z) != CUFFT_SUCCESS)
    return fail(cudaErrorUnknown);
  have_plan = true;
  cufftSetStream(plan, c->work);
  k_sample_kernel<<<blocks_for(nreal), kThreads, 0, c->work>>>(g, samp, 0);
  if (cufftExecD2Z(plan, samp, reinterpret_cast<cufftDoubleComplex*>(sf)) != CUFFT_SUCCESS)
    return fail(cudaErrorUnknown);
  if (g.pm_bc == 1) {
    k_sample_kernel<<<blocks_for(nreal), kThreads, 0, c->work>>>(g, samp, 1);
    if (cufftExecD2Z(plan, samp, reinterpret_cast<cufftDoubleComplex*>(si)) != CUFFT_SUCCESS)
      return fail(cudaErrorUnknown);
  }
  // scale: k_e q / (Mx My Mz); the mesh holds assignment weights, the inverse FFT is unnormalised
  const double scale = g.ke * g.q / static_cast<double>(nreal);
  if (c->fp32)
    k_finish_kernels<float><<<blocks_for(ncplx), kThreads, 0, c->work>>>(
        g, sf, si, static_cast<float*>(c->khat_f), static_cast<float2*>(c->khat_i), scale,
        c->prm.influence);
  else
    k_finish_kernels<double><<<blocks_for(ncplx), kThreads, 0, c->work>>>(
        g, sf, si, static_cast<double*>(c->khat_f), static_cast<double2*>(c->khat_i), scale,
        c->prm.influence);
  err = cudaStreamSynchronize(c->work);
  if (err == cudaSuccess) err = cudaGetLastError();
  return fail(err);
}

void launch_zero_block(const p3m_ctx* c) {
  const size_t es = c->fp32 ? sizeof(float) : sizeof(double);
  cudaPitchedPtr pp = make_cudaPitchedPtr(c->qpad, es * c->g.M[0], es * c->g.M[0], c->g.M[1]);
  cudaMemset3DAsync(pp, 0, make_cudaExtent(es * c->g.n[0], c->g.n[1], c->g.n[2]), c->work);
}

void launch_deposit_det(const p3m_ctx* c, int64_t n, const double* w) {
  const uint32_t* total = c->starts + c->nkeys;
  const size_t nn = static_cast<size_t>(c->g.n[0]) * c->g.n[1] * c->g.n[2];
  cudaMemsetAsync(c->q128, 0, 2 * sizeof(unsigned long long) * nn, c->work);
  const auto* recm = static_cast<const Rec64*>(c->recm);
  const auto* recp = static_cast<const Rec64*>(c->recp);
  if (w) {
    cudaMemsetAsync(c->dbound, 0, sizeof(unsigned long long), c->work);
    if (n > 0)
      k_dipole_bound<<<blocks_for(n), kThreads, 0, c->work>>>(c->g, total, recp, w, c->dbound);
    if (n > 0)
      k_deposit_det<true><<<blocks_for(n), kThreads, 0, c->work>>>(c->g, total, recm, recp, w,
                                                                     c->dbound, c->q128);
    k_q128_to_mesh<true><<<blocks_for(nn), kThreads, 0, c->work>>>(
        c->g, c->q128, c->dbound, static_cast<double*>(c->qpad));
  } else {
    if (n > 0)
      k_deposit_det<false><<<blocks_for(n), kThreads, 0, c->work>>>(c->g, total, recm, recp,
                                                                      nullptr, c->dbound, c->q128);
    k_q128_to_mesh<false><<<blocks_for(nn), kThreads, 0, c->work>>>(
        c->g, c->q128, c->dbound, static_cast<double*>(c->qpad));
  }
}

void launch_det_sum_pp(const p3m_ctx* c, int64_t n, cudaStream_t s) {
  (void)n;
  k_det_part_pp<<<kDetBlocks, kThreads, 0, s>>>(c->starts + c->nkeys,
                                                 static_cast<const D4*>(c->fpp), c->dred);
  k_det_combine<<<1, kThreads, 0, s>>>(c->dred, c->energy_acc);
}

void launch_det_sum_mesh(const p3m_ctx* c) {
  k_det_part_mesh<<<kDetBlocks, kThreads, 0, c->work>>>(
      c->g, static_cast<const double*>(c->qpad), static_cast<const double*>(c->phireal),
      c->dred + kDetBlocks);
  k_det_combine<<<1, kThreads, 0, c->work>>>(c->dred + kDetBlocks, c->energy_acc + 1);
}

void launch_deposit(const p3m_ctx* c, int64_t n) {
  if (c->det) {
    launch_deposit_det(c, n, nullptr);
    return;
  }
  if (n == 0) return;
  const uint32_t* total = c->starts + c->nkeys;
  const unsigned blocks = static_cast<unsigned>((n + kDepPerBlock - 1) / kDepPerBlock);
  if (c->fp32)
    k_deposit_tiled<float, false><<<blocks, kDepThreads, 0, c->work>>>(
        c->g, total, static_cast<const float4*>(c->recp), static_cast<const float4*>(c->recp),
        nullptr, static_cast<float*>(c->qpad));
  else
    k_deposit_tiled<double, false><<<blocks, kDepThreads, 0, c->work>>>(
        c->g, total, static_cast<const Rec64*>(c->recm), static_cast<const Rec64*>(c->recp),
        nullptr, static_cast<double*>(c->qpad));
}

void launch_dipole_deposit(const p3m_ctx* c, int64_t n, const double* w) {
  if (c->det) {
    launch_deposit_det(c, n, w);
    return;
  }
  if (n == 0) return;
  const uint32_t* total = c->starts + c->nkeys;
  const unsigned blocks = static_cast<unsigned>((n + kDepPerBlock - 1) / kDepPerBlock);
  if (c->fp32)
    k_deposit_tiled<float, true><<<blocks, kDepThreads, 0, c->work>>>(
        c->g, total, static_cast<const float4*>(c->recp), static_cast<const float4*>(c->recp), w,
        static_cast<float*>(c->qpad));
  else
    k_deposit_tiled<double, true><<<blocks, kDepThreads, 0, c->work>>>(
        c->g, total, static_cast<const Rec64*>(c->recm), static_cast<const Rec64*>(c->recp), w,
        static_cast<double*>(c->qpad));
}

void launch_green_multiply(const p3m_ctx* c, bool want_phi, bool want_diff, bool want_energy) {
  const Geom& g = c->g;
  const dim3 grid(blocks_for(static_cast<uint64_t>(g.M[0] / 2 + 1) * g.M[1]), g.M[2] / 2 + 1);
  double* en = want_energy ? c->energy_acc + 1 : nullptr;
  if (c->fp32)
    k_green_multiply<float><<<grid, kThreads, 0, c->work>>>(
        g, static_cast<const float2*>(c->qhat2), static_cast<const float*>(c->khat_f),
        static_cast<const float2*>(c->khat_i), c->dfac,
        want_diff ? static_cast<float2*>(c->fhat) : nullptr,
        want_phi ? static_cast<float2*>(c->phihat) : nullptr, en, c->n_cplx);
  else
    k_green_multiply<double><<<grid, kThreads, 0, c->work>>>(
        g, static_cast<const double2*>(c->qhat2), static_cast<const double*>(c->khat_f),
        static_cast<const double2*>(c->khat_i), nullptr, nullptr,
        want_phi ? static_cast<double2*>(c->phihat) : nullptr, en, c->n_cplx);
}

void launch_interp(const p3m_ctx* c, int64_t n, double* f, int parts) {
  if (n == 0) return;
  const uint32_t* total = c->starts + c->nkeys;
  const double pp_scale = c->g.ke * c->g.q * c->g.q / (c->g.rc * c->g.rc);
  if (c->fp32) {
    k_interp<float><<<blocks_for(n), kThreads, 0, c->work>>>(
        c->g, total, static_cast<const float4*>(c->recp), static_cast<const float*>(c->freal),
        c->n_real, c->fpp, c->fplo, c->fplo + c->n_max, parts, static_cast<float>(pp_scale),
        pp_scale);
    k_unpermute<float><<<blocks_for(n), kThreads, 0, c->work>>>(c->keys, n, c->fpp, f);
  } else {
    k_interp<double><<<blocks_for(n), kThreads, 0, c->work>>>(
        c->g, total, static_cast<const Rec64*>(c->recm), static_cast<const double*>(c->phireal),
        c->n_real, c->fpp, nullptr, nullptr, parts, static_cast<float>(pp_scale), pp_scale);
    k_unpermute<double><<<blocks_for(n), kThreads, 0, c->work>>>(c->keys, n, c->fpp, f);
  }
}

void launch_vjp_gather(const p3m_ctx* c, int64_t n, int pass, const double* w, double* out) {
  if (n == 0) return;
  const uint32_t* total = c->starts + c->nkeys;
  if (c->fp32)
    k_vjp_gather<float><<<blocks_for(n), kThreads, 0, c->work>>>(
        c->g, total, static_cast<const float4*>(c->recp), static_cast<const float4*>(c->recp),
        static_cast<const float*>(c->freal), c->n_real, w, c->acc, out, pass,
        static_cast<const float4*>(c->fpp),
        c->g.ke * c->g.q * c->g.q / (c->g.rc * c->g.rc * c->g.rc));
  else
    k_vjp_gather<double><<<blocks_for(n), kThreads, 0, c->work>>>(
        c->g, total, static_cast<const Rec64*>(c->recm), static_cast<const Rec64*>(c->recp),
        static_cast<const double*>(c->phireal), c->n_real, w, c->acc, out, pass, nullptr, 0.0);
}

void launch_get_mesh(const p3m_ctx* c, int which, double* out) {
  const size_t total = static_cast<size_t>(c->g.n[0]) * c->g.n[1] * c->g.n[2];
  const void* src = which == 0   ? c->qpad
                    : which == 1 ? c->phireal
                                 : static_cast<const void*>(static_cast<const float*>(c->freal) +
                                                            (which - 2) * c->n_real);
  const double scale = which == 0 ? c->g.q : 1.0;
  if (c->fp32)
    k_get_mesh<float><<<blocks_for(total), kThreads, 0, c->work>>>(
        c->g, static_cast<const float*>(src), scale, out);
  else
    k_get_mesh<double><<<blocks_for(total), kThreads, 0, c->work>>>(
        c->g, static_cast<const double*>(src), scale, out);
}

}  // namespace p3m
