// Short-range (particle-particle) half of P3M, eq. (summation_short) with the screened kernel
// G^S(r) = erfc(a r)/r of eq. (ewald_split); the self term is omitted. For r = |xi_i - xi_j|
// below the cutoff r_c the force on i is
//   k_e q^2 [erfc(a r)/r + (2a/sqrt(pi)) e^{-a^2 r^2}] (xi_i - xi_j) / r^2.
// With pp_bc = 1 the cathode also enters the short range (Sec. 3.1.1): each particle j has an
// image of charge -q at S(xi_j) (its own image included) that acts through the same kernel.
//
// Work is in cutoff units (rho = r / r_c, kappa = a r_c): the force is
// (k_e q^2 / r_c^2) P(kappa rho) rho_vec / rho^3 with P(x) = erfc(x) + (2x/sqrt(pi)) e^{-x^2}.
// Positions are cell-local offsets, so FP32 differences keep ~1e-7 of r_c absolute accuracy.
// The FP32 path sums each row of three neighbour cells in FP32 and folds the row sums into a
// two-float (TwoSum) accumulator, which keeps the per-particle sum compensated at the cost of a
// few additions per row instead of per pair.
#include <cmath>

#include "p3m_internal.cuh"

namespace p3m {
namespace {

constexpr int kThreads = 128;

template <typename T>
struct Vec3 {
  T x, y, z;
};

// two-float accumulator (hi + lo) with Knuth's TwoSum
struct Acc2 {
  float hi, lo;
  __device__ __forceinline__ void add(float v) {
    const float s = hi + v;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (v - bp);
    hi = s;
    lo += err;
  }
  __device__ __forceinline__ float value() const { return hi + lo; }
};

__device__ __forceinline__ void pair_terms(float r2, float kappa, float c2k, float& fco,
                                           float& pot) {
  const float rinv = rsqrtf(r2);
  const float x = kappa * (r2 * rinv);
  const float ec = erfcf(x);
  const float ex = __expf(-x * x);
  pot = ec * rinv;
  fco = (pot + c2k * ex) * (rinv * rinv);
}

__device__ __forceinline__ void pair_terms(double r2, double kappa, double c2k, double& fco,
                                           double& pot) {
  const double r = sqrt(r2);
  const double x = kappa * r;
  const double ec = erfc(x);
  const double ex = exp(-x * x);
  pot = ec / r;
  fco = (pot + c2k * ex) / r2;
}

template <typename T>
struct SumT;
template <>
struct SumT<float> {
  Acc2 v[4];
  __device__ void zero() {
    for (int k = 0; k < 4; ++k) v[k].hi = v[k].lo = 0.f;
  }
  __device__ void fold(const float r[4]) {
    for (int k = 0; k < 4; ++k) v[k].add(r[k]);
  }
  __device__ float get(int k) const { return v[k].value(); }
};
template <>
struct SumT<double> {
  double v[4];
  __device__ void zero() {
    for (int k = 0; k < 4; ++k) v[k] = 0.0;
  }
  __device__ void fold(const double r[4]) {
    for (int k = 0; k < 4; ++k) v[k] += r[k];
  }
  __device__ double get(int k) const { return v[k]; }
};

template <typename T>
__device__ __forceinline__ void block_reduce_add(double v, double* dst) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __shared__ double ws[kThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = threadIdx.x < kThreads / 32 ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(dst, s);
  }
}

__device__ __forceinline__ void warp_add_u64(unsigned long long v, unsigned long long* dst) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// One thread per sorted particle; the 27 neighbour cells are read through L1/L2.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_pp(Geom g, const uint32_t* __restrict__ total, const typename RecT<T>::type* __restrict__ rec,
         const uint32_t* __restrict__ skey, const uint32_t* __restrict__ starts,
         void* __restrict__ fpp, double* __restrict__ energy,
         unsigned long long* __restrict__ pairs) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t N = *total;
  const T kappa = static_cast<T>(g.kappa_eff);
  const T c2k = static_cast<T>(2.0 * g.kappa_eff * 0.56418958354775628695);
  const T ax = static_cast<T>(g.a[0]), ay = static_cast<T>(g.a[1]), az = static_cast<T>(g.a[2]);
  double pot_out = 0.0;
  unsigned long long np = 0, ni = 0;
  if (i < N) {
    T ui[3];
    long long idx;
    load_rec(rec + 0, i, ui, idx);
    int cx, cy, cz;
    cell_decode(g, skey[i], cx, cy, cz);
    const T px = ui[0] * ax, py = ui[1] * ay, pz = ui[2] * az;
    SumT<T> sum;
    sum.zero();
    for (int dz = -1; dz <= 1; ++dz) {
      const int nz = cz + dz;
      if (nz < 0 || nz >= g.nc[2]) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int ny = cy + dy;
        if (ny < 0 || ny >= g.nc[1]) continue;
        T row[4] = {T(0), T(0), T(0), T(0)};
        for (int dx = -1; dx <= 1; ++dx) {
          const int nx = cx + dx;
          if (nx < 0 || nx >= g.nc[0]) continue;
          const uint32_t key = cell_key(g, nx, ny, nz);
          const uint32_t j0 = starts[key], j1 = starts[key + 1];
          const T sx = static_cast<T>(dx * g.kc[0]) * ax;
          const T sy = static_cast<T>(dy * g.kc[1]) * ay;
          const T sz = static_cast<T>(dz * g.kc[2]) * az;
          for (uint32_t j = j0; j < j1; ++j) {
            if (j == i) continue;
            T uj[3];
            long long jdx;
            load_rec(rec, j, uj, jdx);
            const T rx = px - (uj[0] * ax + sx);
            const T ry = py - (uj[1] * ay + sy);
            const T rz = pz - (uj[2] * az + sz);
            const T r2 = rx * rx + ry * ry + rz * rz;
            if (r2 < T(1) && r2 > T(0)) {
              T fco, pot;
              pair_terms(r2, kappa, c2k, fco, pot);
              row[0] += fco * rx;
              row[1] += fco * ry;
              row[2] += fco * rz;
              row[3] += pot;
              ++np;
            }
          }
        }
        sum.fold(row);
      }
    }
    if (g.pp_bc) {
      // images of the sources within r_c: only particles less than r_c above the cathode
      const double szi = static_cast<double>(cz * g.kc[2]) + static_cast<double>(ui[2]);
      const double above = (szi - g.s_cath) * g.h[2];
      if (above < g.rc) {
        const double mz = 2.0 * g.s_cath - szi;  // mirrored query point, mesh units
        const double reach = g.rc / g.h[2];
        int z0 = static_cast<int>(floor((mz - reach) / g.kc[2]));
        int z1 = static_cast<int>(floor((mz + reach) / g.kc[2]));
        z0 = max(z0, 0);
        z1 = min(z1, g.nc[2] - 1);
        for (int nz = z0; nz <= z1; ++nz) {
          const T base = static_cast<T>(static_cast<double>((cz + nz) * g.kc[2]) - 2.0 * g.s_cath);
          for (int dy = -1; dy <= 1; ++dy) {
            const int ny = cy + dy;
            if (ny < 0 || ny >= g.nc[1]) continue;
            T row[4] = {T(0), T(0), T(0), T(0)};
            for (int dx = -1; dx <= 1; ++dx) {
              const int nx = cx + dx;
              if (nx < 0 || nx >= g.nc[0]) continue;
              const uint32_t key = cell_key(g, nx, ny, nz);
              const uint32_t j0 = starts[key], j1 = starts[key + 1];
              const T sx = static_cast<T>(dx * g.kc[0]) * ax;
              const T sy = static_cast<T>(dy * g.kc[1]) * ay;
              for (uint32_t j = j0; j < j1; ++j) {
                T uj[3];
                long long jdx;
                load_rec(rec, j, uj, jdx);
                const T rx = px - (uj[0] * ax + sx);
                const T ry = py - (uj[1] * ay + sy);
                const T rz = (base + ui[2] + uj[2]) * az;  // z_i - (2 z_c - z_j)
                const T r2 = rx * rx + ry * ry + rz * rz;
                if (r2 < T(1) && r2 > T(0)) {
                  T fco, pot;
                  pair_terms(r2, kappa, c2k, fco, pot);
                  row[0] -= fco * rx;
                  row[1] -= fco * ry;
                  row[2] -= fco * rz;
                  row[3] -= pot;
                  ++ni;
                }
              }
            }
            sum.fold(row);
          }
        }
      }
    }
    if constexpr (sizeof(T) == 4) {
      reinterpret_cast<float4*>(fpp)[i] =
          make_float4(sum.get(0), sum.get(1), sum.get(2), sum.get(3));
    } else {
      reinterpret_cast<D4*>(fpp)[i] = D4{sum.get(0), sum.get(1), sum.get(2), sum.get(3)};
    }
    pot_out = static_cast<double>(sum.get(3));
  }
  if (energy) block_reduce_add<T>(pot_out, energy);
  warp_add_u64(np, pairs);
  warp_add_u64(ni, pairs + 1);
}

// Vector-Jacobian product of the short-range force map, accumulated into acc (sorted order):
//   free pairs:  acc_i += H(d_ij) (w_i - w_j)
//   image pairs: acc_i += H'(d_ij) (w_i - S w_j)   (H' of the -q image; S = diag(1, 1, -1))
// H(d) = C [phi(rho) I + (phi'(rho)/rho) d d^T]; the force map is the gradient of an energy,
// so its Jacobian is symmetric and this gather form equals the transpose product.
template <typename T>
__device__ __forceinline__ void pair_hess(T r2, T kappa, T c2k, T& fco, T& dfr) {
  const T r = sqrt(r2);
  const T x = kappa * r;
  const T ex = exp(-x * x);
  const T ec = erfc(x);
  const T A = ec / r + c2k * ex;
  const T dA = -c2k * ex / r - ec / r2 - T(2) * kappa * kappa * r * c2k * ex;
  fco = A / r2;
  dfr = (dA / r2 - T(2) * A / (r2 * r)) / r;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_pp_vjp(Geom g, const uint32_t* __restrict__ total,
             const typename RecT<T>::type* __restrict__ rec, const uint32_t* __restrict__ skey,
             const uint32_t* __restrict__ starts, const double* __restrict__ w,
             double* __restrict__ acc, double scale) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *total) return;
  const T kappa = static_cast<T>(g.kappa_eff);
  const T c2k = static_cast<T>(2.0 * g.kappa_eff * 0.56418958354775628695);
  const T ax = static_cast<T>(g.a[0]), ay = static_cast<T>(g.a[1]), az = static_cast<T>(g.a[2]);
  T ui[3];
  long long idx;
  load_rec(rec, i, ui, idx);
  int cx, cy, cz;
  cell_decode(g, skey[i], cx, cy, cz);
  const T px = ui[0] * ax, py = ui[1] * ay, pz = ui[2] * az;
  const T wi[3] = {static_cast<T>(w[3 * idx]), static_cast<T>(w[3 * idx + 1]),
                   static_cast<T>(w[3 * idx + 2])};
  double out[3] = {0.0, 0.0, 0.0};
  for (int dz = -1; dz <= 1; ++dz) {
    const int nz = cz + dz;
    if (nz < 0 || nz >= g.nc[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int ny = cy + dy;
      if (ny < 0 || ny >= g.nc[1]) continue;
      T row[3] = {T(0), T(0), T(0)};
      for (int dx = -1; dx <= 1; ++dx) {
        const int nx = cx + dx;
        if (nx < 0 || nx >= g.nc[0]) continue;
        const uint32_t key = cell_key(g, nx, ny, nz);
        const T sx = static_cast<T>(dx * g.kc[0]) * ax;
        const T sy = static_cast<T>(dy * g.kc[1]) * ay;
        const T sz = static_cast<T>(dz * g.kc[2]) * az;
        for (uint32_t j = starts[key]; j < starts[key + 1]; ++j) {
          if (j == i) continue;
          T uj[3];
          long long jdx;
          load_rec(rec, j, uj, jdx);
          const T rx = px - (uj[0] * ax + sx);
          const T ry = py - (uj[1] * ay + sy);
          const T rz = pz - (uj[2] * az + sz);
          const T r2 = rx * rx + ry * ry + rz * rz;
          if (r2 < T(1) && r2 > T(0)) {
            T fco, dfr;
            pair_hess(r2, kappa, c2k, fco, dfr);
            const T v0 = wi[0] - static_cast<T>(w[3 * jdx]);
            const T v1 = wi[1] - static_cast<T>(w[3 * jdx + 1]);
            const T v2 = wi[2] - static_cast<T>(w[3 * jdx + 2]);
            const T dv = rx * v0 + ry * v1 + rz * v2;
            row[0] += fco * v0 + dfr * dv * rx;
            row[1] += fco * v1 + dfr * dv * ry;
            row[2] += fco * v2 + dfr * dv * rz;
          }
        }
      }
      for (int d = 0; d < 3; ++d) out[d] += static_cast<double>(row[d]);
    }
  }
  if (g.pp_bc) {
    const double szi = static_cast<double>(cz * g.kc[2]) + static_cast<double>(ui[2]);
    if ((szi - g.s_cath) * g.h[2] < g.rc) {
      const double mz = 2.0 * g.s_cath - szi;
      const double reach = g.rc / g.h[2];
      const int z0 = max(static_cast<int>(floor((mz - reach) / g.kc[2])), 0);
      const int z1 = min(static_cast<int>(floor((mz + reach) / g.kc[2])), g.nc[2] - 1);
      for (int nz = z0; nz <= z1; ++nz) {
        const T base = static_cast<T>(static_cast<double>((cz + nz) * g.kc[2]) - 2.0 * g.s_cath);
        for (int dy = -1; dy <= 1; ++dy) {
          const int ny = cy + dy;
          if (ny < 0 || ny >= g.nc[1]) continue;
          for (int dx = -1; dx <= 1; ++dx) {
            const int nx = cx + dx;
            if (nx < 0 || nx >= g.nc[0]) continue;
            const uint32_t key = cell_key(g, nx, ny, nz);
            const T sx = static_cast<T>(dx * g.kc[0]) * ax;
            const T sy = static_cast<T>(dy * g.kc[1]) * ay;
            for (uint32_t j = starts[key]; j < starts[key + 1]; ++j) {
              T uj[3];
              long long jdx;
              load_rec(rec, j, uj, jdx);
              const T rx = px - (uj[0] * ax + sx);
              const T ry = py - (uj[1] * ay + sy);
              const T rz = (base + ui[2] + uj[2]) * az;
              const T r2 = rx * rx + ry * ry + rz * rz;
              if (r2 < T(1) && r2 > T(0)) {
                T fco, dfr;
                pair_hess(r2, kappa, c2k, fco, dfr);
                const T v0 = wi[0] - static_cast<T>(w[3 * jdx]);
                const T v1 = wi[1] - static_cast<T>(w[3 * jdx + 1]);
                const T v2 = wi[2] + static_cast<T>(w[3 * jdx + 2]);  // w_i - S w_j
                const T dv = rx * v0 + ry * v1 + rz * v2;
                out[0] -= static_cast<double>(fco * v0 + dfr * dv * rx);
                out[1] -= static_cast<double>(fco * v1 + dfr * dv * ry);
                out[2] -= static_cast<double>(fco * v2 + dfr * dv * rz);
              }
            }
          }
        }
      }
    }
  }
  acc[3 * i] = scale * out[0];
  acc[3 * i + 1] = scale * out[1];
  acc[3 * i + 2] = scale * out[2];
}

}  // namespace

void launch_pp(const p3m_ctx* c, int64_t n, cudaStream_t s) {
  if (n == 0) return;
  const unsigned blocks = static_cast<unsigned>((n + kThreads - 1) / kThreads);
  const uint32_t* total = c->starts + c->nkeys;
  if (c->fp32)
    k_pp<float><<<blocks, kThreads, 0, s>>>(c->g, total, static_cast<const float4*>(c->rec),
                                            c->skey, c->starts, c->fpp, c->energy_acc,
                                            c->pair_acc);
  else
    k_pp<double><<<blocks, kThreads, 0, s>>>(c->g, total, static_cast<const Rec64*>(c->rec),
                                             c->skey, c->starts, c->fpp, c->energy_acc,
                                             c->pair_acc);
}

void launch_pp_vjp(const p3m_ctx* c, int64_t n, const double* w, cudaStream_t s) {
  if (n == 0) return;
  const unsigned blocks = static_cast<unsigned>((n + kThreads - 1) / kThreads);
  const uint32_t* total = c->starts + c->nkeys;
  // d/dxi of (k_e q^2 / r_c^2) f(rho): one more factor 1/r_c
  const double scale = c->g.ke * c->g.q * c->g.q / (c->g.rc * c->g.rc * c->g.rc);
  if (c->fp32)
    k_pp_vjp<float><<<blocks, kThreads, 0, s>>>(c->g, total, static_cast<const float4*>(c->rec),
                                                c->skey, c->starts, w, c->acc, scale);
  else
    k_pp_vjp<double><<<blocks, kThreads, 0, s>>>(c->g, total, static_cast<const Rec64*>(c->rec),
                                                 c->skey, c->starts, w, c->acc, scale);
}

}  // namespace p3m
