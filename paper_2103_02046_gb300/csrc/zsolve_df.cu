// FP64-path long-range solve along z, fused and in double-float arithmetic: for each (kx, ky)
// column of the x-y transformed charge, the forward transform along z, the Green's-function
// multiply of eq. (phi_L) with the cathode image term of eq. (GreenFunc_planar_cathode), and the
// inverse transform of the potential spectrum, keeping only the n_z planes that the x-y inverse
// transform reads. The FP64 path's numbers enter and leave as doubles; inside, every real is an
// unevaluated sum hi + lo of two FP32 numbers (about 48 significant bits), so the butterflies
// run on GB300's FP32 pipes instead of its scarce FP64 units, with a rounding error of a few
// 1e-15 per operation (the FP64 path's bound against the oracle is 1e-12).
//
// Mesh layout as in the FP32 fused solve: element (z, ky, kx) of a spectrum at (z My + ky) Hx +
// kx, Hx = Mx/2 + 1; the charge is non-zero only in planes z < n_z <= Mz / 2. With
// base = Kf Q - Ki Q(-kz) (Ki absent without the cathode), phihat = base.
//
// Transforms: power-of-two Mz in [64, 2048], radix-8 Stockham autosort passes (then one radix-4
// or radix-2 pass when log2 Mz is not a multiple of 3) in shared memory; twiddles from a table
// computed in FP64 on the host and split into double-float. A block holds C = 2048 / Mz columns
// of consecutive kx (one 8-point butterfly per thread and pass, 256 threads). The Green's spectra
// are held in double-float from context creation on, and the charge spectrum is split by
// integer operations, so that no FP64 instruction runs per element but the final conversion.
#include <algorithm>
#include <cmath>
#include <vector>

#include "df_math.cuh"
#include "p3m_internal.cuh"

namespace p3m {
namespace {

using dfm::F2;

constexpr double kTwoPiD = 6.28318530717958647692;
constexpr int kDThreads = 256;
constexpr int kDElems = 2048;  // columns per block x Mz

// complex double-float
struct CD {
  F2 x, y;
};

// Double-float sum with one error-free transformation of the leading parts: its error is
// bounded by a few units of 2^-48 times |a| + |b| (a normwise bound, which is what a transform's
// error analysis uses), at half the cost of the fully renormalised sum.
__device__ __forceinline__ F2 dadd(F2 a, F2 b) {
  const F2 s = dfm::two_sum(a.hi, b.hi);
  return dfm::fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ F2 dsub(F2 a, F2 b) { return dadd(a, dfm::neg(b)); }

__device__ __forceinline__ CD cd_add(CD a, CD b) { return CD{dadd(a.x, b.x), dadd(a.y, b.y)}; }
__device__ __forceinline__ CD cd_sub(CD a, CD b) { return CD{dsub(a.x, b.x), dsub(a.y, b.y)}; }
__device__ __forceinline__ CD cd_mul(CD a, CD b) {
  return CD{dsub(dfm::mul(a.x, b.x), dfm::mul(a.y, b.y)),
            dadd(dfm::mul(a.x, b.y), dfm::mul(a.y, b.x))};
}
// a * (s i), s = +-1 (exact)
__device__ __forceinline__ CD cd_mul_si(CD a, float s) {
  return s > 0.f ? CD{dfm::neg(a.y), a.x} : CD{a.y, dfm::neg(a.x)};
}
__device__ __forceinline__ CD cd_zero() { return CD{F2{0.f, 0.f}, F2{0.f, 0.f}}; }
__device__ __forceinline__ double d_of(F2 a) {
  return static_cast<double>(a.hi) + static_cast<double>(a.lo);
}
__device__ __forceinline__ double2 cd_to(CD a) { return make_double2(d_of(a.x), d_of(a.y)); }
// the charge spectrum's doubles, split without FP64 instructions
__device__ __forceinline__ CD cd_split(double2 v) {
  return CD{dfm::split_double(v.x), dfm::split_double(v.y)};
}

// sqrt(1/2) in double-float
__device__ __forceinline__ F2 half_sqrt2() {
  return F2{0.70710677f, 1.21016175e-08f};  // the leading 24 bits and the next 24
}

// (a.x - s a.y, a.y + s a.x) sqrt(1/2): a times the eighth root h (1 + s i)
__device__ __forceinline__ CD w8_1(CD a, float s) {
  const F2 h = half_sqrt2();
  const F2 re = s > 0.f ? dsub(a.x, a.y) : dadd(a.x, a.y);
  const F2 im = s > 0.f ? dadd(a.y, a.x) : dsub(a.y, a.x);
  return CD{dfm::mul(re, h), dfm::mul(im, h)};
}
// (-a.x - s a.y, -a.y + s a.x) sqrt(1/2): a times h (-1 + s i)
__device__ __forceinline__ CD w8_3(CD a, float s) {
  const F2 h = half_sqrt2();
  const F2 re = s > 0.f ? dfm::neg(dadd(a.x, a.y)) : dsub(a.y, a.x);
  const F2 im = s > 0.f ? dsub(a.x, a.y) : dfm::neg(dadd(a.y, a.x));
  return CD{dfm::mul(re, h), dfm::mul(im, h)};
}

// R-point DFTs in registers: u_s <- sum_r u_r e^{sign 2 pi i r s / R}.
__device__ __forceinline__ void ddft2(CD& a, CD& b) {
  const CD t = a;
  a = cd_add(t, b);
  b = cd_sub(t, b);
}

__device__ __forceinline__ void ddft4(CD& u0, CD& u1, CD& u2, CD& u3, float sign) {
  const CD t0 = cd_add(u0, u2), t1 = cd_sub(u0, u2);
  const CD t2 = cd_add(u1, u3), t3 = cd_mul_si(cd_sub(u1, u3), sign);
  u0 = cd_add(t0, t2);
  u2 = cd_sub(t0, t2);
  u1 = cd_add(t1, t3);
  u3 = cd_sub(t1, t3);
}

// even and odd halves as two 4-point DFTs, joined with the eighth roots of unity
__device__ __forceinline__ void ddft8_join(CD (&u)[8], CD e0, CD e1, CD e2, CD e3, CD o0, CD o1,
                                           CD o2, CD o3, float sign) {
  o1 = w8_1(o1, sign);
  o2 = cd_mul_si(o2, sign);
  o3 = w8_3(o3, sign);
  u[0] = cd_add(e0, o0);
  u[4] = cd_sub(e0, o0);
  u[1] = cd_add(e1, o1);
  u[5] = cd_sub(e1, o1);
  u[2] = cd_add(e2, o2);
  u[6] = cd_sub(e2, o2);
  u[3] = cd_add(e3, o3);
  u[7] = cd_sub(e3, o3);
}

__device__ __forceinline__ void ddft8(CD (&u)[8], float sign) {
  CD e0 = u[0], e1 = u[2], e2 = u[4], e3 = u[6];
  CD o0 = u[1], o1 = u[3], o2 = u[5], o3 = u[7];
  ddft4(e0, e1, e2, e3, sign);
  ddft4(o0, o1, o2, o3, sign);
  ddft8_join(u, e0, e1, e2, e3, o0, o1, o2, o3, sign);
}

// ddft8 for u_4 .. u_7 = 0: the even and odd 4-point DFTs each have two non-zero inputs
__device__ __forceinline__ void ddft8_lower_inputs(CD (&u)[8], float sign) {
  const CD x0 = u[0], x1 = u[1], x2 = u[2], x3 = u[3];
  const CD x2s = cd_mul_si(x2, sign), x3s = cd_mul_si(x3, sign);
  ddft8_join(u, cd_add(x0, x2), cd_add(x0, x2s), cd_sub(x0, x2), cd_sub(x0, x2s), cd_add(x1, x3),
             cd_add(x1, x3s), cd_sub(x1, x3), cd_sub(x1, x3s), sign);
}

// shared-memory index with one pad element per 16
__host__ __device__ __forceinline__ int dpad(int i) { return i + (i >> 4); }

enum DPassKind { kDGeneral = 0, kDFirstHalf = 1, kDLastLower = 2 };

// One Stockham pass of radix R on one column of length N = 2^logN after passes whose radices
// multiply to p = 2^logp: butterfly i (of N / R) reads u_r = x[i + r N/R], applies the twiddles
// e^{sign 2 pi i r k / (p R)}, k = i mod p, takes the R-point DFT and writes
// y[(i - k) R + k + r p]. Each thread does 8 / R butterflies; reads and writes are separated by
// a barrier, so the pass runs in place. kDFirstHalf: inputs r >= R/2 are zero (and p = 1);
// kDLastLower: only outputs r < R/2 are kept.
template <int R, int kKind>
__device__ __forceinline__ void dpass(CD* a, int logN, int logp, int i0, int tpc, float sign,
                                      const CD* __restrict__ tw) {
  constexpr int kB = 8 / R;
  constexpr int kLogR = R == 8 ? 3 : (R == 4 ? 2 : 1);
  constexpr int kIn = kKind == kDFirstHalf ? R / 2 : R;
  constexpr int kOut = kKind == kDLastLower ? R / 2 : R;
  const int T = (1 << logN) >> kLogR;
  CD u[kB][R];
#pragma unroll
  for (int q = 0; q < kB; ++q)
#pragma unroll
    for (int r = 0; r < R; ++r) u[q][r] = r < kIn ? a[dpad(i0 + q * tpc + r * T)] : cd_zero();
  __syncthreads();
  const int p = 1 << logp;
  const int tshift = logN - logp - kLogR;  // twiddle table step N / (p R)
#pragma unroll
  for (int q = 0; q < kB; ++q) {
    const int i = i0 + q * tpc;
    const int k = i & (p - 1);
    if (kKind != kDFirstHalf && logp > 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        CD w = tw[(r * k) << tshift];            // e^{-2 pi i r k / (p R)}
        if (sign > 0.f) w.y = dfm::neg(w.y);     // conjugate for the inverse
        u[q][r] = cd_mul(u[q][r], w);
      }
    }
    if constexpr (R == 8) {
      if constexpr (kKind == kDFirstHalf)
        ddft8_lower_inputs(u[q], sign);
      else
        ddft8(u[q], sign);
    } else if constexpr (R == 4) {
      ddft4(u[q][0], u[q][1], u[q][2], u[q][3], sign);
    } else {
      ddft2(u[q][0], u[q][1]);
    }
    const int j = ((i - k) << kLogR) + k;
#pragma unroll
    for (int r = 0; r < kOut; ++r) a[dpad(j + r * p)] = u[q][r];
  }
  __syncthreads();
}

template <int kKind>
__device__ __forceinline__ void drun_pass(int R, CD* a, int logN, int logp, int i0, int tpc,
                                          float sign, const CD* __restrict__ tw) {
  if (R == 8)
    dpass<8, kKind>(a, logN, logp, i0, tpc, sign, tw);
  else if (R == 4)
    dpass<4, kKind>(a, logN, logp, i0, tpc, sign, tw);
  else
    dpass<2, kKind>(a, logN, logp, i0, tpc, sign, tw);
}

// Forward transform (sign -1) of a column that is zero in its upper half, or inverse transform
// (sign +1) of which only the lower half is kept; unnormalised, length 2^logN >= 64.
template <bool kForward>
__device__ void dcolumn_fft(CD* a, int logN, int i0, int tpc, const CD* __restrict__ tw) {
  const float sign = kForward ? -1.f : 1.f;
  const int npass = (logN + 2) / 3;
  for (int q = 0, logp = 0; q < npass; ++q) {
    const int logR = (logN - logp) >= 3 ? 3 : logN - logp;
    const int R = 1 << logR;
    if (kForward && q == 0)
      drun_pass<kDFirstHalf>(R, a, logN, logp, i0, tpc, sign, tw);
    else if (!kForward && q == npass - 1)
      drun_pass<kDLastLower>(R, a, logN, logp, i0, tpc, sign, tw);
    else
      drun_pass<kDGeneral>(R, a, logN, logp, i0, tpc, sign, tw);
    logp += logR;
  }
}

// One block: columns kx0 .. kx0 + C - 1 (clipped to Hx) at one ky.
__global__ void __launch_bounds__(kDThreads, 2)
    k_zsolve_df(Geom g, int logN, int padN, const double2* __restrict__ qhat,
                const F2* __restrict__ kf, const CD* __restrict__ ki,
                const CD* __restrict__ tw_g, double2* __restrict__ phihat,
                double* __restrict__ energy) {
  extern __shared__ CD zd[];
  const int N = 1 << logN;
  const int logC = 11 - logN;  // C = 2048 / N
  const int C = 1 << logC;
  const int tpc = N >> 3;      // threads per column
  CD* A = zd;                  // the columns, then their spectra, then the potential
  CD* tw = zd + C * padN;      // e^{-2 pi i t / N}, t < N
  const int Hx = g.M[0] / 2 + 1, My = g.M[1], nz = g.n[2];
  const int nxb = (Hx + C - 1) >> logC;
  const int ky = blockIdx.x / nxb;
  const int kx0 = (blockIdx.x - ky * nxb) << logC;
  const size_t plane = static_cast<size_t>(My) * Hx;
  const size_t row = static_cast<size_t>(ky) * Hx;
  const int tid = threadIdx.x;
  for (int t = tid; t < N; t += kDThreads) tw[t] = tw_g[t];
  // the charged planes z < n_z of the columns, zero above
  for (int idx = tid; idx < kDElems; idx += kDThreads) {
    const int z = idx >> logC, kx = kx0 + (idx & (C - 1));
    A[(idx & (C - 1)) * padN + dpad(z)] =
        (z < nz && kx < Hx) ? cd_split(qhat[z * plane + row + kx]) : cd_zero();
  }
  __syncthreads();
  const int c = tid / tpc, i0 = tid - c * tpc;
  CD* col = A + c * padN;
  dcolumn_fft<true>(col, logN, i0, tpc, tw);
  // Green's-function multiply, kz paired with -kz (the image term reads Q(-kz))
  double e = 0.0;
  const int nmul = (N / 2 + 1) << logC;  // (kz, -kz) pairs x columns
  for (int idx = tid; idx < nmul; idx += kDThreads) {
    const int cc = idx & (C - 1), kz = idx >> logC;
    const int kz2 = (N - kz) & (N - 1);
    const int kxx = kx0 + cc;
    if (kxx >= Hx) continue;
    CD* cl = A + cc * padN;
    const CD a = cl[dpad(kz)], b = cl[dpad(kz2)];
    const size_t ia = kz * plane + row + kxx, ib = kz2 * plane + row + kxx;
    const F2 fa = kf[ia], fb = kf[ib];
    CD ba{dfm::mul(a.x, fa), dfm::mul(a.y, fa)};
    CD bb{dfm::mul(b.x, fb), dfm::mul(b.y, fb)};
    if (ki) {
      ba = cd_sub(ba, cd_mul(ki[ia], b));
      bb = cd_sub(bb, cd_mul(ki[ib], a));
    }
    if (energy) {
      const double wx = (kxx == 0 || 2 * kxx == g.M[0]) ? 1.0 : 2.0;
      double ee = wx * (d_of(dadd(dfm::mul(a.x, ba.x), dfm::mul(a.y, ba.y))));
      if (kz2 != kz) ee += wx * d_of(dadd(dfm::mul(b.x, bb.x), dfm::mul(b.y, bb.y)));
      e += ee;
    }
    cl[dpad(kz)] = ba;
    if (kz2 != kz) cl[dpad(kz2)] = bb;
  }
  __syncthreads();
  dcolumn_fft<false>(col, logN, i0, tpc, tw);
  // the planes z < n_z of the potential spectrum
  for (int idx = tid; idx < (nz << logC); idx += kDThreads) {
    const int z = idx >> logC, cc = idx & (C - 1);
    const int kxx = kx0 + cc;
    if (kxx >= Hx) continue;
    phihat[z * plane + row + kxx] = cd_to(A[cc * padN + dpad(z)]);
  }
  if (energy) {
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((tid & 31) == 0 && e != 0.0) atomicAdd(energy, e);
  }
}

// The Green's spectra, FP64 as built, to double-float in place (8 bytes each either way), once
// at context creation: the fused solve is then their only reader.
__global__ void k_spectra_to_df(double* __restrict__ v, size_t n) {
  const size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (i < n) {
    const F2 d = dfm::split_double_fp64(v[i]);
    reinterpret_cast<F2*>(v)[i] = d;
  }
}

size_t zsolve_df_smem_bytes(int N) {
  return sizeof(CD) * (static_cast<size_t>(kDElems / N) * dpad(N) + N);
}

}  // namespace

bool zsolve_df_supported(const p3m_ctx* c) {
  const int N = c->g.M[2];
  return !c->fp32 && !c->det && c->g.pm_bc != 2 && N >= 64 && N <= 2048 && (N & (N - 1)) == 0;
}

cudaError_t zsolve_df_setup(p3m_ctx* c) {
  const int N = c->g.M[2];
  std::vector<float> tw(4 * static_cast<size_t>(N));
  for (int t = 0; t < N; ++t) {
    const double ang = -kTwoPiD * static_cast<double>(t) / N;
    const double v[2] = {std::cos(ang), std::sin(ang)};
    for (int d = 0; d < 2; ++d) {
      const float h = static_cast<float>(v[d]);
      tw[4 * t + 2 * d] = h;
      tw[4 * t + 2 * d + 1] = static_cast<float>(v[d] - static_cast<double>(h));
    }
  }
  static_assert(sizeof(CD) == 4 * sizeof(float), "complex double-float layout");
  cudaError_t e = cudaMalloc(&c->ztw, sizeof(CD) * N);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->ztw, tw.data(), sizeof(CD) * N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_zsolve_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(zsolve_df_smem_bytes(N)));
  // the spectra: n_cplx reals (free kernel) and n_cplx complex values (image kernel)
  auto convert = [&](void* p, size_t n) {
    if (p == nullptr || e != cudaSuccess) return;
    k_spectra_to_df<<<static_cast<unsigned>((n + 255) / 256), 256, 0, c->work>>>(
        static_cast<double*>(p), n);
    e = cudaGetLastError();
  };
  convert(c->khat_f, c->n_cplx);
  convert(c->khat_i, 2 * c->n_cplx);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->work);
  return e;
}

void launch_zsolve_df(const p3m_ctx* c, bool want_energy) {
  const Geom& g = c->g;
  const int N = g.M[2];
  int logN = 0;
  while ((1 << logN) < N) ++logN;
  const int C = kDElems / N;
  const int Hx = g.M[0] / 2 + 1;
  const unsigned blocks = static_cast<unsigned>(((Hx + C - 1) / C) * g.M[1]);
  double* en = want_energy ? c->energy_acc + 1 : nullptr;
  k_zsolve_df<<<blocks, kDThreads, zsolve_df_smem_bytes(N), c->work>>>(
      g, logN, dpad(N), static_cast<const double2*>(c->qhat),
      static_cast<const F2*>(c->khat_f), static_cast<const CD*>(c->khat_i),
      reinterpret_cast<const CD*>(c->ztw), static_cast<double2*>(c->phihat), en);
}

}  // namespace p3m
