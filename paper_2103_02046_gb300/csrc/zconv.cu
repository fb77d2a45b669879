// FP32 long-range solve along z, fused: for each (kx, ky) column of the x-y transformed charge,
// the forward transform along z, the Green's-function multiply of eq. (phi_L) with the cathode
// image term of eq. (GreenFunc_planar_cathode), and the inverse transforms along z of the
// forward-difference spectra, keeping only the n_z planes that the x-y inverse transforms read.
//
// Mesh layout (doubled mesh M = 2n, half spectrum in x): element (z, ky, kx) of a spectrum is at
// (z My + ky) Hx + kx, Hx = Mx/2 + 1. The charge is non-zero only in planes z < n_z, so the
// column is loaded from those planes and zero-padded to Mz. With base = Kf Q - Ki Q(-kz):
//   D_x = base (e^{2 pi i kx/Mx} - 1),  D_y = base (e^{2 pi i ky/My} - 1),
//   D_z = base (e^{2 pi i kz/Mz} - 1).
// The x and y factors are constant along a column, so D_x and D_y come from one inverse
// transform (of base) and D_z from a second: two inverse transforms instead of three.
//
// Transforms: power-of-two Mz in [64, 2048], radix-8 Stockham autosort passes (then one radix-4
// or radix-2 pass when log2 Mz is not a multiple of 3) in shared memory, twiddles from a table
// computed in FP64 on the host. A block holds C = 4096 / Mz columns of consecutive kx (one
// 8-point butterfly per thread and pass, 512 threads), so loads and stores along kx coalesce.
#include <algorithm>
#include <cmath>
#include <vector>

#include "p3m_internal.cuh"

namespace p3m {
namespace {

constexpr double kTwoPi = 6.28318530717958647692;
constexpr int kZThreads = 512;
constexpr int kZElems = 4096;  // columns per block x Mz

__device__ __forceinline__ float2 c_add(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) {
  return make_float2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 c_scale(float2 a, float s) {
  return make_float2(a.x * s, a.y * s);
}
// a * (s i), s = +-1
__device__ __forceinline__ float2 c_mul_si(float2 a, float s) {
  return make_float2(-s * a.y, s * a.x);
}

// R-point DFT in registers: u_s <- sum_r u_r e^{sign 2 pi i r s / R}.
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  const float2 t = a;
  a = c_add(t, b);
  b = c_sub(t, b);
}

__device__ __forceinline__ void dft4(float2& u0, float2& u1, float2& u2, float2& u3, float sign) {
  const float2 t0 = c_add(u0, u2), t1 = c_sub(u0, u2);
  const float2 t2 = c_add(u1, u3), t3 = c_mul_si(c_sub(u1, u3), sign);
  u0 = c_add(t0, t2);
  u2 = c_sub(t0, t2);
  u1 = c_add(t1, t3);
  u3 = c_sub(t1, t3);
}

// Even and odd halves as two 4-point DFTs, joined with the eighth roots of unity.
__device__ __forceinline__ void dft8(float2 (&u)[8], float sign) {
  float2 e0 = u[0], e1 = u[2], e2 = u[4], e3 = u[6];
  float2 o0 = u[1], o1 = u[3], o2 = u[5], o3 = u[7];
  dft4(e0, e1, e2, e3, sign);
  dft4(o0, o1, o2, o3, sign);
  const float h = 0.70710678118654752440f;
  // W^1 = h (1 + sign i), W^2 = sign i, W^3 = h (-1 + sign i)
  o1 = c_scale(make_float2(o1.x - sign * o1.y, o1.y + sign * o1.x), h);
  o2 = c_mul_si(o2, sign);
  o3 = c_scale(make_float2(-o3.x - sign * o3.y, -o3.y + sign * o3.x), h);
  u[0] = c_add(e0, o0);
  u[4] = c_sub(e0, o0);
  u[1] = c_add(e1, o1);
  u[5] = c_sub(e1, o1);
  u[2] = c_add(e2, o2);
  u[6] = c_sub(e2, o2);
  u[3] = c_add(e3, o3);
  u[7] = c_sub(e3, o3);
}

// dft8 for u_4 .. u_7 = 0: the even and odd 4-point DFTs each have two non-zero inputs.
__device__ __forceinline__ void dft8_lower_inputs(float2 (&u)[8], float sign) {
  const float2 x0 = u[0], x1 = u[1], x2 = u[2], x3 = u[3];
  // E = DFT4(x0, x2, 0, 0), O = DFT4(x1, x3, 0, 0)
  const float2 e0 = c_add(x0, x2), e2 = c_sub(x0, x2);
  const float2 e1 = c_add(x0, c_mul_si(x2, sign)), e3 = c_sub(x0, c_mul_si(x2, sign));
  float2 o0 = c_add(x1, x3), o2 = c_sub(x1, x3);
  float2 o1 = c_add(x1, c_mul_si(x3, sign)), o3 = c_sub(x1, c_mul_si(x3, sign));
  const float h = 0.70710678118654752440f;
  o1 = c_scale(make_float2(o1.x - sign * o1.y, o1.y + sign * o1.x), h);
  o2 = c_mul_si(o2, sign);
  o3 = c_scale(make_float2(-o3.x - sign * o3.y, -o3.y + sign * o3.x), h);
  u[0] = c_add(e0, o0);
  u[4] = c_sub(e0, o0);
  u[1] = c_add(e1, o1);
  u[5] = c_sub(e1, o1);
  u[2] = c_add(e2, o2);
  u[6] = c_sub(e2, o2);
  u[3] = c_add(e3, o3);
  u[7] = c_sub(e3, o3);
}

// Shared-memory index with one pad element per 16: a half-warp reading 16 consecutive
// elements of a column then touches 16 distinct two-bank slots, and the strided stores of the
// Stockham passes spread over the banks.
__host__ __device__ __forceinline__ int zpad(int i) { return i + (i >> 4); }

// Pass variants: kGeneral; kFirstHalf, the first pass of a forward transform whose input is
// zero in its upper half (the zero-padded charge column: inputs r >= R/2 of every butterfly
// vanish; the first pass has no twiddles); kLastLower, the last pass of an inverse transform
// of which only outputs below N/2 are kept (those are outputs r < R/2 of every butterfly).
enum PassKind { kGeneral = 0, kFirstHalf = 1, kLastLower = 2 };

// One Stockham pass of radix R on one column (and, with kTwo, the same pass on a second
// column), for a transform of length N = 2^logN after passes whose radices multiply to
// p = 2^logp. Butterfly i (of N / R) reads u_r = x[i + r N/R], applies the twiddles
// e^{sign 2 pi i r k / (p R)}, k = i mod p (all 1 when p = 1), takes the R-point DFT and
// writes y[(i - k) R + k + r p]. Each thread does 8 / R butterflies; reads and writes are
// separated by a barrier, so the pass runs in place.
template <int R, bool kTwo, int kKind>
__device__ __forceinline__ void stockham_pass(float2* a, float2* b, int logN, int logp, int i0,
                                              int tpc, float sign, const float2* __restrict__ tw) {
  constexpr int kB = 8 / R;
  constexpr int kLogR = R == 8 ? 3 : (R == 4 ? 2 : 1);
  constexpr int kIn = kKind == kFirstHalf ? R / 2 : R;    // inputs that can be non-zero
  constexpr int kOut = kKind == kLastLower ? R / 2 : R;   // outputs that are kept
  const int T = (1 << logN) >> kLogR;
  float2 u[kB][R], v[kB][R];
#pragma unroll
  for (int q = 0; q < kB; ++q)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r < kIn) {
        const int src = zpad(i0 + q * tpc + r * T);
        u[q][r] = a[src];
        if (kTwo) v[q][r] = b[src];
      } else {
        u[q][r] = make_float2(0.f, 0.f);
        if (kTwo) v[q][r] = make_float2(0.f, 0.f);
      }
    }
  __syncthreads();
  const int p = 1 << logp;
  const int tshift = logN - logp - kLogR;  // twiddle table step N / (p R)
#pragma unroll
  for (int q = 0; q < kB; ++q) {
    const int i = i0 + q * tpc;
    const int k = i & (p - 1);
    if (kKind != kFirstHalf && logp > 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = tw[(r * k) << tshift];  // e^{-2 pi i r k / (p R)}
        w.y *= -sign;                       // conjugate for the inverse (sign = +1)
        u[q][r] = c_mul(u[q][r], w);
        if (kTwo) v[q][r] = c_mul(v[q][r], w);
      }
    }
    if constexpr (R == 8) {
      if constexpr (kKind == kFirstHalf) {
        dft8_lower_inputs(u[q], sign);
        if (kTwo) dft8_lower_inputs(v[q], sign);
      } else {
        dft8(u[q], sign);
        if (kTwo) dft8(v[q], sign);
      }
    } else if constexpr (R == 4) {
      dft4(u[q][0], u[q][1], u[q][2], u[q][3], sign);
      if (kTwo) dft4(v[q][0], v[q][1], v[q][2], v[q][3], sign);
    } else {
      dft2(u[q][0], u[q][1]);
      if (kTwo) dft2(v[q][0], v[q][1]);
    }
    const int j = ((i - k) << kLogR) + k;
#pragma unroll
    for (int r = 0; r < kOut; ++r) {
      const int dst = zpad(j + r * p);
      a[dst] = u[q][r];
      if (kTwo) b[dst] = v[q][r];
    }
  }
  __syncthreads();
}

template <bool kTwo, int kKind>
__device__ __forceinline__ void run_pass(int R, float2* a, float2* b, int logN, int logp, int i0,
                                         int tpc, float sign, const float2* __restrict__ tw) {
  if (R == 8)
    stockham_pass<8, kTwo, kKind>(a, b, logN, logp, i0, tpc, sign, tw);
  else if (R == 4)
    stockham_pass<4, kTwo, kKind>(a, b, logN, logp, i0, tpc, sign, tw);
  else
    stockham_pass<2, kTwo, kKind>(a, b, logN, logp, i0, tpc, sign, tw);
}

// Forward transform of a column that is zero in its upper half (sign -1), or inverse
// transform (sign +1) of which only the lower half is kept; unnormalised, length 2^logN >= 64:
// radix-8 passes, then one radix-4 or radix-2 pass when log2 N is not a multiple of 3.
template <bool kTwo, bool kForward>
__device__ void column_fft(float2* a, float2* b, int logN, int i0, int tpc,
                           const float2* __restrict__ tw) {
  const float sign = kForward ? -1.f : 1.f;
  const int npass = (logN + 2) / 3;
  for (int q = 0, logp = 0; q < npass; ++q) {
    const int logR = (logN - logp) >= 3 ? 3 : logN - logp;
    const int R = 1 << logR;
    if (kForward && q == 0)
      run_pass<kTwo, kFirstHalf>(R, a, b, logN, logp, i0, tpc, sign, tw);
    else if (!kForward && q == npass - 1)
      run_pass<kTwo, kLastLower>(R, a, b, logN, logp, i0, tpc, sign, tw);
    else
      run_pass<kTwo, kGeneral>(R, a, b, logN, logp, i0, tpc, sign, tw);
    logp += logR;
  }
}

constexpr int kMulItems = 5;  // multiply items per thread: ceil((N/2 + 1) C / 512) <= 5

// One block: columns kx0 .. kx0 + C - 1 (clipped to Hx) at one ky. kImage: the cathode's image
// kernel is present.
template <bool kImage>
__global__ void __launch_bounds__(kZThreads, 2)
    k_zconv(Geom g, int logN, int padN, const float2* __restrict__ qhat,
            const float* __restrict__ kf, const float2* __restrict__ ki,
            const float2* __restrict__ dfac, const float2* __restrict__ tw_g,
            float2* __restrict__ fhat, size_t ncplx, double* __restrict__ energy) {
  extern __shared__ float2 zs[];
  const int N = 1 << logN;
  const int logC = 12 - logN;  // C = 4096 / N
  const int C = 1 << logC;
  const int tpc = N >> 3;      // threads per column
  float2* A = zs;              // base, then its inverse transform
  float2* Bz = zs + C * padN;  // base (e^{2 pi i kz/Mz} - 1), then its inverse transform
  float2* tw = Bz + C * padN;  // e^{-2 pi i t / N}, t < N
  const int Hx = g.M[0] / 2 + 1, My = g.M[1], nz = g.n[2];
  const int nxb = (Hx + C - 1) >> logC;
  const int ky = blockIdx.x / nxb;
  const int kx0 = (blockIdx.x - ky * nxb) << logC;
  const size_t plane = static_cast<size_t>(My) * Hx;
  const size_t row = static_cast<size_t>(ky) * Hx;
  const int tid = threadIdx.x;
  const int nmul = (N / 2 + 1) << logC;  // (kz, -kz) pairs x columns
  for (int t = tid; t < N; t += kZThreads) tw[t] = tw_g[t];
  // load the charged planes z < n_z of the columns (zero above): all of a thread's loads are
  // issued before the first store
  {
    float2 v[kZElems / kZThreads];
#pragma unroll
    for (int q = 0; q < kZElems / kZThreads; ++q) {
      const int idx = tid + q * kZThreads;
      const int z = idx >> logC, kx = kx0 + (idx & (C - 1));
      v[q] = (z < nz && kx < Hx) ? qhat[z * plane + row + kx] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < kZElems / kZThreads; ++q) {
      const int idx = tid + q * kZThreads;
      A[(idx & (C - 1)) * padN + zpad(idx >> logC)] = v[q];
    }
  }
  // the kernel spectra this thread multiplies with, fetched now so that their latency overlaps
  // the forward transform
  float kfa[kMulItems], kfb[kMulItems];
  float2 kia[kMulItems], kib[kMulItems];
#pragma unroll
  for (int q = 0; q < kMulItems; ++q) {
    const int idx = tid + q * kZThreads;
    const int kz = idx >> logC, kxx = kx0 + (idx & (C - 1));
    const int kz2 = (N - kz) & (N - 1);
    const bool ok = idx < nmul && kxx < Hx;
    const size_t ia = kz * plane + row + kxx, ib = kz2 * plane + row + kxx;
    kfa[q] = ok ? kf[ia] : 0.f;
    kfb[q] = ok ? kf[ib] : 0.f;
    if (kImage) {
      kia[q] = ok ? ki[ia] : make_float2(0.f, 0.f);
      kib[q] = ok ? ki[ib] : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  const int c = tid / tpc, i0 = tid - c * tpc;
  float2* colA = A + c * padN;
  float2* colB = Bz + c * padN;
  column_fft<false, true>(colA, nullptr, logN, i0, tpc, tw);
  // Green's-function multiply, kz paired with -kz (the image term reads Q(-kz)); the columns
  // of one kz are adjacent lanes, so the kernel spectra are read along kx
  const float2* fz = dfac + Hx + My;
  double e = 0.0;
#pragma unroll
  for (int q = 0; q < kMulItems; ++q) {
    const int idx = tid + q * kZThreads;
    if (idx >= nmul) break;
    const int cc = idx & (C - 1), kz = idx >> logC;
    const int kz2 = (N - kz) & (N - 1);
    const int kxx = kx0 + cc;
    float2* ca = A + cc * padN;
    float2* cb = Bz + cc * padN;
    const float2 a = ca[zpad(kz)], b = ca[zpad(kz2)];
    float2 ba = c_scale(a, kfa[q]), bb = c_scale(b, kfb[q]);
    if (kImage) {
      ba = c_sub(ba, c_mul(kia[q], b));
      bb = c_sub(bb, c_mul(kib[q], a));
    }
    if (energy && kxx < Hx) {
      const float wx = (kxx == 0 || 2 * kxx == g.M[0]) ? 1.f : 2.f;
      float ee = wx * (a.x * ba.x + a.y * ba.y);
      if (kz2 != kz) ee += wx * (b.x * bb.x + b.y * bb.y);
      e += static_cast<double>(ee);
    }
    ca[zpad(kz)] = ba;
    cb[zpad(kz)] = c_mul(ba, fz[kz]);
    if (kz2 != kz) {
      ca[zpad(kz2)] = bb;
      cb[zpad(kz2)] = c_mul(bb, fz[kz2]);
    }
  }
  __syncthreads();
  column_fft<true, false>(colA, colB, logN, i0, tpc, tw);
  // store the planes z < n_z of the three difference spectra
  const float2* fx = dfac;
  const float2 fyk = dfac[Hx + ky];
  for (int idx = tid; idx < (nz << logC); idx += kZThreads) {
    const int z = idx >> logC, cc = idx & (C - 1);
    const int kxx = kx0 + cc;
    if (kxx >= Hx) continue;
    const float2 av = A[cc * padN + zpad(z)];
    const size_t o = z * plane + row + kxx;
    fhat[o] = c_mul(av, fx[kxx]);
    fhat[ncplx + o] = c_mul(av, fyk);
    fhat[2 * ncplx + o] = Bz[cc * padN + zpad(z)];
  }
  if (energy) {
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((tid & 31) == 0 && e != 0.0) atomicAdd(energy, e);
  }
}

}  // namespace

bool zconv_supported(const p3m_ctx* c) {
  const int N = c->g.M[2];
  return c->fp32 && N >= 64 && N <= 2048 && (N & (N - 1)) == 0;
}

// Column stride (float2 elements) for a block of C = 4096 / N columns: the smallest stride
// >= zpad(N) whose warp rows -- C columns by 32 / C values of z, at z and at -z (the Green's
// multiply) -- need the fewest shared-memory wavefronts, counted per half-warp as the largest
// number of distinct elements falling in one 4-byte bank.
int zcol_stride(int N) {
  const int C = kZElems / N;
  int best = 0, best_w = 1 << 30;
  for (int P = zpad(N); P < zpad(N) + 16; ++P) {
    int w = 0;
    for (int dir = 0; dir < 2; ++dir)
      for (int z0 = 0; z0 < std::max(1, 64 / C); z0 += std::max(1, 32 / C)) {
        for (int h = 0; h < 2; ++h) {
          int count[32] = {}, last[32];
          for (int b = 0; b < 32; ++b) last[b] = -1;
          int worst = 0;
          for (int l = 16 * h; l < 16 * h + 16; ++l) {
            const int col = l & (C - 1), z = z0 + l / C;
            const int e = col * P + zpad(dir ? (N - z) & (N - 1) : z);
            for (int half = 0; half < 2; ++half) {
              const int bank = (2 * e + half) & 31;
              if (last[bank] != e) {  // distinct elements of a bank (each lane's once)
                last[bank] = e;
                worst = std::max(worst, ++count[bank]);
              }
            }
          }
          w += worst;
        }
      }
    if (w < best_w) best_w = w, best = P;
  }
  return best;
}

size_t zconv_smem_bytes(int N) {
  return sizeof(float2) * (2 * static_cast<size_t>(kZElems / N) * zcol_stride(N) + N);
}

cudaError_t zconv_setup(p3m_ctx* c) {
  const int N = c->g.M[2];
  std::vector<float2> tw(N);
  for (int t = 0; t < N; ++t) {
    const double ang = -kTwoPi * static_cast<double>(t) / N;
    tw[t] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
  }
  cudaError_t e = cudaMalloc(&c->ztw, sizeof(float2) * N);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->ztw, tw.data(), sizeof(float2) * N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_zconv<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(zconv_smem_bytes(N)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_zconv<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(zconv_smem_bytes(N)));
  return e;
}

void launch_zconv(const p3m_ctx* c, bool want_energy) {
  const Geom& g = c->g;
  const int N = g.M[2];
  int logN = 0;
  while ((1 << logN) < N) ++logN;
  const int C = kZElems / N;
  const int Hx = g.M[0] / 2 + 1;
  const unsigned blocks = static_cast<unsigned>(((Hx + C - 1) / C) * g.M[1]);
  double* en = want_energy ? c->energy_acc + 1 : nullptr;
  auto run = [&](auto kern) {
    kern<<<blocks, kZThreads, zconv_smem_bytes(N), c->work>>>(
        g, logN, zcol_stride(N), static_cast<const float2*>(c->qhat),
        static_cast<const float*>(c->khat_f), static_cast<const float2*>(c->khat_i), c->dfac,
        c->ztw, static_cast<float2*>(c->fhat), c->n_cplx, en);
  };
  if (c->khat_i)
    run(k_zconv<true>);
  else
    run(k_zconv<false>);
}

}  // namespace p3m
