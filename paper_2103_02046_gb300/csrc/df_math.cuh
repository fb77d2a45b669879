// Double-float evaluation of the short-range pair function for the FP64 path.
//
// The FP64 short range spends most of its time in the pair function of eq. (summation_short)
// with the screened kernel of eq. (ewald_split): erfc, exp, a square root and divisions, each a
// long chain of FP64 operations on a part whose FP64 units run at a small fraction of its FP32
// rate. Here the same function is evaluated in double-float arithmetic: every quantity is an
// unevaluated sum hi + lo of two FP32 numbers (about 48 significant bits), formed with the
// error-free transformations of Knuth (TwoSum), Dekker (Fast2Sum) and the FMA product split,
// so the pair function costs FP32 instructions only and keeps a relative error of a few 1e-15,
// far inside the FP64 path's 1e-12 bound.
//
// In cutoff units (rho = r / r_c, kappa = alpha r_c, x = kappa rho):
//   pot(rho) = erfc(x) / rho,   fco(rho) = [erfc(x) / rho + (2 kappa / sqrt(pi)) e^{-x^2}] / rho^2
// with erfc(x) = R(x) e^{-x^2}, R(x) = erfc(x) e^{x^2} (smooth and slowly varying on [0, kappa]):
//   * 1/rho: the FP32 reciprocal square root refined by two Newton steps in double-float;
//   * R(x): [0, kappa] cut into intervals of equal width w <= 0.375, on each a polynomial in
//     t = 2 (x - x_q) / w - 1 (Chebyshev interpolation of R at 96 nodes, converted to the
//     monomial basis in long double on the host), evaluated by Horner's rule;
//   * e^{-y}, y = kappa^2 rho^2: y = k ln2/16 + r with |r| <= ln2/32, the product k ln2/16 taken
//     exactly from a three-part split of ln2/16 (12, 12 and 24 bits), e^{-r} from its Taylor
//     series (degrees 4 to 9 in FP32, where they are below 1e-8, degrees 0 to 3 in
//     double-float), times 2^{-j/16} (a table) and 2^{-(k >> 4)} (exact scaling).
//
// Everything here is plain arithmetic on floats, written so that it compiles as host code too
// (the host evaluation backs a CPU test of the accuracy against long-double erfc and exp).
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#if defined(__CUDACC__)
#define DFM_HD __host__ __device__ __forceinline__
#else
#define DFM_HD inline
#endif

namespace dfm {

struct F2 {
  float hi, lo;
};

// Rounded FP32 operations that the compiler may not contract into FMAs or reassociate (the
// error-free transformations depend on each rounding). Host builds are compiled without FP
// contraction.
DFM_HD float add_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
DFM_HD float sub_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
DFM_HD float mul_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
DFM_HD float fma_rn(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}

// a + b = s + e exactly (Knuth)
DFM_HD F2 two_sum(float a, float b) {
  const float s = add_rn(a, b);
  const float bb = sub_rn(s, a);
  return F2{s, add_rn(sub_rn(a, sub_rn(s, bb)), sub_rn(b, bb))};
}
// s + e renormalised, |s| >= |e| (Dekker)
DFM_HD F2 fast_two_sum(float s, float e) {
  const float h = add_rn(s, e);
  return F2{h, sub_rn(e, sub_rn(h, s))};
}
// a b = p + e exactly (FMA)
DFM_HD F2 two_prod(float a, float b) {
  const float p = mul_rn(a, b);
  return F2{p, fma_rn(a, b, -p)};
}

DFM_HD F2 add(F2 a, F2 b) {
  const F2 s = two_sum(a.hi, b.hi);
  const F2 t = two_sum(a.lo, b.lo);
  const F2 u = fast_two_sum(s.hi, add_rn(s.lo, t.hi));
  return fast_two_sum(u.hi, add_rn(u.lo, t.lo));
}
DFM_HD F2 neg(F2 a) { return F2{-a.hi, -a.lo}; }
DFM_HD F2 sub(F2 a, F2 b) { return add(a, neg(b)); }
DFM_HD F2 mul(F2 a, F2 b) {
  const F2 p = two_prod(a.hi, b.hi);
  float e = fma_rn(a.hi, b.lo, p.lo);
  e = fma_rn(a.lo, b.hi, e);
  return fast_two_sum(p.hi, e);
}
DFM_HD F2 mul_f(F2 a, float b) {
  const F2 p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, fma_rn(a.lo, b, p.lo));
}
// Bit views (the device intrinsics, or a copy of the bytes on the host).
DFM_HD uint64_t bits_of(double v) {
#if defined(__CUDA_ARCH__)
  return static_cast<uint64_t>(__double_as_longlong(v));
#else
  uint64_t b;
  memcpy(&b, &v, sizeof b);
  return b;
#endif
}
DFM_HD float float_of(uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float v;
  memcpy(&v, &b, sizeof v);
  return v;
#endif
}

// A double as hi + lo by FP64 conversions (hi its FP32 rounding, lo the rest rounded).
DFM_HD F2 split_double_fp64(double v) {
  const float h = static_cast<float>(v);
  return F2{h, static_cast<float>(v - static_cast<double>(h))};
}

// A double as hi + lo by integer operations on its bits, with no FP64 instruction (GB300's FP64
// pipe runs at a small fraction of its FP32 rate): hi holds the sign, the exponent and the
// leading 23 stored significand bits (truncated, so exact in FP32); the remaining 29 bits,
// r = r1 2^6 + r0 (r1 < 2^23 and r0 < 2^6, each exact in FP32 through the 2^23 magic number), give
// lo = (r1 2^6 + r0) 2^(e - 1075), rounded once to FP32, with v's sign. So |lo| < ulp(hi) and
// hi + lo = v to 2^-47 relative. Zero and subnormal doubles give zero (of v's sign); |v| outside
// [2^-74, 2^128) takes the FP64 conversion.
DFM_HD F2 split_double(double v) {
  const uint64_t b = bits_of(v);
  const int e = static_cast<int>((b >> 52) & 0x7ffu);
  const uint32_t sgn = static_cast<uint32_t>(b >> 32) & 0x80000000u;
  if (e == 0) return F2{float_of(sgn), 0.f};
  if (e < 949 || e > 1150) return split_double_fp64(v);
  const uint32_t mh = static_cast<uint32_t>(b >> 29) & 0x7fffffu;
  const float hi = float_of(sgn | (static_cast<uint32_t>(e - 1023 + 127) << 23) | mh);
  const uint32_t r = static_cast<uint32_t>(b) & 0x1fffffffu;
  const float r1 = sub_rn(float_of(0x4b000000u | (r >> 6)), 8388608.f);
  const float r0 = sub_rn(float_of(0x4b000000u | (r & 63u)), 8388608.f);
  const float scale = float_of(sgn | (static_cast<uint32_t>(e - 1075 + 127) << 23));
  return F2{hi, mul_rn(fma_rn(r1, 64.f, r0), scale)};
}

// a 2^n for -126 < n <= 0 on normal results (exact)
DFM_HD F2 scale_pow2(F2 a, int n) {
  const float s = ldexpf(1.0f, n);
  return F2{a.hi * s, a.lo * s};
}

// Interval polynomials of R(x) = erfc(x) e^{x^2} and the constants of the pair function.
constexpr int kMaxIntervals = 32;
constexpr int kMaxDegree = 16;
constexpr float kMaxWidth = 0.375f;

// ln 2 / 16 in three parts: 12, 12 and 24 significant bits, so that k * L1 and k * L2 are exact
// for k < 2^11 and L1 + L2 + L3 agrees with ln2/16 to 2^-48 of its value.
struct Ln2Parts {
  float l1, l2, l3;
};

struct PairConsts {
  int nint;                     // intervals of [0, kappa]
  int deg;                      // polynomial degree on each
  float inv_w;                  // 1 / w (FP32: chooses the interval)
  F2 two_over_w;                // 2 / w
  F2 kappa;                     // kappa = alpha r_c
  F2 kappa2;                    // kappa^2
  F2 c2k;                       // 2 kappa / sqrt(pi)
  F2 exp2m[16];                 // 2^{-j/16}
  Ln2Parts ln2;                 // ln2 / 16 in three parts
};

using Coef = F2[kMaxDegree + 1];  // monomial coefficients in t, lowest degree first

struct PairDF {
  PairConsts k;
  Coef coef[kMaxIntervals];
  double max_rel_err;           // of the fitted R over [0, kappa] (host check, reported)
};

// e^{-y} for y = kappa^2 rho^2 in [0, kappa^2], kappa^2 < 88 (k < 2^11)
DFM_HD F2 exp_neg(const PairConsts& T, F2 y) {
  const Ln2Parts& L = T.ln2;
  const float kf = rintf(mul_rn(y.hi, 23.083120654223414f));  // 16 / ln 2
  const float a = sub_rn(y.hi, mul_rn(kf, L.l1));               // exact (Sterbenz)
  F2 r = add(F2{a, y.lo}, F2{-mul_rn(kf, L.l2), 0.f});
  r = add(r, two_prod(-kf, L.l3));
  // e^{-r} = sum (-r)^n / n!: the tail n >= 4 in FP32 (|r|^4 / 24 < 1e-8), the rest in
  // double-float
  const float rh = r.hi;
  float tail = fma_rn(rh, -2.7557319e-6f, 2.4801587e-5f);  // -1/9!, 1/8!
  tail = fma_rn(rh, tail, -1.9841270e-4f);                  // -1/7!
  tail = fma_rn(rh, tail, 1.3888889e-3f);                   // 1/6!
  tail = fma_rn(rh, tail, -8.3333333e-3f);                  // -1/5!
  tail = fma_rn(rh, tail, 4.1666667e-2f);                   // 1/4!
  F2 p = F2{tail, 0.f};
  p = add(mul(p, r), F2{-0.16666667f, 4.9670538e-9f});       // -1/6
  p = add(mul(p, r), F2{0.5f, 0.f});
  p = add(mul(p, r), F2{-1.f, 0.f});
  p = add(mul(p, r), F2{1.f, 0.f});
  const int k = static_cast<int>(kf);
  return scale_pow2(mul(p, T.exp2m[k & 15]), -(k >> 4));
}

// R(x) on the interval that holds x (x in [0, kappa])
DFM_HD F2 erfcx_poly(const PairConsts& T, const Coef* coef, F2 x) {
  int q = static_cast<int>(mul_rn(x.hi, T.inv_w));
  q = q < 0 ? 0 : (q >= T.nint ? T.nint - 1 : q);
  const F2 t = sub(mul(x, T.two_over_w), F2{static_cast<float>(2 * q + 1), 0.f});
  F2 acc = coef[q][T.deg];
  for (int k = T.deg - 1; k >= 0; --k) acc = add(mul(acc, t), coef[q][k]);
  return acc;
}

// 1/rho from s = rho^2 (s > 0): FP32 estimate, two Newton steps y <- y + y (1 - s y^2) / 2
DFM_HD F2 rsqrt_df(F2 s) {
#if defined(__CUDA_ARCH__)
  const float y0 = rsqrtf(s.hi);
#else
  const float y0 = 1.0f / sqrtf(s.hi);
#endif
  F2 y{y0, 0.f};
  for (int it = 0; it < 2; ++it) {
    const F2 e = sub(F2{1.f, 0.f}, mul(s, mul(y, y)));
    y = add(y, mul(mul_f(e, 0.5f), y));
  }
  return y;
}

// Pair terms for s = rho^2 in (0, 1]: fco = [erfc(x)/rho + c2k e^{-x^2}]/rho^2, pot = erfc(x)/rho
struct PairOut {
  F2 fco, pot, ex, rinv, rho, R;
};

DFM_HD PairOut pair_df(const PairConsts& T, const Coef* coef, F2 s) {
  PairOut o;
  o.rinv = rsqrt_df(s);
  o.rho = mul(s, o.rinv);
  const F2 x = mul(o.rho, T.kappa);
  o.R = erfcx_poly(T, coef, x);
  o.ex = exp_neg(T, mul(T.kappa2, s));
  o.pot = mul(mul(o.R, o.ex), o.rinv);                 // erfc(x) / rho
  const F2 A = add(o.pot, mul(T.c2k, o.ex));            // rho^2 fco
  o.fco = mul(A, mul(o.rinv, o.rinv));
  return o;
}

// The pair energy's Hessian terms for the adjoint: with A(rho) = erfc(x)/rho + c2k e^{-x^2},
//   fco = A / rho^2,   dfr = (A'(rho) / rho^2 - 2 A / rho^3) / rho,
//   A'(rho) = -c2k e^{-x^2} / rho - erfc(x) / rho^2 - 2 kappa^2 rho c2k e^{-x^2}.
DFM_HD void pair_hess_df(const PairConsts& T, const Coef* coef, F2 s, F2& fco, F2& dfr) {
  const PairOut o = pair_df(T, coef, s);
  fco = o.fco;
  const F2 cex = mul(T.c2k, o.ex);
  const F2 A = add(o.pot, cex);
  // A' = -(cex + pot) / rho - 2 kappa^2 rho cex
  const F2 dA = neg(add(mul(add(cex, o.pot), o.rinv), mul_f(mul(mul(T.kappa2, o.rho), cex), 2.f)));
  const F2 r2inv = mul(o.rinv, o.rinv);
  dfr = mul(mul(sub(dA, mul_f(mul(A, o.rinv), 2.f)), r2inv), o.rinv);
}

// ---- host side: the fit ----
inline F2 split_ld(long double v) {
  const float h = static_cast<float>(v);
  return F2{h, static_cast<float>(v - static_cast<long double>(h))};
}

inline Ln2Parts ln2_parts() {
  const long double L = 0.6931471805599453094172321214581765680755L / 16.0L;
  // round L to 12 significant bits, then the remainder to 12, then to 24
  auto round_bits = [](long double v, int bits) -> float {
    int e;
    const long double m = frexpl(v, &e);  // v = m 2^e, 0.5 <= |m| < 1
    const long double q = ldexpl(1.0L, bits);
    return static_cast<float>(ldexpl(roundl(m * q) / q, e));
  };
  Ln2Parts p;
  p.l1 = round_bits(L, 12);
  p.l2 = round_bits(L - p.l1, 12);
  p.l3 = static_cast<float>(L - p.l1 - static_cast<long double>(p.l2));
  return p;
}

// Fits R on [0, kappa] for kappa in (0, 9.3] (kappa^2 < 88 for the exponential's table range).
// Returns false for kappa outside that range.
inline bool fit_pair_df(double kappa, PairDF& P) {
  PairConsts& T = P.k;
  if (!(kappa > 0.0) || kappa > 9.3) return false;
  T.ln2 = ln2_parts();
  int nint = static_cast<int>(ceil(kappa / kMaxWidth - 1e-12));
  if (nint < 1) nint = 1;
  if (nint > kMaxIntervals) return false;
  const long double w = static_cast<long double>(kappa) / nint;
  T.nint = nint;
  T.inv_w = static_cast<float>(1.0L / w);
  T.two_over_w = split_ld(2.0L / w);
  T.kappa = split_ld(kappa);
  T.kappa2 = split_ld(static_cast<long double>(kappa) * kappa);
  T.c2k = split_ld(2.0L * kappa / sqrtl(3.14159265358979323846264338327950288L));
  for (int j = 0; j < 16; ++j) T.exp2m[j] = split_ld(powl(2.0L, -j / 16.0L));
  constexpr int N = 96;
  const long double pi = 3.14159265358979323846264338327950288L;
  auto R = [](long double x) { return erfcl(x) * expl(x * x); };
  std::vector<long double> fv(static_cast<size_t>(nint) * N);  // R at the Chebyshev nodes
  for (int q = 0; q < nint; ++q)
    for (int j = 0; j < N; ++j)
      fv[q * N + j] = R(q * w + (cosl(pi * (j + 0.5L) / N) + 1.0L) * w / 2);
  for (int deg = 12; deg <= kMaxDegree; ++deg) {
    T.deg = deg;
    double worst = 0.0;
    for (int q = 0; q < nint; ++q) {
      const long double a = q * w;
      // Chebyshev coefficients from the values at the Chebyshev nodes
      long double ch[kMaxDegree + 1] = {};
      for (int k = 0; k <= deg; ++k) {
        long double acc = 0.0L;
        for (int j = 0; j < N; ++j) acc += fv[q * N + j] * cosl(k * pi * (j + 0.5L) / N);
        ch[k] = acc * 2.0L / N;
      }
      ch[0] *= 0.5L;
      // Chebyshev -> monomial in t: T_0 = 1, T_1 = t, T_{k+1} = 2 t T_k - T_{k-1}
      long double mono[kMaxDegree + 1] = {}, tm1[kMaxDegree + 1] = {}, tk[kMaxDegree + 1] = {},
                  tp1[kMaxDegree + 1] = {};
      tm1[0] = 1.0L;
      tk[1] = 1.0L;
      mono[0] += ch[0];
      mono[1] += ch[1];
      for (int k = 1; k < deg; ++k) {
        for (int m = 0; m <= deg; ++m) tp1[m] = (m > 0 ? 2.0L * tk[m - 1] : 0.0L) - tm1[m];
        for (int m = 0; m <= deg; ++m) {
          mono[m] += ch[k + 1] * tp1[m];
          tm1[m] = tk[m];
          tk[m] = tp1[m];
        }
      }
      for (int m = 0; m <= deg; ++m) P.coef[q][m] = split_ld(mono[m]);
      for (int m = deg + 1; m <= kMaxDegree; ++m) P.coef[q][m] = F2{0.f, 0.f};
      for (int u = 0; u <= 400; ++u) {
        const long double t = -1.0L + u / 200.0L;
        long double p = 0.0L;
        for (int m = deg; m >= 0; --m)
          p = p * t + (static_cast<long double>(P.coef[q][m].hi) + P.coef[q][m].lo);
        const long double ref = R(a + (t + 1.0L) * w / 2);
        worst = fmax(worst, static_cast<double>(fabsl(p / ref - 1.0L)));
      }
    }
    P.max_rel_err = worst;
    if (worst < 2e-15) break;
  }
  for (int q = nint; q < kMaxIntervals; ++q)
    for (int m = 0; m <= kMaxDegree; ++m) P.coef[q][m] = F2{0.f, 0.f};
  return true;
}

}  // namespace dfm
