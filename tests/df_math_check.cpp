// Host check of the FP64 path's double-float pair function (paper_2103_02046_gb300/csrc/
// df_math.cuh) against long-double erfc and exp: for kappa = alpha r_c given on the command
// line, the largest relative errors of the potential erfc(x)/rho, the force coefficient
// [erfc(x)/rho + (2 kappa/sqrt(pi)) e^{-x^2}]/rho^2 and the Hessian term of the adjoint over
// rho in (0, 1] (eq. (ewald_split), eq. (summation_short)), printed as one JSON line.
// With the argument "split": the bit-level split of doubles into double-float that the FP64
// path's fused z solve applies to the charge spectrum, against the doubles themselves.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <random>

#include "df_math.cuh"

// Largest relative error of hi + lo over seeded random doubles whose magnitudes span
// 10^-22 .. 10^37 (the fast path; smaller and larger ones take the FP64 conversion), how many
// violate |lo| < ulp(hi) or carry the wrong sign, and the special values.
static int split_check() {
  std::mt19937_64 gen(20210302);
  std::normal_distribution<double> nd(0.0, 1.0);
  std::uniform_real_distribution<double> ud(-22.0, 37.0);
  double worst = 0.0, worst_slow = 0.0;
  long bad_ulp = 0, bad_sign = 0, fast = 0;
  for (int k = 0; k < 400000; ++k) {
    const double v = nd(gen) * std::pow(10.0, ud(gen));
    if (v == 0.0) continue;
    const dfm::F2 d = dfm::split_double(v);
    const double err = std::fabs((static_cast<double>(d.hi) + d.lo - v) / v);
    const int e = static_cast<int>((dfm::bits_of(v) >> 52) & 0x7ff);
    if (e >= 949 && e <= 1150) {
      ++fast;
      worst = std::fmax(worst, err);
      if (std::fabs(d.lo) >= std::ldexp(std::fabs(d.hi), -23)) ++bad_ulp;
      if ((d.hi < 0) != (v < 0) || (d.lo != 0 && (d.lo < 0) != (v < 0))) ++bad_sign;
    } else {
      worst_slow = std::fmax(worst_slow, err);
    }
  }
  const dfm::F2 z = dfm::split_double(0.0), nz = dfm::split_double(-0.0);
  const dfm::F2 one = dfm::split_double(1.0), third = dfm::split_double(-1.0 / 3.0);
  const double sub = std::ldexp(1.0, -1050);  // subnormal
  const dfm::F2 s = dfm::split_double(sub);
  const double edge = std::ldexp(1.0, -74);  // smallest value on the fast path
  const dfm::F2 ed = dfm::split_double(edge * 1.2345);
  std::printf("{\"fast\": %ld, \"worst\": %.3e, \"worst_slow\": %.3e, \"bad_ulp\": %ld, "
              "\"bad_sign\": %ld, \"zero\": %d, \"neg_zero\": %d, \"one\": %d, "
              "\"third_err\": %.3e, \"subnormal\": %d, \"edge_err\": %.3e}\n",
              fast, worst, worst_slow, bad_ulp, bad_sign,
              z.hi == 0.f && z.lo == 0.f && !std::signbit(z.hi),
              nz.hi == 0.f && std::signbit(nz.hi), one.hi == 1.f && one.lo == 0.f,
              std::fabs((static_cast<double>(third.hi) + third.lo) * 3.0 + 1.0),
              s.hi == 0.f && s.lo == 0.f,
              std::fabs((static_cast<double>(ed.hi) + ed.lo) / (edge * 1.2345) - 1.0));
  return 0;
}

int main(int argc, char** argv) {
  if (argc > 1 && std::strcmp(argv[1], "split") == 0) return split_check();
  const double kappa = argc > 1 ? std::atof(argv[1]) : 3.0;
  std::unique_ptr<dfm::PairDF> P(new dfm::PairDF());
  if (!dfm::fit_pair_df(kappa, *P)) {
    std::printf("{\"kappa\": %g, \"fit\": false}\n", kappa);
    return 0;
  }
  const long double pi = 3.14159265358979323846264338327950288L;
  const long double c2k = 2.0L * kappa / sqrtl(pi);
  double wp = 0, wf = 0, wd = 0;
  for (int u = 1; u <= 100000; ++u) {
    // a uniform grid on (0, 1] and a finer one on (0, 0.01]
    const double rho = (u % 5 == 0) ? u / 100000.0 * 0.01 : u / 100000.0;
    const double s = rho * rho;
    const dfm::F2 sd{static_cast<float>(s), static_cast<float>(s - static_cast<float>(s))};
    const dfm::PairOut o = dfm::pair_df(P->k, P->coef, sd);
    dfm::F2 hf, hd;
    dfm::pair_hess_df(P->k, P->coef, sd, hf, hd);
    const long double sl = static_cast<long double>(sd.hi) + sd.lo;
    const long double r = sqrtl(sl), x = kappa * r, ex = expl(-x * x), ec = erfcl(x);
    const long double pot = ec / r, A = pot + c2k * ex, fco = A / sl;
    const long double dA = -c2k * ex / r - ec / sl - 2.0L * kappa * kappa * r * c2k * ex;
    const long double dfr = (dA / sl - 2.0L * A / (sl * r)) / r;
    auto rel = [](dfm::F2 v, long double ref) {
      return static_cast<double>(fabsl((static_cast<long double>(v.hi) + v.lo) / ref - 1.0L));
    };
    wp = std::fmax(wp, rel(o.pot, pot));
    wf = std::fmax(wf, rel(o.fco, fco));
    wd = std::fmax(wd, rel(hd, dfr));
  }
  std::printf("{\"kappa\": %g, \"fit\": true, \"intervals\": %d, \"degree\": %d, "
              "\"fit_err\": %.3e, \"pot\": %.3e, \"fco\": %.3e, \"dfr\": %.3e}\n",
              kappa, P->k.nint, P->k.deg, P->max_rel_err, wp, wf, wd);
  return 0;
}
