// Host check of the FP64 path's double-float pair function (paper_2103_02046_gb300/csrc/
// df_math.cuh) against long-double erfc and exp: for kappa = alpha r_c given on the command
// line, the largest relative errors of the potential erfc(x)/rho, the force coefficient
// [erfc(x)/rho + (2 kappa/sqrt(pi)) e^{-x^2}]/rho^2 and the Hessian term of the adjoint over
// rho in (0, 1] (eq. (ewald_split), eq. (summation_short)), printed as one JSON line.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <memory>

#include "df_math.cuh"

int main(int argc, char** argv) {
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
