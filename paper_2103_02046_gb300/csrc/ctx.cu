// C ABI of the GB300 P3M library: parameter checks, the context (all scratch memory, FFT plans,
// streams) and the orchestration of one force evaluation, the leapfrog push and its reverse pass.
//
// One force evaluation (eq. (eom_p3m_coord) right-hand side), all stream-ordered:
//   bin + counting sort --(fork)--> short range on a side stream
//                       \--> zero mesh, deposit, R2C, Green multiply, C2R (long range)
//   join --> interpolation + combination, written in the caller's particle order.
// The short range (ALU-bound, the longest stage) runs at high priority; the mesh chain fills
// the SMs its blocks leave free, mostly in its tail.
#include <algorithm>
#include <memory>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "df_math.cuh"
#include "p3m_internal.cuh"

using namespace p3m;

namespace {

constexpr double kEps0 = 8.8541878128e-12;  // F/m, CODATA 2018
constexpr double kPi = 3.14159265358979323846;
constexpr double kElectronMass = 9.1093837015e-31;
constexpr double kElementaryCharge = 1.602176634e-19;
constexpr double kSpeedOfLight = 299792458.0;

p3m_status fail(p3m_ctx* c, p3m_status s, const char* msg) {
  if (c) c->last_error = msg;
  return s;
}

p3m_status cuda_fail(p3m_ctx* c, cudaError_t e, const char* where) {
  if (c) {
    c->last_error = std::string(where) + ": " + cudaGetErrorString(e);
  }
  return P3M_ECUDA;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

p3m_status validate(const p3m_params* p, std::string* why) {
  for (int d = 0; d < 3; ++d) {
    if (p->n[d] < 8 || p->n[d] > kMaxMesh) { *why = "mesh n must be in [8, 1024] per axis"; return P3M_EINVAL; }
    if (!finite_pos(p->h[d])) { *why = "mesh spacing h must be finite and > 0"; return P3M_EINVAL; }
    if (!std::isfinite(p->lo[d])) { *why = "mesh origin lo must be finite"; return P3M_EINVAL; }
  }
  if (!(p->rc_over_h >= 0.25) || !std::isfinite(p->rc_over_h)) { *why = "rc_over_h must be >= 0.25"; return P3M_EINVAL; }
  if (!(p->alpha > 0.0) && !finite_pos(p->kappa)) { *why = "kappa must be > 0 (or alpha > 0)"; return P3M_EINVAL; }
  if (p->assign_order != 1 && p->assign_order != 2) { *why = "assign_order must be 1 or 2"; return P3M_EINVAL; }
  if (p->pm_bc < 0 || p->pm_bc > 2 || (p->pp_bc != 0 && p->pp_bc != 1)) { *why = "pm_bc must be 0, 1 or 2 and pp_bc 0 or 1"; return P3M_EINVAL; }
  if (p->pm_bc == 2 && (p->precision != P3M_FP64 || p->pp_bc != 0 || p->influence != 0)) {
    *why = "the grounded box (pm_bc = 2) runs on the FP64 path with pp_bc = 0, influence = 0";
    return P3M_EINVAL;
  }
  if (!std::isfinite(p->z_cathode)) { *why = "z_cathode must be finite"; return P3M_EINVAL; }
  if (p->influence < 0 || p->influence > 2) { *why = "influence must be 0, 1 or 2"; return P3M_EINVAL; }
  if (p->precision != P3M_FP64 && p->precision != P3M_FP32_MIXED) { *why = "precision must be 0 or 1"; return P3M_EINVAL; }
  if (p->deterministic != 0 && p->deterministic != 1) { *why = "deterministic must be 0 or 1"; return P3M_EINVAL; }
  if (p->deterministic && p->precision != P3M_FP64) {
    *why = "deterministic = 1 runs on the FP64 path";
    return P3M_EINVAL;
  }
  if (p->deterministic && p->pm_bc == 2) {
    *why = "deterministic = 1 does not cover the grounded box";
    return P3M_EINVAL;
  }
  if (p->force_diff != 0 && p->force_diff != 1) { *why = "force_diff must be 0 or 1"; return P3M_EINVAL; }
  if (p->search_rows < 0 || p->search_rows > 3) { *why = "search_rows must be 0, 1, 2 or 3"; return P3M_EINVAL; }
  if (p->search_xcells < 0 || p->search_xcells > 32 ||
      (p->search_xcells & (p->search_xcells - 1)) != 0) {
    *why = "search_xcells must be 0, 1, 2, 4, 8, 16 or 32";
    return P3M_EINVAL;
  }
  if (p->adj_slots < 0 || p->adj_segment < 0 || (p->adj_slots > 0 && p->adj_segment < 1)) { *why = "adj_slots/adj_segment invalid"; return P3M_EINVAL; }
  if (!std::isfinite(p->q) || p->q == 0.0) { *why = "q must be finite and nonzero"; return P3M_EINVAL; }
  if (!finite_pos(p->mass)) { *why = "mass must be > 0"; return P3M_EINVAL; }
  return P3M_OK;
}

Geom make_geom(const p3m_params* p, int64_t n_max) {
  Geom g{};
  double hmax = 0.0;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = p->n[d];
    g.M[d] = 2 * p->n[d];
    g.lo[d] = p->lo[d];
    g.h[d] = p->h[d];
    hmax = std::max(hmax, p->h[d]);
  }
  g.rc = p->rc_over_h * hmax;
  g.alpha = p->alpha > 0.0 ? p->alpha : p->kappa / g.rc;
  g.kappa_eff = g.alpha * g.rc;
  // cells: y and z edges r_c (1 + 4 slack) / rows, x edges r_c / nsub, at most
  // max(4 n_max, 2^20) cells. rows = 2 (a tighter search) while the budget allows nsub = 4;
  // otherwise rows = 1, which keeps x edges r_c / 4 with 4x fewer cells: at low density the
  // per-particle row setup (13 neighbour rows of the half shell, or 5) and the x rounding of the
  // runs outweigh the pairs. A particle's row is computed in FP32 and may be off by one within
  // rounding (< slack / 3) of a row boundary; with rows (1 + 4 slack) r_c / rows wide, two
  // particles closer than r_c still sit at most `rows` rows apart, so the (2 rows + 1)^2 row
  // block around a particle's row holds all of its neighbours.
  double ext[3];
  double ext_max = 0.0;
  for (int d = 0; d < 3; ++d) {
    g.a[d] = g.h[d] / g.rc;
    ext[d] = (g.n[d] - 1) * g.a[d];
    ext_max = std::max(ext_max, ext[d]);
  }
  g.slack = std::max(1e-4, 1e-6 * ext_max);
  const double cap = std::max<double>(4.0 * static_cast<double>(n_max), 1 << 20);
  auto layout = [&](int rows, int nsub) {
    g.rows = rows;
    g.cw[0] = (1.0 + 1e-9) / nsub;
    g.cw[1] = g.cw[2] = (1.0 + 4.0 * g.slack) / rows;
    double cells = 1.0;
    for (int d = 0; d < 3; ++d) {
      g.inv_cw[d] = 1.0 / g.cw[d];
      g.nc[d] = static_cast<int>(std::floor(ext[d] * g.inv_cw[d])) + 1;
      cells *= g.nc[d];
    }
    return cells;
  };
  // Dense bunches: with hundreds of neighbours per particle the per-particle setup of more rows
  // is cheap next to the pairs, and narrower rows with shorter x cells cut the records tested
  // that are not pairs (in a uniform-density model, 46% of the records a particle tests are
  // pairs with rows r_c/2 and x cells r_c/4, 61% with rows r_c/3 and x cells r_c/16). The
  // neighbour estimate takes n_max particles over the mesh volume (a Gaussian bunch's core is
  // denser still).
  const double vol = std::max(ext[0], 1e-3) * std::max(ext[1], 1e-3) * std::max(ext[2], 1e-3);
  const double neighbours = static_cast<double>(n_max) * 4.18879020478639 / vol;
  if (p->search_rows > 0) {
    int nsub = p->search_xcells > 0 ? p->search_xcells : (p->search_rows == 3 ? 16 : 4);
    while (layout(p->search_rows, nsub) > cap && p->search_xcells == 0 && nsub > 1) nsub /= 2;
    if (layout(p->search_rows, nsub) > cap) g.rows = 0;  // refused by p3m_create
  } else {
    bool dense = false;
    if (neighbours >= 200.0)
      for (int nsub = p->search_xcells > 0 ? p->search_xcells : 16; nsub >= 4 && !dense; nsub /= 2)
        dense = layout(3, nsub) <= cap;
    if (!dense) {
      const int nsub0 = p->search_xcells > 0 ? p->search_xcells : 4;
      if (layout(2, nsub0) > cap) {
        // (with nsub = 1 the layout stands even over the budget; p3m_create still refuses
        // 2^32 cells or more)
        int nsub = nsub0;
        while (layout(1, nsub) > cap && nsub > 1 && p->search_xcells == 0) nsub /= 2;
        if (p->search_xcells > 0 && layout(1, nsub) > cap) g.rows = 0;
      }
    }
  }
  for (int d = 0; d < 3; ++d) {
    g.cw_f[d] = static_cast<float>(g.cw[d]);
    g.inv_cw_f[d] = static_cast<float>(g.inv_cw[d]);
  }
  g.slack_f = static_cast<float>(g.slack);
  auto df = [](double v, float out[2]) {
    out[0] = static_cast<float>(v);
    out[1] = static_cast<float>(v - static_cast<double>(out[0]));
  };
  for (int d = 0; d < 3; ++d) {
    df(g.lo[d], g.lo_df[d]);
    df(1.0 / g.h[d], g.inv_h_df[d]);
  }
  df(1.0 / g.rc, g.inv_rc_df);
  for (int d = 0; d < 3; ++d) {
    g.fscale_f[d] = static_cast<float>(-p->q / g.h[d]);
    df(g.rc / g.h[d], g.rch_df[d]);
  }
  g.order = p->assign_order;
  g.pm_bc = p->pm_bc;
  g.force_diff = p->force_diff;
  g.pp_bc = p->pp_bc;
  g.zc = p->z_cathode;
  g.img_c = 2.0 * (p->z_cathode - p->lo[2]) / g.rc;
  g.inv_rc = 1.0 / g.rc;
  for (int d = 0; d < 3; ++d) {
    g.inv_h[d] = 1.0 / g.h[d];
    g.inv_h_f[d] = static_cast<float>(g.inv_h[d]);
    g.inv_cell_f[d] = static_cast<float>(g.inv_cw[d] / g.rc);
    g.fscale[d] = -p->q / g.h[d];
  }
  g.q = p->q;
  g.mass = p->mass;
  g.ke = 1.0 / (4.0 * kPi * kEps0);
  return g;
}

// Polynomial for the FP32 pair kernel: R(x) = erfc(x) e^{x^2} on [0, kappa] in the variable
// t = 1 / (1 + p x) of Abramowitz & Stegun's form of erfc (7.1.26), p = 0.47, in which R is close
// to t times a low-degree polynomial: R(x) = t P(u), u = t - t_c, t_c the midpoint of
// [t_min, 1], t_min = 1 / (1 + p kappa) (the subtraction is exact where t and t_c are within a
// factor 2 of each other, i.e. for kappa up to about 4). P is fitted by Chebyshev interpolation
// at 96 nodes and converted to monomials in u. Evaluated as the kernel does in FP32, the erfc
// error falls with the degree to a floor of about 2e-7 set by FP32 rounding; the lowest degree
// whose error is below 2e-7 absolute, or within 30% of that floor, is kept (a force error of the
// same relative size, since erfc(x) <= 1 multiplies 1/rho^2 in the pair force): degree 6 for
// kappa = 3, where a polynomial in x itself needs degree 12.
PairPoly fit_pair_poly(double kappa) {
  PairPoly pp{};
  const double p = 0.47;
  const double tmin = 1.0 / (1.0 + p * kappa);
  const int N = 96;
  std::vector<double> un(N), fn(N);
  for (int j = 0; j < N; ++j) {
    un[j] = std::cos(kPi * (j + 0.5) / N);
    const double t = tmin + 0.5 * (un[j] + 1.0) * (1.0 - tmin);
    const double x = (1.0 / t - 1.0) / p;
    fn[j] = std::erfc(x) * std::exp(x * x) / t;
  }
  const double tc = 0.5 * (1.0 + tmin), hw = 0.5 * (1.0 - tmin);
  pp.pk = static_cast<float>(p * kappa);
  pp.tc = static_cast<float>(tc);
  std::vector<std::vector<float>> coefs(kMaxPoly);
  std::vector<double> errs(kMaxPoly, 1.0);
  for (int deg = 4; deg < kMaxPoly; ++deg) {
    std::vector<double> ch(deg + 1);
    for (int k = 0; k <= deg; ++k) {
      double acc = 0.0;
      for (int j = 0; j < N; ++j) acc += fn[j] * std::cos(k * std::acos(un[j]));
      ch[k] = acc * 2.0 / N;
    }
    ch[0] *= 0.5;
    // Chebyshev -> monomial in v = (t - t_c) / hw: T_0 = 1, T_1 = v, T_{k+1} = 2 v T_k - T_{k-1}
    std::vector<double> mono(deg + 1, 0.0), tkm1(deg + 1, 0.0), tk(deg + 1, 0.0), tkp1(deg + 1);
    tkm1[0] = 1.0;
    tk[1] = 1.0;
    mono[0] += ch[0];
    if (deg >= 1) mono[1] += ch[1];
    for (int k = 1; k < deg; ++k) {
      for (int m = 0; m <= deg; ++m) tkp1[m] = (m > 0 ? 2.0 * tk[m - 1] : 0.0) - tkm1[m];
      for (int m = 0; m <= deg; ++m) mono[m] += ch[k + 1] * tkp1[m];
      tkm1 = tk;
      tk = tkp1;
    }
    // then in u = t - t_c: coefficient m scaled by hw^-m
    coefs[deg].resize(deg + 1);
    for (int m = 0; m <= deg; ++m) coefs[deg][m] = static_cast<float>(mono[m] / std::pow(hw, m));
    double err = 0.0;
    for (int q = 0; q <= 4000; ++q) {
      const double x = kappa * q / 4000.0;
      const float rho = static_cast<float>(x / kappa);
      const float t = 1.0f / std::fma(pp.pk, rho, 1.0f);
      const float u = t - pp.tc;
      float r = coefs[deg][deg];
      for (int m = deg - 1; m >= 0; --m) r = std::fma(r, u, coefs[deg][m]);
      r *= t;
      err = std::max(err, std::fabs(static_cast<double>(r) * std::exp(-x * x) - std::erfc(x)));
    }
    errs[deg] = err;
  }
  const double floor_err = *std::min_element(errs.begin() + 4, errs.end());
  int deg = kMaxPoly - 1;
  for (int d = 4; d < kMaxPoly; ++d)
    if (errs[d] < 2e-7 || errs[d] <= 1.3 * floor_err) {
      deg = d;
      break;
    }
  pp.deg = deg;
  for (int m = 0; m <= deg; ++m) pp.c[m] = coefs[deg][m];
  pp.max_abs_err = static_cast<float>(errs[deg]);
  pp.kappa2_log2e = static_cast<float>(kappa * kappa * 1.4426950408889634);
  pp.kappa2 = static_cast<float>(kappa * kappa);
  pp.c2k = static_cast<float>(2.0 * kappa / std::sqrt(kPi));
  return pp;
}

template <typename T>
cudaError_t alloc(T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void**>(ptr), sizeof(T) * count);
}

void free_all(p3m_ctx* c) {
  void* bufs[] = {c->counts, c->starts, c->bsum, c->keys, c->ranks, c->recp, c->recm, c->fpp,
                  c->fplo, c->pdf,
                  c->acc, c->qpad, c->qhat, c->qhat2, c->khat_f, c->khat_i, c->fhat, c->freal,
                  c->phihat, c->phireal, c->dfac, c->ztw, c->box_real, c->box_spec, c->box_mult,
                  c->energy_acc, c->pair_acc,
                  c->pp_tile, c->err_dev, c->ckpt, c->seg, c->lam_x, c->lam_p, c->xw, c->pw,
                  c->tmp3, c->tmp3b, c->f_work, c->red, c->ered, c->q128, c->dbound, c->dred};
  for (void* b : bufs) cudaFree(b);
  if (c->err_host) cudaFreeHost(c->err_host);
  if (c->have_xy_f) cufftDestroy(c->plan_xy_f);
  if (c->have_z) cufftDestroy(c->plan_z);
  if (c->have_xy_i) cufftDestroy(c->plan_xy_i);
  if (c->have_box_f) cufftDestroy(c->plan_box_f);
  if (c->have_box_i) cufftDestroy(c->plan_box_i);
  if (c->s_pp) cudaStreamDestroy(c->s_pp);
  if (c->work) cudaStreamDestroy(c->work);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  for (auto& e : c->tev)
    if (e) cudaEventDestroy(e);
}

// Every call orders its work after the caller's stream (enter) and makes the caller's stream
// wait for it (finish); the work itself runs on the context's own streams.
void enter(p3m_ctx* c) {
  cudaEventRecord(c->ev_in, c->stream);
  cudaStreamWaitEvent(c->work, c->ev_in, 0);
}

// Returns a device error latched by earlier calls (and clears it), from the pinned mirror that
// every call refreshes asynchronously at its end. Also orders the call after the caller's stream.
p3m_status take_deferred(p3m_ctx* c) {
  enter(c);
  const int e = *reinterpret_cast<volatile int*>(c->err_host);
  if (!e) return P3M_OK;
  *c->err_host = 0;
  cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->work);
  if (e & kErrTimeout) return fail(c, P3M_ETIMEOUT, "a bounded device wait ran out");
  if (e & kErrNaN) return fail(c, P3M_EINVAL, "a particle position is NaN");
  return fail(c, P3M_ERANGE, "a particle lies outside the mesh's valid range or below the cathode");
}

p3m_status finish(p3m_ctx* c) {
  cudaMemcpyAsync(c->err_host, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->work);
  cudaEventRecord(c->ev_out, c->work);
  cudaStreamWaitEvent(c->stream, c->ev_out, 0);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
  return P3M_OK;
}

p3m_status check_n(p3m_ctx* c, int64_t n) {
  if (n < 0 || n > c->n_max) return fail(c, P3M_EINVAL, "n must be in [0, n_max]");
  return P3M_OK;
}

void sort_particles(p3m_ctx* c, const double* x, int64_t n, double* f_zero) {
  launch_bin(c, x, n, f_zero);
  launch_scan(c);
  launch_scatter(c, x, n);
  c->last_n = n;
}

p3m_status fft_r2c(p3m_ctx* c) {
  cufftResult r;
  if (c->fp32) {
    r = cufftExecR2C(c->plan_xy_f, static_cast<cufftReal*>(c->qpad),
                     static_cast<cufftComplex*>(c->qhat));
    if (r == CUFFT_SUCCESS)
      r = cufftExecC2C(c->plan_z, static_cast<cufftComplex*>(c->qhat),
                       static_cast<cufftComplex*>(c->qhat2), CUFFT_FORWARD);
  } else {
    r = cufftExecD2Z(c->plan_xy_f, static_cast<cufftDoubleReal*>(c->qpad),
                     static_cast<cufftDoubleComplex*>(c->qhat));
    if (r == CUFFT_SUCCESS)
      r = cufftExecZ2Z(c->plan_z, static_cast<cufftDoubleComplex*>(c->qhat),
                       static_cast<cufftDoubleComplex*>(c->qhat2), CUFFT_FORWARD);
  }
  return r == CUFFT_SUCCESS ? P3M_OK : fail(c, P3M_ECUFFT, "cuFFT forward transform failed");
}

// Inverse transform of one spectrum (destroyed) into the planes z < n_z of a real field.
cufftResult fft_c2r(p3m_ctx* c, void* spec, void* real) {
  cufftResult r;
  if (c->fp32) {
    r = cufftExecC2C(c->plan_z, static_cast<cufftComplex*>(spec),
                     static_cast<cufftComplex*>(spec), CUFFT_INVERSE);
    if (r == CUFFT_SUCCESS)
      r = cufftExecC2R(c->plan_xy_i, static_cast<cufftComplex*>(spec),
                       static_cast<cufftReal*>(real));
  } else {
    r = cufftExecZ2Z(c->plan_z, static_cast<cufftDoubleComplex*>(spec),
                     static_cast<cufftDoubleComplex*>(spec), CUFFT_INVERSE);
    if (r == CUFFT_SUCCESS)
      r = cufftExecZ2D(c->plan_xy_i, static_cast<cufftDoubleComplex*>(spec),
                       static_cast<cufftDoubleReal*>(real));
  }
  return r;
}

// Solve on the current qpad: FP64 -> potential; FP32 -> difference fields (and the potential
// when want_phi).
p3m_status mesh_solve(p3m_ctx* c, bool want_phi, bool want_diff, bool want_energy) {
  if (c->g.pm_bc == 2) {  // grounded box (FP64): the potential, on the interior nodes
    const p3m_status s = box_solve(c, want_energy);
    if (s != P3M_OK) return fail(c, s, "grounded-box solve failed");
    c->phi_valid = true;
    return P3M_OK;
  }
  if (c->zconv && want_diff && !want_phi) {
    // FP32 forces: x-y transforms of the charged planes, the fused z solve, x-y inverses
    if (cufftExecR2C(c->plan_xy_f, static_cast<cufftReal*>(c->qpad),
                     static_cast<cufftComplex*>(c->qhat)) != CUFFT_SUCCESS)
      return fail(c, P3M_ECUFFT, "cuFFT forward transform failed");
    launch_zconv(c, want_energy);
    for (int d = 0; d < 3; ++d) {
      auto* spec = static_cast<cufftComplex*>(c->fhat) + d * c->n_cplx;
      auto* real = static_cast<cufftReal*>(c->freal) + d * c->n_real;
      if (cufftExecC2R(c->plan_xy_i, spec, real) != CUFFT_SUCCESS)
        return fail(c, P3M_ECUFFT, "cuFFT inverse transform failed");
    }
    c->diff_valid = true;
    return P3M_OK;
  }
  if (c->zsolve_df) {
    // FP64 potential: x-y transforms of the charged planes, the fused z solve in double-float,
    // x-y inverses of the planes z < n_z
    if (cufftExecD2Z(c->plan_xy_f, static_cast<cufftDoubleReal*>(c->qpad),
                     static_cast<cufftDoubleComplex*>(c->qhat)) != CUFFT_SUCCESS)
      return fail(c, P3M_ECUFFT, "cuFFT forward transform failed");
    launch_zsolve_df(c, want_energy);
    if (cufftExecZ2D(c->plan_xy_i, static_cast<cufftDoubleComplex*>(c->phihat),
                     static_cast<cufftDoubleReal*>(c->phireal)) != CUFFT_SUCCESS)
      return fail(c, P3M_ECUFFT, "cuFFT inverse transform failed");
    c->phi_valid = true;
    return P3M_OK;
  }
  p3m_status s = fft_r2c(c);
  if (s != P3M_OK) return s;
  if (!c->fp32) want_phi = true, want_diff = false;
  // deterministic contexts form the mesh energy from the potential, in a fixed order
  launch_green_multiply(c, want_phi, want_diff, want_energy && !c->det);
  if (want_phi) {
    if (fft_c2r(c, c->phihat, c->phireal) != CUFFT_SUCCESS)
      return fail(c, P3M_ECUFFT, "cuFFT inverse transform failed");
    c->phi_valid = true;
    if (c->det && want_energy) launch_det_sum_mesh(c);
  }
  if (want_diff) {
    for (int d = 0; d < 3; ++d) {
      void* spec = static_cast<float2*>(c->fhat) + d * c->n_cplx;
      void* real = static_cast<float*>(c->freal) + d * c->n_real;
      if (fft_c2r(c, spec, real) != CUFFT_SUCCESS)
        return fail(c, P3M_ECUFFT, "cuFFT inverse transform failed");
    }
    c->diff_valid = true;
  }
  return P3M_OK;
}

p3m_status forces_impl(p3m_ctx* c, const double* x, int64_t n, double* f, double* energy,
                       int parts) {
  cudaStream_t st = c->work;
  cudaMemsetAsync(c->energy_acc, 0, 2 * sizeof(double), st);
  cudaMemsetAsync(c->pair_acc, 0, 3 * sizeof(unsigned long long), st);
  cudaEventRecord(c->tev[0], st);
  sort_particles(c, x, n, f);
  cudaEventRecord(c->tev[1], st);
  if (parts & 1) {
    cudaEventRecord(c->ev_fork, st);
    cudaStreamWaitEvent(c->s_pp, c->ev_fork, 0);
    cudaEventRecord(c->tev[6], c->s_pp);
    launch_pp(c, n, c->s_pp, energy != nullptr);
    cudaEventRecord(c->tev[7], c->s_pp);
    cudaEventRecord(c->ev_join, c->s_pp);
  }
  cudaEventRecord(c->tev[2], st);
  if (parts & 2) {
    launch_zero_block(c);
    launch_deposit(c, n);
    c->deposited = true;
    cudaEventRecord(c->tev[3], st);
    p3m_status s = mesh_solve(c, false, true, energy != nullptr);
    if (s != P3M_OK) return s;
  } else {
    cudaEventRecord(c->tev[3], st);
  }
  cudaEventRecord(c->tev[4], st);
  if (parts & 1) cudaStreamWaitEvent(st, c->ev_join, 0);
  launch_interp(c, n, f, parts);
  cudaEventRecord(c->tev[5], st);
  if (energy) launch_energy_out(c, energy);
  c->last_parts = parts;
  return P3M_OK;
}

// out = (dF/dx)^T w
p3m_status vjp_impl(p3m_ctx* c, const double* x, int64_t n, const double* w, double* out) {
  sort_particles(c, x, n, out);
  launch_pp_vjp(c, n, w, c->work);  // acc = short-range part
  launch_zero_block(c);
  launch_deposit(c, n);
  p3m_status s = mesh_solve(c, false, true, false);
  if (s != P3M_OK) return s;
  launch_vjp_gather(c, n, 0, w, out);
  launch_zero_block(c);
  launch_dipole_deposit(c, n, w);
  s = mesh_solve(c, false, true, false);
  if (s != P3M_OK) return s;
  launch_vjp_gather(c, n, 1, w, out);
  c->deposited = false;  // the mesh now holds the dipole deposit
  c->phi_valid = false;
  c->diff_valid = false;
  return P3M_OK;
}

p3m_status push_impl(p3m_ctx* c, double* x, double* p, int64_t n, double dt, int32_t nsteps,
                     double* f, bool f_valid) {
  if (!f_valid) {
    p3m_status s = forces_impl(c, x, n, f, nullptr, 3);
    if (s != P3M_OK) return s;
  }
  for (int32_t k = 0; k < nsteps; ++k) {
    launch_kick_drift(x, p, f, n, 0.5 * dt, dt / c->g.mass, c->work);
    p3m_status s = forces_impl(c, x, n, f, nullptr, 3);
    if (s != P3M_OK) return s;
    launch_kick_drift(x, p, f, n, 0.5 * dt, 0.0, c->work);
  }
  return P3M_OK;
}

}  // namespace

extern "C" {

p3m_status p3m_default_params(p3m_params* p) {
  if (!p) return P3M_EINVAL;
  std::memset(p, 0, sizeof(*p));
  for (int d = 0; d < 3; ++d) {
    p->n[d] = 64;
    p->lo[d] = 0.0;
    p->h[d] = 1e-5;
  }
  p->rc_over_h = 2.0;
  p->kappa = 3.0;
  p->alpha = 0.0;
  p->assign_order = 2;
  p->pm_bc = 0;
  p->pp_bc = 0;
  p->z_cathode = 0.0;
  p->influence = 0;
  p->force_diff = 0;
  p->search_rows = 0;
  p->search_xcells = 0;
  p->precision = P3M_FP64;
  p->deterministic = 0;
  p->adj_slots = 0;
  p->adj_segment = 0;
  p->q = 1e-15;
  p->mass = p->q / kElementaryCharge * kElectronMass;
  return P3M_OK;
}

p3m_status p3m_auto_mesh(const double* x, int64_t n, p3m_params* inout, void* stream) {
  if (!x || !inout || n < 1) return P3M_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (inout->n[d] < 8) return P3M_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* red = nullptr;
  if (cudaMalloc(&red, 8 * sizeof(double)) != cudaSuccess) return P3M_ENOMEM;
  launch_bbox(x, n, red, st);
  unsigned long long keys[6];
  int bad = 0;
  cudaError_t e = cudaMemcpyAsync(keys, red, sizeof(keys), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, red + 6, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(red);
  if (e != cudaSuccess) return P3M_ECUDA;
  if (bad) return P3M_EINVAL;
  for (int d = 0; d < 3; ++d) {
    auto unkey = [](unsigned long long k) {
      const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
      double v;
      std::memcpy(&v, &b, sizeof(v));
      return v;
    };
    const double a = unkey(keys[d]), b = unkey(keys[3 + d]);
    const double h = (b - a) / (inout->n[d] - 5);
    if (!(h > 0.0) || !std::isfinite(h)) return P3M_EINVAL;
    inout->h[d] = h;
    inout->lo[d] = a - 2.0 * h;
  }
  return P3M_OK;
}

p3m_status p3m_create(const p3m_params* params, int64_t n_max, void* stream, p3m_ctx** out) {
  if (!params || !out) return P3M_EINVAL;
  *out = nullptr;
  std::string why;
  if (validate(params, &why) != P3M_OK) {
    std::fprintf(stderr, "p3m_create: %s\n", why.c_str());
    return P3M_EINVAL;
  }
  if (n_max < 1 || n_max > 2147483647LL) return P3M_EINVAL;
  auto* c = new p3m_ctx();
  c->prm = *params;
  c->g = make_geom(params, n_max);
  if (c->g.rows == 0) {
    std::fprintf(stderr, "p3m_create: the short-range search layout exceeds the cell budget\n");
    delete c;
    return P3M_EINVAL;
  }
  c->poly = fit_pair_poly(c->g.kappa_eff);
  c->n_max = n_max;
  c->fp32 = params->precision == P3M_FP32_MIXED;
  c->det = params->deterministic != 0;
  c->stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&c->device);
  const Geom& g = c->g;
  c->nkeys = static_cast<uint64_t>(g.nc[0]) * g.nc[1] * g.nc[2];
  if (c->nkeys >= 0xFFFFFFF0ull ||
      static_cast<uint64_t>(g.nc[1]) * static_cast<uint64_t>(g.nc[2]) > kRowMask) {
    delete c;
    return P3M_EINVAL;
  }
  c->n_real = static_cast<size_t>(g.M[0]) * g.M[1] * g.M[2];
  c->n_cplx = static_cast<size_t>(g.M[0] / 2 + 1) * g.M[1] * g.M[2];
  const size_t es = c->fp32 ? 4 : 8;
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  const uint64_t tiles = (c->nkeys + 4095) / 4096;
  A(alloc(&c->counts, c->nkeys));
  A(alloc(&c->starts, c->nkeys + 1));
  A(alloc(&c->bsum, tiles));
  A(alloc(&c->keys, n_max));
  A(alloc(&c->ranks, n_max));
  A(cudaMalloc(&c->recp, 32 * static_cast<size_t>(n_max)));
  if (!c->fp32) A(cudaMalloc(&c->recm, 32 * static_cast<size_t>(n_max)));  // FP32: in recp
  // short-range result: FP64 {F, phi} (32 B); FP32 float4
  A(cudaMalloc(&c->fpp, (c->fp32 ? 16 : 32) * static_cast<size_t>(n_max)));
  if (c->fp32) A(alloc(&c->fplo, 2 * n_max));  // fine parts, then big terms
  A(alloc(&c->acc, 3 * n_max));
  A(cudaMalloc(&c->qpad, es * c->n_real));
  A(cudaMalloc(&c->qhat, 2 * es * c->n_cplx));
  A(cudaMalloc(&c->qhat2, 2 * es * c->n_cplx));
  A(cudaMalloc(&c->khat_f, es * c->n_cplx));
  if (g.pm_bc == 1) A(cudaMalloc(&c->khat_i, 2 * es * c->n_cplx));
  A(cudaMalloc(&c->phihat, 2 * es * c->n_cplx));
  A(cudaMalloc(&c->phireal, es * c->n_real));
  if (c->fp32) {
    A(cudaMalloc(&c->fhat, 3 * 2 * es * c->n_cplx));
    A(cudaMalloc(&c->freal, 3 * es * c->n_real));
    A(alloc(&c->dfac, static_cast<size_t>(g.M[0] / 2 + 1 + g.M[1] + g.M[2])));
  }
  A(alloc(&c->energy_acc, 2));
  A(alloc(&c->pair_acc, 3));
  A(alloc(&c->pp_tile, 1));
  A(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  A(alloc(&c->err_dev, 1));
  A(alloc(&c->red, 32));
  A(alloc(&c->ered, static_cast<size_t>(kEmitBlocks) * 16));
  if (params->deterministic) {
    const size_t nn = static_cast<size_t>(g.n[0]) * g.n[1] * g.n[2];
    A(alloc(&c->q128, 2 * nn));
    A(alloc(&c->dbound, 1));
    A(alloc(&c->dred, 2 * 1024));
  }
  A(alloc(&c->f_work, 3 * n_max));
  // FP64 path: the pair function in double-float arithmetic (kappa up to 6.5, where its relative
  // error stays below about 2e-13; beyond, the FP64 pair function)
  if (!c->fp32 && c->g.kappa_eff <= 6.5 && e == cudaSuccess) {
    std::unique_ptr<dfm::PairDF> tab(new dfm::PairDF());  // filled on the host, then copied
    if (dfm::fit_pair_df(c->g.kappa_eff, *tab)) {
      A(alloc(&c->pdf, 1));
      if (e == cudaSuccess)
        e = cudaMemcpy(c->pdf, tab.get(), sizeof(dfm::PairDF), cudaMemcpyHostToDevice);
    }
  }
  if (params->adj_slots > 0) {
    A(alloc(&c->ckpt, static_cast<size_t>(params->adj_slots) * 6 * n_max));
    A(alloc(&c->seg, static_cast<size_t>(params->adj_segment + 1) * 3 * n_max));
    A(alloc(&c->lam_x, 3 * n_max));
    A(alloc(&c->lam_p, 3 * n_max));
    A(alloc(&c->xw, 3 * n_max));
    A(alloc(&c->pw, 3 * n_max));
    A(alloc(&c->tmp3, 3 * n_max));
    A(alloc(&c->tmp3b, 3 * n_max));
  }
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&c->err_host), sizeof(int), 0);
  int prio_low = 0, prio_high = 0;
  cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  if (e == cudaSuccess)
    e = cudaStreamCreateWithPriority(&c->work, cudaStreamNonBlocking, prio_low);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->s_pp, cudaStreamNonBlocking, prio_high);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
  for (auto& ev : c->tev)
    if (e == cudaSuccess) e = cudaEventCreate(&ev);
  if (e != cudaSuccess) {
    free_all(c);
    delete c;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? P3M_ENOMEM : P3M_ECUDA;
  }
  *c->err_host = 0;
  cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->work);
  cudaMemsetAsync(c->qpad, 0, es * c->n_real, c->work);
  cudaMemsetAsync(c->qhat, 0, 2 * es * c->n_cplx, c->work);  // planes z >= n_z stay zero
  if (c->fp32) {
    std::vector<float2> fac(g.M[0] / 2 + 1 + g.M[1] + g.M[2]);
    size_t o = 0;
    auto put = [&](int M, int count) {
      for (int k = 0; k < count; ++k) {
        const double s = std::sin(kPi * k / M), co = std::cos(kPi * k / M);
        fac[o++] = make_float2(static_cast<float>(-2.0 * s * s), static_cast<float>(2.0 * s * co));
      }
    };
    put(g.M[0], g.M[0] / 2 + 1);
    put(g.M[1], g.M[1]);
    put(g.M[2], g.M[2]);
    cudaMemcpyAsync(c->dfac, fac.data(), sizeof(float2) * fac.size(), cudaMemcpyHostToDevice,
                    c->work);
  }
  // FFT plans (see p3m_internal.cuh: pruned to the planes that carry charge or are read back)
  {
    const int Hx = g.M[0] / 2 + 1;
    int xy[2] = {g.M[1], g.M[0]};
    int in_r[2] = {g.M[1], g.M[0]}, in_c[2] = {g.M[1], Hx};
    int zlen[1] = {g.M[2]};
    const long long col = static_cast<long long>(g.M[1]) * Hx;
    cufftResult r = cufftPlanMany(&c->plan_xy_f, 2, xy, in_r, 1, g.M[1] * g.M[0], in_c, 1,
                                  g.M[1] * Hx, c->fp32 ? CUFFT_R2C : CUFFT_D2Z, g.n[2]);
    c->have_xy_f = r == CUFFT_SUCCESS;
    if (r == CUFFT_SUCCESS) {
      r = cufftPlanMany(&c->plan_z, 1, zlen, zlen, static_cast<int>(col), 1, zlen,
                        static_cast<int>(col), 1, c->fp32 ? CUFFT_C2C : CUFFT_Z2Z,
                        static_cast<int>(col));
      c->have_z = r == CUFFT_SUCCESS;
    }
    if (r == CUFFT_SUCCESS) {
      r = cufftPlanMany(&c->plan_xy_i, 2, xy, in_c, 1, g.M[1] * Hx, in_r, 1, g.M[1] * g.M[0],
                        c->fp32 ? CUFFT_C2R : CUFFT_Z2D, g.n[2]);
      c->have_xy_i = r == CUFFT_SUCCESS;
    }
    if (r != CUFFT_SUCCESS) {
      free_all(c);
      delete c;
      return r == CUFFT_ALLOC_FAILED ? P3M_ENOMEM : P3M_ECUFFT;
    }
    cufftSetStream(c->plan_xy_f, c->work);
    cufftSetStream(c->plan_z, c->work);
    cufftSetStream(c->plan_xy_i, c->work);
  }
  e = g.pm_bc == 2 ? cudaSuccess : build_green(c);
  if (e == cudaSuccess && g.pm_bc == 2) {
    const p3m_status bs = box_setup(c);
    if (bs != P3M_OK) {
      free_all(c);
      delete c;
      cudaGetLastError();
      return bs;
    }
  }
  if (e == cudaSuccess && zconv_supported(c)) {
    e = zconv_setup(c);
    c->zconv = e == cudaSuccess;
  }
  if (e == cudaSuccess && zsolve_df_supported(c)) {
    e = zsolve_df_setup(c);
    c->zsolve_df = e == cudaSuccess;
  }
  if (e != cudaSuccess) {
    free_all(c);
    delete c;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? P3M_ENOMEM : P3M_ECUFFT;
  }
  *out = c;
  return P3M_OK;
}

p3m_status p3m_destroy(p3m_ctx* c) {
  if (!c) return P3M_OK;
  cudaStreamSynchronize(c->work);
  cudaStreamSynchronize(c->s_pp);
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
  return P3M_OK;
}

p3m_status p3m_set_stream(p3m_ctx* c, void* stream) {
  if (!c) return P3M_EINVAL;
  c->stream = static_cast<cudaStream_t>(stream);
  return P3M_OK;
}

p3m_status p3m_deposit(p3m_ctx* c, const double* x, int64_t n) {
  if (!c) return P3M_EINVAL;
  if (!x && n > 0) return fail(c, P3M_EINVAL, "x is NULL");
  p3m_status s = take_deferred(c);
  if (s != P3M_OK) return s;
  if ((s = check_n(c, n)) != P3M_OK) return s;
  sort_particles(c, x, n, nullptr);
  launch_zero_block(c);
  launch_deposit(c, n);
  c->deposited = true;
  c->phi_valid = false;
  c->diff_valid = false;
  return finish(c);
}

p3m_status p3m_solve(p3m_ctx* c) {
  if (!c) return P3M_EINVAL;
  p3m_status s = take_deferred(c);
  if (s != P3M_OK) return s;
  if (!c->deposited) return fail(c, P3M_ESTATE, "p3m_solve needs a deposit first");
  cudaMemsetAsync(c->energy_acc, 0, 2 * sizeof(double), c->work);
  s = mesh_solve(c, true, c->fp32, true);
  if (s != P3M_OK) return s;
  return finish(c);
}

p3m_status p3m_get_mesh(p3m_ctx* c, int32_t which, double* out) {
  if (!c || !out || which < 0 || which > 4) return P3M_EINVAL;
  if (which == 0 && !c->deposited) return fail(c, P3M_ESTATE, "no deposit");
  if (which == 1 && !c->phi_valid) return fail(c, P3M_ESTATE, "no potential (call p3m_solve)");
  if (which >= 2 && !(c->fp32 && c->diff_valid))
    return fail(c, P3M_ESTATE, "no difference fields (FP32 path, after p3m_forces)");
  enter(c);
  launch_get_mesh(c, which, out);
  return finish(c);
}

p3m_status p3m_forces_ex(p3m_ctx* c, const double* x, int64_t n, double* f, double* energy,
                         int32_t parts) {
  if (!c) return P3M_EINVAL;
  if ((!x || !f) && n > 0) return fail(c, P3M_EINVAL, "x or f is NULL");
  if (parts < 1 || parts > 3) return fail(c, P3M_EINVAL, "parts must be 1, 2 or 3");
  if (x == f && n > 0) return fail(c, P3M_EINVAL, "f may not alias x");
  p3m_status s = take_deferred(c);
  if (s != P3M_OK) return s;
  if ((s = check_n(c, n)) != P3M_OK) return s;
  s = forces_impl(c, x, n, f, energy, parts);
  if (s != P3M_OK) return s;
  if (parts & 2) c->phi_valid = !c->fp32;
  return finish(c);
}

p3m_status p3m_forces(p3m_ctx* c, const double* x, int64_t n, double* f, double* energy) {
  return p3m_forces_ex(c, x, n, f, energy, 3);
}

p3m_status p3m_pair_count(p3m_ctx* c, int64_t* pairs, int64_t* image_pairs) {
  if (!c || !pairs) return P3M_EINVAL;
  unsigned long long v[2] = {0, 0};
  enter(c);
  cudaError_t e = cudaMemcpyAsync(v, c->pair_acc, sizeof(v), cudaMemcpyDeviceToHost, c->work);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->work);
  if (e != cudaSuccess) return cuda_fail(c, e, "p3m_pair_count");
  *pairs = static_cast<int64_t>(v[0]);
  if (image_pairs) *image_pairs = static_cast<int64_t>(v[1]);
  return P3M_OK;
}

p3m_status p3m_candidate_count(p3m_ctx* c, int64_t* candidates) {
  if (!c || !candidates) return P3M_EINVAL;
  unsigned long long v = 0;
  enter(c);
  launch_pp_count(c, c->last_n, c->pair_acc + 2, c->work);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&v, c->pair_acc + 2, sizeof(v), cudaMemcpyDeviceToHost, c->work);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->work);
  if (e != cudaSuccess) return cuda_fail(c, e, "p3m_candidate_count");
  *candidates = static_cast<int64_t>(v);
  return P3M_OK;
}

p3m_status p3m_search_layout(const p3m_ctx* c, int32_t* rows, int32_t* xcells) {
  if (!c || !rows || !xcells) return P3M_EINVAL;
  *rows = c->g.rows;
  *xcells = static_cast<int32_t>(std::lround(1.0 / c->g.cw[0]));
  return P3M_OK;
}

p3m_status p3m_push_ex(p3m_ctx* c, double* x, double* p, int64_t n, double dt, int32_t nsteps,
                       double* f, int32_t f_valid) {
  if (!c) return P3M_EINVAL;
  if ((!x || !p || !f) && n > 0) return fail(c, P3M_EINVAL, "x, p or f is NULL");
  if (nsteps < 0 || !std::isfinite(dt)) return fail(c, P3M_EINVAL, "bad dt or nsteps");
  p3m_status s = take_deferred(c);
  if (s != P3M_OK) return s;
  if ((s = check_n(c, n)) != P3M_OK) return s;
  s = push_impl(c, x, p, n, dt, nsteps, f, f_valid != 0);
  if (s != P3M_OK) return s;
  return finish(c);
}

p3m_status p3m_push(p3m_ctx* c, double* x, double* p, int64_t n, double dt, int32_t nsteps,
                    double* f) {
  if (!c) return P3M_EINVAL;
  // f given: it holds F(x0) and receives F(x_end); NULL: the forces live in the context's
  // scratch (f_work, not otherwise in use during a push)
  if (f) return p3m_push_ex(c, x, p, n, dt, nsteps, f, 1);
  return p3m_push_ex(c, x, p, n, dt, nsteps, c->f_work, 0);
}

p3m_status p3m_force_vjp(p3m_ctx* c, const double* x, int64_t n, const double* w, double* out) {
  if (!c) return P3M_EINVAL;
  if ((!x || !w || !out) && n > 0) return fail(c, P3M_EINVAL, "NULL argument");
  if (c->g.force_diff)
    return fail(c, P3M_ESTATE, "the adjoint needs the variational force (force_diff = 0)");
  p3m_status s = take_deferred(c);
  if (s != P3M_OK) return s;
  if ((s = check_n(c, n)) != P3M_OK) return s;
  s = vjp_impl(c, x, n, w, out);
  if (s != P3M_OK) return s;
  return finish(c);
}

p3m_status p3m_backward(p3m_ctx* c, const double* x0, const double* p0, int64_t n, double dt,
                        int32_t nsteps, int32_t ckpt_every, const double* gx_T,
                        const double* gp_T, double* gx0, double* gp0) {
  if (!c) return P3M_EINVAL;
  if ((!x0 || !p0 || !gx_T || !gp_T || !gx0 || !gp0) && n > 0)
    return fail(c, P3M_EINVAL, "NULL argument");
  if (c->prm.adj_slots <= 0) return fail(c, P3M_ESTATE, "context created with adj_slots = 0");
  if (c->g.force_diff)
    return fail(c, P3M_ESTATE, "the adjoint needs the variational force (force_diff = 0)");
  // checkpoints every ckpt_every steps (0: adj_segment); the segment buffer holds adj_segment
  if (ckpt_every < 0 || ckpt_every > c->prm.adj_segment)
    return fail(c, P3M_EINVAL, "ckpt_every must be in [0, adj_segment]");
  const int C = ckpt_every > 0 ? ckpt_every : c->prm.adj_segment;
  if (nsteps < 1 || static_cast<int64_t>(c->prm.adj_slots) * C < nsteps || !std::isfinite(dt))
    return fail(c, P3M_EINVAL, "nsteps must be in [1, adj_slots * ckpt_every]");
  p3m_status s = take_deferred(c);
  if (s != P3M_OK) return s;
  if ((s = check_n(c, n)) != P3M_OK) return s;
  cudaStream_t st = c->work;
  const size_t n3 = 3 * static_cast<size_t>(n);
  const size_t bytes = n3 * sizeof(double);
  const size_t slot = 6 * static_cast<size_t>(c->n_max);
  const int K = (nsteps + C - 1) / C;
  // forward sweep: checkpoints of (x, p) at the start of every segment
  cudaMemcpyAsync(c->xw, x0, bytes, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(c->pw, p0, bytes, cudaMemcpyDeviceToDevice, st);
  bool f_valid = false;
  for (int k = 0; k < K; ++k) {
    cudaMemcpyAsync(c->ckpt + k * slot, c->xw, bytes, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(c->ckpt + k * slot + 3 * c->n_max, c->pw, bytes, cudaMemcpyDeviceToDevice, st);
    const int steps = std::min(C, nsteps - k * C);
    if (k < K - 1) {
      if ((s = push_impl(c, c->xw, c->pw, n, dt, steps, c->f_work, f_valid)) != P3M_OK) return s;
      f_valid = true;
    }
  }
  // reverse sweep
  cudaMemcpyAsync(c->lam_x, gx_T, bytes, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(c->lam_p, gp_T, bytes, cudaMemcpyDeviceToDevice, st);
  bool first = true;
  for (int k = K - 1; k >= 0; --k) {
    const int steps = std::min(C, nsteps - k * C);
    cudaMemcpyAsync(c->xw, c->ckpt + k * slot, bytes, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(c->pw, c->ckpt + k * slot + 3 * c->n_max, bytes, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(c->seg, c->xw, bytes, cudaMemcpyDeviceToDevice, st);
    bool fv = false;
    for (int t = 1; t <= steps; ++t) {
      if ((s = push_impl(c, c->xw, c->pw, n, dt, 1, c->f_work, fv)) != P3M_OK) return s;
      fv = true;
      cudaMemcpyAsync(c->seg + t * 3 * c->n_max, c->xw, bytes, cudaMemcpyDeviceToDevice, st);
    }
    for (int t = steps - 1; t >= 0; --t) {
      const int64_t gstep = static_cast<int64_t>(k) * C + t;
      if (first) {  // end-of-step kick of the last step: lam_x += J(x_T)^T (dt/2 lam_p)
        launch_scale(c->tmp3, c->lam_p, n3, 0.5 * dt, st);
        if ((s = vjp_impl(c, c->seg + (t + 1) * 3 * c->n_max, n, c->tmp3, c->tmp3b)) != P3M_OK)
          return s;
        launch_axpy(c->lam_x, c->tmp3b, n3, 1.0, st);
        first = false;
      }
      launch_axpy(c->lam_p, c->lam_x, n3, dt / c->g.mass, st);  // drift
      // start-of-step kick of this step merged with the end-of-step kick of the previous one
      const double coef = gstep > 0 ? dt : 0.5 * dt;
      launch_scale(c->tmp3, c->lam_p, n3, coef, st);
      if ((s = vjp_impl(c, c->seg + t * 3 * c->n_max, n, c->tmp3, c->tmp3b)) != P3M_OK) return s;
      launch_axpy(c->lam_x, c->tmp3b, n3, 1.0, st);
    }
  }
  cudaMemcpyAsync(gx0, c->lam_x, bytes, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(gp0, c->lam_p, bytes, cudaMemcpyDeviceToDevice, st);
  return finish(c);
}

p3m_status p3m_emittance(p3m_ctx* c, const double* x, const double* p, int64_t n, double* eps3,
                         double* gx, double* gp) {
  if (!c) return P3M_EINVAL;
  if (!x || !p || !eps3 || n < 2) return fail(c, P3M_EINVAL, "bad argument");
  p3m_status s = take_deferred(c);
  if (s != P3M_OK) return s;
  launch_emittance(x, p, n, c->g.mass * kSpeedOfLight, eps3, gx, gp, c->ered, c->red, c->work);
  return finish(c);
}

p3m_status p3m_sync(p3m_ctx* c) {
  if (!c) return P3M_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->work);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_pp);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "p3m_sync");
  int v = 0;
  e = cudaMemcpy(&v, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "p3m_sync");
  *c->err_host = v;
  return take_deferred(c);
}

p3m_status p3m_get_timings(p3m_ctx* c, double* ms, int32_t cap, int32_t* count) {
  if (!c || !ms || cap < 0) return P3M_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->work);
  if (e != cudaSuccess) return cuda_fail(c, e, "p3m_get_timings");
  float t[6] = {0, 0, 0, 0, 0, 0};
  cudaEventElapsedTime(&t[0], c->tev[0], c->tev[1]);
  if (c->last_parts & 1) cudaEventElapsedTime(&t[1], c->tev[6], c->tev[7]);
  if (c->last_parts & 2) {
    cudaEventElapsedTime(&t[2], c->tev[2], c->tev[3]);
    cudaEventElapsedTime(&t[3], c->tev[3], c->tev[4]);
  }
  cudaEventElapsedTime(&t[4], c->tev[4], c->tev[5]);
  cudaEventElapsedTime(&t[5], c->tev[0], c->tev[5]);
  cudaGetLastError();
  const int k = std::min<int32_t>(cap, 6);
  for (int i = 0; i < k; ++i) ms[i] = t[i];
  if (count) *count = 6;
  return P3M_OK;
}

const char* p3m_last_error(const p3m_ctx* c) {
  if (!c) return "null context";
  return c->last_error.c_str();
}

}  // extern "C"
