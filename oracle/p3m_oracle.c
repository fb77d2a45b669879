/*
 * p3m_oracle.c -- plain FP64 CPU oracle of the P3M space-charge force evaluation.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file's library. The product path never calls it and shares no
 * code, header, table or constant with it. Every routine here is the plain definition of
 * one step of the method, written for a reader to check against the paper
 * (Wyssling & Adelmann, "On Boundary Conditions in the sub-mesh interaction of the P3M
 * algorithm", arXiv 2103.02046), in double precision, without blocking, fusion or reordering.
 *
 * Conventions (the paper's readings, stated once):
 *   * SI units. k_e = 1/(4 pi eps0). The paper's Poisson equation and Green's function carry
 *     sign and 4 pi slips (Sec. 2.1 and Sec. 3, eq. (greens_function_for_poisson)); here the
 *     potential of a charge q at distance r is k_e q / r.
 *   * Ewald split (Sec. 2.2, eq. (ewald_split)): 1/r = erfc(a r)/r + erf(a r)/r, with
 *     erf the standard error function (the integral printed in the text is erfc/4; the
 *     complement relation printed next to it is the one used).
 *   * Grounded planar cathode at z = zc (Sec. 3.1, eq. (GreenFunc_planar_cathode) and
 *     eq. (symmetry_planar_cathode)): G(x,y) = G^F(x,y) - G^F(x,S(y)), S(x,y,z) = (x,y,2zc-z).
 *   * Mesh (Sec. 2.4.2): node g at lo + g*h per axis, arrays stored x fastest:
 *     index (gz*ny + gy)*nx + gx. Assignment W = product of 1D B-splines in mesh units,
 *     order 1 (cloud-in-cell, eq. (interpolation_splines_b0)) or 2 (TSC, one order higher).
 *   * Node charges Q_g = q sum_i W(x_g - xi_i). The cell volume factors of eq. (eom_p3m_poiss_L)
 *     and eq. (phi_L) cancel between the charge density and the discrete convolution.
 *   * A particle is valid when its TSC nearest node (floor(s+1/2)) lies in [1, n-2] on every
 *     axis (CIC: floor(s) in [0, n-2]); invalid particles are skipped and counted.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_EPS0 8.8541878128e-12 /* F/m, CODATA 2018 */
#define ORACLE_PI 3.14159265358979323846

static double coulomb_k(void) { return 1.0 / (4.0 * ORACLE_PI * ORACLE_EPS0); }

double oracle_coulomb_constant(void) { return coulomb_k(); }

/* ------------------------------------------------------------------------------------------
 * B-spline assignment along one axis, Sec. 2.4.2 (eq. (WL), eq. (interpolation_splines_b0)).
 * s = (xi - lo)/h is the particle position in mesh units. Returns the first node index g0 of
 * the support; w[k] is the weight of node g0+k, dw[k] its derivative d/ds and d2w[k] its
 * second derivative d2/ds2 (all in mesh units).
 * TSC: c = floor(s + 1/2), u = s - c in [-1/2, 1/2):
 *      w = { (1/2 - u)^2 / 2, 3/4 - u^2, (1/2 + u)^2 / 2 }  on nodes c-1, c, c+1.
 * CIC: c = floor(s), f = s - c:  w = { 1 - f, f } on nodes c, c+1.
 * ------------------------------------------------------------------------------------------ */
static int spline_1d(double s, int order, double *w, double *dw, double *d2w) {
  if (order == 2) {
    double c = floor(s + 0.5);
    double u = s - c;
    w[0] = 0.5 * (0.5 - u) * (0.5 - u);
    w[1] = 0.75 - u * u;
    w[2] = 0.5 * (0.5 + u) * (0.5 + u);
    dw[0] = -(0.5 - u);
    dw[1] = -2.0 * u;
    dw[2] = 0.5 + u;
    d2w[0] = 1.0;
    d2w[1] = -2.0;
    d2w[2] = 1.0;
    return (int)c - 1;
  } else {
    double c = floor(s);
    double f = s - c;
    w[0] = 1.0 - f;
    w[1] = f;
    dw[0] = -1.0;
    dw[1] = 1.0;
    d2w[0] = 0.0;
    d2w[1] = 0.0;
    w[2] = dw[2] = d2w[2] = 0.0;
    return (int)c;
  }
}

static int support(int order) { return order == 2 ? 3 : 2; }

/* Fills g0[3] and the per-axis weights for particle position p; returns 0 if the particle is
 * valid (whole support inside the mesh), 1 otherwise. */
static int particle_weights(const double *p, const int32_t *n, const double *lo, const double *h,
                            int order, int *g0, double w[3][3], double dw[3][3],
                            double d2w[3][3]) {
  int bad = 0;
  for (int d = 0; d < 3; ++d) {
    double s = (p[d] - lo[d]) / h[d];
    if (!(s == s)) return 1; /* NaN */
    g0[d] = spline_1d(s, order, w[d], dw[d], d2w[d]);
    if (g0[d] < 0 || g0[d] + support(order) - 1 > n[d] - 1) bad = 1;
  }
  return bad;
}

static int64_t mesh_index(const int32_t *n, int gx, int gy, int gz) {
  return ((int64_t)gz * n[1] + gy) * n[0] + gx;
}

/* Charge assignment, eq. (rho_L) with W = W^L: Q_g = q sum_i W(x_g - xi_i).
 * Q (n0*n1*n2) is overwritten. Returns the number of skipped (invalid) particles. */
int64_t oracle_deposit(int64_t N, const double *x, double q, const int32_t *n, const double *lo,
                       const double *h, int order, double *Q) {
  int64_t nm = (int64_t)n[0] * n[1] * n[2];
  memset(Q, 0, sizeof(double) * nm);
  int64_t bad = 0;
  int S = support(order);
  for (int64_t i = 0; i < N; ++i) {
    int g0[3];
    double w[3][3], dw[3][3], d2w[3][3];
    if (particle_weights(x + 3 * i, n, lo, h, order, g0, w, dw, d2w)) { ++bad; continue; }
    for (int c = 0; c < S; ++c)
      for (int b = 0; b < S; ++b)
        for (int a = 0; a < S; ++a)
          Q[mesh_index(n, g0[0] + a, g0[1] + b, g0[2] + c)] += q * w[0][a] * w[1][b] * w[2][c];
  }
  return bad;
}

/* Adjoint helper: psi_g = sum_i grad_xi W(x_g - xi_i) . w_i  (a dipole deposit).
 * grad_xi W = (dw_d / h_d) * (weights of the other two axes). */
int64_t oracle_dipole_deposit(int64_t N, const double *x, const double *wv, const int32_t *n,
                              const double *lo, const double *h, int order, double *psi) {
  int64_t nm = (int64_t)n[0] * n[1] * n[2];
  memset(psi, 0, sizeof(double) * nm);
  int64_t bad = 0;
  int S = support(order);
  for (int64_t i = 0; i < N; ++i) {
    int g0[3];
    double w[3][3], dw[3][3], d2w[3][3];
    if (particle_weights(x + 3 * i, n, lo, h, order, g0, w, dw, d2w)) { ++bad; continue; }
    for (int c = 0; c < S; ++c)
      for (int b = 0; b < S; ++b)
        for (int a = 0; a < S; ++a) {
          double gx = dw[0][a] / h[0] * w[1][b] * w[2][c];
          double gy = w[0][a] * dw[1][b] / h[1] * w[2][c];
          double gz = w[0][a] * w[1][b] * dw[2][c] / h[2];
          psi[mesh_index(n, g0[0] + a, g0[1] + b, g0[2] + c)] +=
              gx * wv[3 * i] + gy * wv[3 * i + 1] + gz * wv[3 * i + 2];
        }
  }
  return bad;
}

/* Long-range force, eq. (eom_p3m_coord) first term, with the analytic derivative of W:
 * F_i = -q sum_g phi_g grad_xi W(x_g - xi_i). Optionally the interpolated potential
 * phi_at[i] = sum_g phi_g W(x_g - xi_i). Invalid particles get F = 0. */
int64_t oracle_interp(int64_t N, const double *x, double q, const double *phi, const int32_t *n,
                      const double *lo, const double *h, int order, double *F, double *phi_at) {
  int64_t bad = 0;
  int S = support(order);
  for (int64_t i = 0; i < N; ++i) {
    int g0[3];
    double w[3][3], dw[3][3], d2w[3][3];
    double f[3] = {0, 0, 0}, pa = 0.0;
    if (particle_weights(x + 3 * i, n, lo, h, order, g0, w, dw, d2w)) {
      ++bad;
    } else {
      for (int c = 0; c < S; ++c)
        for (int b = 0; b < S; ++b)
          for (int a = 0; a < S; ++a) {
            double p = phi[mesh_index(n, g0[0] + a, g0[1] + b, g0[2] + c)];
            f[0] += p * dw[0][a] / h[0] * w[1][b] * w[2][c];
            f[1] += p * w[0][a] * dw[1][b] / h[1] * w[2][c];
            f[2] += p * w[0][a] * w[1][b] * dw[2][c] / h[2];
            pa += p * w[0][a] * w[1][b] * w[2][c];
          }
    }
    F[3 * i] = -q * f[0];
    F[3 * i + 1] = -q * f[1];
    F[3 * i + 2] = -q * f[2];
    if (phi_at) phi_at[i] = pa;
  }
  return bad;
}

/* Vector-Jacobian product of the long-range force map xi -> F^L(xi) for cotangent w:
 *   out_k = -q sum_g phi_g (grad grad W)(x_g - xi_k) w_k  -  q^2 sum_g chi_g grad W(x_g - xi_k)
 * where phi is the mesh potential of the charges and chi the mesh potential (same solve) of
 * the dipole deposit psi of w (oracle_dipole_deposit). The solve is symmetric because both
 * the free and the image Green's function are symmetric in their two arguments. */
int64_t oracle_interp_vjp(int64_t N, const double *x, double q, const double *phi,
                          const double *chi, const double *wv, const int32_t *n, const double *lo,
                          const double *h, int order, double *out) {
  int64_t bad = 0;
  int S = support(order);
  for (int64_t i = 0; i < N; ++i) {
    int g0[3];
    double w[3][3], dw[3][3], d2w[3][3];
    double hess[3][3] = {{0}}, gchi[3] = {0, 0, 0};
    if (particle_weights(x + 3 * i, n, lo, h, order, g0, w, dw, d2w)) {
      ++bad;
      out[3 * i] = out[3 * i + 1] = out[3 * i + 2] = 0.0;
      continue;
    }
    for (int c = 0; c < S; ++c)
      for (int b = 0; b < S; ++b)
        for (int a = 0; a < S; ++a) {
          int64_t g = mesh_index(n, g0[0] + a, g0[1] + b, g0[2] + c);
          double p = phi[g], ch = chi[g];
          /* first and second derivatives of the tensor-product weight */
          double W1[3] = {dw[0][a] / h[0] * w[1][b] * w[2][c], w[0][a] * dw[1][b] / h[1] * w[2][c],
                          w[0][a] * w[1][b] * dw[2][c] / h[2]};
          double W2[3][3];
          W2[0][0] = d2w[0][a] / (h[0] * h[0]) * w[1][b] * w[2][c];
          W2[1][1] = w[0][a] * d2w[1][b] / (h[1] * h[1]) * w[2][c];
          W2[2][2] = w[0][a] * w[1][b] * d2w[2][c] / (h[2] * h[2]);
          W2[0][1] = W2[1][0] = dw[0][a] / h[0] * dw[1][b] / h[1] * w[2][c];
          W2[0][2] = W2[2][0] = dw[0][a] / h[0] * w[1][b] * dw[2][c] / h[2];
          W2[1][2] = W2[2][1] = w[0][a] * dw[1][b] / h[1] * dw[2][c] / h[2];
          for (int r = 0; r < 3; ++r) {
            gchi[r] += ch * W1[r];
            for (int s = 0; s < 3; ++s) hess[r][s] += p * W2[r][s];
          }
        }
    for (int r = 0; r < 3; ++r) {
      double hw = hess[r][0] * wv[3 * i] + hess[r][1] * wv[3 * i + 1] + hess[r][2] * wv[3 * i + 2];
      out[3 * i + r] = -q * hw - q * q * gchi[r];
    }
  }
  return bad;
}

/* ------------------------------------------------------------------------------------------
 * Short-range (particle-particle) part, eq. (summation_short) with the screened kernel
 * G^S(r) = erfc(a r)/r of eq. (ewald_split); the self term is omitted. For an ordered pair
 * (i, j), r = |xi_i - xi_j| < rc strictly, the force on i is
 *   k_e q_i q_j [erfc(a r)/r + (2a/sqrt(pi)) exp(-a^2 r^2)] (xi_i - xi_j) / r^2.
 * With the cathode applied to the short range as well (pp_bc = 1, Sec. 3.1.1), every particle j
 * (including j = i) also has an image of charge -q at S(xi_j) that acts on i with the same
 * screened kernel when |xi_i - S(xi_j)| < rc.
 * ------------------------------------------------------------------------------------------ */

/* pair quantities at squared distance r2: screened potential kernel erfc(a r)/r and the
 * force coefficient [erfc(a r)/r + (2a/sqrt(pi)) e^{-a^2 r^2}] / r^2. */
static void screened_pair(double r2, double alpha, double *pot, double *fco) {
  double r = sqrt(r2);
  double ec = erfc(alpha * r);
  *pot = ec / r;
  *fco = (ec / r + 2.0 * alpha / sqrt(ORACLE_PI) * exp(-alpha * alpha * r2)) / r2;
}

/* d/dr of the force coefficient phi(r) = A(r)/r^2, A = erfc(a r)/r + c e^{-a^2 r^2}. */
static void screened_pair_hess(double r2, double alpha, double *fco, double *dfco_over_r) {
  double r = sqrt(r2);
  double c = 2.0 * alpha / sqrt(ORACLE_PI);
  double ex = exp(-alpha * alpha * r2);
  double ec = erfc(alpha * r);
  double A = ec / r + c * ex;
  double dA = -c * ex / r - ec / r2 - 2.0 * alpha * alpha * r * c * ex;
  *fco = A / r2;
  double dphi = dA / r2 - 2.0 * A / (r2 * r);
  *dfco_over_r = dphi / r;
}

/* A plain uniform cell list over all particles, cell side >= rc. */
typedef struct {
  double lo[3];
  double s;
  int nc[3];
  int64_t *start; /* nc0*nc1*nc2 + 1 */
  int64_t *idx;   /* particle indices grouped by cell */
} cell_list;

static void cells_build(cell_list *cl, int64_t N, const double *x, double rc) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < N; ++i)
    for (int d = 0; d < 3; ++d) {
      if (x[3 * i + d] < lo[d]) lo[d] = x[3 * i + d];
      if (x[3 * i + d] > hi[d]) hi[d] = x[3 * i + d];
    }
  double ext = 0.0;
  for (int d = 0; d < 3; ++d) ext = fmax(ext, hi[d] - lo[d]);
  double s = rc;
  if (ext / s > 400.0) s = ext / 400.0; /* keeps the cell count bounded; still s >= rc */
  cl->s = s;
  int64_t ncell = 1;
  for (int d = 0; d < 3; ++d) {
    cl->lo[d] = lo[d];
    cl->nc[d] = (N > 0) ? (int)floor((hi[d] - lo[d]) / s) + 1 : 1;
    ncell *= cl->nc[d];
  }
  cl->start = (int64_t *)calloc(ncell + 1, sizeof(int64_t));
  cl->idx = (int64_t *)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
  int64_t *key = (int64_t *)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
  for (int64_t i = 0; i < N; ++i) {
    int k[3];
    for (int d = 0; d < 3; ++d) {
      k[d] = (int)floor((x[3 * i + d] - cl->lo[d]) / s);
      if (k[d] < 0) k[d] = 0;
      if (k[d] > cl->nc[d] - 1) k[d] = cl->nc[d] - 1;
    }
    key[i] = ((int64_t)k[2] * cl->nc[1] + k[1]) * cl->nc[0] + k[0];
    cl->start[key[i] + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) cl->start[c + 1] += cl->start[c];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (ncell + 1));
  memcpy(fill, cl->start, sizeof(int64_t) * (ncell + 1));
  for (int64_t i = 0; i < N; ++i) cl->idx[fill[key[i]]++] = i;
  free(fill);
  free(key);
}

static void cells_free(cell_list *cl) {
  free(cl->start);
  free(cl->idx);
}

/* inclusive cell range along axis d that covers [v - rc, v + rc], clamped to the grid */
static void cell_range(const cell_list *cl, double v, double rc, int d, int *a, int *b) {
  double fa = floor((v - rc - cl->lo[d]) / cl->s), fb = floor((v + rc - cl->lo[d]) / cl->s);
  if (fa < 0) fa = 0;
  if (fb > cl->nc[d] - 1) fb = cl->nc[d] - 1;
  *a = (int)fa;
  *b = (int)fb;
}

/* Adds the screened interaction of all sources within rc of point P to acc (force per unit
 * target charge, i.e. field, and potential), with source charge sign sgn. If mirror, the source
 * positions are S(xi_j) instead of xi_j (the query is then made at S(P), which is equivalent
 * because |P - S(xi_j)| = |S(P) - xi_j|). Source `skip` (if >= 0 and not mirror) is excluded. */
static void pp_gather(const cell_list *cl, const double *x, const double *P, int64_t skip,
                      double alpha, double rc, int mirror, double zc, double *field,
                      double *pot, int64_t *npairs, int64_t *ncoinc) {
  double Q[3] = {P[0], P[1], mirror ? 2.0 * zc - P[2] : P[2]};
  int a[3], b[3];
  for (int d = 0; d < 3; ++d) cell_range(cl, Q[d], rc, d, &a[d], &b[d]);
  double rc2 = rc * rc;
  for (int kz = a[2]; kz <= b[2]; ++kz)
    for (int ky = a[1]; ky <= b[1]; ++ky)
      for (int kx = a[0]; kx <= b[0]; ++kx) {
        int64_t c = ((int64_t)kz * cl->nc[1] + ky) * cl->nc[0] + kx;
        for (int64_t t = cl->start[c]; t < cl->start[c + 1]; ++t) {
          int64_t j = cl->idx[t];
          if (!mirror && j == skip) continue;
          const double *y = x + 3 * j;
          double src[3] = {y[0], y[1], mirror ? 2.0 * zc - y[2] : y[2]};
          double d0 = P[0] - src[0], d1 = P[1] - src[1], d2 = P[2] - src[2];
          double r2 = d0 * d0 + d1 * d1 + d2 * d2;
          if (!(r2 < rc2)) continue;
          if (r2 == 0.0) { ++*ncoinc; continue; }
          double pt, fc;
          screened_pair(r2, alpha, &pt, &fc);
          field[0] += (mirror ? -1.0 : 1.0) * fc * d0;
          field[1] += (mirror ? -1.0 : 1.0) * fc * d1;
          field[2] += (mirror ? -1.0 : 1.0) * fc * d2;
          *pot += (mirror ? -1.0 : 1.0) * pt;
          ++*npairs;
        }
      }
}

/* Short-range forces on a sample of particles (sample == NULL: all N), each computed from
 * every one of the N particles through a cell list. F is [n_out, 3]; phi (nullable) is the
 * short-range potential at the particle [V]; counts[0] = ordered in-cutoff pairs,
 * counts[1] = image pairs, counts[2] = coincident pairs skipped. */
void oracle_pp(int64_t N, const double *x, double q, double alpha, double rc, int pp_bc,
               double zc, int64_t n_out, const int64_t *sample, double *F, double *phi,
               int64_t *counts) {
  cell_list cl;
  cells_build(&cl, N, x, rc);
  double ke = coulomb_k();
  int64_t np = 0, ni = 0, nc = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : np, ni, nc)
  for (int64_t t = 0; t < n_out; ++t) {
    int64_t i = sample ? sample[t] : t;
    double field[3] = {0, 0, 0}, pot = 0.0;
    int64_t a = 0, b = 0, c = 0;
    pp_gather(&cl, x, x + 3 * i, i, alpha, rc, 0, zc, field, &pot, &a, &c);
    if (pp_bc) pp_gather(&cl, x, x + 3 * i, i, alpha, rc, 1, zc, field, &pot, &b, &c);
    for (int d = 0; d < 3; ++d) F[3 * t + d] = ke * q * q * field[d];
    if (phi) phi[t] = ke * q * pot;
    np += a;
    ni += b;
    nc += c;
  }
  counts[0] = np;
  counts[1] = ni;
  counts[2] = nc;
  cells_free(&cl);
}

/* The same sum by brute force over all pairs, without a cell list (a pin for oracle_pp). */
void oracle_pp_brute(int64_t N, const double *x, double q, double alpha, double rc, int pp_bc,
                     double zc, double *F, double *phi, int64_t *counts) {
  double ke = coulomb_k(), rc2 = rc * rc;
  int64_t np = 0, ni = 0, nc = 0;
  for (int64_t i = 0; i < N; ++i) {
    double f[3] = {0, 0, 0}, pot = 0.0;
    for (int64_t j = 0; j < N; ++j) {
      for (int m = 0; m <= pp_bc; ++m) {
        if (m == 0 && j == i) continue;
        double sz = m ? 2.0 * zc - x[3 * j + 2] : x[3 * j + 2];
        double d0 = x[3 * i] - x[3 * j], d1 = x[3 * i + 1] - x[3 * j + 1], d2 = x[3 * i + 2] - sz;
        double r2 = d0 * d0 + d1 * d1 + d2 * d2;
        if (!(r2 < rc2)) continue;
        if (r2 == 0.0) { ++nc; continue; }
        double pt, fc, sg = m ? -1.0 : 1.0;
        screened_pair(r2, alpha, &pt, &fc);
        f[0] += sg * fc * d0;
        f[1] += sg * fc * d1;
        f[2] += sg * fc * d2;
        pot += sg * pt;
        if (m) ++ni; else ++np;
      }
    }
    for (int d = 0; d < 3; ++d) F[3 * i + d] = ke * q * q * f[d];
    if (phi) phi[i] = ke * q * pot;
  }
  counts[0] = np;
  counts[1] = ni;
  counts[2] = nc;
}

/* Vector-Jacobian product of the short-range force map for cotangent w (all N particles).
 * A pair term f(d) = C phi(r) d, d = xi_i - src, has Jacobian H(d) = C [phi I + (phi'/r) d d^T].
 * Free pairs (src = xi_j, C = k_e q^2): out_i += H (w_i - w_j).
 * Image pairs (src = S(xi_j), C = -k_e q^2, j = i included): out_i += H w_i and
 * out_j += -S H w_i, with S = diag(1, 1, -1). */
void oracle_pp_vjp(int64_t N, const double *x, double q, double alpha, double rc, int pp_bc,
                   double zc, const double *wv, double *out) {
  double ke = coulomb_k(), rc2 = rc * rc;
  memset(out, 0, sizeof(double) * 3 * N);
  cell_list cl;
  cells_build(&cl, N, x, rc);
  for (int64_t i = 0; i < N; ++i) {
    for (int m = 0; m <= pp_bc; ++m) {
      double P[3] = {x[3 * i], x[3 * i + 1], m ? 2.0 * zc - x[3 * i + 2] : x[3 * i + 2]};
      int a[3], b[3];
      for (int d = 0; d < 3; ++d) cell_range(&cl, P[d], rc, d, &a[d], &b[d]);
      for (int kz = a[2]; kz <= b[2]; ++kz)
        for (int ky = a[1]; ky <= b[1]; ++ky)
          for (int kx = a[0]; kx <= b[0]; ++kx) {
            int64_t c = ((int64_t)kz * cl.nc[1] + ky) * cl.nc[0] + kx;
            for (int64_t t = cl.start[c]; t < cl.start[c + 1]; ++t) {
              int64_t j = cl.idx[t];
              if (m == 0 && j == i) continue;
              double src[3] = {x[3 * j], x[3 * j + 1], m ? 2.0 * zc - x[3 * j + 2] : x[3 * j + 2]};
              double dv[3] = {x[3 * i] - src[0], x[3 * i + 1] - src[1], x[3 * i + 2] - src[2]};
              double r2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
              if (!(r2 < rc2) || r2 == 0.0) continue;
              double fc, dfr;
              screened_pair_hess(r2, alpha, &fc, &dfr);
              double C = (m ? -1.0 : 1.0) * ke * q * q;
              if (m == 0) {
                double u[3] = {wv[3 * i] - wv[3 * j], wv[3 * i + 1] - wv[3 * j + 1],
                               wv[3 * i + 2] - wv[3 * j + 2]};
                double du = dv[0] * u[0] + dv[1] * u[1] + dv[2] * u[2];
                for (int d = 0; d < 3; ++d) out[3 * i + d] += C * (fc * u[d] + dfr * du * dv[d]);
              } else {
                const double *u = wv + 3 * i;
                double du = dv[0] * u[0] + dv[1] * u[1] + dv[2] * u[2];
                double Hu[3];
                for (int d = 0; d < 3; ++d) Hu[d] = C * (fc * u[d] + dfr * du * dv[d]);
                for (int d = 0; d < 3; ++d) out[3 * i + d] += Hu[d];
                out[3 * j] -= Hu[0];
                out[3 * j + 1] -= Hu[1];
                out[3 * j + 2] += Hu[2];
              }
            }
          }
    }
  }
  cells_free(&cl);
}

/* Exact (unsplit) Coulomb forces and potentials by brute force, the "true" interaction the
 * method approximates (Sec. 3.1.1, Phi = R (x) rho). bc = 1 adds the image charge -q at
 * S(xi_j) of every particle j, the particle's own image included. */
void oracle_coulomb_brute(int64_t N, const double *x, double q, int bc, double zc, double *F,
                          double *phi) {
  double ke = coulomb_k();
  for (int64_t i = 0; i < N; ++i) {
    double f[3] = {0, 0, 0}, pot = 0.0;
    for (int64_t j = 0; j < N; ++j) {
      for (int m = 0; m <= bc; ++m) {
        if (m == 0 && j == i) continue;
        double sz = m ? 2.0 * zc - x[3 * j + 2] : x[3 * j + 2];
        double d0 = x[3 * i] - x[3 * j], d1 = x[3 * i + 1] - x[3 * j + 1], d2 = x[3 * i + 2] - sz;
        double r2 = d0 * d0 + d1 * d1 + d2 * d2;
        if (r2 == 0.0) continue;
        double r = sqrt(r2), sg = m ? -1.0 : 1.0;
        f[0] += sg * d0 / (r2 * r);
        f[1] += sg * d1 / (r2 * r);
        f[2] += sg * d2 / (r2 * r);
        pot += sg / r;
      }
    }
    for (int d = 0; d < 3; ++d) F[3 * i + d] = ke * q * q * f[d];
    if (phi) phi[i] = ke * q * pot;
  }
}

/* Long-range kernel of eq. (ewald_split): G^L(r) = erf(a r)/r, with its limit 2a/sqrt(pi) at 0. */
static double g_long(double r, double alpha) {
  return r > 0.0 ? erf(alpha * r) / r : 2.0 * alpha / sqrt(ORACLE_PI);
}

/* Mesh potential by direct summation over node pairs, eq. (phi_L) with the planar-cathode
 * Green's function eq. (GreenFunc_planar_cathode) when bc = 1:
 *   phi_g = k_e sum_g' Q_g' [G^L(|x_g - x_g'|) - bc G^L(|x_g - S(x_g')|)].
 * O(M^2); a pin for the FFT convolution on small meshes. */
void oracle_mesh_direct(const int32_t *n, const double *lo, const double *h, double alpha, int bc,
                        double zc, const double *Q, double *phi) {
  double ke = coulomb_k();
  int64_t nm = (int64_t)n[0] * n[1] * n[2];
  for (int64_t g = 0; g < nm; ++g) {
    int gx = (int)(g % n[0]), gy = (int)((g / n[0]) % n[1]), gz = (int)(g / ((int64_t)n[0] * n[1]));
    double X[3] = {lo[0] + gx * h[0], lo[1] + gy * h[1], lo[2] + gz * h[2]};
    double acc = 0.0;
    for (int64_t k = 0; k < nm; ++k) {
      if (Q[k] == 0.0) continue;
      int kx = (int)(k % n[0]), ky = (int)((k / n[0]) % n[1]), kz = (int)(k / ((int64_t)n[0] * n[1]));
      double Y[3] = {lo[0] + kx * h[0], lo[1] + ky * h[1], lo[2] + kz * h[2]};
      double d0 = X[0] - Y[0], d1 = X[1] - Y[1], d2 = X[2] - Y[2];
      acc += Q[k] * g_long(sqrt(d0 * d0 + d1 * d1 + d2 * d2), alpha);
      if (bc) {
        double e2 = X[2] - (2.0 * zc - Y[2]);
        acc -= Q[k] * g_long(sqrt(d0 * d0 + d1 * d1 + e2 * e2), alpha);
      }
    }
    phi[g] = ke * acc;
  }
}
