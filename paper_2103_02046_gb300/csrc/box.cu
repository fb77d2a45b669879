// Long range in a grounded box (pm_bc = 2, FP64 path): the discrete Poisson equation
// D_xyz phi = -rho_L / eps0 of eq. (def_G_L), D_xyz the 7-point Laplacian of
// eq. (3dim_second_order_fin_diff), on the interior nodes 1 .. n_d - 2 of the mesh, with phi = 0
// on the six faces (nodes 0 and n_d - 1: grounded conductors). rho_L = q W / (h_x h_y h_z) is
// screened by the Gaussian of the charge splitting, applied in the sine basis as
// gamma^(k) = exp(-|k|^2 / (4 alpha^2)).
//
// The sine transform is taken as a real FFT of the odd extension: along each axis the node
// values f_0 .. f_{n-1} (f_0 = f_{n-1} = 0) are continued to period B = 2 (n - 1) with
// f_{B-i} = -f_i. Its spectrum is diagonal in D_xyz with eigenvalue
// lambda(j) = sum_d (2 cos(2 pi j_d / B_d) - 2) / h_d^2, and a real multiplier even in every j_d
// keeps the odd symmetry, so the inverse transform returns the odd extension of the solution.
#include <cmath>

#include "p3m_internal.cuh"

namespace p3m {
namespace {

// node index along one axis of the odd extension -> (node in [0, n), sign); sign 0 on faces
__device__ __forceinline__ int odd_fold(int i, int n, int B, int& sign) {
  if (i == 0 || i == n - 1) {
    sign = 0;
    return 0;
  }
  if (i < n - 1) {
    sign = 1;
    return i;
  }
  sign = -1;
  return B - i;
}

__global__ void k_box_extend(Geom g, const double* __restrict__ qpad, double* __restrict__ ext,
                             int Bx, int By, int Bz) {
  const size_t total = static_cast<size_t>(Bx) * By * Bz;
  const size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (e >= total) return;
  const int ix = static_cast<int>(e % Bx);
  const int iy = static_cast<int>((e / Bx) % By);
  const int iz = static_cast<int>(e / (static_cast<size_t>(Bx) * By));
  int sx, sy, sz;
  const int x = odd_fold(ix, g.n[0], Bx, sx);
  const int y = odd_fold(iy, g.n[1], By, sy);
  const int z = odd_fold(iz, g.n[2], Bz, sz);
  const int s = sx * sy * sz;
  ext[e] = s == 0 ? 0.0 : s * qpad[real_index(g, x, y, z)];
}

__global__ void k_box_multiply(double2* __restrict__ spec, const double* __restrict__ mult,
                               size_t ncplx) {
  const size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (e >= ncplx) return;
  const double m = mult[e];
  spec[e].x *= m;
  spec[e].y *= m;
}

// phi on the n^3 block (faces exactly 0) into the doubled-mesh potential array the
// interpolation reads; and sum_g W_g phi_g for the long-range energy
__global__ void k_box_extract(Geom g, const double* __restrict__ ext,
                              const double* __restrict__ qpad, double* __restrict__ phireal,
                              int Bx, int By, double* __restrict__ energy) {
  const size_t total = static_cast<size_t>(g.n[0]) * g.n[1] * g.n[2];
  const size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  double e = 0.0;
  if (t < total) {
    const int x = static_cast<int>(t % g.n[0]);
    const int y = static_cast<int>((t / g.n[0]) % g.n[1]);
    const int z = static_cast<int>(t / (static_cast<size_t>(g.n[0]) * g.n[1]));
    const bool face = x == 0 || y == 0 || z == 0 || x == g.n[0] - 1 || y == g.n[1] - 1 ||
                      z == g.n[2] - 1;
    const double v = face ? 0.0 : ext[(static_cast<size_t>(z) * By + y) * Bx + x];
    const size_t r = real_index(g, x, y, z);
    phireal[r] = v;
    if (energy) e = qpad[r] * v;
  }
  if (energy) {
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0 && e != 0.0) atomicAdd(energy, e);
  }
}

// multiplier per spectrum element: -gamma^(k) q / (eps0 h_x h_y h_z lambda(k)) / (Bx By Bz),
// 1 / eps0 = 4 pi k_e; 0 where some j_d is 0 or B_d / 2 (modes that vanish on the odd extension)
__global__ void k_box_mult_build(Geom g, int Bx, int By, int Bz, double* __restrict__ mult) {
  const int Hx = Bx / 2 + 1;
  const size_t total = static_cast<size_t>(Hx) * By * Bz;
  const size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (e >= total) return;
  const int j[3] = {static_cast<int>(e % Hx), static_cast<int>((e / Hx) % By),
                    static_cast<int>(e / (static_cast<size_t>(Hx) * By))};
  const int B[3] = {Bx, By, Bz};
  const double pi = 3.14159265358979323846;
  double lam = 0.0, k2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    if (j[d] == 0 || 2 * j[d] == B[d]) {
      mult[e] = 0.0;
      return;
    }
    const int js = j[d] <= B[d] / 2 ? j[d] : j[d] - B[d];
    lam += (2.0 * cospi(2.0 * js / B[d]) - 2.0) / (g.h[d] * g.h[d]);
    const double k = 2.0 * pi * js / (B[d] * g.h[d]);
    k2 += k * k;
  }
  const double vol = g.h[0] * g.h[1] * g.h[2];
  const double gam = exp(-k2 / (4.0 * g.alpha * g.alpha));
  mult[e] = -gam * g.q * 4.0 * pi * g.ke / (vol * lam) / (static_cast<double>(Bx) * By * Bz);
}

inline unsigned grid_of(size_t n) { return static_cast<unsigned>((n + 255) / 256); }

}  // namespace

p3m_status box_setup(p3m_ctx* c) {
  const Geom& g = c->g;
  const int Bx = 2 * (g.n[0] - 1), By = 2 * (g.n[1] - 1), Bz = 2 * (g.n[2] - 1);
  const size_t nreal = static_cast<size_t>(Bx) * By * Bz;
  const size_t ncplx = static_cast<size_t>(Bx / 2 + 1) * By * Bz;
  cudaError_t e = cudaMalloc(&c->box_real, sizeof(double) * nreal);
  if (e == cudaSuccess) e = cudaMalloc(&c->box_spec, sizeof(double2) * ncplx);
  if (e == cudaSuccess) e = cudaMalloc(&c->box_mult, sizeof(double) * ncplx);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? P3M_ENOMEM : P3M_ECUDA;
  cufftResult r = cufftPlan3d(&c->plan_box_f, Bz, By, Bx, CUFFT_D2Z);
  c->have_box_f = r == CUFFT_SUCCESS;
  if (r == CUFFT_SUCCESS) {
    r = cufftPlan3d(&c->plan_box_i, Bz, By, Bx, CUFFT_Z2D);
    c->have_box_i = r == CUFFT_SUCCESS;
  }
  if (r != CUFFT_SUCCESS) return r == CUFFT_ALLOC_FAILED ? P3M_ENOMEM : P3M_ECUFFT;
  cufftSetStream(c->plan_box_f, c->work);
  cufftSetStream(c->plan_box_i, c->work);
  k_box_mult_build<<<grid_of(ncplx), 256, 0, c->work>>>(g, Bx, By, Bz, c->box_mult);
  return cudaGetLastError() == cudaSuccess ? P3M_OK : P3M_ECUDA;
}

p3m_status box_solve(p3m_ctx* c, bool want_energy) {
  const Geom& g = c->g;
  const int Bx = 2 * (g.n[0] - 1), By = 2 * (g.n[1] - 1), Bz = 2 * (g.n[2] - 1);
  const size_t nreal = static_cast<size_t>(Bx) * By * Bz;
  const size_t ncplx = static_cast<size_t>(Bx / 2 + 1) * By * Bz;
  k_box_extend<<<grid_of(nreal), 256, 0, c->work>>>(g, static_cast<const double*>(c->qpad),
                                                     c->box_real, Bx, By, Bz);
  if (cufftExecD2Z(c->plan_box_f, c->box_real, c->box_spec) != CUFFT_SUCCESS) return P3M_ECUFFT;
  k_box_multiply<<<grid_of(ncplx), 256, 0, c->work>>>(c->box_spec, c->box_mult, ncplx);
  if (cufftExecZ2D(c->plan_box_i, c->box_spec, c->box_real) != CUFFT_SUCCESS) return P3M_ECUFFT;
  const size_t nb = static_cast<size_t>(g.n[0]) * g.n[1] * g.n[2];
  k_box_extract<<<grid_of(nb), 256, 0, c->work>>>(g, c->box_real,
                                                   static_cast<const double*>(c->qpad),
                                                   static_cast<double*>(c->phireal), Bx, By,
                                                   want_energy ? c->energy_acc + 1 : nullptr);
  return cudaGetLastError() == cudaSuccess ? P3M_OK : P3M_ECUDA;
}

}  // namespace p3m
