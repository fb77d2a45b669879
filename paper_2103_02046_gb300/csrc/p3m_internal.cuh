// Internal declarations of the GB300 P3M library (not part of the C ABI).
//
// Data layout in HBM (one context, up to n_max particles, mesh n = (nx, ny, nz), n_d <= 1024):
//   * Cells for the short-range search are rows along x: edge a hair above r_c / rows in y and z
//     (rows = 2, or 1 at low density), r_c / nsub in x, keys x-fastest, so the cells of one (y, z)
//     row within any x-interval hold a contiguous run of sorted particles. Each of the
//     (2 rows + 1)^2 neighbour rows of a particle is then one index range, pruned by the
//     particle's distance to the row.
//   * Sorted records (counting sort by cell key):
//       recp  positions in cutoff units from the mesh origin, (x - lo) / r_c, 32 B each:
//             FP32 two float4 {hi_x, hi_y, hi_z, bits(original index)} {lo_x, lo_y, lo_z, 0},
//             lo the rounding remainders, so that (hi_i - hi_j) + (lo_i - lo_j) is the
//             separation to FP32 relative accuracy however close the pair is; FP64
//             {x, y, z, index};
//       recm  assignment data in mesh units: the node c = floor(s + 1/2) (TSC) or floor(s)
//             (CIC) packed 10 bits per axis, and the offset u = s - c, s = (x - lo) / h, computed
//             in FP64 exactly as the definition reads (FP32 float4 or FP64 {u, node}).
//   * Mesh arrays use the doubled (2n)^3 layout of the FFT convolution, x fastest:
//     index (gz * My + gy) * Mx + gx; half spectra have Mx/2 + 1 entries along x.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>
#include <string>

#include "p3m.h"

namespace dfm {
struct PairDF;
}

namespace p3m {

constexpr uint32_t kInvalidKey = 0xFFFFFFFFu;
constexpr int kMaxMesh = 1024;

enum ErrBits : int { kErrRange = 1, kErrNaN = 2, kErrTimeout = 4 };

// Geometry, passed by value to kernels.
struct Geom {
  int n[3];      // mesh nodes per axis
  int M[3];      // doubled mesh 2 n
  int nc[3];     // cells per axis
  int rows;      // cell rows per cutoff length in y and z (1, 2 or 3)
  int order;     // 1 CIC, 2 TSC
  int pm_bc, pp_bc;
  int force_diff;  // 1: long-range force from central differences of the mesh potential
  double lo[3], h[3];
  double rc, alpha, zc;
  double q, mass, ke;
  double a[3];       // h_d / r_c
  double cw[3];      // cell edges in cutoff units (y, z: (1 + 4 slack) / rows; x: 1 / nsub)
  double inv_cw[3];
  double inv_h[3];   // 1 / h_d
  float inv_h_f[3];  // 1 / h_d, FP32
  float inv_cell_f[3];  // 1 / (r_c cw_d): metres from lo -> cell index, FP32
  double inv_rc;     // 1 / r_c
  double fscale[3];  // -q / h_d: long-range force per volt of mesh-unit gradient
  double img_c;      // 2 (z_c - lo_z) / r_c: the image of z (cutoff units) is img_c - z
  double kappa_eff;  // alpha * r_c
  // Search slack (cutoff units): bounds every rounding in where a particle is placed (the sort
  // bins in FP32, the short range works from FP32 hi parts): 1e-6 of the largest mesh extent,
  // at least 1e-4, while those errors stay below 3.1e-7 of the extent.
  double slack;
  float cw_f[3], inv_cw_f[3], slack_f;  // FP32 copies for the FP32 short range
  // double-float (hi + lo, each FP32) copies for the FP32 path's binning and records
  float lo_df[3][2];     // mesh origin lo_d
  float inv_rc_df[2];    // 1 / r_c
  float inv_h_df[3][2];  // 1 / h_d
  float fscale_f[3];     // -q / h_d in FP32
  float rch_df[3][2];    // r_c / h_d: cutoff units -> mesh units
};

// FP32 records: the lo part's w packs the particle's row (rz nc_y + ry, below 2^26) and, in the
// top 6 bits, a node correction of -1, 0 or +1 per axis (2 bits each, stored + 1) that turns the
// node recomputed from the position into the exact one near a knot.
constexpr uint32_t kRowBits = 26;
constexpr uint32_t kRowMask = (1u << kRowBits) - 1u;

// ------------------------------------------------------------------------------------------
// Double-float arithmetic: a value held as an unevaluated sum hi + lo of two floats, |lo| <=
// ulp(hi) / 2, about 48 significant bits. The FP32 path uses it instead of FP64, whose
// throughput on this part is a small fraction of FP32's.
// ------------------------------------------------------------------------------------------
struct DF {
  float hi, lo;
};

// The double-float steps below use the _rn intrinsics so that the compiler cannot contract a
// product and a sum into one FMA, which would break the exact error terms.

// Exact sum a + b = s + e (Knuth's TwoSum).
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// Renormalises s + e when |s| >= |e| (Dekker's Fast2Sum).
__device__ __forceinline__ DF df_fast_two_sum(float s, float e) {
  const float h = __fadd_rn(s, e);
  return DF{h, __fsub_rn(e, __fsub_rn(h, s))};
}

// (a.hi + a.lo) - (b.hi + b.lo), error about 2^-46 of the larger operand.
__device__ __forceinline__ DF df_sub(DF a, DF b) {
  const DF s = df_two_sum(a.hi, -b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo)));
}

// (a.hi + a.lo) (c.hi + c.lo), relative error about 2^-46; the product a.hi c.hi is split
// exactly with an FMA.
__device__ __forceinline__ DF df_mul(DF a, const float c[2]) {
  const float p = __fmul_rn(a.hi, c[0]);
  float e = __fmaf_rn(a.hi, c[0], -p);
  e = __fmaf_rn(a.hi, c[1], e);
  e = __fmaf_rn(a.lo, c[0], e);
  return df_fast_two_sum(p, e);
}

// Exact widening of a float to double with integer operations (zero, subnormals, infinities
// and NaN take the conversion route).
static __device__ __noinline__ double float_to_double_slow(float v) {
  return static_cast<double>(v);
}
static __device__ __noinline__ DF df_from_double_slow(double v) {
  const float h = static_cast<float>(v);
  return DF{h, static_cast<float>(v - static_cast<double>(h))};
}

__device__ __forceinline__ double float_to_double_exact(float v) {
  const unsigned int b = __float_as_uint(v);
  const unsigned int e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return float_to_double_slow(v);  // rare: a call, not predicated
  const unsigned long long d = (static_cast<unsigned long long>(b & 0x80000000u) << 32) |
                               (static_cast<unsigned long long>(e + 896u) << 52) |
                               (static_cast<unsigned long long>(b & 0x7fffffu) << 29);
  return __longlong_as_double(static_cast<long long>(d));
}

// Splits a double into hi + lo with integer operations only: hi is v truncated to its leading
// 24 significant bits (exactly a float), lo the remaining 29 bits rounded to a float, so
// |v - hi - lo| <= 2^-48 |v|. Values whose exponent a float cannot hold (zero, below 2^-74,
// above 2^127, not finite) take the conversion route instead.
__device__ __forceinline__ DF df_from_double(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const int e = static_cast<int>((b >> 52) & 0x7ffull);  // biased exponent
  if (e < 1023 - 74 || e > 1023 + 127) return df_from_double_slow(v);  // rare: a real branch
  const unsigned int sign = static_cast<unsigned int>(b >> 32) & 0x80000000u;
  const unsigned int hb = sign | (static_cast<unsigned int>(e - 1023 + 127) << 23) |
                          static_cast<unsigned int>((b >> 29) & 0x7fffffull);
  const unsigned int rem = static_cast<unsigned int>(b & 0x1fffffffull);  // below hi's last bit
  // rem * 2^(e - 1075): the scale is a normal float for e >= 949
  const float scale = __uint_as_float(static_cast<unsigned int>(e - 1075 + 127) << 23);
  const float lo = __uint_as_float(__float_as_uint(static_cast<float>(rem) * scale) | sign);
  return DF{__uint_as_float(hb), lo};
}

// FP32 pair kernel: erfc(x) e^{x^2} on x in [0, kappa_eff] as t P(u), t = 1 / (1 + pk rho),
// u = t - tc, P a polynomial (Horner, highest degree first), fitted at context creation.
constexpr int kMaxPoly = 16;
struct PairPoly {
  int deg;
  float c[kMaxPoly];
  float pk, tc;        // p kappa_eff; the midpoint of t's range
  float kappa2_log2e;  // kappa_eff^2 log2(e): e^{-kappa^2 rho^2} = 2^{-kappa2_log2e rho^2}
  float kappa2;        // kappa_eff^2
  float c2k;           // 2 kappa_eff / sqrt(pi)
  float max_abs_err;   // fit error of erfc over [0, kappa_eff] (reported, not used)
};

__host__ __device__ inline uint32_t cell_key(const Geom& g, int cx, int cy, int cz) {
  return (static_cast<uint32_t>(cz) * g.nc[1] + cy) * g.nc[0] + cx;
}

// element (x, y, z) of a real field on the doubled mesh (x fastest)
__host__ __device__ inline size_t real_index(const Geom& g, int x, int y, int z) {
  return (static_cast<size_t>(z) * g.M[1] + y) * g.M[0] + x;
}

__host__ __device__ inline uint32_t pack_node(int cx, int cy, int cz) {
  return static_cast<uint32_t>(cx) | (static_cast<uint32_t>(cy) << 10) |
         (static_cast<uint32_t>(cz) << 20);
}

struct Rec64 {
  double u[3];
  long long idx;
};

// FP64 short-range result per sorted particle: force (x, y, z) and potential (w)
struct alignas(32) D4 {
  double x, y, z, w;
};

template <typename T>
struct RecT;
template <>
struct RecT<float> {
  using type = float4;
};
template <>
struct RecT<double> {
  using type = Rec64;
};

#ifdef __CUDACC__
__device__ __forceinline__ void load_rec(const float4* rec, uint32_t i, float u[3],
                                         long long& idx) {
  const float4 r = rec[i];
  u[0] = r.x;
  u[1] = r.y;
  u[2] = r.z;
  idx = __float_as_int(r.w);
}
__device__ __forceinline__ void load_rec(const Rec64* rec, uint32_t i, double u[3],
                                         long long& idx) {
  const Rec64 r = rec[i];
  u[0] = r.u[0];
  u[1] = r.u[1];
  u[2] = r.u[2];
  idx = r.idx;
}
#endif

}  // namespace p3m

// The opaque context of the C ABI.
struct p3m_ctx {
  p3m_params prm{};
  p3m::Geom g{};
  p3m::PairPoly poly{};
  dfm::PairDF* pdf = nullptr;   // FP64 path: device copy of the double-float pair-function fit
                                // (kappa <= 6.5; otherwise nullptr and the FP64 pair function)
  int64_t n_max = 0;
  int device = 0;
  bool fp32 = false;
  bool det = false;             // deterministic = 1 (FP64 path): run-to-run identical results
  cudaStream_t stream = nullptr;  // caller's stream (not owned)
  cudaStream_t work = nullptr;    // owned, low priority: sort, mesh chain, combination
  cudaStream_t s_pp = nullptr;    // owned, high priority: the short range (the longest stage),
                                  // so the mesh chain only takes SMs its blocks leave free
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_in = nullptr, ev_out = nullptr;
  cudaEvent_t tev[8] = {};

  // binning / counting sort
  uint64_t nkeys = 0;
  uint32_t* counts = nullptr;   // [nkeys]
  uint32_t* starts = nullptr;   // [nkeys + 1]
  uint32_t* bsum = nullptr;     // scan block sums
  uint32_t* keys = nullptr;     // [n_max] key of each input particle
  uint32_t* ranks = nullptr;    // [n_max] rank within its cell
  void* recp = nullptr;         // [n_max] sorted positions, cutoff units (2 float4 / Rec64)
  void* recm = nullptr;         // [n_max] FP64 path: sorted assignment records (Rec64)
  void* fpp = nullptr;          // [n_max] short-range result, sorted (FP32 float4, FP64 D4)
  float4* fplo = nullptr;       // [2 n_max] FP32 path: the fine x and y parts of the
                                // short-range terms (float2 [n]), then (from n_max on) the rare
                                // big terms; fpp holds the coarse x, y, z parts (summed exactly)
                                // and the fine z part
  double* acc = nullptr;        // [3 n_max] adjoint accumulator, sorted order

  // mesh
  size_t n_real = 0;            // Mx My Mz
  size_t n_cplx = 0;            // Mz My (Mx/2 + 1)
  void* qpad = nullptr;         // real, doubled mesh, zero outside the n^3 block
  void* qhat = nullptr;         // x-y transformed planes z < n_z (planes above stay zero)
  void* khat_f = nullptr;       // real spectrum of the free kernel (scaled)
  void* khat_i = nullptr;       // complex spectrum of the image kernel (scaled, phase folded)
  void* fhat = nullptr;         // FP32: 3 difference spectra; FP64: unused
  void* freal = nullptr;        // FP32: 3 forward-difference fields
  void* phihat = nullptr;       // potential spectrum
  void* phireal = nullptr;      // potential on the doubled mesh
  float2* dfac = nullptr;       // FP32: difference factors e^{2 pi i k/M} - 1 per axis (Mx/2+1 + My + Mz)
  float2* ztw = nullptr;        // fused z solve: e^{-2 pi i t / Mz}, t < Mz (FP32 path: float2;
                                // FP64 path: double-float, two float2 per entry)
  // grounded box (pm_bc = 2, FP64): odd extension (2(n-1))^3, its half spectrum, multiplier
  double* box_real = nullptr;
  double2* box_spec = nullptr;
  double* box_mult = nullptr;
  cufftHandle plan_box_f = 0, plan_box_i = 0;
  bool have_box_f = false, have_box_i = false;
  bool zconv = false;           // FP32 forces use the fused z solve
  bool zsolve_df = false;       // the FP64 potential uses the double-float fused z solve
  // Pruned transforms of the doubled mesh: the charge is non-zero, and the fields are needed,
  // only in the n^3 block, so the x-y plane transforms run on the first n_z planes only and
  // the z transforms are strided 1D batches over all (kx, ky) columns.
  void* qhat2 = nullptr;        // full spectrum of qpad (z transformed, out of place)
  cufftHandle plan_xy_f = 0;    // 2D R2C (or D2Z) on planes z < n_z: qpad -> qhat
  cufftHandle plan_z = 0;       // 1D C2C (or Z2Z) along z, stride My (Mx/2 + 1), all columns
  cufftHandle plan_xy_i = 0;    // 2D C2R (or Z2D) on planes z < n_z: spectrum -> real field
  bool have_xy_f = false, have_z = false, have_xy_i = false;

  // diagnostics
  double* energy_acc = nullptr;              // device [2]
  unsigned long long* pair_acc = nullptr;    // device [3]: pairs, image pairs, candidates
  uint32_t* pp_tile = nullptr;               // device [1]: next tile of the persistent short range
  int num_sms = 0;
  int* err_dev = nullptr;                    // device error bits
  int* err_host = nullptr;                   // pinned mirror of err_dev

  // adjoint checkpoints: adj_slots (x, p) states + adj_segment + 1 positions
  double* ckpt = nullptr;
  double* seg = nullptr;
  double* lam_x = nullptr;
  double* lam_p = nullptr;
  double* xw = nullptr;                     // [3 n_max] working state of the reverse pass
  double* pw = nullptr;
  double* tmp3 = nullptr;                   // [3 n_max] scratch cotangent
  double* tmp3b = nullptr;                  // [3 n_max] scratch product
  double* f_work = nullptr;                 // [3 n_max]
  double* red = nullptr;                    // device reduction scratch [32]
  double* ered = nullptr;                   // emittance partial sums [blocks][16]
  // deterministic = 1: 128-bit fixed-point node sums [n^3][2], the dipole scale bound, and the
  // partial sums of the fixed-order energy reductions [2][1024]
  unsigned long long* q128 = nullptr;
  unsigned long long* dbound = nullptr;
  double* dred = nullptr;

  // state
  bool deposited = false, solved = false, phi_valid = false;
  bool diff_valid = false;  // FP32: freal holds the difference fields of the current deposit
  int64_t last_n = 0;
  int last_parts = 0;
  std::string last_error;
};

namespace p3m {

// ---- launch helpers (defined in the .cu files) ----
// binning and sort (sort.cu)
void launch_bin(const p3m_ctx* c, const double* x, int64_t n, double* f_zero);
void launch_scan(const p3m_ctx* c);
void launch_scatter(const p3m_ctx* c, const double* x, int64_t n);

// mesh (pm.cu)
cudaError_t build_green(p3m_ctx* c);
void launch_zero_block(const p3m_ctx* c);
void launch_deposit(const p3m_ctx* c, int64_t n);
void launch_dipole_deposit(const p3m_ctx* c, int64_t n, const double* w);
void launch_green_multiply(const p3m_ctx* c, bool want_phi, bool want_diff, bool want_energy);
// fused z transforms + Green's multiply of the FP32 path (power-of-two Mz in [64, 2048])
bool zconv_supported(const p3m_ctx* c);
cudaError_t zconv_setup(p3m_ctx* c);
void launch_zconv(const p3m_ctx* c, bool want_energy);
// FP64 path: forward z transform, Green's multiply (with the cathode image term) and inverse z
// transform of the potential, fused, in double-float arithmetic (zsolve_df.cu)
bool zsolve_df_supported(const p3m_ctx* c);
cudaError_t zsolve_df_setup(p3m_ctx* c);
void launch_zsolve_df(const p3m_ctx* c, bool want_energy);
// grounded box (pm_bc = 2): discrete-Laplacian solve of the deposit into phireal
p3m_status box_setup(p3m_ctx* c);
p3m_status box_solve(p3m_ctx* c, bool want_energy);
void launch_interp(const p3m_ctx* c, int64_t n, double* f, int parts);
// deterministic = 1: fixed-order energies (short range from the per-particle potentials, mesh
// from (1/2) sum_g Q_g phi_g) into energy_acc[0] and energy_acc[1]
void launch_det_sum_pp(const p3m_ctx* c, int64_t n, cudaStream_t s);
void launch_det_sum_mesh(const p3m_ctx* c);
void launch_vjp_gather(const p3m_ctx* c, int64_t n, int pass, const double* w, double* out);
void launch_get_mesh(const p3m_ctx* c, int which, double* out);

// short range (pp.cu)
// want_energy: the short-range energy is asked for (the FP64 path skips the pair potentials
// otherwise)
void launch_pp(const p3m_ctx* c, int64_t n, cudaStream_t s, bool want_energy);
// (particle, record) distance tests of the FP32 short range on the current sorted records,
// into *out (FP64 contexts: nothing; their short range counts as it runs)
void launch_pp_count(const p3m_ctx* c, int64_t n, unsigned long long* out, cudaStream_t s);
void launch_pp_vjp(const p3m_ctx* c, int64_t n, const double* w, cudaStream_t s);

// particles (particles.cu)
void launch_bbox(const double* x, int64_t n, double* red, cudaStream_t s);
void launch_kick_drift(double* x, double* p, const double* f, int64_t n, double kick, double drift,
                       cudaStream_t s);
void launch_axpy(double* y, const double* x, int64_t n3, double a, cudaStream_t s);
void launch_scale(double* y, const double* x, int64_t n3, double a, cudaStream_t s);
// fixed-order reductions (deterministic for every context): part holds kEmitBlocks x 16 partial
// sums, red the 16 totals
constexpr int kEmitBlocks = 1216;
void launch_emittance(const double* x, const double* p, int64_t n, double mc, double* eps3,
                      double* gx, double* gp, double* part, double* red, cudaStream_t s);
void launch_energy_out(const p3m_ctx* c, double* energy);

}  // namespace p3m
