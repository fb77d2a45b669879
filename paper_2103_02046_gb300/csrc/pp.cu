// Short-range (particle-particle) half of P3M, eq. (summation_short) with the screened kernel
// G^S(r) = erfc(a r)/r of eq. (ewald_split); the self term is omitted. For r = |xi_i - xi_j|
// below the cutoff r_c the force on i is
//   k_e q^2 [erfc(a r)/r + (2a/sqrt(pi)) e^{-a^2 r^2}] (xi_i - xi_j) / r^2.
// With pp_bc = 1 the cathode also enters the short range (Sec. 3.1.1): each particle j has an
// image of charge -q at S(xi_j) (its own image included) that acts through the same kernel.
//
// Work is in cutoff units (rho = r / r_c, kappa = a r_c): the force is
// (k_e q^2 / r_c^2) [erfc(kappa rho)/rho + (2 kappa/sqrt(pi)) e^{-kappa^2 rho^2}] rho_vec / rho^2.
//
// Search: cells are rows along x (r_c / R wide in y and z, R = Geom::rows = 2, or 1 at low
// density; r_c / nsub in x; keys x-fastest). For particle i and each of the (2R + 1)^2
// neighbour rows, the distance d from i to the row's (y, z) rectangle bounds |dx| < sqrt(1 - d^2),
// which selects one contiguous run of sorted particles; rows with d >= 1 are skipped. With R = 2
// this visits about 8 r_c^3 of volume per particle (the cutoff sphere is 4.19 r_c^3) instead of
// the 27 r_c^3 of a plain 27-cell stencil.
//
// FP32: every candidate's separation is (hi_i - hi_j) + (lo_i - lo_j) of the cutoff-unit
// positions, exact to FP32 relative rounding at any distance. Partial sums are folded into a
// two-float (TwoSum) accumulator every few steps, so the per-particle sum is compensated at a
// small fraction of an addition per pair.
#include <algorithm>
#include <cmath>

#include "p3m_internal.cuh"

namespace p3m {
namespace {

constexpr int kThreads = 128;

// Row geometry for kRows cell rows per cutoff length in y and z (Geom::rows, 1 or 2): the
// neighbour rows of a particle's row are the (2 kRows + 1)^2 rows around it, numbered y fastest;
// the particle's own row is number `first`, and the half shell walked by the short range is
// rows first .. last - 1 (13 of 25 rows, or 5 of 9).
template <int kRows>
struct Rows {
  static constexpr int reach = kRows;
  static constexpr int span = 2 * kRows + 1;
  static constexpr int first = span * span / 2;
  static constexpr int last = span * span;
  static constexpr int half = last - first;
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

__device__ __forceinline__ void pair_terms(double r2, double kappa, double c2k, double& fco,
                                           double& pot) {
  const double r = sqrt(r2);
  const double x = kappa * r;
  const double ec = erfc(x);
  const double ex = exp(-x * x);
  pot = ec / r;
  fco = (pot + c2k * ex) / r2;
}

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

// Calls visit(j0, j1) for every neighbour row of the query point (px, py, pz) (cutoff units)
// that can hold particles within distance 1, with [j0, j1) the sorted range of its cells whose
// x-extent meets (px - w, px + w), w = sqrt(1 - d^2) + slack, d the point's distance to the
// row's (y, z) rectangle less the slack. The slack (Geom::slack) exceeds every rounding in where
// the sort placed a particle, so no particle within distance 1 is left out.
template <typename T, typename V>
__device__ __forceinline__ void for_rows(const Geom& g, const uint32_t* __restrict__ starts, T px,
                                         T py, T pz, V&& visit) {
  const T slack = static_cast<T>(g.slack);
  const T cwy = static_cast<T>(g.cw[1]), cwz = static_cast<T>(g.cw[2]);
  const T iwx = static_cast<T>(g.inv_cw[0]), iwy = static_cast<T>(g.inv_cw[1]),
          iwz = static_cast<T>(g.inv_cw[2]);
  const int y0 = max(static_cast<int>(floor((py - T(1) - slack) * iwy)), 0);
  const int y1 = min(static_cast<int>(floor((py + T(1) + slack) * iwy)), g.nc[1] - 1);
  const int z0 = max(static_cast<int>(floor((pz - T(1) - slack) * iwz)), 0);
  const int z1 = min(static_cast<int>(floor((pz + T(1) + slack) * iwz)), g.nc[2] - 1);
  for (int rz = z0; rz <= z1; ++rz) {
    const T zl = static_cast<T>(rz) * cwz, zh = zl + cwz;
    const T dz = max((pz < zl ? zl - pz : (pz > zh ? pz - zh : T(0))) - slack, T(0));
    for (int ry = y0; ry <= y1; ++ry) {
      const T yl = static_cast<T>(ry) * cwy, yh = yl + cwy;
      const T dy = max((py < yl ? yl - py : (py > yh ? py - yh : T(0))) - slack, T(0));
      const T d2 = dy * dy + dz * dz;
      if (d2 >= T(1)) continue;
      const T w = sqrt(T(1) - d2) + slack;
      const int c0 = max(static_cast<int>(floor((px - w) * iwx)), 0);
      const int c1 = min(static_cast<int>(floor((px + w) * iwx)), g.nc[0] - 1);
      if (c0 > c1) continue;
      const uint32_t base = (static_cast<uint32_t>(rz) * g.nc[1] + ry) * g.nc[0];
      visit(starts[base + c0], starts[base + c1 + 1]);
    }
  }
}

// ------------------------------------------------------------------------------------------
// Position access for the FP64 adjoint kernel.
// ------------------------------------------------------------------------------------------
struct PosD {
  const Rec64* __restrict__ r;
};

// ------------------------------------------------------------------------------------------
// FP32 short range: each unordered pair once (Newton's third law), each lane holding two
// particles and walking their candidate lists in lockstep with the other lanes.
//
// Pairs: particle i takes the pairs (i, j) with j > i in sorted order. Sorted order is row-major
// over (z row, y row, x cell), so these are the later part of i's own row and the neighbour
// rows after it (dz > 0, or dz = 0 and dy > 0) -- 13 of 25 rows, or 5 of 9. i's row is the one
// the sort put it in (stored with the record), so every pair is taken by exactly one of its
// particles.
//
// Lanes: lane l of a tile holds the sorted particles a = 2l and b = 2l + 1 (adjacent in sorted
// order, so nearly always in the same row and a quarter cutoff apart or less). Per neighbour row
// the lane walks the hull of the two particles' runs and tests every loaded record against
// both: one 256-bit load serves two particles, which halves the record traffic of the short
// range (the L1 data pipe bounds this kernel). Each pair is still taken exactly once: a pair
// (i, j) counts only when j > i and |xi_i - xi_j| < r_c, and the hull holds no record twice.
// When a and b lie in different rows (a row boundary) the lane keeps both run lists, each
// tested against its own particle only.
//
// The force on a and b accumulates in registers; the reaction on j (both particles' share) goes
// to j by one predicated vector reduction (red.global.add.v4.f32) into the zeroed result array,
// and a's and b's own sums are added the same way at the end.
//
// Walk: each lane first writes its non-empty runs (at most 13, or 26 across a row boundary) to
// shared memory, then the warp steps through them together, two records per lane per step; a
// lane moves on to its next run as soon as one ends. Lanes with nothing left re-read record 0
// with every result masked. The step is straight-line code: the pair function runs for every
// lane and candidate and its results are selected by the hit predicate, since with 64 lane
// candidates per step some lane nearly always holds a pair. Separations are exact to FP32
// relative rounding ((hi_i - hi_j) + (lo_i - lo_j)). FP32 partial sums are folded into a
// two-float (TwoSum) accumulator every 16 steps.
// The pair function uses one ex2 for both e^{-kappa^2 rho^2} terms and the fitted polynomial
// R(x) = erfc(x) e^{x^2}: erfc(kappa rho) = R * e^{-kappa^2 rho^2}; rsqrt and ex2 are the
// hardware approximations (flush-to-zero: every argument here is a normal number).
// ------------------------------------------------------------------------------------------
constexpr int kPpBlocksPerSm = 6;    // resident blocks per SM of the short range (80 registers)
constexpr int kVjpBlocksPerSm = 10;  // resident blocks per SM of its adjoint (48 registers)

// One 32-byte record (hi and lo float4) in a single 256-bit load through the read-only path.
// The records array is 32-byte aligned and not written while the short range runs.
__device__ __forceinline__ void load_rec32(const float4* p, float4& h, float4& l) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(h.x), "=f"(h.y), "=f"(h.z), "=f"(h.w), "=f"(l.x), "=f"(l.y), "=f"(l.z), "=f"(l.w)
      : "l"(p));
}

__device__ __forceinline__ void red_add_v4(float4* dst, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}

// predicated form: the reduction happens only where p holds (no branch around it)
__device__ __forceinline__ void red_add_v4_if(bool p, float4* dst, float a, float b, float c,
                                              float d) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %5, 0;\n\t"
      "@q red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n\t}" ::"l"(dst),
      "f"(a), "f"(b), "f"(c), "f"(d), "r"(static_cast<int>(p))
      : "memory");
}

__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float ex2_ftz(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// pair_poly on the hardware approximations; r2 in (0, 1]
template <int kDeg>
__device__ __forceinline__ void pair_poly_hw(const PairPoly& P, float r2, float& fco,
                                             float& pot) {
  const float rinv = rsqrt_ftz(r2);
  const float rho = r2 * rinv;
  const float t = fmaf(2.f, rho, -1.f);
  float R = P.c[kDeg];
#pragma unroll
  for (int m = kDeg - 1; m >= 0; --m) R = fmaf(R, t, P.c[m]);
  const float ex = ex2_ftz(-P.kappa2_log2e * r2);
  pot = R * ex * rinv;
  fco = fmaf(P.c2k, ex, pot) * (rinv * rinv);
}

template <int kDeg>
__device__ __forceinline__ void pair_poly(const PairPoly& P, float r2, float& fco, float& pot) {
  const float rinv = rsqrtf(r2);
  const float rho = r2 * rinv;
  const float t = fmaf(2.f, rho, -1.f);
  float R = P.c[kDeg];
#pragma unroll
  for (int m = kDeg - 1; m >= 0; --m) R = fmaf(R, t, P.c[m]);
  const float ex = exp2f(-P.kappa2_log2e * r2);
  pot = R * ex * rinv;
  fco = fmaf(P.c2k, ex, pot) * (rinv * rinv);
}

// Sorted range [j0, j1) of neighbour row r (y fastest, Rows::first = the particle's own row
// (cy, cz)) that can hold particles within distance 1 of (px, py, pz); empty if none can. The
// rectangle distance and the x half-width carry the search slack, as in for_rows.
template <int kRows>
__device__ __forceinline__ void row_range(const Geom& g, const uint32_t* __restrict__ starts,
                                          float px, float py, float pz, int cy, int cz, int r,
                                          uint32_t& j0, uint32_t& j1) {
  using R = Rows<kRows>;
  j0 = j1 = 0;
  const int ry = cy + (r % R::span) - R::reach, rz = cz + (r / R::span) - R::reach;
  if (ry < 0 || ry >= g.nc[1] || rz < 0 || rz >= g.nc[2]) return;
  const float slack = g.slack_f;
  const float cwy = g.cw_f[1], cwz = g.cw_f[2];
  const float yl = ry * cwy, yh = yl + cwy, zl = rz * cwz, zh = zl + cwz;
  const float dy = fmaxf((py < yl ? yl - py : (py > yh ? py - yh : 0.f)) - slack, 0.f);
  const float dz = fmaxf((pz < zl ? zl - pz : (pz > zh ? pz - zh : 0.f)) - slack, 0.f);
  const float d2 = dy * dy + dz * dz;
  if (d2 >= 1.f) return;
  const float w = sqrtf(1.f - d2) + slack;
  const float iwx = g.inv_cw_f[0];
  const int c0 = max(static_cast<int>(floorf((px - w) * iwx)), 0);
  const int c1 = min(static_cast<int>(floorf((px + w) * iwx)), g.nc[0] - 1);
  if (c0 > c1) return;
  const uint32_t base = (static_cast<uint32_t>(rz) * g.nc[1] + ry) * g.nc[0];
  j0 = starts[base + c0];
  j1 = starts[base + c1 + 1];
}

// The runs of the lane holding sorted particles a = ia and b = ia + 1 (b only if alive_b),
// in walk order: emit(j0, j1) for each non-empty run. With a and b in one row (same) each run is
// the hull of the two particles' runs in one neighbour row and is tested against both;
// otherwise a's runs come first (split of them) and are tested against a only, then b's.
template <int kRows, typename Emit>
__device__ __forceinline__ void pair_runs(const Geom& g, const uint32_t* __restrict__ starts,
                                          const float4& pa, const float4& la, const float4& pb,
                                          const float4& lb, uint32_t ia, bool alive_b, bool& same,
                                          int& split, Emit&& emit) {
  constexpr int kFirst = Rows<kRows>::first, kLast = Rows<kRows>::last;  // half shell
  const uint32_t ib = ia + 1;
  const uint32_t row_a = __float_as_uint(la.w) & kRowMask;
  const uint32_t row_b = __float_as_uint(lb.w) & kRowMask;
  same = !alive_b || row_a == row_b;
  const int cya = static_cast<int>(row_a % static_cast<uint32_t>(g.nc[1]));
  const int cza = static_cast<int>(row_a / static_cast<uint32_t>(g.nc[1]));
  int n = 0;
#pragma unroll 1
  for (int r = kFirst; r < kLast; ++r) {
    uint32_t j0, j1;
    row_range<kRows>(g, starts, pa.x, pa.y, pa.z, cya, cza, r, j0, j1);
    j0 = max(j0, ia + 1);  // own row: only the particles after a (a no-op for later rows)
    if (same && alive_b) {
      uint32_t k0, k1;
      row_range<kRows>(g, starts, pb.x, pb.y, pb.z, cya, cza, r, k0, k1);
      k0 = max(k0, ib + 1);
      if (k0 < k1) {
        j0 = j0 < j1 ? min(j0, k0) : k0;
        j1 = max(j1, k1);
      }
    }
    if (j0 < j1) {
      emit(j0, j1);
      ++n;
    }
  }
  split = n;
  if (!same) {
    const int cyb = static_cast<int>(row_b % static_cast<uint32_t>(g.nc[1]));
    const int czb = static_cast<int>(row_b / static_cast<uint32_t>(g.nc[1]));
#pragma unroll 1
    for (int r = kFirst; r < kLast; ++r) {
      uint32_t j0, j1;
      row_range<kRows>(g, starts, pb.x, pb.y, pb.z, cyb, czb, r, j0, j1);
      j0 = max(j0, ib + 1);
      if (j0 < j1) emit(j0, j1);
    }
  }
}

// ------------------------------------------------------------------------------------------
// FP32 short range with the candidate tests separated from the pair evaluations.
//
// Pairs: as above, particle i takes the pairs (i, j) with j > i in sorted order. Lane l of a
// tile holds the adjacent sorted particles a = 2l and b = a + 1 when they share a cell row;
// otherwise b goes to a list that a second launch works through, one particle per lane (so no
// lane of the first launch carries two run lists). Per neighbour row the lane walks the hull of
// a's and b's runs (13 rows of the half shell, or 5 with rows r_c wide), one candidate record
// per step, and tests it against both particles.
//
// Tests read the 16-byte search records (SearchRec): a separation is three subtractions from
// cell-local coordinates, accurate to a few 1e-8 cutoff lengths. A record within the cutoff of
// a or b is pushed, with a's separation and the two hit flags, into the lane's ring of pending
// pairs in shared memory. When some lane's ring is full the warp evaluates one pending entry per
// lane: the pair function for a and b side by side in the two-wide FP32 instructions, the force
// on a and b added to their sums in registers and the reaction on j (both particles' share)
// added to j's result by one vector reduction. The pair function thus runs on pairs only (a ring
// entry holds at least one), instead of on every lane's candidate as a lockstep walk would.
//
// Accumulation: the sums of a and b are folded into two-float (TwoSum) accumulators every 16
// evaluations. Reactions are FP32 reductions: a particle with m reactions gets at most m
// roundings of half an ulp of its running sum (FP64 reductions would need FP64 conversions and
// additions in every evaluation, which this part runs at a small fraction of the FP32 rate).
// Pairs closer than 1e-2 r_c (about one in a million) take their separation from the 32-byte
// hi + lo records instead, exact to FP32 relative rounding.
// ------------------------------------------------------------------------------------------
// resident blocks per SM of the FP32 short range (its register budget: 65536 / (128 x blocks));
// a build-time tuning value
#ifndef P3M_PP32_BLOCKS
#define P3M_PP32_BLOCKS 5
#endif
constexpr int kPp32BlocksPerSm = P3M_PP32_BLOCKS;

__device__ __forceinline__ float4 ldg_nc(const float4* p) {
  float4 v;
  asm("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p));
  return v;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// packed squared distance of (a, b): the same operations in the tests and in the evaluations,
// so that an evaluation sees the r^2 its test saw
__device__ __forceinline__ float2 dist2(float2 dx, float2 dy, float2 dz) {
  float2 r2 = __fmul2_rn(dx, dx);
  r2 = __ffma2_rn(dy, dy, r2);
  return __ffma2_rn(dz, dz, r2);
}

// the pair function of pair_poly_hw for two pairs at once (r2 in (0, 1] in both lanes)
template <int kDeg>
__device__ __forceinline__ void pair_poly_hw2(const PairPoly& P, float2 r2, float2& fco,
                                              float2& pot) {
  const float2 rinv = f2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
  const float2 rho = __fmul2_rn(r2, rinv);
  const float2 t = __ffma2_rn(f2(2.f, 2.f), rho, f2(-1.f, -1.f));
  float2 R = f2(P.c[kDeg], P.c[kDeg]);
#pragma unroll
  for (int m = kDeg - 1; m >= 0; --m) R = __ffma2_rn(R, t, f2(P.c[m], P.c[m]));
  const float2 arg = __fmul2_rn(f2(-P.kappa2_log2e, -P.kappa2_log2e), r2);
  const float2 ex = f2(ex2_ftz(arg.x), ex2_ftz(arg.y));
  pot = __fmul2_rn(__fmul2_rn(R, ex), rinv);
  fco = __fmul2_rn(__ffma2_rn(f2(P.c2k, P.c2k), ex, pot), __fmul2_rn(rinv, rinv));
}

// exact separation of sorted particles i and j from the 32-byte records (hi + lo)
__device__ __forceinline__ void exact_sep(const float4* __restrict__ rec, uint32_t i, uint32_t j,
                                          float& dx, float& dy, float& dz) {
  const float4 hi = rec[2 * static_cast<size_t>(i)], li = rec[2 * static_cast<size_t>(i) + 1];
  const float4 hj = rec[2 * static_cast<size_t>(j)], lj = rec[2 * static_cast<size_t>(j) + 1];
  dx = (hi.x - hj.x) + (li.x - lj.x);
  dy = (hi.y - hj.y) + (li.y - lj.y);
  dz = (hi.z - hj.z) + (li.z - lj.z);
}

template <int kDeg, int kRows, bool kLeft>
__global__ void __launch_bounds__(kThreads, kPp32BlocksPerSm)
    k_pp_f32(Geom g, PairPoly P, const uint32_t* __restrict__ total,
             const float4* __restrict__ recs, const float4* __restrict__ rec,
             const uint32_t* __restrict__ starts, float4* __restrict__ fs,
             uint32_t* __restrict__ next_tile, uint32_t* __restrict__ left,
             double* __restrict__ energy, unsigned long long* __restrict__ pairs,
             uint32_t sentinel) {
  using RW = Rows<kRows>;
  constexpr int kW = kThreads / 32;
  constexpr int kR = RW::half;
  constexpr uint32_t kTile = kLeft ? 32u : 64u;  // particles per warp tile
  // per warp: the owners' runs, the owners' particle data and the owners' sums (each owner's
  // particles a and b: x, y, z, phi)
  __shared__ uint2 run_s[kW][kR][32];      // {j0, length}
  __shared__ uint8_t rrow_s[kW][kR][32];   // the run's row in the half shell
  __shared__ uint8_t nrun_s[kW][32];       // runs per owner
  __shared__ float4 own_s[kW][2][32];      // {x_loc, y_loc, z_loc, x_org}, {b - a, b alive}
  // the owners' sums, gathered without atomics: a lane's chunk covers its first owner's
  // candidates in part (sum in first_s[lane]), owners in the middle in full (mid_s[owner]) and
  // its last owner in part (last_s[lane]); fo_s / lo_s name the first and last owner
  __shared__ float mid_s[kW][8][32];
  __shared__ float first_s[kW][8][32];
  __shared__ float last_s[kW][8][32];
  __shared__ uint8_t fo_s[kW][32], lo_s[kW][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t N = kLeft ? left[0] : *total;
  const uint32_t nc1 = static_cast<uint32_t>(g.nc[1]);
  float e_hi = 0.f, e_lo = 0.f;  // sum of the particles' potentials (compensated)
  unsigned long long np = 0, ni = 0;
  for (;;) {
    uint32_t tile = 0;
    if (lane == 0) tile = atomicAdd(next_tile, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (static_cast<uint64_t>(tile) * kTile >= N) break;
    // ---- the owner: particles a and b of this lane ----
    uint32_t a, b;
    bool alive_a, alive_b;
    if (kLeft) {
      const uint32_t t = tile * kTile + lane;
      alive_a = t < N;
      a = alive_a ? left[1 + t] : 0u;
      b = a;
      alive_b = false;
    } else {
      a = tile * kTile + 2 * lane;
      b = a + 1;
      alive_a = a < N;
      alive_b = b < N;
    }
    const uint32_t ea = alive_a ? a : 0u;
    const uint32_t rowa = __float_as_uint(rec[2 * static_cast<size_t>(ea) + 1].w) & kRowMask;
    if (alive_b) {
      const uint32_t rowb = __float_as_uint(rec[2 * static_cast<size_t>(b) + 1].w) & kRowMask;
      if (rowb != rowa) {  // a row boundary between a and b: b to the second pass
        left[1 + atomicAdd(left, 1u)] = b;
        alive_b = false;
      }
    }
    const uint32_t eb = alive_b ? b : ea;
    const float4 sa = recs[ea], sb = recs[eb];
    const int cya = static_cast<int>(rowa % nc1), cza = static_cast<int>(rowa / nc1);
    // runs: per neighbour row of the half shell, the hull of a's and b's runs
    uint32_t L = 0;  // this owner's candidates
    int nr = 0;
    if (alive_a) {
      // positions for the row search (FP32 in cutoff units; the search slack covers rounding)
      const float ry0 = static_cast<float>(cya) * g.cw_f[1];
      const float rz0 = static_cast<float>(cza) * g.cw_f[2];
      const float pax = sa.w + sa.x, pay = ry0 + sa.y, paz = rz0 + sa.z;
      const float pbx = sb.w + sb.x, pby = ry0 + sb.y, pbz = rz0 + sb.z;
#pragma unroll 1
      for (int r = RW::first; r < RW::last; ++r) {
        uint32_t j0, j1;
        row_range<kRows>(g, starts, pax, pay, paz, cya, cza, r, j0, j1);
        j0 = max(j0, a + 1);
        if (alive_b) {
          uint32_t k0, k1;
          row_range<kRows>(g, starts, pbx, pby, pbz, cya, cza, r, k0, k1);
          k0 = max(k0, b + 1);
          if (k0 < k1) {
            j0 = j0 < j1 ? min(j0, k0) : k0;
            j1 = max(j1, k1);
          }
        }
        if (j0 < j1) {
          run_s[w][nr][lane] = make_uint2(j0, j1 - j0);
          rrow_s[w][nr][lane] = static_cast<uint8_t>(r);
          L += j1 - j0;
          ++nr;
        }
      }
    }
    nrun_s[w][lane] = static_cast<uint8_t>(nr);
    own_s[w][0][lane] = sa;
    own_s[w][1][lane] = make_float4(
        __fadd_rn(__fsub_rn(sb.x, sa.x), __fsub_rn(sb.w, sa.w)), __fsub_rn(sb.y, sa.y),
        __fsub_rn(sb.z, sa.z), alive_b ? 1.f : 0.f);
    for (int c = 0; c < 8; ++c) mid_s[w][c][lane] = 0.f;
    fo_s[w][lane] = lo_s[w][lane] = 0xff;
    __syncwarp();
    // ---- balanced chunks: the warp's candidates, owner by owner, cut into 32 equal parts ----
    uint32_t incl = L;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t c0 = static_cast<uint32_t>((static_cast<uint64_t>(lane) * T) >> 5);
    const uint32_t c1 = static_cast<uint32_t>((static_cast<uint64_t>(lane + 1) * T) >> 5);
    uint32_t rem = c1 - c0;  // candidates left in this lane's chunk
    // owner of candidate c0: the first lane whose inclusive prefix exceeds c0
    int o = 0;
    {
      int lo = 0, hi = 31;
#pragma unroll
      for (int it = 0; it < 5; ++it) {
        const int mid = (lo + hi) >> 1;
        const uint32_t pm = __shfl_sync(0xffffffffu, incl, mid);
        if (pm > c0) hi = mid; else lo = mid + 1;
      }
      o = lo;
    }
    const uint32_t before = __shfl_sync(0xffffffffu, incl - L, o);  // exclusive prefix of o
    // run and offset of c0 within owner o (only lanes with work read the owner's runs)
    int k = 0;
    uint32_t ptr = 0, rrem = 0;
    float4 oa = make_float4(0.f, 0.f, 0.f, 0.f), od = oa;
    float yo = 0.f, zo = 0.f;
    auto load_run = [&]() {
      const uint2 q = run_s[w][k][o];
      const int r = rrow_s[w][k][o];
      // offsets toward row (cya + dy, cza + dz) of the owner: k cw is exact for |k| <= 2
      yo = __fsub_rn(oa.y, static_cast<float>((r % RW::span) - RW::reach) * g.cw_f[1]);
      zo = __fsub_rn(oa.z, static_cast<float>((r / RW::span) - RW::reach) * g.cw_f[2]);
      return q;
    };
    if (rem > 0) {
      oa = own_s[w][0][o];
      od = own_s[w][1][o];
      uint32_t off = c0 - before;
      uint2 q = load_run();
      while (off >= q.y) {
        off -= q.y;
        ++k;
        q = load_run();
      }
      ptr = q.x + off;
      rrem = q.y - off;
    }
    // ---- candidate tests and pair evaluations, one candidate record per lane and step ----
    float2 qx = f2(0.f, 0.f), qy = qx, qz = qx, qp = qx;  // (a, b) partial sums
    Acc2 sum[8];                                          // a: x y z phi, b: x y z phi
    for (int c = 0; c < 8; ++c) sum[c].hi = sum[c].lo = 0.f;
    float nhit = 0.f;  // pairs evaluated by this lane (exact as a float below 2^24 per tile)
    auto fold = [&]() {
      sum[0].add(qx.x);
      sum[1].add(qy.x);
      sum[2].add(qz.x);
      sum[3].add(qp.x);
      sum[4].add(qx.y);
      sum[5].add(qy.y);
      sum[6].add(qz.y);
      sum[7].add(qp.y);
      qx = qy = qz = qp = f2(0.f, 0.f);
    };
    // a finished owner segment: the lane's first one to first_s, a middle one (the owner's
    // candidates all in this chunk) to mid_s, the last one to last_s
    int seg = 0;
    auto store_segment = [&](int owner, bool last) {
      fold();
      float* dst;
      if (seg == 0) {
        dst = &first_s[w][0][lane];
        fo_s[w][lane] = static_cast<uint8_t>(owner);
      } else if (last) {
        dst = &last_s[w][0][lane];
        lo_s[w][lane] = static_cast<uint8_t>(owner);
      } else {
        dst = &mid_s[w][0][owner];
      }
      for (int c = 0; c < 8; ++c) {
        dst[32 * c] = sum[c].value();
        sum[c].hi = sum[c].lo = 0.f;
      }
      ++seg;
    };
    // the next candidate's record is loaded one step ahead
    float4 rj = ldg_nc(recs + (rem > 0 ? ptr : sentinel));
    int step = 0;
    while (__any_sync(0xffffffffu, rem > 0)) {
      const bool v = rem > 0;
      const float4 cur = rj;
      const uint32_t jc = ptr;
      const int oc = o;
      const float xo = oa.x, xw = oa.w, yc = yo, zc = zo;
      const float4 dc = od;
      // advance: the next candidate of this run, of the owner's next run, or of the next owner
      // (lanes whose chunk is done keep their counters at zero)
      if (v) {
        --rem;
        --rrem;
        ++ptr;
      }
      if (v && rem > 0 && rrem == 0) {
        ++k;
        while (k >= nrun_s[w][o]) {
          ++o;
          k = 0;
          oa = own_s[w][0][o];
          od = own_s[w][1][o];
        }
        const uint2 q = load_run();
        ptr = q.x;
        rrem = q.y;
      }
      rj = ldg_nc(recs + (rem > 0 ? ptr : sentinel));
      // the current candidate against the owner's a and b (b's separation is a's plus b - a)
      const float dxa = __fadd_rn(__fsub_rn(xo, cur.x), __fsub_rn(xw, cur.w));
      const float dya = __fsub_rn(yc, cur.y), dza = __fsub_rn(zc, cur.z);
      float2 DX = f2(dxa, __fadd_rn(dxa, dc.x)), DY = f2(dya, __fadd_rn(dya, dc.y)),
             DZ = f2(dza, __fadd_rn(dza, dc.z));
      float2 R2 = dist2(DX, DY, DZ);
      // hit masks in FP32 (1 or 0): 0 < r2 < 1  <=>  r2 (1 - r2) > 0, saturated; a lane with
      // nothing left reads the sentinel record far away (r2 ~ 1e36), b only if alive
      const float2 t = __ffma2_rn(f2(-R2.x, -R2.y), R2, R2);
      float2 m = f2(__saturatef(t.x * 1e38f), __saturatef(t.y * 1e38f) * dc.w);
      // masked lanes evaluate the pair function at r2 = 1/2
      float2 R2m = __ffma2_rn(__fadd2_rn(R2, f2(-0.5f, -0.5f)), m, f2(0.5f, 0.5f));
      if (fminf(R2m.x, R2m.y) < 1e-4f) {
        bool fa = m.x != 0.f, fb = m.y != 0.f;
        // very close pair: the exact separation from the hi + lo records
        const uint32_t ia = kLeft ? left[1 + tile * kTile + oc] : tile * kTile + 2 * oc;
        float x0, y0, z0;
        if (fa) {
          exact_sep(rec, ia, jc, x0, y0, z0);
          DX.x = x0, DY.x = y0, DZ.x = z0;
        }
        if (fb) {
          exact_sep(rec, ia + 1, jc, x0, y0, z0);
          DX.y = x0, DY.y = y0, DZ.y = z0;
        }
        R2 = dist2(DX, DY, DZ);
        fa = fa && R2.x > 0.f && R2.x < 1.f;
        fb = fb && R2.y > 0.f && R2.y < 1.f;
        m = f2(fa ? 1.f : 0.f, fb ? 1.f : 0.f);
        R2m = f2(fa ? R2.x : 0.5f, fb ? R2.y : 0.5f);
      }
      float2 FCO, POT;
      pair_poly_hw2<kDeg>(P, R2m, FCO, POT);
      FCO = __fmul2_rn(FCO, m);
      POT = __fmul2_rn(POT, m);
      const float2 FX = __fmul2_rn(FCO, DX), FY = __fmul2_rn(FCO, DY), FZ = __fmul2_rn(FCO, DZ);
      qx = __fadd2_rn(qx, FX);
      qy = __fadd2_rn(qy, FY);
      qz = __fadd2_rn(qz, FZ);
      qp = __fadd2_rn(qp, POT);
      const float hits = m.x + m.y;
      red_add_v4_if(hits != 0.f, fs + jc, -__fadd_rn(FX.x, FX.y), -__fadd_rn(FY.x, FY.y),
                    -__fadd_rn(FZ.x, FZ.y), 0.f);
      nhit += hits;
      if (oc != o) store_segment(oc, false);  // the owner's last candidate of this chunk
      if ((++step & 15) == 0) fold();
    }
    if (c1 > c0) store_segment(o, true);
    np += static_cast<unsigned long long>(nhit);
    __syncwarp();
    // the owner's sums: its segments from the lanes whose chunks cover its candidates
    Acc2 own[8];
    for (int c = 0; c < 8; ++c) own[c].hi = own[c].lo = 0.f;
    if (L > 0) {
      const uint32_t pf = incl - L, pl = incl - 1;  // the owner's first and last candidate
      // lane whose chunk holds candidate c: the largest l with l T < 32 (c + 1)
      const int l0 = static_cast<int>((32ull * (pf + 1) - 1) / T);
      const int l1 = static_cast<int>((32ull * (pl + 1) - 1) / T);
      for (int l = l0; l <= l1; ++l) {
        const float* src;
        if (fo_s[w][l] == lane)
          src = &first_s[w][0][l];
        else if (lo_s[w][l] == lane)
          src = &last_s[w][0][l];
        else
          src = &mid_s[w][0][lane];  // one lane's chunk holds all of the owner's candidates
        for (int c = 0; c < 8; ++c) own[c].add(src[32 * c]);
      }
    }
    __syncwarp();  // the segment arrays are reused by the next tile
    // ---- the owner's images and its own sums, energy ----
    const float pair_pot_a = own[3].value(), pair_pot_b = own[7].value();
    // images within r_c of particles less than r_c above the cathode (rare): plain loop over
    // all rows around the image point; image pairs act on the particle only
    auto images = [&](uint32_t i, Acc2* acc) {
      const float4 pi = rec[2 * static_cast<size_t>(i)], li = rec[2 * static_cast<size_t>(i) + 1];
      const double zi = static_cast<double>(pi.z) + static_cast<double>(li.z);
      if (zi - 0.5 * g.img_c >= 1.0) return;
      const float mz = static_cast<float>(g.img_c - zi);
      const float ch = static_cast<float>(g.img_c);
      const float cl = static_cast<float>(g.img_c - static_cast<double>(ch));
      for_rows<float>(g, starts, pi.x, pi.y, mz, [&](uint32_t ja, uint32_t jb) {
        float rowv[4] = {0.f, 0.f, 0.f, 0.f};
        for (uint32_t jj = ja; jj < jb; ++jj) {
          const float4 hj = rec[2 * jj], lj = rec[2 * jj + 1];
          const float ax = (pi.x - hj.x) + (li.x - lj.x);
          const float ay = (pi.y - hj.y) + (li.y - lj.y);
          const float s = pi.z + hj.z;
          const float bp = s - pi.z;
          const float e = (pi.z - (s - bp)) + (hj.z - bp);
          const float az = ((s - ch) + e) + ((li.z + lj.z) - cl);
          const float r2 = ax * ax + ay * ay + az * az;
          if (r2 < 1.f && r2 > 0.f) {
            float fco, pot;
            pair_poly<kDeg>(P, r2, fco, pot);
            rowv[0] -= fco * ax;
            rowv[1] -= fco * ay;
            rowv[2] -= fco * az;
            rowv[3] -= pot;
            ++ni;
          }
        }
        for (int c = 0; c < 4; ++c) acc[c].add(rowv[c]);
      });
    };
    if (g.pp_bc) {
      if (alive_a) images(a, own);
      if (alive_b) images(b, own + 4);
    }
    // own sums (reactions from other lanes arrive concurrently, by the same reduction)
    auto add_energy = [&](float v) {
      const DF t = df_two_sum(e_hi, v);
      e_hi = t.hi;
      e_lo += t.lo;
    };
    if (alive_a) {
      red_add_v4(fs + a, own[0].value(), own[1].value(), own[2].value(), 0.f);
      add_energy(own[3].value());
      add_energy(pair_pot_a);
    }
    if (alive_b) {
      red_add_v4(fs + b, own[4].value(), own[5].value(), own[6].value(), 0.f);
      add_energy(own[7].value());
      add_energy(pair_pot_b);
    }
  }
  if (energy) block_reduce_add(static_cast<double>(e_hi) + static_cast<double>(e_lo), energy);
  warp_add_u64(2ull * np, pairs);
  warp_add_u64(ni, pairs + 1);
}

// (particle, record) distance tests k_pp_f32 makes on the current sorted records: the same
// runs, summed instead of walked (a run shared by a and b counts twice). Run on request only,
// so that the short range itself carries no counter.
template <int kRows>
__global__ void k_pp_count_f32(Geom g, const uint32_t* __restrict__ total,
                               const float4* __restrict__ rec,
                               const uint32_t* __restrict__ starts,
                               unsigned long long* __restrict__ out) {
  const uint32_t N = *total;
  const uint32_t lane_pair = blockIdx.x * static_cast<uint32_t>(blockDim.x) + threadIdx.x;
  const uint32_t ia = 2 * lane_pair, ib = ia + 1;
  unsigned long long n = 0;
  if (ia < N) {
    const bool alive_b = ib < N;
    const uint32_t eb = alive_b ? ib : ia;
    const float4 pa = rec[2 * ia], la = rec[2 * ia + 1];
    const float4 pb = rec[2 * eb], lb = rec[2 * eb + 1];
    bool same = true;
    int split = 0;
    pair_runs<kRows>(g, starts, pa, la, pb, lb, ia, alive_b, same, split,
                     [&](uint32_t j0, uint32_t j1) { n += j1 - j0; });
    if (same && alive_b) n *= 2;
  }
  warp_add_u64(n, out);
}

// ------------------------------------------------------------------------------------------
// FP32 vector-Jacobian product of the short-range force map, each unordered pair once: for a
// pair (i, j), j > i, with d = xi_i - xi_j and H(d) = fco(rho) I + dfr(rho) d d^T (the pair
// energy's Hessian, even in d), i gets H(d) (w_i - w_j) and j gets its negative. Same walk as
// k_pp_f32 (persistent blocks, runs in shared memory, 256-bit record loads); w in sorted
// order as float4 (ws). The result goes to acc4 (zeroed, cutoff units); image pairs (pp_bc)
// act on i only: acc_i -= H(d)(w_i - S w_j), d = xi_i - S xi_j.
// ------------------------------------------------------------------------------------------
template <int kDeg>
__device__ __forceinline__ void pair_hess_poly(const PairPoly& P, float r2, float& fco,
                                               float& dfr) {
  const float rinv = rsqrtf(r2);
  const float rho = r2 * rinv;
  const float t = fmaf(2.f, rho, -1.f);
  float R = P.c[kDeg];
#pragma unroll
  for (int m = kDeg - 1; m >= 0; --m) R = fmaf(R, t, P.c[m]);
  const float ex = exp2f(-P.kappa2_log2e * r2);
  const float pot = R * ex * rinv;           // erfc(kappa rho) / rho
  const float cex = P.c2k * ex;
  const float A = pot + cex;                 // rho^2 times the force coefficient
  const float rinv2 = rinv * rinv;
  fco = A * rinv2;
  // dA/drho = -c2k e/rho - erfc/rho^2 - 2 kappa^2 rho c2k e; dfr = (dA/rho^2 - 2 A/rho^3)/rho
  const float dA = -(cex + pot) * rinv - 2.f * P.kappa2 * rho * cex;
  dfr = (dA - 2.f * A * rinv) * rinv2 * rinv;
}

template <int kDeg, int kRows>
__global__ void __launch_bounds__(kThreads, kVjpBlocksPerSm)
    k_pp_vjp_f32(Geom g, PairPoly P, const uint32_t* __restrict__ total,
                 const float4* __restrict__ rec, const uint32_t* __restrict__ starts,
                 const float4* __restrict__ ws, float4* __restrict__ acc4,
                 uint32_t* __restrict__ next_tile) {
  using R = Rows<kRows>;
  __shared__ uint32_t run_j0[R::half][kThreads], run_j1[R::half][kThreads];
  __shared__ uint32_t tile_s;
  const int tid = threadIdx.x;
  const uint32_t N = *total;
  for (;;) {
    if (tid == 0) tile_s = atomicAdd(next_tile, 1u);
    __syncthreads();
    const uint32_t tile = tile_s;
    __syncthreads();
    if (static_cast<uint64_t>(tile) * kThreads >= N) break;
    const uint32_t i = tile * kThreads + tid;
    const bool alive = i < N;
    const uint32_t ie = alive ? i : 0u;
    const float4 pi = rec[2 * ie], li = rec[2 * ie + 1];
    const float4 wi = ws[ie];
    int cnt = 0;
    if (alive) {
      const uint32_t row = __float_as_uint(li.w) & kRowMask;
      const int cy = static_cast<int>(row % static_cast<uint32_t>(g.nc[1]));
      const int cz = static_cast<int>(row / static_cast<uint32_t>(g.nc[1]));
      for (int r = R::first; r < R::last; ++r) {
        uint32_t j0, j1;
        row_range<kRows>(g, starts, pi.x, pi.y, pi.z, cy, cz, r, j0, j1);
        j0 = max(j0, i + 1);
        if (j0 < j1) {
          run_j0[cnt][tid] = j0;
          run_j1[cnt][tid] = j1;
          ++cnt;
        }
      }
    }
    uint32_t ptr = 0, end = 0;
    if (cnt > 0) {
      ptr = run_j0[0][tid];
      end = run_j1[0][tid];
    }
    int k = 0;
    Acc2 sum[3];
    for (int c = 0; c < 3; ++c) sum[c].hi = sum[c].lo = 0.f;
    float part[3] = {0.f, 0.f, 0.f};
    auto pair = [&](bool hit, float r2, float rx, float ry, float rz, uint32_t j) {
      float fco, dfr;
      pair_hess_poly<kDeg>(P, hit ? r2 : 0.5f, fco, dfr);
      const float4 wj = ws[hit ? j : ie];
      const float v0 = wi.x - wj.x, v1 = wi.y - wj.y, v2 = wi.z - wj.z;
      const float dv = hit ? dfr * (rx * v0 + ry * v1 + rz * v2) : 0.f;
      fco = hit ? fco : 0.f;
      const float c0 = fmaf(fco, v0, dv * rx), c1 = fmaf(fco, v1, dv * ry),
                  c2 = fmaf(fco, v2, dv * rz);
      part[0] += c0;
      part[1] += c1;
      part[2] += c2;
      if (hit) red_add_v4(acc4 + j, -c0, -c1, -c2, 0.f);
    };
    int step = 0;
    while (__any_sync(0xffffffffu, ptr < end)) {
      const bool va = ptr < end, vb = ptr + 1 < end;
      const float4* pa = va ? rec + 2 * static_cast<size_t>(ptr) : rec;
      const float4* pb = vb ? rec + 2 * static_cast<size_t>(ptr + 1) : rec;
      float4 ha, la, hb, lb;
      load_rec32(pa, ha, la);
      load_rec32(pb, hb, lb);
      const float ax = (pi.x - ha.x) + (li.x - la.x), ay = (pi.y - ha.y) + (li.y - la.y),
                  az = (pi.z - ha.z) + (li.z - la.z);
      const float bx = (pi.x - hb.x) + (li.x - lb.x), by = (pi.y - hb.y) + (li.y - lb.y),
                  bz = (pi.z - hb.z) + (li.z - lb.z);
      const float ra = ax * ax + ay * ay + az * az, rb = bx * bx + by * by + bz * bz;
      const bool hita = va && ra < 1.f && ra > 0.f;
      const bool hitb = vb && rb < 1.f && rb > 0.f;
      if (__any_sync(0xffffffffu, hita)) pair(hita, ra, ax, ay, az, ptr);
      if (__any_sync(0xffffffffu, hitb)) pair(hitb, rb, bx, by, bz, ptr + 1);
      ptr += 2;
      {
        // the next run without a branch: slot k stays in bounds (k < cnt, or k = 0)
        const bool sw = ptr >= end && k + 1 < cnt;
        k += sw ? 1 : 0;
        const uint32_t nj0 = run_j0[k][tid], nj1 = run_j1[k][tid];
        ptr = sw ? nj0 : ptr;
        end = sw ? nj1 : end;
      }
      if ((++step & 7) == 0) {
        for (int c = 0; c < 3; ++c) {
          sum[c].add(part[c]);
          part[c] = 0.f;
        }
      }
    }
    for (int c = 0; c < 3; ++c) sum[c].add(part[c]);
    if (alive && g.pp_bc) {
      const double zi = static_cast<double>(pi.z) + static_cast<double>(li.z);
      if (zi - 0.5 * g.img_c < 1.0) {
        const float mz = static_cast<float>(g.img_c - zi);
        const float ch = static_cast<float>(g.img_c);
        const float cl = static_cast<float>(g.img_c - static_cast<double>(ch));
        for_rows<float>(g, starts, pi.x, pi.y, mz, [&](uint32_t ja, uint32_t jb) {
          float rowv[3] = {0.f, 0.f, 0.f};
          for (uint32_t jj = ja; jj < jb; ++jj) {
            const float4 hj = rec[2 * jj], lj = rec[2 * jj + 1];
            const float ax = (pi.x - hj.x) + (li.x - lj.x);
            const float ay = (pi.y - hj.y) + (li.y - lj.y);
            const float s = pi.z + hj.z;
            const float bp = s - pi.z;
            const float e = (pi.z - (s - bp)) + (hj.z - bp);
            const float az = ((s - ch) + e) + ((li.z + lj.z) - cl);
            const float r2 = ax * ax + ay * ay + az * az;
            if (r2 < 1.f && r2 > 0.f) {
              float fco, dfr;
              pair_hess_poly<kDeg>(P, r2, fco, dfr);
              const float4 wj = ws[jj];
              const float v0 = wi.x - wj.x, v1 = wi.y - wj.y, v2 = wi.z + wj.z;  // w_i - S w_j
              const float dv = dfr * (ax * v0 + ay * v1 + az * v2);
              rowv[0] -= fmaf(fco, v0, dv * ax);
              rowv[1] -= fmaf(fco, v1, dv * ay);
              rowv[2] -= fmaf(fco, v2, dv * az);
            }
          }
          for (int c = 0; c < 3; ++c) sum[c].add(rowv[c]);
        });
      }
    }
    if (alive) red_add_v4(acc4 + i, sum[0].value(), sum[1].value(), sum[2].value(), 0.f);
  }
}

// w (input order, FP64) -> ws (sorted order, float4): the weights the FP32 VJP pairs read.
__global__ void k_gather_w(const uint32_t* __restrict__ total, const float4* __restrict__ rec,
                           const double* __restrict__ w, float4* __restrict__ ws) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *total) return;
  const long long idx = __float_as_int(rec[2 * i].w);
  ws[i] = make_float4(static_cast<float>(w[3 * idx]), static_cast<float>(w[3 * idx + 1]),
                      static_cast<float>(w[3 * idx + 2]), 0.f);
}

// ------------------------------------------------------------------------------------------
// FP64 short range: each unordered pair once, as in the FP32 kernel: particle i takes the pairs
// with j > i in sorted order (every one of the 25 neighbour rows is clipped to j > i, so this
// holds however the row of i was rounded) and adds the reaction to j with FP64 reductions into
// the zeroed result. Rows are walked in lockstep. The FP64 pair function (erfc, exp, division)
// costs far more than finding a pair on this part, so pairs found wait in a per-lane ring in
// shared memory and are evaluated, a batch of one per lane, whenever some lane's ring is full:
// the pair function then runs with most lanes busy.
// ------------------------------------------------------------------------------------------
constexpr int kRing64 = 4;

template <int kRows>
__device__ __forceinline__ void row_range64(const Geom& g, const uint32_t* __restrict__ starts,
                                            double px, double py, double pz, int cy, int cz,
                                            int r, uint32_t& j0, uint32_t& j1) {
  using R = Rows<kRows>;
  j0 = j1 = 0;
  const int ry = cy + (r % R::span) - R::reach, rz = cz + (r / R::span) - R::reach;
  if (ry < 0 || ry >= g.nc[1] || rz < 0 || rz >= g.nc[2]) return;
  const double slack = g.slack;
  const double yl = ry * g.cw[1], yh = yl + g.cw[1], zl = rz * g.cw[2], zh = zl + g.cw[2];
  const double dy = fmax((py < yl ? yl - py : (py > yh ? py - yh : 0.0)) - slack, 0.0);
  const double dz = fmax((pz < zl ? zl - pz : (pz > zh ? pz - zh : 0.0)) - slack, 0.0);
  const double d2 = dy * dy + dz * dz;
  if (d2 >= 1.0) return;
  const double w = sqrt(1.0 - d2) + slack;
  const int c0 = max(static_cast<int>(floor((px - w) * g.inv_cw[0])), 0);
  const int c1 = min(static_cast<int>(floor((px + w) * g.inv_cw[0])), g.nc[0] - 1);
  if (c0 > c1) return;
  const uint32_t base = (static_cast<uint32_t>(rz) * g.nc[1] + ry) * g.nc[0];
  j0 = starts[base + c0];
  j1 = starts[base + c1 + 1];
}

// kDet (deterministic = 1): every ordered pair is evaluated by its own particle (all rows of the
// block, j != i), with no reductions: each particle's sum runs in the fixed sorted order and is
// stored as is, together with its potential (w), from which the energy is summed in a fixed
// order afterwards.
template <int kRows, bool kDet>
__global__ void __launch_bounds__(kThreads)
    k_pp_f64(Geom g, const uint32_t* __restrict__ total, const Rec64* __restrict__ rec,
             const Rec64* __restrict__ recm, const uint32_t* __restrict__ starts,
             D4* __restrict__ fpp, double* __restrict__ energy,
             unsigned long long* __restrict__ pairs) {
  __shared__ D4 ring_s[kThreads / 32][kRing64][32];
  __shared__ uint32_t ringj_s[kThreads / 32][kRing64][32];
  D4(*ring)[32] = ring_s[threadIdx.x >> 5];
  uint32_t(*ringj)[32] = ringj_s[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const uint32_t N = *total;
  const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
  const bool alive = i < N;
  const double kappa = g.kappa_eff;
  const double c2k = 2.0 * g.kappa_eff * 0.56418958354775628695;
  // lanes past the last particle compare record 0 with itself (separation 0, never a pair)
  const uint32_t ie = alive ? i : 0u;
  const Rec64 me = rec[ie];
  const double px = me.u[0], py = me.u[1], pz = me.u[2];
  // the row the sort put the particle in (two particles closer than r_c sit in sort rows at most
  // kRows apart, whatever the rounding of either binning)
  const uint32_t row = static_cast<uint32_t>(static_cast<unsigned long long>(recm[ie].idx) >> 32);
  const int cy = static_cast<int>(row % static_cast<uint32_t>(g.nc[1]));
  const int cz = static_cast<int>(row / static_cast<uint32_t>(g.nc[1]));
  double sum[4] = {0.0, 0.0, 0.0, 0.0};
  unsigned int np = 0, ncand = 0;  // pairs found, records tested
  int head = 0, cnt = 0;
  auto evaluate = [&]() {
    const bool has = cnt > 0;
    D4 e = ring[head & (kRing64 - 1)][lane];
    const uint32_t j = ringj[head & (kRing64 - 1)][lane];
    if (!has) e = D4{0.0, 0.0, 0.0, 0.5};
    double fco, pot;
    pair_terms(e.w, kappa, c2k, fco, pot);
    if (has) {
      const double fx = fco * e.x, fy = fco * e.y, fz = fco * e.z;
      sum[0] += fx;
      sum[1] += fy;
      sum[2] += fz;
      sum[3] += pot;
      if (!kDet) {
        double* fj = &fpp[j].x;
        // the potential is summed on the owner's side only: j's fourth component stays unused
        atomicAdd(fj, -fx);
        atomicAdd(fj + 1, -fy);
        atomicAdd(fj + 2, -fz);
      }
    }
    head += has;
    cnt -= has;
  };
  for (int r = 0; r < Rows<kRows>::last; ++r) {
    uint32_t j0 = 0, j1 = 0;
    if (alive) {
      row_range64<kRows>(g, starts, px, py, pz, cy, cz, r, j0, j1);
      if (!kDet) j0 = max(j0, i + 1);
      j1 = max(j1, j0);
    }
    const int len = static_cast<int>(j1 - j0);
    ncand += static_cast<unsigned>(len);
    int maxlen = len;
    for (int o = 16; o > 0; o >>= 1) maxlen = max(maxlen, __shfl_xor_sync(0xffffffffu, maxlen, o));
    for (int t = 0; t < maxlen; ++t) {
      const uint32_t j = t < len ? j0 + t : ie;  // an idle lane re-reads itself: no pair
      const Rec64 rj = rec[j];
      const double rx = px - rj.u[0], ry = py - rj.u[1], rz = pz - rj.u[2];
      const double r2 = rx * rx + ry * ry + rz * rz;
      if (alive && j != i && r2 < 1.0 && r2 > 0.0) {
        ring[(head + cnt) & (kRing64 - 1)][lane] = D4{rx, ry, rz, r2};
        ringj[(head + cnt) & (kRing64 - 1)][lane] = j;
        ++cnt;
        ++np;
      }
      if (__any_sync(0xffffffffu, cnt == kRing64)) evaluate();
    }
  }
  while (__any_sync(0xffffffffu, cnt > 0)) evaluate();
  const double pair_pot = sum[3];
  unsigned long long ni = 0;
  if (alive && g.pp_bc && pz - 0.5 * g.img_c < 1.0) {
    // images within r_c of particles less than r_c above the cathode (rare): plain loop
    for_rows<double>(g, starts, px, py, g.img_c - pz, [&](uint32_t ja, uint32_t jb) {
      for (uint32_t jj = ja; jj < jb; ++jj) {
        const Rec64 rj = rec[jj];
        const double ax = px - rj.u[0], ay = py - rj.u[1], az = pz + rj.u[2] - g.img_c;
        const double r2 = ax * ax + ay * ay + az * az;
        if (r2 < 1.0 && r2 > 0.0) {
          double fco, pot;
          pair_terms(r2, kappa, c2k, fco, pot);
          sum[0] -= fco * ax;
          sum[1] -= fco * ay;
          sum[2] -= fco * az;
          sum[3] -= pot;
          ++ni;
        }
      }
    });
  }
  if (kDet) {
    // sum_i phi_i is formed from w in a fixed order by the caller
    if (alive) fpp[i] = D4{sum[0], sum[1], sum[2], sum[3]};
  } else {
    if (alive) {
      double* fi = &fpp[i].x;
      for (int c = 0; c < 3; ++c) atomicAdd(fi + c, sum[c]);  // the potential: energy only
    }
    // sum_i phi_i over ordered pairs: each pair's potential was taken once here, plus images
    if (energy) block_reduce_add(alive ? sum[3] + pair_pot : 0.0, energy);
  }
  warp_add_u64(kDet ? np : 2ull * np, pairs);
  warp_add_u64(ni, pairs + 1);
  warp_add_u64(ncand, pairs + 2);
}

// Vector-Jacobian product of the short-range force map, into acc (sorted order):
//   free pairs:  acc_i += H(d_ij) (w_i - w_j)
//   image pairs: acc_i -= H(d_ij) (w_i - S w_j)   (S = diag(1, 1, -1), image charge -q)
// H(d) = [phi(rho) I + (phi'(rho)/rho) d d^T] (times k_e q^2 / r_c^3). The force map is the
// gradient of an energy, so its Jacobian is symmetric and this gather equals J^T w.
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

// FP64 vector-Jacobian product of the short-range force map (every ordered pair, one thread
// per particle): acc_i = scale sum_j H(d_ij) (w_i - w_j) - scale sum_j H(d_ij') (w_i - S w_j)
// over image pairs (pp_bc).
__global__ void __launch_bounds__(kThreads)
    k_pp_vjp(Geom g, const uint32_t* __restrict__ total, PosD pos,
             const uint32_t* __restrict__ starts, const double* __restrict__ w,
             double* __restrict__ acc, double scale) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *total) return;
  const double kappa = g.kappa_eff;
  const double c2k = 2.0 * g.kappa_eff * 0.56418958354775628695;
  const Rec64 me = pos.r[i];
  const double pi[3] = {me.u[0], me.u[1], me.u[2]};
  const long long idx = me.idx;
  const double wi[3] = {w[3 * idx], w[3 * idx + 1], w[3 * idx + 2]};
  double out[3] = {0.0, 0.0, 0.0};
  for_rows<double>(g, starts, pi[0], pi[1], pi[2], [&](uint32_t j0, uint32_t j1) {
    for (uint32_t j = j0; j < j1; ++j) {
      if (j == i) continue;
      const Rec64 rj = pos.r[j];
      const double rx = pi[0] - rj.u[0], ry = pi[1] - rj.u[1], rz = pi[2] - rj.u[2];
      const double r2 = rx * rx + ry * ry + rz * rz;
      if (r2 < 1.0 && r2 > 0.0) {
        double fco, dfr;
        pair_hess(r2, kappa, c2k, fco, dfr);
        const double v0 = wi[0] - w[3 * rj.idx];
        const double v1 = wi[1] - w[3 * rj.idx + 1];
        const double v2 = wi[2] - w[3 * rj.idx + 2];
        const double dv = rx * v0 + ry * v1 + rz * v2;
        out[0] += fco * v0 + dfr * dv * rx;
        out[1] += fco * v1 + dfr * dv * ry;
        out[2] += fco * v2 + dfr * dv * rz;
      }
    }
  });
  if (g.pp_bc && pi[2] - 0.5 * g.img_c < 1.0) {
    for_rows<double>(g, starts, pi[0], pi[1], g.img_c - pi[2], [&](uint32_t j0, uint32_t j1) {
      for (uint32_t j = j0; j < j1; ++j) {
        const Rec64 rj = pos.r[j];
        const double rx = pi[0] - rj.u[0], ry = pi[1] - rj.u[1];
        const double rz = pi[2] + rj.u[2] - g.img_c;
        const double r2 = rx * rx + ry * ry + rz * rz;
        if (r2 < 1.0 && r2 > 0.0) {
          double fco, dfr;
          pair_hess(r2, kappa, c2k, fco, dfr);
          const double v0 = wi[0] - w[3 * rj.idx];
          const double v1 = wi[1] - w[3 * rj.idx + 1];
          const double v2 = wi[2] + w[3 * rj.idx + 2];  // w_i - S w_j
          const double dv = rx * v0 + ry * v1 + rz * v2;
          out[0] -= fco * v0 + dfr * dv * rx;
          out[1] -= fco * v1 + dfr * dv * ry;
          out[2] -= fco * v2 + dfr * dv * rz;
        }
      }
    });
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
  if (c->fp32) {
    // the kernel adds each pair's force to both particles: the result starts at zero
    cudaMemsetAsync(c->fpp, 0, sizeof(float4) * static_cast<size_t>(n), s);
    cudaMemsetAsync(c->pp_tile, 0, sizeof(uint32_t), s);
    cudaMemsetAsync(c->left, 0, sizeof(uint32_t), s);
    // persistent grids of a few blocks per SM; the second launch takes the particles the first
    // left over (those whose sorted neighbour starts a new cell row)
    const int64_t tiles = (n + 2 * kThreads - 1) / (2 * kThreads);  // two particles a thread
    const int64_t cap = static_cast<int64_t>(kPp32BlocksPerSm) * c->num_sms;
    const unsigned wblocks = static_cast<unsigned>(std::min<int64_t>(tiles, cap));
    const int64_t ltiles = (n / 2 + kThreads) / kThreads;
    const unsigned lblocks = static_cast<unsigned>(std::min<int64_t>(ltiles, cap));
    auto run = [&](auto k_rows1, auto k_rows2, auto l_rows1, auto l_rows2) {
      const bool one = c->g.rows == 1;
      auto kern = one ? k_rows1 : k_rows2;
      auto lern = one ? l_rows1 : l_rows2;
      const auto* recs = c->recs;
      const auto* rec = static_cast<const float4*>(c->recp);
      float4* fs = static_cast<float4*>(c->fpp);
      // recs[n_max] holds a record far from every particle: lanes with nothing to test read it
      const uint32_t sentinel = static_cast<uint32_t>(c->n_max);
      kern<<<wblocks, kThreads, 0, s>>>(c->g, c->poly, total, recs, rec, c->starts, fs,
                                        c->pp_tile, c->left, c->energy_acc, c->pair_acc,
                                        sentinel);
      cudaMemsetAsync(c->pp_tile, 0, sizeof(uint32_t), s);
      lern<<<lblocks, kThreads, 0, s>>>(c->g, c->poly, total, recs, rec, c->starts, fs,
                                        c->pp_tile, c->left, c->energy_acc, c->pair_acc,
                                        sentinel);
    };
#define P3M_PP_CASE(D)                                                                   \
  case D:                                                                               \
    run(k_pp_f32<D, 1, false>, k_pp_f32<D, 2, false>, k_pp_f32<D, 1, true>,             \
        k_pp_f32<D, 2, true>);                                                          \
    break;
    switch (c->poly.deg) {
      P3M_PP_CASE(6)
      P3M_PP_CASE(7)
      P3M_PP_CASE(8)
      P3M_PP_CASE(9)
      P3M_PP_CASE(10)
      P3M_PP_CASE(11)
      P3M_PP_CASE(12)
      P3M_PP_CASE(13)
      P3M_PP_CASE(14)
      default:
        run(k_pp_f32<15, 1, false>, k_pp_f32<15, 2, false>, k_pp_f32<15, 1, true>,
            k_pp_f32<15, 2, true>);
        break;
    }
#undef P3M_PP_CASE
  } else {
    auto kern = c->det ? (c->g.rows == 1 ? k_pp_f64<1, true> : k_pp_f64<2, true>)
                       : (c->g.rows == 1 ? k_pp_f64<1, false> : k_pp_f64<2, false>);
    if (!c->det) cudaMemsetAsync(c->fpp, 0, sizeof(D4) * static_cast<size_t>(n), s);
    kern<<<blocks, kThreads, 0, s>>>(c->g, total, static_cast<const Rec64*>(c->recp),
                                     static_cast<const Rec64*>(c->recm), c->starts,
                                     static_cast<D4*>(c->fpp), c->energy_acc, c->pair_acc);
    if (c->det) launch_det_sum_pp(c, n, s);
  }
}

void launch_pp_count(const p3m_ctx* c, int64_t n, unsigned long long* out, cudaStream_t s) {
  if (!c->fp32) return;  // FP64: the short range counts as it walks
  cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (n == 0) return;
  const int64_t lane_pairs = (n + 1) / 2;
  auto kern = c->g.rows == 1 ? k_pp_count_f32<1> : k_pp_count_f32<2>;
  kern<<<static_cast<unsigned>((lane_pairs + kThreads - 1) / kThreads), kThreads, 0, s>>>(
      c->g, c->starts + c->nkeys, static_cast<const float4*>(c->recp), c->starts, out);
}

void launch_pp_vjp(const p3m_ctx* c, int64_t n, const double* w, cudaStream_t s) {
  if (n == 0) return;
  const unsigned blocks = static_cast<unsigned>((n + kThreads - 1) / kThreads);
  const uint32_t* total = c->starts + c->nkeys;
  if (c->fp32) {
    // weights in sorted order (in acc, free until the mesh gather), result in fpp (cutoff
    // units; the mesh gather scales it)
    float4* ws = reinterpret_cast<float4*>(c->acc);
    k_gather_w<<<blocks, kThreads, 0, s>>>(total, static_cast<const float4*>(c->recp), w, ws);
    cudaMemsetAsync(c->fpp, 0, sizeof(float4) * static_cast<size_t>(n), s);
    cudaMemsetAsync(c->pp_tile, 0, sizeof(uint32_t), s);
    const unsigned wblocks = static_cast<unsigned>(
        std::min<int64_t>(blocks, static_cast<int64_t>(kVjpBlocksPerSm) * c->num_sms));
    auto run = [&](auto k_rows1, auto k_rows2) {
      auto kern = c->g.rows == 1 ? k_rows1 : k_rows2;
      kern<<<wblocks, kThreads, 0, s>>>(c->g, c->poly, total,
                                        static_cast<const float4*>(c->recp), c->starts, ws,
                                        static_cast<float4*>(c->fpp), c->pp_tile);
    };
    switch (c->poly.deg) {
      case 6: run(k_pp_vjp_f32<6, 1>, k_pp_vjp_f32<6, 2>); break;
      case 7: run(k_pp_vjp_f32<7, 1>, k_pp_vjp_f32<7, 2>); break;
      case 8: run(k_pp_vjp_f32<8, 1>, k_pp_vjp_f32<8, 2>); break;
      case 9: run(k_pp_vjp_f32<9, 1>, k_pp_vjp_f32<9, 2>); break;
      case 10: run(k_pp_vjp_f32<10, 1>, k_pp_vjp_f32<10, 2>); break;
      case 11: run(k_pp_vjp_f32<11, 1>, k_pp_vjp_f32<11, 2>); break;
      case 12: run(k_pp_vjp_f32<12, 1>, k_pp_vjp_f32<12, 2>); break;
      case 13: run(k_pp_vjp_f32<13, 1>, k_pp_vjp_f32<13, 2>); break;
      case 14: run(k_pp_vjp_f32<14, 1>, k_pp_vjp_f32<14, 2>); break;
      default: run(k_pp_vjp_f32<15, 1>, k_pp_vjp_f32<15, 2>); break;
    }
  } else {
    // d/dxi of (k_e q^2 / r_c^2) f(rho): one more factor 1/r_c
    const double scale = c->g.ke * c->g.q * c->g.q / (c->g.rc * c->g.rc * c->g.rc);
    k_pp_vjp<<<blocks, kThreads, 0, s>>>(
        c->g, total, PosD{static_cast<const Rec64*>(c->recp)}, c->starts, w, c->acc, scale);
  }
}

}  // namespace p3m
