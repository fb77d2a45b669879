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
#include <type_traits>

#include "df_math.cuh"
#include "p3m_internal.cuh"

namespace p3m {
namespace {

constexpr int kThreads = 128;

// Row geometry for kRows cell rows per cutoff length in y and z (Geom::rows, 1, 2 or 3): the
// neighbour rows of a particle's row are the (2 kRows + 1)^2 rows around it, numbered y fastest;
// the particle's own row is number `first`, and the half shell walked by the short range is
// rows first .. last - 1 (5 of 9, 13 of 25 or 25 of 49 rows).
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

template <int kBlk = kThreads>
__device__ __forceinline__ void block_reduce_add(double v, double* dst) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __shared__ double ws[kBlk / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = threadIdx.x < kBlk / 32 ? ws[threadIdx.x] : 0.0;
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
// The pair function uses one ex2 for both e^{-kappa^2 rho^2} terms and the fitted form
// R(x) = erfc(x) e^{x^2} = t P(u), t = 1 / (1 + p x): erfc(kappa rho) = R * e^{-kappa^2 rho^2};
// rsqrt, rcp and ex2 are the hardware approximations (flush-to-zero: every argument here is a
// normal number).
// ------------------------------------------------------------------------------------------
constexpr int kPpThreads = 128;     // threads per block of the FP32 short range
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

// Error-free split of a short-range force component about the grid of multiples of
// kSplitQ = 2^-6 (the kernel's force unit is the pair force at a cutoff length's scale, so the
// terms are O(1) and a particle's sums stay far below 2^24 kSplitQ even with tens of thousands
// of neighbours): v = c + f exactly, with c a multiple of kSplitQ and |f| <= kSplitQ / 2.
// Adding kSplitC = 1.5 * 2^23 * kSplitQ rounds v to that grid (the sum's last mantissa bit is
// worth kSplitQ); subtracting it again is exact (Sterbenz), and so is v - c. The coarse parts c
// of one particle's terms are multiples of kSplitQ, so their FP32 atomic sum is exact, and
// independent of the order, while it stays below 2^24 kSplitQ in magnitude; only the small
// parts f are rounded when summed.
constexpr float kSplitQ = 0.015625f;
constexpr float kSplitC = 1.5f * 8388608.f * kSplitQ;
// A term of magnitude 2^21 kSplitQ or more (a pair closer than about 0.006 cutoff lengths)
// would take the coarse sum out of its exact range: it goes whole to a third array (big), where
// a particle rarely has more than one term.
constexpr float kBigTerm = 2097152.f * kSplitQ;
// (in PTX, so that no compiler pass folds (v + C) - C into v)
__device__ __forceinline__ void split_q(float v, float& c, float& f) {
  float t;
  asm("add.rn.f32 %0, %1, %2;" : "=f"(t) : "f"(v), "f"(kSplitC));
  asm("sub.rn.f32 %0, %1, %2;" : "=f"(c) : "f"(t), "f"(kSplitC));
  asm("sub.rn.f32 %0, %1, %2;" : "=f"(f) : "f"(v), "f"(c));
}

__device__ __forceinline__ bool big_term(float a, float b, float c) {
  return fmaf(a, a, fmaf(b, b, c * c)) >= kBigTerm * kBigTerm;
}

// 2-wide reduction (the fine x and y parts)
__device__ __forceinline__ void red_add_v2_if(bool p, float2* dst, float a, float b) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t"
      "@q red.global.add.v2.f32 [%0], {%1, %2};\n\t}" ::"l"(dst),
      "f"(a), "f"(b), "r"(static_cast<int>(p))
      : "memory");
}

// One particle's short-range force held in three arrays: co (float4: the coarse x, y, z parts and
// the fine z part), fi (float2: the fine x and y parts) and bg (float4: big terms). Each added
// term is split; the coarse parts and the fine z part go out in one 4-wide reduction into co, the
// fine x and y parts in one 2-wide reduction into fi (24 bytes a term; the fourth coarse slot
// would otherwise carry a zero), or, if the term is big, it is reduced whole into bg. The result
// is the exact sum up to the rounding of the fine sums, whose terms are at most kSplitQ / 2, and
// of the (rare) big terms. `big` may be set for terms below kBigTerm too (a cheaper test that
// never misses a big term).
__device__ __forceinline__ void split_add_v4_if(bool p, bool big, float4* co, float2* fi,
                                                float4* bg, float a, float b, float c) {
  // x and y split on the two-wide FP32 instructions, z on the scalar ones (the same steps)
  const float2 ab = make_float2(a, b);
  const float2 abc = __fadd2_rn(__fadd2_rn(ab, make_float2(kSplitC, kSplitC)),
                                make_float2(-kSplitC, -kSplitC));
  const float2 abf = __fadd2_rn(ab, make_float2(-abc.x, -abc.y));
  float cc, cf;
  split_q(c, cc, cf);
  red_add_v4_if(p && !big, co, abc.x, abc.y, cc, cf);
  red_add_v2_if(p && !big, fi, abf.x, abf.y);
  if (p && big) red_add_v4(bg, abc.x + abf.x, abc.y + abf.y, cc + cf, 0.f);  // (a, b, c); rare
}
// the same for a compensated sum hi + lo (lo far below hi): hi is split, lo joins the fine part
__device__ __forceinline__ void split_add_v4(float4* co, float2* fi, float4* bg, float a, float b,
                                             float c, float la, float lb, float lc) {
  if (big_term(a, b, c)) {
    red_add_v4(bg, a, b, c, 0.f);
    red_add_v4(co, 0.f, 0.f, 0.f, lc);
    red_add_v2_if(true, fi, la, lb);
    return;
  }
  float ac, af, bc, bf, cc, cf;
  split_q(a, ac, af);
  split_q(b, bc, bf);
  split_q(c, cc, cf);
  red_add_v4(co, ac, bc, cc, __fadd_rn(cf, lc));
  red_add_v2_if(true, fi, __fadd_rn(af, la), __fadd_rn(bf, lb));
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

__device__ __forceinline__ float rcp_ftz(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// R(x) = erfc(x) e^{x^2}, x = kappa rho, as t P(u): t = 1 / (1 + p kappa rho), u = t - t_c
template <int kDeg, bool kHw>
__device__ __forceinline__ float erfcx_poly(const PairPoly& P, float rho) {
  const float t = kHw ? rcp_ftz(fmaf(P.pk, rho, 1.f)) : 1.f / fmaf(P.pk, rho, 1.f);
  const float u = t - P.tc;
  float R = P.c[kDeg];
#pragma unroll
  for (int m = kDeg - 1; m >= 0; --m) R = fmaf(R, u, P.c[m]);
  return R * t;
}

// pair_poly on the hardware approximations; r2 in (0, 1]
template <int kDeg>
__device__ __forceinline__ void pair_poly_hw(const PairPoly& P, float r2, float& fco,
                                             float& pot) {
  const float rinv = rsqrt_ftz(r2);
  const float rho = r2 * rinv;
  const float R = erfcx_poly<kDeg, true>(P, rho);
  const float ex = ex2_ftz(-P.kappa2_log2e * r2);
  pot = R * ex * rinv;
  fco = fmaf(P.c2k, ex, pot) * (rinv * rinv);
}

template <int kDeg>
__device__ __forceinline__ void pair_poly(const PairPoly& P, float r2, float& fco, float& pot) {
  const float rinv = rsqrtf(r2);
  const float rho = r2 * rinv;
  const float R = erfcx_poly<kDeg, false>(P, rho);
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

// b's own runs (particle ib in row row_b), for a lane whose two particles sit in different rows
template <int kRows, typename Emit>
__device__ __forceinline__ void b_runs(const Geom& g, const uint32_t* __restrict__ starts,
                                       const float4& pb, const float4& lb, uint32_t ib,
                                       Emit&& emit) {
  constexpr int kFirst = Rows<kRows>::first, kLast = Rows<kRows>::last;  // half shell
  const uint32_t row_b = __float_as_uint(lb.w) & kRowMask;
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

// The runs of the lane holding sorted particles a = ia and b = ia + 1 (b only if alive_b),
// in walk order: emit(j0, j1) for each non-empty run. With a and b in one row (same) each run is
// the hull of the two particles' runs in one neighbour row and is tested against both;
// otherwise a's runs come first (split of them) and are tested against a only, then b's
// (unless kOnlyA: the caller then takes b's runs later, from b_runs).
template <int kRows, bool kOnlyA = false, typename Emit>
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
  if (!kOnlyA && !same) b_runs<kRows>(g, starts, pb, lb, ib, emit);
}

// Run slots per lane of k_pp_f32: a's and b's runs, up to twice the half shell when their rows
// differ. With 3 rows per cutoff (25 half-shell rows) that would not fit beside 6 blocks per
// SM: a lane whose particles sit in different rows then walks a's runs first and b's after
// them, in the same slots.
__host__ __device__ constexpr int pp_pair_runs(int rows) {
  return (rows >= 3 ? 1 : 2) * ((2 * rows + 1) * (2 * rows + 1) - (2 * rows + 1) * (2 * rows + 1) / 2);
}
inline size_t pp_run_bytes(int rows) {
  return 2 * sizeof(uint32_t) * static_cast<size_t>(pp_pair_runs(rows)) * kPpThreads;
}

// Work stealing inside a warp: once at least kStealMin lanes have walked all their runs, each
// of them takes work from a lane that still has some: that lane's last unstarted run, or else
// the back half of its current run if at least 2 kStealRecs records are left of it. The thief
// first sends the sums of the pair it held to their force arrays, then adopts the donor's pair
// (positions, index, which of the two the run is tested against) with zeroed sums, which it
// sends out in turn when it is done or steals again; the reduction targets are shared, so the
// owner's force is the sum of its holders' parts. This takes the warp's step count from the
// maximum of its lanes' walks towards their mean.
constexpr int kStealMin = 8;
constexpr uint32_t kStealRecs = 4;

__device__ __forceinline__ float4 shfl_f4(float4 v, int src) {
  v.x = __shfl_sync(0xffffffffu, v.x, src);
  v.y = __shfl_sync(0xffffffffu, v.y, src);
  v.z = __shfl_sync(0xffffffffu, v.z, src);
  v.w = __shfl_sync(0xffffffffu, v.w, src);
  return v;
}

template <int kDeg, int kRows>
__global__ void __launch_bounds__(kPpThreads, kPpBlocksPerSm)
    k_pp_f32(Geom g, PairPoly P, const uint32_t* __restrict__ total,
             const float4* __restrict__ rec, const uint32_t* __restrict__ starts,
             float4* __restrict__ fpp, float2* __restrict__ flo, float4* __restrict__ fbig,
             uint32_t* __restrict__ next_tile,
             double* __restrict__ energy, unsigned long long* __restrict__ pairs) {
  constexpr uint32_t kTile = 2 * kPpThreads;  // particles per tile
  constexpr bool kPhased = kRows >= 3;
  constexpr int kPairRuns = pp_pair_runs(kRows);
  static_assert(kPairRuns == (kPhased ? 1 : 2) * Rows<kRows>::half, "run slots");
  // the lanes' runs, [kPairRuns][kPpThreads] each, in dynamic shared memory
  extern __shared__ uint32_t pp_runs[];
  uint32_t(*run_j0)[kPpThreads] = reinterpret_cast<uint32_t(*)[kPpThreads]>(pp_runs);
  uint32_t(*run_j1)[kPpThreads] = run_j0 + kPairRuns;
  __shared__ uint8_t donor_s[kPpThreads / 32][32];
  __shared__ uint32_t tile_s;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const uint32_t N = *total;
  double e_acc = 0.0;
  unsigned long long np = 0, ni = 0;
  // persistent blocks: each takes the next tile of kTile sorted particles until none is left
  // (the block's four warps work on adjacent particles, which share most of their neighbours
  // in L1)
  for (;;) {
    if (tid == 0) tile_s = atomicAdd(next_tile, 1u);
    __syncthreads();
    const uint32_t tile = tile_s;
    __syncthreads();
    if (static_cast<uint64_t>(tile) * kTile >= N) break;
    // the pair the lane holds: a = ia, b = ia + 1 (a thief adopts another lane's pair)
    uint32_t ia = tile * kTile + 2 * tid;
    bool alive_a = ia < N, alive_b = ia + 1 < N;
    // lanes past the last particle read record 0 (in bounds) and take part in the lockstep
    // loop with every result masked out
    const uint32_t ea = alive_a ? ia : 0u, eb = alive_b ? ia + 1 : ea;
    float4 pa = rec[2 * ea], la = rec[2 * ea + 1];
    float4 pb = rec[2 * eb], lb = rec[2 * eb + 1];
    // runs: with a and b in one row, the hull of their two runs per neighbour row (tested
    // against both); otherwise a's runs [0, split) and b's runs [split, cnt) (kPhased: a's
    // runs, then b's in their place once they are walked, while pending_b)
    int cnt = 0, split = 0;
    bool same = true;
    auto emit = [&](uint32_t j0, uint32_t j1) {
      run_j0[cnt][tid] = j0;
      run_j1[cnt][tid] = j1;
      ++cnt;
    };
    if (alive_a)
      pair_runs<kRows, kPhased>(g, starts, pa, la, pb, lb, ia, alive_b, same, split, emit);
    bool pending_b = kPhased && alive_a && !same;
    uint32_t ptr = 0, end = 0;
    int k = 0;
    if (cnt > 0) {
      ptr = run_j0[0][tid];
      end = run_j1[0][tid];
    }
    bool ta = same || split > 0;                               // the current run is tested against a
    bool tb = alive_b && (same || (!kPhased && split == 0));   // ... and against b
    Acc2 sa[4], sb[4];
    for (int c = 0; c < 4; ++c) sa[c].hi = sa[c].lo = sb[c].hi = sb[c].lo = 0.f;
    float qa[4] = {0.f, 0.f, 0.f, 0.f}, qb[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t np_part = 0;
    // images within r_c of particles less than r_c above the cathode (rare): plain loop over
    // all rows around the image point; image pairs act on the particle only. Taken before the
    // walk, for the lane's own pair; their potential goes straight to the energy (once)
    auto images = [&](const float4 pi, const float4 li, Acc2* sum) {
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
        for (int c = 0; c < 3; ++c) sum[c].add(rowv[c]);
        e_acc += static_cast<double>(rowv[3]);
      });
    };
    if (g.pp_bc) {
      if (alive_a) images(pa, la, sa);
      if (alive_b) images(pb, lb, sb);
    }
    // the held pair's sums (hi + lo of the compensated accumulators) to its force arrays, split
    // like the reactions, and zeroed; sum_i phi_i over ordered pairs takes each unordered
    // pair's potential twice
    auto flush = [&]() {
      for (int c = 0; c < 4; ++c) {
        sa[c].add(qa[c]);
        sb[c].add(qb[c]);
        qa[c] = qb[c] = 0.f;
      }
      if (alive_a) {
        split_add_v4(fpp + ia, flo + ia, fbig + ia, sa[0].hi, sa[1].hi, sa[2].hi, sa[0].lo,
                     sa[1].lo, sa[2].lo);
        e_acc += 2.0 * static_cast<double>(sa[3].value());
      }
      if (alive_b) {
        split_add_v4(fpp + ia + 1, flo + ia + 1, fbig + ia + 1, sb[0].hi, sb[1].hi, sb[2].hi,
                     sb[0].lo, sb[1].lo, sb[2].lo);
        e_acc += 2.0 * static_cast<double>(sb[3].value());
      }
      for (int c = 0; c < 4; ++c) sa[c].hi = sa[c].lo = sb[c].hi = sb[c].lo = 0.f;
    };
    // one candidate record j (hj, lj) against a and b
    auto cand = [&](bool v, uint32_t j, const float4& hj, const float4& lj) {
      const float ax = (pa.x - hj.x) + (la.x - lj.x);
      const float ay = (pa.y - hj.y) + (la.y - lj.y);
      const float az = (pa.z - hj.z) + (la.z - lj.z);
      const float bx = (pb.x - hj.x) + (lb.x - lj.x);
      const float by = (pb.y - hj.y) + (lb.y - lj.y);
      const float bz = (pb.z - hj.z) + (lb.z - lj.z);
      const float r2a = ax * ax + ay * ay + az * az;
      const float r2b = bx * bx + by * by + bz * bz;
      // coincident particles (r2 == 0) are skipped
      const bool ha = v && ta && r2a < 1.f && r2a > 0.f;
      const bool hb = v && tb && r2b < 1.f && r2b > 0.f;
      float fa, ua, fb, ub;
      pair_poly_hw<kDeg>(P, ha ? r2a : 0.5f, fa, ua);
      pair_poly_hw<kDeg>(P, hb ? r2b : 0.5f, fb, ub);
      fa = ha ? fa : 0.f;
      ua = ha ? ua : 0.f;
      fb = hb ? fb : 0.f;
      ub = hb ? ub : 0.f;
      const float fax = fa * ax, fay = fa * ay, faz = fa * az;
      const float fbx = fb * bx, fby = fb * by, fbz = fb * bz;
      qa[0] += fax;
      qa[1] += fay;
      qa[2] += faz;
      qa[3] += ua;
      qb[0] += fbx;
      qb[1] += fby;
      qb[2] += fbz;
      qb[3] += ub;
      np_part += static_cast<uint32_t>(ha) + static_cast<uint32_t>(hb);
      // the reaction on j, split into coarse and fine parts (j's potential is summed on the
      // owner side only); it is big only if fa + fb is, as separations are below 1
      split_add_v4_if(ha || hb, fa + fb >= kBigTerm, fpp + j, flo + j, fbig + j, -(fax + fbx),
                      -(fay + fby), -(faz + fbz));
    };
    int step = 0;
    while (__any_sync(0xffffffffu, ptr < end || pending_b)) {
      // a lane without a candidate reads record 0, as every such lane does, so that the load
      // costs the warp one extra sector at most; its results are masked out
      const bool va = ptr < end, vb = ptr + 1 < end;
      const uint32_t ja = va ? ptr : 0u, jb = vb ? ptr + 1 : 0u;
      float4 h0, l0, h1, l1;  // both loads in flight before either record is used
      load_rec32(rec + 2 * static_cast<size_t>(ja), h0, l0);
      load_rec32(rec + 2 * static_cast<size_t>(jb), h1, l1);
      cand(va, ja, h0, l0);
      cand(vb, jb, h1, l1);
      ptr += 2;
      {
        // the next run without a branch: slot k stays in bounds (k < cnt, or k = 0)
        const bool sw = ptr >= end && k + 1 < cnt;
        k += sw ? 1 : 0;
        const uint32_t nj0 = run_j0[k][tid], nj1 = run_j1[k][tid];
        ptr = sw ? nj0 : ptr;
        end = sw ? nj1 : end;
        if constexpr (!kPhased) {
          ta = same || k < split;
          tb = alive_b && (same || k >= split);
        }
      }
      if constexpr (kPhased) {
        // a's runs walked (rare: a and b in different rows): b's runs take their slots
        const bool go = pending_b && ptr >= end;
        if (__any_sync(0xffffffffu, go)) {
          if (go) {
            cnt = 0;
            b_runs<kRows>(g, starts, pb, lb, ia + 1, emit);
            k = 0;
            pending_b = false;
            ta = false;
            tb = true;
            ptr = cnt > 0 ? run_j0[0][tid] : 0u;
            end = cnt > 0 ? run_j1[0][tid] : 0u;
          }
        }
      }
      {
        const bool idle = ptr >= end && !pending_b;
        const unsigned im = __ballot_sync(0xffffffffu, idle);
        if (__popc(im) >= kStealMin) {
          const bool spare = k + 1 < cnt;  // an unstarted run (runs are never empty)
          const bool halve = !spare && ptr < end && end - ptr >= 2 * kStealRecs;
          const bool offer = spare || halve;
          const unsigned om = __ballot_sync(0xffffffffu, offer);
          if (om != 0u) {
            // the offered run [g0, g1) and whom it is tested against (bit 0: a, bit 1: b);
            // bit 2: b exists
            uint32_t g0 = 0, g1 = 0, gf = alive_b ? 4u : 0u;
            if (spare) {
              const int kk = cnt - 1;
              g0 = run_j0[kk][tid];
              g1 = run_j1[kk][tid];
              if constexpr (kPhased)  // all runs of the current phase are tested alike
                gf |= (ta ? 1u : 0u) | (tb ? 2u : 0u);
              else
                gf |= ((same || kk < split) ? 1u : 0u) |
                      ((alive_b && (same || kk >= split)) ? 2u : 0u);
            } else if (halve) {
              g0 = ptr + (((end - ptr) >> 1) & ~1u);  // the donor keeps an even count
              g1 = end;
              gf |= (ta ? 1u : 0u) | (tb ? 2u : 0u);
            }
            // the r-th idle lane takes from the r-th offering lane
            const unsigned lt = (1u << lane) - 1u;
            const int nt = __popc(im), no = __popc(om);
            const int orank = __popc(om & lt), trank = __popc(im & lt);
            if (offer) donor_s[tid >> 5][orank] = static_cast<uint8_t>(lane);
            __syncwarp();
            const bool take = idle && trank < no;
            const int src = take ? static_cast<int>(donor_s[tid >> 5][trank]) : lane;
            __syncwarp();
            if (offer && orank < nt) {
              if (spare)
                --cnt;
              else
                end = g0;
            }
            if (take) flush();  // the sums of the pair held so far
            // every lane takes part; a lane that takes nothing reads its own values
            pa = shfl_f4(pa, src);
            la = shfl_f4(la, src);
            pb = shfl_f4(pb, src);
            lb = shfl_f4(lb, src);
            ia = __shfl_sync(0xffffffffu, ia, src);
            g0 = __shfl_sync(0xffffffffu, g0, src);
            g1 = __shfl_sync(0xffffffffu, g1, src);
            gf = __shfl_sync(0xffffffffu, gf, src);
            if (take) {
              alive_a = true;
              alive_b = (gf & 4u) != 0u;
              ta = (gf & 1u) != 0u;
              tb = (gf & 2u) != 0u;
              // the run-switch formulas above then keep (ta, tb) for this single run (an idle
              // lane has no b runs pending)
              same = ta && tb;
              split = ta ? 1 : 0;
              k = 0;
              cnt = 0;
              ptr = g0;
              end = g1;
            }
          }
        }
      }
      // the own sums: plain FP32 over at most 32 terms (16 steps of two records), then folded
      // into the TwoSum accumulators; so the rounding of a particle's own sum is at most
      // 31 * 2^-24 times the largest 32-term partial sum, per fold, instead of growing with the
      // neighbour count
      if ((++step & 15) == 0) {
        for (int c = 0; c < 4; ++c) {
          sa[c].add(qa[c]);
          sb[c].add(qb[c]);
          qa[c] = qb[c] = 0.f;
        }
        np += np_part;
        np_part = 0;
      }
    }
    np += np_part;
    flush();
  }
  if (energy) block_reduce_add<kPpThreads>(e_acc, energy);
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
  const float R = erfcx_poly<kDeg, false>(P, rho);
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
// the zeroed result. Rows are walked in lockstep. FP64 arithmetic is scarce on this part, so the
// walk itself runs in FP32: the row search and a distance prefilter on the leading 24 bits of
// each coordinate (within the search slack of the exact test). Candidates that pass wait in a
// per-lane ring in shared memory and are evaluated, a batch of one per lane, whenever some lane's
// ring is full: the exact FP64 separation decides the pair (r^2 < 1 in FP64, as the definition
// reads), and the pair terms follow (in double-float, or FP64 for large kappa), with most lanes
// busy.
// ------------------------------------------------------------------------------------------
constexpr int kRingJ = 16;  // queued candidates per lane of the FP64 short range

// The FP64 path's pair function in double-float arithmetic (df_math.cuh): the fit table copied
// into shared memory by the block (only the intervals and degrees in use), s = rho^2 split into
// two floats with integer operations, the results widened exactly and summed in FP64.
struct DFTable {
  dfm::PairConsts k;
  dfm::Coef coef[dfm::kMaxIntervals];
};

__device__ __forceinline__ void load_df_table(const dfm::PairDF* __restrict__ src, DFTable& dst) {
  constexpr int kWords = sizeof(dfm::PairConsts) / sizeof(uint32_t);
  static_assert(sizeof(dfm::PairConsts) % sizeof(uint32_t) == 0, "copied in words");
  const uint32_t* s = reinterpret_cast<const uint32_t*>(&src->k);
  uint32_t* d = reinterpret_cast<uint32_t*>(&dst.k);
  for (int t = threadIdx.x; t < kWords; t += blockDim.x) d[t] = s[t];
  const int nint = src->k.nint, deg1 = src->k.deg + 1;
  for (int t = threadIdx.x; t < nint * deg1; t += blockDim.x)
    dst.coef[t / deg1][t % deg1] = src->coef[t / deg1][t % deg1];
  __syncthreads();
}

__device__ __forceinline__ double df_to_double(dfm::F2 v) {
  return float_to_double_exact(v.hi) + float_to_double_exact(v.lo);
}

__device__ __forceinline__ void pair_terms_df(const DFTable& T, double r2, double& fco,
                                              double& pot) {
  const DF sd = df_from_double(r2);
  const dfm::PairOut o = dfm::pair_df(T.k, T.coef, dfm::F2{sd.hi, sd.lo});
  fco = df_to_double(o.fco);
  pot = df_to_double(o.pot);
}

// the force coefficient alone (no potential: the energy is not asked for)
__device__ __forceinline__ double pair_fco_df(const DFTable& T, double r2) {
  const DF sd = df_from_double(r2);
  return df_to_double(dfm::pair_df(T.k, T.coef, dfm::F2{sd.hi, sd.lo}).fco);
}

__device__ __forceinline__ void pair_hess_dfd(const DFTable& T, double r2, double& fco,
                                              double& dfr) {
  const DF sd = df_from_double(r2);
  dfm::F2 f, d;
  dfm::pair_hess_df(T.k, T.coef, dfm::F2{sd.hi, sd.lo}, f, d);
  fco = df_to_double(f);
  dfr = df_to_double(d);
}

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
template <int kRows, bool kDet, bool kDF, bool kPot>
__global__ void __launch_bounds__(kThreads)
    k_pp_f64(Geom g, const uint32_t* __restrict__ total, const Rec64* __restrict__ rec,
             const Rec64* __restrict__ recm, const uint32_t* __restrict__ starts,
             D4* __restrict__ fpp, double* __restrict__ energy,
             unsigned long long* __restrict__ pairs, const dfm::PairDF* __restrict__ dftab) {
  __shared__ typename std::conditional<kDF, DFTable, char>::type dft_s[1];
  if constexpr (kDF) load_df_table(dftab, dft_s[0]);
  __shared__ uint32_t ringj_s[kThreads / 32][kRingJ][32];
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
  // FP32 copies (the leading 24 bits) for the search and the distance prefilter; the search
  // slack exceeds their truncation error (2^-23 of the coordinate, twice, on each axis)
  const float pxf = df_from_double(px).hi, pyf = df_from_double(py).hi,
              pzf = df_from_double(pz).hi;
  const float thr = (1.f + g.slack_f) * (1.f + g.slack_f);
  // the row the sort put the particle in (two particles closer than r_c sit in sort rows at most
  // kRows apart, whatever the rounding of either binning)
  const uint32_t row = static_cast<uint32_t>(static_cast<unsigned long long>(recm[ie].idx) >> 32);
  const int cy = static_cast<int>(row % static_cast<uint32_t>(g.nc[1]));
  const int cz = static_cast<int>(row / static_cast<uint32_t>(g.nc[1]));
  double sum[4] = {0.0, 0.0, 0.0, 0.0};
  unsigned int np = 0, ncand = 0;  // pairs found, records tested
  int head = 0, cnt = 0;
  // one queued candidate per lane: the exact FP64 separation decides, then the pair terms
  auto evaluate = [&]() {
    const bool has = cnt > 0;
    const uint32_t j = has ? ringj[head & (kRingJ - 1)][lane] : ie;
    const Rec64 rj = rec[j];
    const double rx = px - rj.u[0], ry = py - rj.u[1], rz = pz - rj.u[2];
    const double r2 = rx * rx + ry * ry + rz * rz;
    const bool hit = has && r2 < 1.0 && r2 > 0.0;
    double fco, pot = 0.0;
    if constexpr (kDF) {
      if constexpr (kPot)
        pair_terms_df(dft_s[0], hit ? r2 : 0.5, fco, pot);
      else
        fco = pair_fco_df(dft_s[0], hit ? r2 : 0.5);
    } else {
      pair_terms(hit ? r2 : 0.5, kappa, c2k, fco, pot);
    }
    if (hit) {
      // the reaction's components, -fco (xi_i - xi_j): the own sum subtracts them
      const double nf = -fco;
      const double gx = nf * rx, gy = nf * ry, gz = nf * rz;
      sum[0] -= gx;
      sum[1] -= gy;
      sum[2] -= gz;
      if constexpr (kPot) sum[3] += pot;
      ++np;
      if (!kDet) {
        double* fj = &fpp[j].x;
        // the potential is summed on the owner's side only: j's fourth component stays unused
        atomicAdd(fj, gx);
        atomicAdd(fj + 1, gy);
        atomicAdd(fj + 2, gz);
      }
    }
    head += has;
    cnt -= has;
  };
  for (int r = 0; r < Rows<kRows>::last; ++r) {
    uint32_t j0 = 0, j1 = 0;
    if (alive) {
      row_range<kRows>(g, starts, pxf, pyf, pzf, cy, cz, r, j0, j1);
      if (!kDet) j0 = max(j0, i + 1);
      j1 = max(j1, j0);
    }
    const int len = static_cast<int>(j1 - j0);
    ncand += static_cast<unsigned>(len);
    int maxlen = len;
    for (int o = 16; o > 0; o >>= 1) maxlen = max(maxlen, __shfl_xor_sync(0xffffffffu, maxlen, o));
    for (int t = 0; t < maxlen; ++t) {
      const bool v = t < len;
      const uint32_t j = v ? j0 + t : ie;
      const Rec64 rj = rec[j];
      const float dx = pxf - df_from_double(rj.u[0]).hi;
      const float dy = pyf - df_from_double(rj.u[1]).hi;
      const float dz = pzf - df_from_double(rj.u[2]).hi;
      if (alive && v && j != i && fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < thr) {
        ringj[(head + cnt) & (kRingJ - 1)][lane] = j;
        ++cnt;
      }
      if (__any_sync(0xffffffffu, cnt == kRingJ)) evaluate();
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
          if constexpr (kDF)
            pair_terms_df(dft_s[0], r2, fco, pot);
          else
            pair_terms(r2, kappa, c2k, fco, pot);
          sum[0] -= fco * ax;
          sum[1] -= fco * ay;
          sum[2] -= fco * az;
          if constexpr (kPot) sum[3] -= pot;
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
template <bool kDF>
__global__ void __launch_bounds__(kThreads)
    k_pp_vjp(Geom g, const uint32_t* __restrict__ total, PosD pos,
             const uint32_t* __restrict__ starts, const double* __restrict__ w,
             double* __restrict__ acc, double scale, const dfm::PairDF* __restrict__ dftab) {
  __shared__ typename std::conditional<kDF, DFTable, char>::type dft_s[1];
  if constexpr (kDF) load_df_table(dftab, dft_s[0]);
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *total) return;
  auto hess = [&](double r2, double& fco, double& dfr) {
    if constexpr (kDF)
      pair_hess_dfd(dft_s[0], r2, fco, dfr);
    else
      pair_hess(r2, g.kappa_eff, 2.0 * g.kappa_eff * 0.56418958354775628695, fco, dfr);
  };
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
        hess(r2, fco, dfr);
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
          hess(r2, fco, dfr);
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

void launch_pp(const p3m_ctx* c, int64_t n, cudaStream_t s, bool want_energy) {
  if (n == 0) return;
  const unsigned blocks = static_cast<unsigned>((n + kThreads - 1) / kThreads);
  const uint32_t* total = c->starts + c->nkeys;
  if (c->fp32) {
    // the kernel adds each pair's force to both particles: the result (coarse, fine and big
    // parts) starts at zero
    float4* fbig = c->fplo + c->n_max;
    cudaMemsetAsync(c->fpp, 0, sizeof(float4) * static_cast<size_t>(n), s);
    cudaMemsetAsync(c->fplo, 0, sizeof(float2) * static_cast<size_t>(n), s);
    cudaMemsetAsync(fbig, 0, sizeof(float4) * static_cast<size_t>(n), s);
    cudaMemsetAsync(c->pp_tile, 0, sizeof(uint32_t), s);
    // persistent grid of a few blocks per SM: the SM resources it leaves free let the mesh
    // chain, on the other stream, run at the same time
    const int64_t tiles = (n + 2 * kPpThreads - 1) / (2 * kPpThreads);  // two particles a thread
    const unsigned wblocks = static_cast<unsigned>(
        std::min<int64_t>(tiles, static_cast<int64_t>(kPpBlocksPerSm) * c->num_sms));
    // the kernel for the context's row geometry (Geom::rows cell rows per cutoff)
    auto run = [&](auto k_rows1, auto k_rows2, auto k_rows3) {
      auto kern = c->g.rows == 1 ? k_rows1 : (c->g.rows == 2 ? k_rows2 : k_rows3);
      const size_t smem = pp_run_bytes(c->g.rows);
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
      kern<<<wblocks, kPpThreads, smem, s>>>(
          c->g, c->poly, total, static_cast<const float4*>(c->recp), c->starts,
          static_cast<float4*>(c->fpp), reinterpret_cast<float2*>(c->fplo), fbig, c->pp_tile,
          c->energy_acc, c->pair_acc);
    };
    switch (c->poly.deg) {
      case 4: run(k_pp_f32<4, 1>, k_pp_f32<4, 2>, k_pp_f32<4, 3>); break;
      case 5: run(k_pp_f32<5, 1>, k_pp_f32<5, 2>, k_pp_f32<5, 3>); break;
      case 6: run(k_pp_f32<6, 1>, k_pp_f32<6, 2>, k_pp_f32<6, 3>); break;
      case 7: run(k_pp_f32<7, 1>, k_pp_f32<7, 2>, k_pp_f32<7, 3>); break;
      case 8: run(k_pp_f32<8, 1>, k_pp_f32<8, 2>, k_pp_f32<8, 3>); break;
      case 9: run(k_pp_f32<9, 1>, k_pp_f32<9, 2>, k_pp_f32<9, 3>); break;
      case 10: run(k_pp_f32<10, 1>, k_pp_f32<10, 2>, k_pp_f32<10, 3>); break;
      case 11: run(k_pp_f32<11, 1>, k_pp_f32<11, 2>, k_pp_f32<11, 3>); break;
      case 12: run(k_pp_f32<12, 1>, k_pp_f32<12, 2>, k_pp_f32<12, 3>); break;
      case 13: run(k_pp_f32<13, 1>, k_pp_f32<13, 2>, k_pp_f32<13, 3>); break;
      case 14: run(k_pp_f32<14, 1>, k_pp_f32<14, 2>, k_pp_f32<14, 3>); break;
      default: run(k_pp_f32<15, 1>, k_pp_f32<15, 2>, k_pp_f32<15, 3>); break;
    }
  } else {
    auto pick = [&](auto k1, auto k2, auto k3) {
      return c->g.rows == 1 ? k1 : (c->g.rows == 2 ? k2 : k3);
    };
    // the pair potentials are summed for the energy or the deterministic mode's fixed-order sum
    const bool pot = c->det || want_energy;
    auto kern = c->pdf
                    ? (c->det ? pick(k_pp_f64<1, true, true, true>, k_pp_f64<2, true, true, true>,
                                     k_pp_f64<3, true, true, true>)
                              : (pot ? pick(k_pp_f64<1, false, true, true>,
                                            k_pp_f64<2, false, true, true>,
                                            k_pp_f64<3, false, true, true>)
                                     : pick(k_pp_f64<1, false, true, false>,
                                            k_pp_f64<2, false, true, false>,
                                            k_pp_f64<3, false, true, false>)))
                    : (c->det ? pick(k_pp_f64<1, true, false, true>, k_pp_f64<2, true, false, true>,
                                     k_pp_f64<3, true, false, true>)
                              : (pot ? pick(k_pp_f64<1, false, false, true>,
                                            k_pp_f64<2, false, false, true>,
                                            k_pp_f64<3, false, false, true>)
                                     : pick(k_pp_f64<1, false, false, false>,
                                            k_pp_f64<2, false, false, false>,
                                            k_pp_f64<3, false, false, false>)));
    if (!c->det) cudaMemsetAsync(c->fpp, 0, sizeof(D4) * static_cast<size_t>(n), s);
    kern<<<blocks, kThreads, 0, s>>>(c->g, total, static_cast<const Rec64*>(c->recp),
                                     static_cast<const Rec64*>(c->recm), c->starts,
                                     static_cast<D4*>(c->fpp), pot ? c->energy_acc : nullptr,
                                     c->pair_acc, c->pdf);
    if (c->det) launch_det_sum_pp(c, n, s);
  }
}

void launch_pp_count(const p3m_ctx* c, int64_t n, unsigned long long* out, cudaStream_t s) {
  if (!c->fp32) return;  // FP64: the short range counts as it walks
  cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (n == 0) return;
  const int64_t lane_pairs = (n + 1) / 2;
  auto kern = c->g.rows == 1   ? k_pp_count_f32<1>
              : c->g.rows == 2 ? k_pp_count_f32<2>
                               : k_pp_count_f32<3>;
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
    auto run = [&](auto k_rows1, auto k_rows2, auto k_rows3) {
      auto kern = c->g.rows == 1 ? k_rows1 : (c->g.rows == 2 ? k_rows2 : k_rows3);
      kern<<<wblocks, kThreads, 0, s>>>(c->g, c->poly, total,
                                        static_cast<const float4*>(c->recp), c->starts, ws,
                                        static_cast<float4*>(c->fpp), c->pp_tile);
    };
    switch (c->poly.deg) {
      case 4: run(k_pp_vjp_f32<4, 1>, k_pp_vjp_f32<4, 2>, k_pp_vjp_f32<4, 3>); break;
      case 5: run(k_pp_vjp_f32<5, 1>, k_pp_vjp_f32<5, 2>, k_pp_vjp_f32<5, 3>); break;
      case 6: run(k_pp_vjp_f32<6, 1>, k_pp_vjp_f32<6, 2>, k_pp_vjp_f32<6, 3>); break;
      case 7: run(k_pp_vjp_f32<7, 1>, k_pp_vjp_f32<7, 2>, k_pp_vjp_f32<7, 3>); break;
      case 8: run(k_pp_vjp_f32<8, 1>, k_pp_vjp_f32<8, 2>, k_pp_vjp_f32<8, 3>); break;
      case 9: run(k_pp_vjp_f32<9, 1>, k_pp_vjp_f32<9, 2>, k_pp_vjp_f32<9, 3>); break;
      case 10: run(k_pp_vjp_f32<10, 1>, k_pp_vjp_f32<10, 2>, k_pp_vjp_f32<10, 3>); break;
      case 11: run(k_pp_vjp_f32<11, 1>, k_pp_vjp_f32<11, 2>, k_pp_vjp_f32<11, 3>); break;
      case 12: run(k_pp_vjp_f32<12, 1>, k_pp_vjp_f32<12, 2>, k_pp_vjp_f32<12, 3>); break;
      case 13: run(k_pp_vjp_f32<13, 1>, k_pp_vjp_f32<13, 2>, k_pp_vjp_f32<13, 3>); break;
      case 14: run(k_pp_vjp_f32<14, 1>, k_pp_vjp_f32<14, 2>, k_pp_vjp_f32<14, 3>); break;
      default: run(k_pp_vjp_f32<15, 1>, k_pp_vjp_f32<15, 2>, k_pp_vjp_f32<15, 3>); break;
    }
  } else {
    // d/dxi of (k_e q^2 / r_c^2) f(rho): one more factor 1/r_c
    const double scale = c->g.ke * c->g.q * c->g.q / (c->g.rc * c->g.rc * c->g.rc);
    auto kern = c->pdf ? k_pp_vjp<true> : k_pp_vjp<false>;
    kern<<<blocks, kThreads, 0, s>>>(c->g, total, PosD{static_cast<const Rec64*>(c->recp)},
                                     c->starts, w, c->acc, scale, c->pdf);
  }
}

}  // namespace p3m
