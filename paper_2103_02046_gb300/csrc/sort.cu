// Binning of particles into cutoff cells and a counting sort by cell.
//
// The short-range sum of eq. (summation_short) needs, for each particle, the particles
// "close to" it (within r_c, Sec. 3.1.1, fig. ShortError). Cells at least r_c / R wide in y and
// z (R = 2, or 1 at low density) turn that search into (2R + 1)^2 rows of cells along x. The
// sort is a counting sort in three passes: histogram with in-cell ranks (atomics), exclusive
// scan of the cell counts, scatter.
// No pass waits on another block, so no inter-block spin is needed.
#include "p3m_internal.cuh"

namespace p3m {
namespace {

constexpr int kBinThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;  // per thread
constexpr int kScanTile = kScanThreads * kScanItems;

// Mesh coordinate s = (x - lo) / h. The product with the reciprocal is used (FP64 division is
// slow on this part) unless it lies within 1e-9 of a point where the assignment changes its
// node (integers for CIC, half-integers for TSC); there the IEEE quotient is taken, so the node
// decision is exactly the one the definition makes.
// Not inlined: the callers reach it only within 1e-3 of a knot, and as a call it stays a real
// branch instead of being predicated into every thread's instruction stream (FP64 is slow here).
static __device__ __noinline__ double mesh_coord(const Geom& g, double v, int d) {
  const double dv = v - g.lo[d];
  const double s = dv * g.inv_h[d];
  const double knot = (g.order == 2) ? floor(s + 0.5) - 0.5 : floor(s);
  const double dist = fmin(fabs(s - knot), fabs(s - knot - 1.0));
  return (dist < 1e-9 * fmax(1.0, fabs(s))) ? dv / g.h[d] : s;
}

// Validity of one particle and its cell. Valid: the assignment support lies inside the mesh
// (TSC: floor(s + 1/2) in [1, n - 2], i.e. s in [1/2, n - 3/2); CIC: floor(s) in [0, n - 2],
// i.e. s in [0, n - 1)) and, with the cathode in the long-range solve, z > z_cathode. The test
// runs in FP32 (the FP64 rate of this part is low) and falls back to the exact FP64 coordinate
// within 1e-3 of a boundary, so the decision is always the definition's. The cell index only
// has to be consistent with the stored positions to within the search slack, so FP32 suffices.
// Returns 0 if valid, else an error bit.
__device__ __forceinline__ int particle_cell(const Geom& g, const double* __restrict__ xi,
                                             int cell[3]) {
  int err = 0;
  for (int d = 0; d < 3; ++d) {
    // x - lo_d in double-float, rounded to FP32 (no FP64 arithmetic)
    const float f = df_sub(df_from_double(xi[d]), DF{g.lo_df[d][0], g.lo_df[d][1]}).hi;
    if (!(f == f)) return kErrNaN;
    const float s = f * g.inv_h_f[d];
    // in the grounded box, and for central differences of phi, the support must also stay off
    // the edge nodes: one node less per side
    const int box = (g.pm_bc == 2 || g.force_diff) ? 1 : 0;
    const float b0 = ((g.order == 2) ? 0.5f : 0.0f) + box;
    const float b1 = static_cast<float>(g.n[d] - box) - ((g.order == 2) ? 1.5f : 1.0f);
    bool ok;
    if (fabsf(s - b0) < 1e-3f || fabsf(s - b1) < 1e-3f) {
      const double se = mesh_coord(g, xi[d], d);
      const double c = (g.order == 2) ? floor(se + 0.5) : floor(se);
      ok = c >= ((g.order == 2) ? 1.0 : 0.0) + box && c <= static_cast<double>(g.n[d] - 2 - box);
    } else {
      ok = s >= b0 && s < b1;
    }
    if (!ok) err = kErrRange;
    cell[d] = min(max(static_cast<int>(floorf(f * g.inv_cell_f[d])), 0), g.nc[d] - 1);
  }
  if (g.pm_bc == 1 && !(xi[2] > g.zc)) err = kErrRange;
  return err;
}

__global__ void k_bin(Geom g, const double* __restrict__ x, int64_t n,
                      uint32_t* __restrict__ counts, uint32_t* __restrict__ keys,
                      uint32_t* __restrict__ ranks, int* __restrict__ err,
                      double* __restrict__ f_zero) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  int cell[3];
  const int e = particle_cell(g, x + 3 * i, cell);
  if (e) {
    keys[i] = kInvalidKey;
    atomicOr(err, e);
    if (f_zero) {
      f_zero[3 * i] = 0.0;
      f_zero[3 * i + 1] = 0.0;
      f_zero[3 * i + 2] = 0.0;
    }
    return;
  }
  const uint32_t key = cell_key(g, cell[0], cell[1], cell[2]);
  keys[i] = key;
  ranks[i] = atomicAdd(counts + key, 1u);
}

// Exclusive scan, level 1: each block scans kScanTile counts and records its total.
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t* __restrict__ in,
                                                             uint32_t* __restrict__ out,
                                                             uint32_t* __restrict__ bsum,
                                                             uint64_t n) {
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  const uint64_t base = blockIdx.x * static_cast<uint64_t>(kScanTile) +
                        threadIdx.x * static_cast<uint64_t>(kScanItems);
  uint32_t v[kScanItems];
  uint32_t run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    const uint32_t t = v[k];
    v[k] = run;
    run += t;
  }
  // block-wide exclusive scan of the per-thread totals
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = (lane < kScanThreads / 32) ? warp_tot[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;  // exclusive
    if (lane == 31) bsum[blockIdx.x] = wi;
  }
  __syncthreads();
  const uint32_t pre = warp_tot[wid] + incl - run;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) out[base + k] = v[k] + pre;
}

// Level 2: one block scans the tile totals in chunks with a running carry; writes the grand
// total to out_total.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint32_t* __restrict__ bsum,
                                                            uint64_t nb,
                                                            uint32_t* __restrict__ out_total) {
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  __shared__ uint32_t carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (uint64_t c0 = 0; c0 < nb; c0 += kScanThreads) {
    const uint64_t i = c0 + threadIdx.x;
    const uint32_t v = (i < nb) ? bsum[i] : 0u;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const uint32_t w = warp_tot[lane];
      uint32_t wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      warp_tot[lane] = wi - w;
    }
    __syncthreads();
    const uint32_t carry = carry_s;
    if (i < nb) bsum[i] = carry + warp_tot[wid] + incl - v;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry_s = carry + warp_tot[wid] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *out_total = carry_s;
}

__global__ void k_scan_add(uint32_t* __restrict__ out, const uint32_t* __restrict__ bsum,
                           uint64_t n) {
  const uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (i < n) out[i] += bsum[i / kScanTile];
}

template <bool kFP32>
__global__ void k_scatter(Geom g, const double* __restrict__ x, int64_t n,
                          uint32_t* __restrict__ keys, const uint32_t* __restrict__ ranks,
                          const uint32_t* __restrict__ starts, void* __restrict__ recp,
                          void* __restrict__ recm) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const uint32_t key = keys[i];
  if (key == kInvalidKey) return;
  const uint32_t pos = starts[key] + ranks[i];
  keys[i] = pos;  // from here on keys[i] is the sorted position of input particle i
  if (kFP32) {
    // FP32 record (one 32-byte sector): the position in cutoff units as hi + lo from
    // double-float arithmetic (about 2^-46 relative), the input index, the row, and per axis
    // the node correction. The mesh kernels recompute the assignment node from hi + lo
    // (s = (hi + lo) r_c / h, node floor(s + 1/2) for TSC, floor(s) for CIC); within 1e-3 of a
    // point where the node changes, the exact FP64 coordinate decides, as in the definition, and
    // the difference to the recomputed node is stored.
    float hi[3], lo[3];
    uint32_t code = 0;
    for (int d = 0; d < 3; ++d) {
      const double v = x[3 * i + d];
      const DF dv = df_sub(df_from_double(v), DF{g.lo_df[d][0], g.lo_df[d][1]});
      const DF xr = df_mul(dv, g.inv_rc_df);
      hi[d] = xr.hi;
      lo[d] = xr.lo;
      const DF sm = df_mul(xr, g.rch_df[d]);
      const float cf = (g.order == 2) ? floorf(sm.hi + 0.5f) : floorf(sm.hi);
      const float kl = (g.order == 2) ? cf - 0.5f : cf;
      int corr = 0;
      if (fabsf(sm.hi - kl) < 1e-3f || fabsf(sm.hi - kl - 1.f) < 1e-3f) {
        const double se = mesh_coord(g, v, d);
        const double cn = (g.order == 2) ? floor(se + 0.5) : floor(se);
        corr = max(-1, min(1, static_cast<int>(cn - static_cast<double>(cf))));
      }
      code |= static_cast<uint32_t>(corr + 1) << (2 * d);
    }
    const uint32_t row = key / static_cast<uint32_t>(g.nc[0]);
    float4* r = reinterpret_cast<float4*>(recp) + 2 * static_cast<size_t>(pos);
    r[0] = make_float4(hi[0], hi[1], hi[2], __int_as_float(static_cast<int>(i)));
    r[1] = make_float4(lo[0], lo[1], lo[2], __uint_as_float(row | (code << kRowBits)));
    return;
  }
  double xr[3], u[3];
  int c[3];
  for (int d = 0; d < 3; ++d) {
    const double v = x[3 * i + d];
    const double dv = v - g.lo[d];
    xr[d] = dv * g.inv_rc;
    // node from an FP32 estimate unless it is within 1e-3 of a knot; then from the exact s
    const float sf = static_cast<float>(dv) * g.inv_h_f[d];
    const float cf = (g.order == 2) ? floorf(sf + 0.5f) : floorf(sf);
    const float kl = (g.order == 2) ? cf - 0.5f : cf;
    double cn;
    if (fabsf(sf - kl) < 1e-3f || fabsf(sf - kl - 1.f) < 1e-3f) {
      const double s = mesh_coord(g, v, d);
      cn = (g.order == 2) ? floor(s + 0.5) : floor(s);
      u[d] = s - cn;
    } else {
      cn = static_cast<double>(cf);
      u[d] = fma(-cn, g.h[d], dv) * g.inv_h[d];
    }
    c[d] = static_cast<int>(cn);
  }
  const uint32_t node = pack_node(c[0], c[1], c[2]);
  {
    Rec64 r;
    r.u[0] = xr[0];
    r.u[1] = xr[1];
    r.u[2] = xr[2];
    r.idx = static_cast<long long>(i);
    reinterpret_cast<Rec64*>(recp)[pos] = r;
    Rec64 m;
    m.u[0] = u[0];
    m.u[1] = u[1];
    m.u[2] = u[2];
    // the node in the low 32 bits; above it the particle's cell row, which the FP64 short range
    // centres its row block on (the row the sort used, so that the search slack argument holds)
    m.idx = static_cast<long long>(node) |
            (static_cast<long long>(key / static_cast<uint32_t>(g.nc[0])) << 32);
    reinterpret_cast<Rec64*>(recm)[pos] = m;
  }
}

// Deterministic order within each cell (FP64 path, deterministic = 1): the counting sort's ranks
// come from atomics, so two particles of one cell can land in either order. One thread per cell
// re-orders its records by input index (insertion sort; cells hold a few particles) and updates
// the sorted position kept in keys. Every later sum then runs in an order fixed by the input.
__global__ void k_cell_order(uint64_t nkeys, const uint32_t* __restrict__ starts,
                             Rec64* __restrict__ recp, Rec64* __restrict__ recm,
                             uint32_t* __restrict__ keys) {
  const uint64_t c = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (c >= nkeys) return;
  const uint32_t j0 = starts[c], j1 = starts[c + 1];
  if (j1 - j0 < 2) return;
  for (uint32_t j = j0 + 1; j < j1; ++j) {
    const Rec64 p = recp[j], m = recm[j];
    uint32_t k = j;
    while (k > j0 && recp[k - 1].idx > p.idx) {
      recp[k] = recp[k - 1];
      recm[k] = recm[k - 1];
      --k;
    }
    recp[k] = p;
    recm[k] = m;
  }
  for (uint32_t j = j0; j < j1; ++j) keys[recp[j].idx] = j;
}

inline unsigned grid_for(int64_t n, int threads) {
  return static_cast<unsigned>((n + threads - 1) / threads);
}

}  // namespace

void launch_bin(const p3m_ctx* c, const double* x, int64_t n, double* f_zero) {
  cudaMemsetAsync(c->counts, 0, sizeof(uint32_t) * c->nkeys, c->work);
  if (n == 0) return;
  k_bin<<<grid_for(n, kBinThreads), kBinThreads, 0, c->work>>>(c->g, x, n, c->counts, c->keys,
                                                                  c->ranks, c->err_dev, f_zero);
}

void launch_scan(const p3m_ctx* c) {
  const uint64_t n = c->nkeys;
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  k_scan_tiles<<<static_cast<unsigned>(tiles), kScanThreads, 0, c->work>>>(c->counts, c->starts,
                                                                             c->bsum, n);
  k_scan_sums<<<1, kScanThreads, 0, c->work>>>(c->bsum, tiles, c->starts + n);
  k_scan_add<<<static_cast<unsigned>((n + 255) / 256), 256, 0, c->work>>>(c->starts, c->bsum,
                                                                            n);
}

void launch_scatter(const p3m_ctx* c, const double* x, int64_t n) {
  if (n == 0) return;
  if (c->fp32)
    k_scatter<true><<<grid_for(n, kBinThreads), kBinThreads, 0, c->work>>>(
        c->g, x, n, c->keys, c->ranks, c->starts, c->recp, c->recm);
  else {
    k_scatter<false><<<grid_for(n, kBinThreads), kBinThreads, 0, c->work>>>(
        c->g, x, n, c->keys, c->ranks, c->starts, c->recp, c->recm);
    if (c->det)
      k_cell_order<<<static_cast<unsigned>((c->nkeys + kBinThreads - 1) / kBinThreads),
                     kBinThreads, 0, c->work>>>(c->nkeys, c->starts, static_cast<Rec64*>(c->recp),
                                                static_cast<Rec64*>(c->recm), c->keys);
  }
}

}  // namespace p3m
