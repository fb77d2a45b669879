// Allocation-free emittance: the same quantity as p3m_emittance, for callers that cannot
// allocate device memory (see include/p3m.h). All scratch lives in one file-scope device array
// of fixed size; nothing here calls cudaMalloc, cudaFree or any allocating library routine.
//
// The reduction is a fixed-order two-level tree (per-block partial sums written to the static
// array, then one block combining them), so every slot that a later step reads has been
// written earlier in the same call: nothing has to be cleared between calls. Calls that run at
// the same time on the GPU (different streams, no ordering) share the array and race.
#include <cuda.h>

#include <mutex>

#include "p3m_internal.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaItems = 16;                                  // particles per thread
constexpr int kNaPerBlock = kNaThreads * kNaItems;            // 4096 particles per block
constexpr int kNaMaxBlocks = 4096;                            // => at most 16,777,216 particles
constexpr int kNaSums = 16;                                   // 6 first + 9 second moments, 1 pad
constexpr int kNaMaxDevices = 64;
static_assert(static_cast<long long>(kNaPerBlock) * kNaMaxBlocks == P3M_NOALLOC_MAX_N,
              "limit in the header must match the scratch size");

// [block][16] partial sums, then 16 totals; 4096 * 16 * 8 B + 128 B = 512.1 KiB per device.
static __device__ __align__(256) double g_na_scratch[kNaMaxBlocks * kNaSums + kNaSums];

// Scratch addresses already looked up, keyed by the CUDA context they belong to. A context ID
// is never reused within a process, so an address cached for a context that was destroyed
// (cudaDeviceReset, or a driver-API context that was popped and freed) is never handed out again.
struct NaSlot {
  unsigned long long ctx_id;
  double* ptr;
};
constexpr int kNaMaxContexts = 64;
std::mutex g_na_mutex;
NaSlot g_na_slots[kNaMaxContexts] = {};
int g_na_used = 0;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sums K per-thread values over the block in a fixed order; thread 0 gets the totals.
template <int K>
__device__ void block_tree(double (&v)[K], double (&ws)[K][kNaThreads / 32]) {
  for (int k = 0; k < K; ++k) {
    const double s = warp_sum(v[k]);
    if ((threadIdx.x & 31) == 0) ws[k][threadIdx.x >> 5] = s;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int k = 0; k < K; ++k) {
      double s = threadIdx.x < kNaThreads / 32 ? ws[k][threadIdx.x] : 0.0;
      v[k] = warp_sum(s);
    }
  }
}

// pass 1: per-block sums of x and p (6 values)
__global__ void __launch_bounds__(kNaThreads)
    k_na_first(const double* __restrict__ x, const double* __restrict__ p, int64_t n,
               double* __restrict__ scratch) {
  __shared__ double ws[6][kNaThreads / 32];
  double v[6] = {0, 0, 0, 0, 0, 0};
  const int64_t b0 = static_cast<int64_t>(blockIdx.x) * kNaPerBlock;
  for (int k = 0; k < kNaItems; ++k) {
    const int64_t i = b0 + k * kNaThreads + threadIdx.x;
    if (i < n)
      for (int d = 0; d < 3; ++d) {
        v[d] += x[3 * i + d];
        v[3 + d] += p[3 * i + d];
      }
  }
  block_tree<6>(v, ws);
  if (threadIdx.x == 0)
    for (int k = 0; k < 6; ++k) scratch[blockIdx.x * kNaSums + k] = v[k];
}

// pass 2/4: one block combines the per-block partials [lo, hi) of every block into the totals
__global__ void __launch_bounds__(kNaThreads)
    k_na_combine(double* __restrict__ scratch, int nblocks, int lo, int hi) {
  __shared__ double ws[kNaSums][kNaThreads / 32];
  double v[kNaSums];
  for (int k = 0; k < kNaSums; ++k) v[k] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kNaThreads)
    for (int k = lo; k < hi; ++k) v[k] += scratch[b * kNaSums + k];
  block_tree<kNaSums>(v, ws);
  if (threadIdx.x == 0)
    for (int k = lo; k < hi; ++k) scratch[kNaMaxBlocks * kNaSums + k] = v[k];
}

// pass 3: per-block centred second moments <du^2>, <dp^2>, <du dp> (9 values)
__global__ void __launch_bounds__(kNaThreads)
    k_na_second(const double* __restrict__ x, const double* __restrict__ p, int64_t n,
                double* __restrict__ scratch) {
  __shared__ double ws[9][kNaThreads / 32];
  const double* tot = scratch + kNaMaxBlocks * kNaSums;
  const double inv = 1.0 / static_cast<double>(n);
  const double mx[3] = {tot[0] * inv, tot[1] * inv, tot[2] * inv};
  const double mp[3] = {tot[3] * inv, tot[4] * inv, tot[5] * inv};
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int64_t b0 = static_cast<int64_t>(blockIdx.x) * kNaPerBlock;
  for (int k = 0; k < kNaItems; ++k) {
    const int64_t i = b0 + k * kNaThreads + threadIdx.x;
    if (i < n)
      for (int d = 0; d < 3; ++d) {
        const double du = x[3 * i + d] - mx[d], dp = p[3 * i + d] - mp[d];
        v[3 * d] += du * du;
        v[3 * d + 1] += dp * dp;
        v[3 * d + 2] += du * dp;
      }
  }
  block_tree<9>(v, ws);
  if (threadIdx.x == 0)
    for (int k = 0; k < 9; ++k) scratch[blockIdx.x * kNaSums + 6 + k] = v[k];
}

// pass 5: eps_u = sqrt(<du^2><dp^2> - <du dp>^2) / (M c) and, if asked, the gradient of
// sum_u eps_u with respect to x and p
__global__ void k_na_finish(const double* __restrict__ x, const double* __restrict__ p,
                            int64_t n, const double* __restrict__ scratch, double mc,
                            double* __restrict__ eps3, double* __restrict__ gx,
                            double* __restrict__ gp) {
  const double* tot = scratch + kNaMaxBlocks * kNaSums;
  const double inv = 1.0 / static_cast<double>(n);
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t < 3 && eps3) {
    const double a = tot[6 + 3 * t] * inv, b = tot[7 + 3 * t] * inv, c = tot[8 + 3 * t] * inv;
    eps3[t] = sqrt(fmax(a * b - c * c, 0.0)) / mc;
  }
  if (!gx && !gp) return;
  if (t >= 3 * n) return;
  const int d = static_cast<int>(t % 3);
  const double a = tot[6 + 3 * d] * inv, b = tot[7 + 3 * d] * inv, c = tot[8 + 3 * d] * inv;
  const double eps = sqrt(fmax(a * b - c * c, 0.0)) / mc;
  const double den = static_cast<double>(n) * mc * mc * eps;
  const double du = x[t] - tot[d] * inv, dp = p[t] - tot[3 + d] * inv;
  if (gx) gx[t] = den > 0.0 ? (du * b - dp * c) / den : 0.0;
  if (gp) gp[t] = den > 0.0 ? (dp * a - du * c) / den : 0.0;
}

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// ID of the CUDA context current on this thread (0 if none is current yet). The two driver
// functions are fetched through the runtime, so the library needs no link to the driver.
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the static scratch in the current context (the caller's device current),
// looked up once per context with cudaGetSymbolAddress and cached under the context's ID.
p3m_status scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return P3M_ECUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  unsigned long long id = current_context_id();
  if (id != 0)
    for (int k = 0; k < g_na_used; ++k)
      if (g_na_slots[k].ctx_id == id) {
        *out = g_na_slots[k].ptr;
        return P3M_OK;
      }
  // not seen yet in this context (or no context bound yet: the lookup binds the device's
  // primary context, whose ID is taken afterwards)
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_na_scratch);
  if (e != cudaSuccess || !ptr) return P3M_ECUDA;
  if (id == 0) id = current_context_id();
  if (id != 0) {
    if (g_na_used < kNaMaxContexts) {
      g_na_slots[g_na_used++] = NaSlot{id, static_cast<double*>(ptr)};
    } else {  // many contexts over the process's life: reuse slots round-robin
      static int next = 0;
      g_na_slots[next] = NaSlot{id, static_cast<double*>(ptr)};
      next = (next + 1) % kNaMaxContexts;
    }
  }
  *out = static_cast<double*>(ptr);
  return P3M_OK;
}

// Launch status of the kernel just launched by this call. `before` is the runtime's pending
// error from the caller's own earlier work (peeked, not cleared): it is left for the caller,
// and only an error that this launch added is taken (and cleared) here.
bool launch_failed(cudaError_t before) {
  const cudaError_t e = cudaPeekAtLastError();
  if (e == cudaSuccess || e == before) return false;
  (void)cudaGetLastError();
  return true;
}

}  // namespace

extern "C" p3m_status p3m_emittance_noalloc(const double* x, const double* p, int64_t n,
                                            double mass, double* eps3, double* gx, double* gp,
                                            void* stream) {
  if (!x || !p || !eps3 || n < 2 || !(mass > 0.0)) return P3M_EINVAL;
  if (n > P3M_NOALLOC_MAX_N) return P3M_EINVAL;
  double* scratch = nullptr;
  const p3m_status s = scratch_address(&scratch);
  if (s != P3M_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nb = static_cast<int>((n + kNaPerBlock - 1) / kNaPerBlock);
  const double mc = mass * 299792458.0;
  const cudaError_t before = cudaPeekAtLastError();
  k_na_first<<<nb, kNaThreads, 0, st>>>(x, p, n, scratch);
  if (launch_failed(before)) return P3M_ECUDA;
  k_na_combine<<<1, kNaThreads, 0, st>>>(scratch, nb, 0, 6);
  if (launch_failed(before)) return P3M_ECUDA;
  k_na_second<<<nb, kNaThreads, 0, st>>>(x, p, n, scratch);
  if (launch_failed(before)) return P3M_ECUDA;
  k_na_combine<<<1, kNaThreads, 0, st>>>(scratch, nb, 6, 15);
  if (launch_failed(before)) return P3M_ECUDA;
  const int64_t work = (gx || gp) ? 3 * n : 3;
  k_na_finish<<<static_cast<unsigned>((work + 255) / 256), 256, 0, st>>>(x, p, n, scratch, mc,
                                                                        eps3, gx, gp);
  return launch_failed(before) ? P3M_ECUDA : P3M_OK;
}
