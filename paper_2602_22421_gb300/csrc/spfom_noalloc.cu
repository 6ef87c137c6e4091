// Allocation-free product sales (spfom_sales_noalloc in include/spfom.h).
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool
// they do not own, embedders whose allocator is reserved for their own
// tensors, or hosts that must not allocate device memory after start-up.
// This entry point computes what one iteration's segment pass computes --
// every segment's exact best response at given margins, the sales summed per
// product and the sum of the segment values -- from device arrays the caller
// passes, and writes into device buffers the caller passes. Its scratch
// lives in the file-scope arrays below, which every GPU that loads the
// library holds until the process exits:
//   g_sales  SPFOM_NOALLOC_MAX_PRODUCTS binary64 sums (1 MiB),
//   g_zpart  kMaxBlocks per-block sums of segment values (8 KiB),
//   g_error  one flag.
// The address of each array is looked up with cudaGetSymbolAddress on the
// first call made in a CUDA context (per device and context: a context made
// after cudaDeviceReset gets its own lookup), with that context current.
// Every call shares the arrays and leaves them holding its last contents;
// each call clears what it accumulates before use. Calls whose work overlaps
// on the GPU (different streams, or different threads on one device) race on
// the arrays and give wrong results.
//
// The kernel is a variant of the general segment kernel: a sub-warp of W
// lanes per segment, binary64 throughout, exact sort and prefix scan, with
// vt = v - w and vt0 = v0 + sum w formed in registers instead of read from
// the ctx's preprocessed arrays.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cstdint>
#include <mutex>

#include "../../include/spfom.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;

static __device__ __align__(256) double g_sales[SPFOM_NOALLOC_MAX_PRODUCTS];
static __device__ __align__(256) double g_zpart[kMaxBlocks];
static __device__ __align__(256) int g_error[1];

struct Scratch {
  double* sales;
  double* zpart;
  int* error;
};

constexpr int kMaxContexts = 64;

struct ScratchEntry {
  int device;
  CUcontext ctx;
  Scratch s;
};

std::mutex g_setup_mutex;
ScratchEntry g_cache[kMaxContexts];
int g_cached = 0;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

// cuCtxGetCurrent through the runtime's driver entry-point query (the library
// does not link the driver library directly).
CtxGetCurrentFn ctx_get_current() {
  static std::once_flag once;
  static CtxGetCurrentFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
  });
  return fn;
}

// Device addresses of the static arrays in the current context: looked up on
// the first call in each (device, context) and kept. A symbol's address
// belongs to one context, so a context created later on the same device (for
// instance after cudaDeviceReset) gets its own lookup.
cudaError_t scratch_for_current_context(Scratch* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  CtxGetCurrentFn get = ctx_get_current();
  if (!get) return cudaErrorDeviceUninitialized;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  CUcontext ctx = nullptr;
  if (get(&ctx) == CUDA_SUCCESS && ctx)  // no context yet: the lookup below makes the primary one current
    for (int k = 0; k < g_cached; ++k)
      if (g_cache[k].device == dev && g_cache[k].ctx == ctx) {
        *out = g_cache[k].s;
        return cudaSuccess;
      }
  Scratch s{};
  e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.sales), g_sales);
  if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.zpart), g_zpart);
  if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.error), g_error);
  if (e != cudaSuccess) return e;
  if (get(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  // A full table (more than kMaxContexts contexts in one process) overwrites a
  // slot; a context that loses its slot is looked up again on its next call.
  const int slot = g_cached < kMaxContexts ? g_cached++ : (int)(reinterpret_cast<uintptr_t>(ctx) % kMaxContexts);
  g_cache[slot] = ScratchEntry{dev, ctx, s};
  *out = s;
  return cudaSuccess;
}

__global__ void k_na_clear(int n, int nblocks, Scratch s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) s.sales[i] = 0.0;
  if (i < nblocks) s.zpart[i] = 0.0;
  if (i == 0) s.error[0] = 0;
}

__device__ double na_block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += sh[k];
  return tot;
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_na_segments(spfom_device_segments D, const double* __restrict__ marg,
                                                          Scratch s) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & (W - 1);
  const int gbase = (threadIdx.x & 31) & ~(W - 1);
  const unsigned mask = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << gbase);
  const long long gpb = kThreads / W, ngroups = (long long)gridDim.x * gpb;
  double zacc = 0.0;
  for (long long l = blockIdx.x * gpb + threadIdx.x / W; l < D.L; l += ngroups) {
    const long long b = D.seg_ptr[l];
    const int K = (int)(D.seg_ptr[l + 1] - b);
    if (K > D.max_set_size) {  // larger than the stated max_set_size: flag it, leave the segment out
      if (lane == 0) s.error[0] = 1;
      continue;
    }
    int j = 0;
    double v = 0.0, w = 0.0, mv = 0.0;
    long long key = -1;
    if (lane < K) {
      j = D.seg_prod[b + lane];
      v = D.v[b + lane];
      w = D.w ? D.w[b + lane] : 0.0;
    }
    const double vt = v - w;
    if (lane < K) {
      const double mj = marg[j];
      if (mj > 0.0) {
        mv = mj * v;
        key = __double_as_longlong(vt == 0.0 ? CUDART_INF : mv / vt);
      }
    }
    double wsum = w;
#pragma unroll
    for (int o = W >> 1; o > 0; o >>= 1) wsum += __shfl_xor_sync(mask, wsum, o, W);
    const double vt0 = D.v0[l] + wsum, lam = D.lam[l];
    int idx = lane;
#pragma unroll
    for (int k = 2; k <= W; k <<= 1)
#pragma unroll
      for (int d = k >> 1; d > 0; d >>= 1) {
        const long long ok = __shfl_xor_sync(mask, key, d, W);
        const int oi = __shfl_xor_sync(mask, idx, d, W);
        const bool other_first = (ok > key) || (ok == key && oi < idx);
        if (((lane & k) == 0) == ((lane & d) == 0) ? other_first : !other_first) {
          key = ok;
          idx = oi;
        }
      }
    const int nc = __popc(__ballot_sync(mask, key >= 0) & mask);
    const double mv_r = __shfl_sync(mask, mv, idx, W), vt_r = __shfl_sync(mask, vt, idx, W);
    const double v_r = __shfl_sync(mask, v, idx, W);
    const int j_r = __shfl_sync(mask, j, idx, W);
    double N = lane < nc ? mv_r : 0.0, Dp = lane < nc ? vt_r : 0.0;
#pragma unroll
    for (int d = 1; d < W; d <<= 1) {
      const double tN = __shfl_up_sync(mask, N, d, W), tD = __shfl_up_sync(mask, Dp, d, W);
      if (lane >= d) {
        N += tN;
        Dp += tD;
      }
    }
    const double Dk = vt0 + Dp;
    long long best = __double_as_longlong(lane < nc ? N / Dk : 0.0);
    int bl = lane;
#pragma unroll
    for (int d = W >> 1; d > 0; d >>= 1) {
      const long long ob = __shfl_xor_sync(mask, best, d, W);
      const int ol = __shfl_xor_sync(mask, bl, d, W);
      if (ob > best || (ob == best && ol < bl)) {
        best = ob;
        bl = ol;
      }
    }
    const int kstar = best > 0 ? bl + 1 : 0;
    const double bestD = __shfl_sync(mask, Dk, bl, W);
    if (lane < kstar) atomicAdd(s.sales + j_r, lam * v_r / bestD);
    if (lane == 0) zacc += lam * __longlong_as_double(best);
  }
  const double tot = na_block_sum(zacc, sh);
  if (threadIdx.x == 0) s.zpart[blockIdx.x] = tot;
}

// Copies the sales out (every entry NaN when a segment exceeded max_set_size:
// the results are then incomplete, and a caller that reads only the sales
// sees it too) and folds the per-block values into *z_out (NaN likewise).
__global__ void k_na_finish(int n, int nblocks, Scratch s, double* __restrict__ sales_out, double* z_out) {
  __shared__ double sh[32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool bad = s.error[0] != 0;
  if (i < n) sales_out[i] = bad ? CUDART_NAN : s.sales[i];
  if (blockIdx.x != 0) return;
  double z = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) z += s.zpart[b];
  z = na_block_sum(z, sh);
  if (threadIdx.x == 0) z_out[0] = bad ? CUDART_NAN : z;
}

}  // namespace

extern "C" spfom_status spfom_sales_noalloc(const spfom_device_segments* seg, const double* margins, double* sales,
                                            double* z_sum, void* stream) {
  if (!seg || !z_sum) return SPFOM_EINVAL;
  if (seg->n < 0 || seg->n > SPFOM_NOALLOC_MAX_PRODUCTS || seg->L < 0 || seg->max_set_size < 0 ||
      seg->max_set_size > 32)
    return SPFOM_EINVAL;
  // seg_prod and v are read only for segments of at most max_set_size products,
  // so with max_set_size == 0 (every segment must be empty) they may be NULL.
  if (!seg->seg_ptr || (seg->n > 0 && (!margins || !sales)) ||
      (seg->L > 0 && (!seg->lam || !seg->v0 || (seg->max_set_size > 0 && (!seg->seg_prod || !seg->v)))))
    return SPFOM_EINVAL;
  // An error already pending on this thread belongs to earlier work: leave it
  // for its owner instead of reporting (and clearing) it as this call's.
  if (cudaPeekAtLastError() != cudaSuccess) return SPFOM_ECUDA;
  Scratch s{};
  if (scratch_for_current_context(&s) != cudaSuccess) return SPFOM_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int W = 1;
  while (W < seg->max_set_size) W <<= 1;
  long long want = (seg->L * W + kThreads - 1) / kThreads;
  const int grid = (int)(want < 1 ? 1 : (want > kMaxBlocks ? kMaxBlocks : want));
  const int span = seg->n > grid ? seg->n : grid;
  k_na_clear<<<(span + kThreads - 1) / kThreads, kThreads, 0, st>>>(seg->n, grid, s);
  switch (W) {
    case 1: k_na_segments<1><<<grid, kThreads, 0, st>>>(*seg, margins, s); break;
    case 2: k_na_segments<2><<<grid, kThreads, 0, st>>>(*seg, margins, s); break;
    case 4: k_na_segments<4><<<grid, kThreads, 0, st>>>(*seg, margins, s); break;
    case 8: k_na_segments<8><<<grid, kThreads, 0, st>>>(*seg, margins, s); break;
    case 16: k_na_segments<16><<<grid, kThreads, 0, st>>>(*seg, margins, s); break;
    default: k_na_segments<32><<<grid, kThreads, 0, st>>>(*seg, margins, s); break;
  }
  const int nb = seg->n > 0 ? (seg->n + kThreads - 1) / kThreads : 1;
  k_na_finish<<<nb, kThreads, 0, st>>>(seg->n, grid, s, sales, z_sum);
  return cudaGetLastError() == cudaSuccess ? SPFOM_OK : SPFOM_ECUDA;
}
