// Row-exact segment kernel for the precision-64 iteration (tiling 4).
//
// The same certified decision as k_seg_fast (Section 4.1 inner problem, GAM
// form: the optimal assortment is S* = {j : m_j v_j > R* vt_j} at the optimal
// rate R*, found by Dinkelbach's iteration in binary32 and certified, with a
// binary64 redo for uncertified segments; see spfom_segments_fast.cu), laid
// out so that no lane issues work for a slot it does not hold:
//
//  * one lane per segment for sets of up to 8 products (32 segments per warp,
//    no shuffles), 2 lanes for up to 16, 4 for up to 32, 8 for up to 64 and 16
//    for up to 128 (kRowsMax = 8 slot rows per lane at most);
//  * the row-exact copy (spfom_sliced.cu) sorts the segments by set size, so a
//    chunk's segments have (nearly) equal sizes, and gives each chunk exactly
//    ceil(largest set / W) slot rows of 32 entries; the kernel is instantiated
//    per (W, rows), and its fully unrolled slot loops hold the binary32 images
//    a_j = m_j v_j, b_j = vt_j of just those rows in registers;
//  * the certificate is tested once, at the converged ratio; a segment that
//    does not pass it is not solved in the chunk loop but listed, and the
//    block's warps solve its listed segments in binary64 after the chunk loop
//    (about 1e-4 of the segments; beyond 64 in a block, a kernel after the
//    pass), so the chunk loop carries no binary64 decision code;
//  * the binary64 work is D* = vt_0 + sum_{S*} vt_j over the chosen slots and
//    the quotient q = lambda / D*, whose warp instructions now serve 32 (or
//    32 / W) segments; the chosen slots' ids, v and vt are read again (L1/L2)
//    for D* and for the sales x_j = q v_j, rounded once to unsigned 64-bit
//    fixed point (from the 106-bit product of the significands; when the
//    rounding position lies in its upper half, as for every workload here,
//    the upper 64 bits decide the rounding exactly) and added per product
//    (shared memory, or global atomics for instances with more products than
//    shared memory holds).
//
// The margins enter the decision as binary32 images prepared with them
// (k_margins): round to nearest for positive margins in binary32's normal
// range, NaN for positive margins outside it (the segment is then not
// certified and redone in binary64 from the binary64 margins), 0 otherwise.
//
// Error budget of the certificate (|a_j - R b_j| > 2^-16 (a_j + R b_j)): the
// images carry at most 2^-23 relative error (v and vt truncated, m rounded),
// a lane sums at most 8 slots in two interleaved partial sums (depth <= 5)
// and a group adds at most 4 shuffle levels, so N, D and R stay within about
// 2e-6 of their exact values, below the 1.5e-5 margin: a certified set is the
// exact-arithmetic optimum.
#include <cuda_runtime.h>

#include <algorithm>

#include "spfom_device.cuh"
#include "spfom_internal.h"

namespace spfom {

namespace {

// Launch shapes of the forms other than shared margins (one 1024-thread block
// per SM). Binary64 on the mid instance (shared sums): 2 x 768 threads (40
// registers, 48 warps) 0.1323 ms, against 0.1397 ms with shared margins
// (1024 threads, 64 registers), 0.1494 at 2 x 512, 0.1377 at 2 x 704 and 0.1355
// at 2 x 1024; binary32 keeps shared margins (0.0556 ms; 0.0577-0.0680 in the
// shared-sums shapes).
#ifndef SPFOM_ROWS_THREADS
#define SPFOM_ROWS_THREADS 768
#endif
#ifndef SPFOM_ROWS32_THREADS
#define SPFOM_ROWS32_THREADS 512
#endif
#ifndef SPFOM_ROWS_MINB
#define SPFOM_ROWS_MINB 2
#endif
#ifndef SPFOM_ROWS_MS_THREADS
#define SPFOM_ROWS_MS_THREADS 1024
#endif
// binary64 with global sums: 2 x 768 threads (40 registers, 48 warps per SM)
// ran 0.426 ms on a 2e6-segment instance of the huge instance's shape against
// 0.469 ms at 2 x 512 (64 registers), 0.429 at 3 x 512, 0.428 at 4 x 384,
// 0.442 at 2 x 1024 and 0.457 at 3 x 640; binary32 keeps 2 x 512 (0.210 ms;
// 0.228-0.266 with more warps and fewer registers)
#ifndef SPFOM_ROWS_G_THREADS
#define SPFOM_ROWS_G_THREADS 768
#endif
#ifndef SPFOM_ROWS_G_MINB
#define SPFOM_ROWS_G_MINB 2
#endif
#ifndef SPFOM_ROWS32_G_THREADS
#define SPFOM_ROWS32_G_THREADS 512
#endif
#ifndef SPFOM_ROWS32_G_MINB
#define SPFOM_ROWS32_G_MINB 2
#endif
constexpr int kRowsMinBlocks = SPFOM_ROWS_MINB;      // blocks per SM of the shared-sums forms (register budget)
constexpr int kRowsMsThreads = SPFOM_ROWS_MS_THREADS;  // block of the shared-margins kernel (one per SM)

// Block size and blocks per SM (the register budget) of each form: shared
// margins and sums (MS), shared sums only (SC = 1), global sums (SC = 2),
// binary64 (F32 = 0) or binary32.
template <int SC, int MS, int F32>
struct RowsCfg {
  static constexpr int threads =
      MS ? kRowsMsThreads
         : (SC == 2 ? (F32 ? SPFOM_ROWS32_G_THREADS : SPFOM_ROWS_G_THREADS)
                    : (F32 ? SPFOM_ROWS32_THREADS : SPFOM_ROWS_THREADS));
  static constexpr int minb = MS ? 1 : (SC == 2 ? (F32 ? SPFOM_ROWS32_G_MINB : SPFOM_ROWS_G_MINB) : kRowsMinBlocks);
};

// round(x 2^G) for binary64 x >= 0 with x 2^G < 2^62 (integer operations only,
// no branch: shift counts are clamped and the cases chosen by selects).
__device__ __forceinline__ long long fx_of(double x, int G) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)(u >> 52);
  const unsigned long long m = (u & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const int sh = 1075 - G - e;  // x 2^G = m 2^-sh
  const int r = sh < 1 ? 1 : (sh > 63 ? 63 : sh);
  const unsigned long long down = (m + (1ull << (r - 1))) >> r;
  const unsigned long long up = m << (sh < 0 ? (-sh > 63 ? 63 : -sh) : 0);
  const unsigned long long v = sh <= 0 ? up : down;
  return (e == 0 || sh > 63) ? 0ll : (long long)v;
}

// round(q v 2^F) for positive normal binary64 q, v (q v 2^F < 2^62), with q's
// significand mq and biased exponent eq decoded once per segment. The product
// of the 53-bit significands is P = hi 2^64 + lo and the result is
// round(P / 2^sh). For sh >= 65 the rounding bit lies in hi and lo < 2^64
// cannot move floor((hi 2^64 + lo + 2^(sh-1)) / 2^sh) = floor((hi + 2^(sh-65)) /
// 2^(sh-64) + lo / 2^sh), so hi alone gives the exact rounding.
__device__ __forceinline__ unsigned long long fixed_q(unsigned long long mq, int eq, double v, int F) {
  const unsigned long long uv = (unsigned long long)__double_as_longlong(v);
  const unsigned long long mv = (uv & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const int sh = 2150 - F - eq - (int)(uv >> 52);
  const unsigned long long hi = __umul64hi(mq, mv);
  if (sh >= 65) return sh > 126 ? 0ull : (hi + (1ull << (sh - 65))) >> (sh - 64);
  if (sh < 43) return 0ull;  // cannot occur below 2^62
  unsigned long long lo = mq * mv, h = hi;
  if (sh <= 64) {
    const unsigned long long half = 1ull << (sh - 1);
    lo += half;
    h += (lo < half) ? 1ull : 0ull;
  }
  return sh < 64 ? (h << (64 - sh)) | (lo >> sh) : h;
}

// Chunk and group of a position of the row-exact copy.
struct RowsPos {
  long long c, e;  // chunk, entry of the group's lane 0 in row 0
  int W, rows;
};
__device__ __forceinline__ RowsPos rows_pos(const SlView& S, long long pos) {
  int k = 0;
  while (k < kRowsClasses - 1 && pos >= S.cls_pos[k + 1]) ++k;
  RowsPos r;
  r.W = 16 >> k;
  const long long rel = pos - S.cls_pos[k], C = 32 / r.W;
  r.c = S.cls_c[k] + rel / C;
  const long long o = S.off[r.c];
  r.rows = (int)((S.off[r.c + 1] - o) >> 5);
  r.e = o + (rel % C) * r.W;
  return r;
}

// One Dinkelbach pass over a lane's R slots at ratio Rr: the set {a_j > Rr b_j},
// with the sums of a and b over it (two interleaved partial sums each). Slots
// that are not candidates hold a = b = 0 and never enter (0 > Rr 0 is false),
// so the pass needs no candidate mask; CERT also tests every candidate
// against the certificate margin.
template <int R, bool CERT>
__device__ __forceinline__ unsigned dk_pass(const float (&af)[R], const float (&bf)[R], unsigned cand, float Rr,
                                            float& N, float& D, bool& cert) {
  unsigned s = 0;
  float N0 = 0.f, N1 = 0.f, D0 = 0.f, D1 = 0.f;
#pragma unroll
  for (int p = 0; p < R; ++p) {
    const float a = af[p], c = Rr * bf[p];
    if (a > c) {
      s |= 1u << p;
      if (p & 1) {
        N1 += a;
        D1 += bf[p];
      } else {
        N0 += a;
        D0 += bf[p];
      }
    }
    if (CERT) cert &= !((cand >> p) & 1u) || fabsf(a - c) > kCertDelta * (a + c);
  }
  N = N0 + N1;
  D = D0 + D1;
  return s;
}

// One segment (W = 1) or one lane of a W-lane segment group, R slot rows.
// sp / vv / vtv point at this lane's entry of row 0 (row stride 32 entries).
// Returns false when the binary32 decision is not certified: nothing is
// added, and the caller lists the segment for the binary64 redo.
template <int W, int R>
__device__ __forceinline__ bool rows_segment(const FastArgs& A, const float* __restrict__ mg,
                                             const int* __restrict__ sp, const double* __restrict__ vv,
                                             const double* __restrict__ vtv, const SlView& S, long long pos,
                                             unsigned gmask, unsigned long long* sums) {
  float af[R], bf[R];
  unsigned cand = 0;
  bool ok = true;
#pragma unroll
  for (int p = 0; p < R; ++p) {
    const int j = sp[32 * p];  // -1: padding (v = vt = 0)
    const double v = vv[32 * p], vt = vtv[32 * p];
    af[p] = 0.f;
    bf[p] = 0.f;
    if (j >= 0) {
      const float m = mg[j];
      if (m > 0.f) {
        cand |= 1u << p;
        af[p] = m * f32_trunc(v, ok);
        bf[p] = f32_trunc(vt, ok);
      } else if (m != m) {
        ok = false;  // positive margin outside binary32's range: decide in binary64
      }
    }
  }
  const double vt0 = S.vt0[pos];
  const float vt0f = f32_trunc(vt0, ok);
  float* rp = S.rprev + pos;
  // Dinkelbach from the carried ratio (the margins move little between
  // iterations, so the second pass confirms almost every set)
  float Rr = *rp, Dsel = 0.f;
  unsigned sel = 0xffffffffu;
  bool conv = false;
#pragma unroll 1
  for (int it = 0; it < R * W + 3; ++it) {
    float N, D;
    bool unused = true;
    const unsigned s = dk_pass<R, false>(af, bf, cand, Rr, N, D, unused);
    if (W == 1 ? s == sel : __all_sync(gmask, s == sel)) {
      conv = true;
      break;
    }
#pragma unroll
    for (int o = W >> 1; o > 0; o >>= 1) {
      N += __shfl_xor_sync(gmask, N, o, W);
      D += __shfl_xor_sync(gmask, D, o, W);
    }
    Rr = __fdividef(N, vt0f + D);
    sel = s;
    Dsel = D;
  }
  // certificate at the final ratio
  bool cert = true;
  {
    float N, D;
    dk_pass<R, true>(af, bf, cand, Rr, N, D, cert);
  }
  bool good = ok && conv && cert;
  if (W == 1 ? !good : !__all_sync(gmask, good)) return false;
  if ((gmask & -gmask) == (1u << (threadIdx.x & 31))) *rp = Rr;  // the group's first lane
  // D* = vt_0 + sum of the chosen vt, each rounded to the segment's unit 2^-G
  // and summed exactly as integers: G puts D* just below 2^61 (from the binary32
  // sum of the chosen images, within 1e-5 of D*), so each term's rounding is
  // below 2^-62 of D*, finer than a binary64 sum's. The chosen slots' vt are
  // read again (L1 or L2) by predicated loads that are all in flight together;
  // the rounding of the sum to binary64 and the quotient are the segment's
  // only binary64 operations.
  const int G = 59 - (int)((__float_as_uint(vt0f + Dsel) >> 23) & 0xFFu) + 127;  // D* < 2^(61 - G)
  long long Dfx = (W == 1 || (gmask & -gmask) == (1u << (threadIdx.x & 31))) ? fx_of(vt0, G) : 0ll;
#pragma unroll
  for (int p = 0; p < R; ++p)
    if ((sel >> p) & 1u) Dfx += fx_of(vtv[32 * p], G);
#pragma unroll
  for (int o = W >> 1; o > 0; o >>= 1) Dfx += __shfl_xor_sync(gmask, Dfx, o, W);
  // Dfx 2^-G: the exponent of the (positive, normal) binary64 image drops by G
  const double Dstar = __longlong_as_double(__double_as_longlong(__ll2double_rn(Dfx)) - ((long long)G << 52));
  const double q = quotient(S.lam[pos], Dstar);
  const unsigned long long uq = (unsigned long long)__double_as_longlong(q);
  const unsigned long long mq = (uq & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const int eq = (int)(uq >> 52);
  const bool qpos = (uq >> 52) != 0ull;  // q > 0 (q is never negative)
  // sales, four slots at a time: their ids and values are loaded before any of their atomics
#pragma unroll
  for (int p0 = 0; p0 < R; p0 += 4) {
    int jc[4];
    double vc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      jc[u] = 0;
      vc[u] = 0.0;
      if (p0 + u < R && ((sel >> (p0 + u)) & 1u)) {
        jc[u] = sp[32 * (p0 + u)];
        vc[u] = vv[32 * (p0 + u)];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (p0 + u < R && qpos && ((sel >> (p0 + u)) & 1u)) atomicAdd(sums + jc[u], fixed_q(mq, eq, vc[u], A.fx_bits));
  }
  return true;
}

// Uncertified segments of a block: listed in shared memory and redone by the
// block's own warps after its chunk loop; beyond kRedoLocal per block they go
// to the global list (redone after the pass).
constexpr int kRedoLocal = 64;
__shared__ long long g_redo_local[kRedoLocal];
__shared__ int g_redo_n;

__device__ void rows_redo_segment(const FastArgs& A, long long pos, unsigned long long* sums, int& fallbacks);

template <int W, int R>
__device__ __forceinline__ void rows_chunk(const FastArgs& A, const float* mg, long long e, long long pos,
                                           unsigned gmask, unsigned long long* sums) {
  const SlView& S = A.rx;
  const bool done = rows_segment<W, R>(A, mg, S.prod + e, S.v + e, S.vt + e, S, pos, gmask, sums);
  if (!done && (gmask & -gmask) == (1u << (threadIdx.x & 31))) {
    const int i = atomicAdd(&g_redo_n, 1);
    if (i < kRedoLocal) g_redo_local[i] = pos;
    else S.redo[atomicAdd(S.redo_ctl, 1u)] = pos;
  }
}

// rows is exactly ceil(largest set / W): 1..kRowsMax for W = 1, above
// kRowsMax / 2 for W >= 2 (and at most ceil(kFastMaxSet / 16) for W = 16).
template <int W>
__host__ __device__ constexpr int rows_lo() { return W == 1 ? 1 : kRowsMax / 2 + 1; }
template <int W>
__host__ __device__ constexpr int rows_hi() { return W == 16 ? (kFastMaxSet + 15) / 16 : kRowsMax; }

template <int W, int R>
__device__ __forceinline__ void rows_dispatch_r(const FastArgs& A, const float* mg, int rows, long long e,
                                                long long pos, unsigned gmask, unsigned long long* sums) {
  if (rows == R) {
    rows_chunk<W, R>(A, mg, e, pos, gmask, sums);
  } else if constexpr (R > rows_lo<W>()) {
    rows_dispatch_r<W, R - 1>(A, mg, rows, e, pos, gmask, sums);
  }  // rows 0 (empty sets) and counts the layout does not produce: nothing to do
}

template <int W>
__device__ __forceinline__ void rows_dispatch(const FastArgs& A, const float* mg, int rows, long long e, long long pos,
                                              unsigned gmask, unsigned long long* sums) {
  rows_dispatch_r<W, rows_hi<W>()>(A, mg, rows, e, pos, gmask, sums);
}

// Binary64 solve of one listed segment by one full warp: lanes r < W hold
// the slots r, r + W, ... of the segment (as in the chunk loop) in registers
// (all loads in flight together), the decision is Dinkelbach's iteration in
// binary64 from the binary64 margins, and the sales go to the global product
// sums; the segment's carried ratio is refreshed.
__device__ void rows_redo_segment(const FastArgs& A, long long pos, unsigned long long* sums, int& fallbacks) {
  const SlView& S = A.rx;
  const RowsPos rp = rows_pos(S, pos);
  const int lane = threadIdx.x & 31;
  const bool in = lane < rp.W;
  int jv[kRowsMax];
  double av[kRowsMax], tv[kRowsMax];
  unsigned cand = 0;
#pragma unroll
  for (int p = 0; p < kRowsMax; ++p) {
    jv[p] = -1;
    av[p] = tv[p] = 0.0;
    if (in && p < rp.rows) {
      const long long k = rp.e + lane + 32ll * p;
      jv[p] = S.prod[k];
      tv[p] = S.vt[k];
      av[p] = S.v[k];
    }
  }
#pragma unroll
  for (int p = 0; p < kRowsMax; ++p)
    if (jv[p] >= 0) {
      const double m = A.marg[jv[p]];
      if (m > 0.0) {
        cand |= 1u << p;
        av[p] *= m;
      }
    }
  const double vt0 = S.vt0[pos];
  double Rd = 0.0;
  unsigned prev = 0xffffffffu;
  for (int it = 0; it < kRowsMax * 16 + 2; ++it) {
    unsigned s = 0;
    double N = 0.0, D = 0.0;
#pragma unroll
    for (int p = 0; p < kRowsMax; ++p)
      if (((cand >> p) & 1u) && av[p] > Rd * tv[p]) {
        s |= 1u << p;
        N += av[p];
        D += tv[p];
      }
    if (__all_sync(0xffffffffu, s == prev)) break;
    for (int o = 16; o > 0; o >>= 1) {
      N += __shfl_xor_sync(0xffffffffu, N, o);
      D += __shfl_xor_sync(0xffffffffu, D, o);
    }
    Rd = N / (vt0 + D);
    prev = s;
  }
  double Dl = 0.0;
#pragma unroll
  for (int p = 0; p < kRowsMax; ++p)
    if ((prev >> p) & 1u) Dl += tv[p];
  for (int o = 16; o > 0; o >>= 1) Dl += __shfl_xor_sync(0xffffffffu, Dl, o);
  const double q = quotient(S.lam[pos], vt0 + Dl);
#pragma unroll
  for (int p = 0; p < kRowsMax; ++p)
    if ((prev >> p) & 1u) atomicAdd(sums + jv[p], fixed_product(q, S.v[rp.e + lane + 32ll * p], A.fx_bits));
  if (lane == 0) {
    S.rprev[pos] = (float)Rd;
    ++fallbacks;
  }
}

// With per-block product sums (SC = 1): the fold of the partial sums into the
// global ones (rows blockIdx.y < chunks, as k_reduce_products) and the binary64
// redo of the listed segments (the last row of blocks, one warp per segment)
// in one launch; both add into s_fx. The last redo block to finish clears the
// list for the next pass.
__global__ void __launch_bounds__(256) k_reduce_redo(FastArgs A, int n, int nparts,
                                                     const unsigned long long* __restrict__ part, int chunks) {
  __shared__ int last;
  if (A.st && A.st->converged) return;
  if ((int)blockIdx.y < chunks) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int per = (nparts + chunks - 1) / chunks;
    const int b0 = blockIdx.y * per, b1 = min(nparts, b0 + per);
    unsigned long long acc = 0ull;
#pragma unroll 8
    for (int b = b0; b < b1; ++b) acc += __ldcg(part + (size_t)b * n + j);
    if (acc) atomicAdd(A.s_fx + j, acc);
    return;
  }
  const SlView& S = A.rx;
  const unsigned cnt = *(volatile unsigned*)S.redo_ctl;
  int fallbacks = 0;
  const unsigned gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), nw = gridDim.x * (blockDim.x >> 5);
  for (unsigned i = gw; i < cnt; i += nw) rows_redo_segment(A, S.redo[i], A.s_fx, fallbacks);
  if (fallbacks && A.fallbacks) atomicAdd(A.fallbacks, (unsigned long long)fallbacks);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(S.redo_ctl + 1, 1u) == gridDim.x - 1;
    if (last) {
      S.redo_ctl[0] = 0u;
      S.redo_ctl[1] = 0u;
    }
  }
}

// The segments the chunk loop listed: one warp per segment; the last block to
// finish clears the list for the next pass.
__global__ void __launch_bounds__(256) k_rows_redo(FastArgs A) {
  __shared__ int last;
  if (A.st && A.st->converged) return;
  const SlView& S = A.rx;
  const unsigned cnt = *(volatile unsigned*)S.redo_ctl;
  int fallbacks = 0;
  const unsigned gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), nw = gridDim.x * (blockDim.x >> 5);
  for (unsigned i = gw; i < cnt; i += nw) rows_redo_segment(A, S.redo[i], A.s_fx, fallbacks);
  if (fallbacks && A.fallbacks) atomicAdd(A.fallbacks, (unsigned long long)fallbacks);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(S.redo_ctl + 1, 1u) == gridDim.x - 1;
    if (last) {
      S.redo_ctl[0] = 0u;
      S.redo_ctl[1] = 0u;
    }
  }
}

// SC = 1: product sums in shared memory, per-block partial sums out
// (k_reduce_products folds them); MS = 1 also copies the binary32 margin
// images into shared memory (one 1024-thread block per SM). SC = 2: global
// atomics into the product sums, margin images read from global memory.
template <int SC, int MS>
__global__ void __launch_bounds__(RowsCfg<SC, MS, 0>::threads, RowsCfg<SC, MS, 0>::minb) k_seg_rows(FastArgs A) {
  extern __shared__ unsigned long long acc[];  // SC == 1: [n] fixed-point sums; MS: + [n] binary32 margins
  if (A.st && A.st->converged) return;
  const int n = A.P.n;
  const float* mg = A.marg32c;
  if (threadIdx.x == 0) g_redo_n = 0;
  if (SC == 1) {
    float* smg = reinterpret_cast<float*>(acc + n);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      acc[j] = 0ull;
      if (MS) smg[j] = A.marg32c[j];
    }
    if (MS) mg = smg;
  }
  __syncthreads();
  unsigned long long* sums = SC == 1 ? acc : A.s_fx;
  const SlView& S = A.rx;
  const int wl = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < S.nchunks; c += nw) {
    const long long o = S.off[c];
    const int rows = (int)((S.off[c + 1] - o) >> 5);
    int k = 0;
    while (k < kRowsClasses - 1 && c >= S.cls_c[k + 1]) ++k;  // warp-uniform
    const int W = 16 >> k;
    const long long pos = S.cls_pos[k] + (c - S.cls_c[k]) * (32 / W) + wl / W;
    const long long e = o + wl;
    const unsigned gmask = W == 1 ? (1u << wl) : (((1u << W) - 1u) << (wl & ~(W - 1)));
    switch (W) {
      case 1: rows_dispatch<1>(A, mg, rows, e, pos, gmask, sums); break;
      case 2: rows_dispatch<2>(A, mg, rows, e, pos, gmask, sums); break;
      case 4: rows_dispatch<4>(A, mg, rows, e, pos, gmask, sums); break;
      case 8: rows_dispatch<8>(A, mg, rows, e, pos, gmask, sums); break;
      default: rows_dispatch<16>(A, mg, rows, e, pos, gmask, sums); break;
    }
  }
  // the block's uncertified segments (about 1e-4 of them), in binary64, one warp each
  __syncthreads();
  {
    const int nl = g_redo_n < kRedoLocal ? g_redo_n : kRedoLocal;
    int fallbacks = 0;
    for (int i = threadIdx.x >> 5; i < nl; i += blockDim.x >> 5) rows_redo_segment(A, g_redo_local[i], sums, fallbacks);
    if (fallbacks && A.fallbacks) atomicAdd(A.fallbacks, (unsigned long long)fallbacks);
  }
  // an iterate pass forms no segment values: the dual step takes sum_l z_l as sum_j m_j s_j
  if (threadIdx.x == 0) A.zpart[blockIdx.x] = 0.0;
  if (SC == 1) {
    __syncthreads();
    unsigned long long* dst = A.part + (size_t)blockIdx.x * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) dst[j] = acc[j];
  }
}

// ---- binary32 bulk pass (precision 32, tiling 9) --------------------------
// The same row-exact layout and Dinkelbach iteration on binary32 copies of the
// inputs (12 B per nonzero), without certificate or binary64 redo: the bulk
// mode's decisions are its binary32 ones, as in k_seg_f32. Every slot's id and
// v stay in registers, so nothing is read twice: q = lambda / (vt_0 + D) from
// the final set's binary32 sum, and each chosen product's sales are the exact
// product q v rounded once to fixed point.
// round(q v 2^F) for non-negative binary32 q, v with q v 2^F < 2^62, q's
// significand mq (24 bits) and biased exponent eq decoded once per segment:
// the 48-bit product of the significands is exact, so the only rounding is the
// final one (no branch: shift counts clamped, cases chosen by selects).
__device__ __forceinline__ unsigned long long fixed32_q(unsigned mq, int eq, float v, int F) {
  const unsigned uv = __float_as_uint(v);
  const int ev = (int)(uv >> 23);
  const unsigned long long prod = (unsigned long long)mq * (unsigned long long)((uv & 0x7FFFFFu) | 0x800000u);
  const int sh = 300 - F - eq - ev;  // q v 2^F = prod / 2^sh
  const int r = sh < 1 ? 1 : (sh > 63 ? 63 : sh);
  const unsigned long long down = (prod + (1ull << (r - 1))) >> r;
  const unsigned long long up = prod << (sh < 0 ? (-sh > 63 ? 63 : -sh) : 0);
  const unsigned long long x = sh <= 0 ? up : down;
  return (eq == 0 || ev == 0 || sh > 63) ? 0ull : x;
}

template <int W, int R>
__device__ __forceinline__ void rows32_segment(const F32Args& A, const float* __restrict__ mg,
                                               const int* __restrict__ sp, const float* __restrict__ vv,
                                               const float* __restrict__ vtv, const SlView& S, long long pos,
                                               unsigned gmask, unsigned long long* sums) {
  int jv[R];
  float vf[R], af[R], bf[R];
  unsigned cand = 0;
#pragma unroll
  for (int p = 0; p < R; ++p) {
    const int j = sp[32 * p];  // -1: padding (v = vt = 0)
    const float v = vv[32 * p], t = vtv[32 * p];
    const float m = mg[j >= 0 ? j : 0];
    const bool c = j >= 0 && m > 0.f;
    jv[p] = j;
    vf[p] = v;
    af[p] = c ? m * v : 0.f;
    bf[p] = c ? t : 0.f;
    cand |= c ? 1u << p : 0u;
  }
  const float vt0 = S.vt0_32[pos];
  float* rp = S.rprev + pos;
  // Dinkelbach from the carried ratio: the first two passes are straight-line
  // code (the second confirms almost every set: the margins move little between
  // iterations); the rare remaining segments go on in a loop
  float N, D;
  bool unused = true;
  unsigned sel = dk_pass<R, false>(af, bf, cand, *rp, N, D, unused);
#pragma unroll
  for (int o = W >> 1; o > 0; o >>= 1) {
    N += __shfl_xor_sync(gmask, N, o, W);
    D += __shfl_xor_sync(gmask, D, o, W);
  }
  float Rr = __fdividef(N, vt0 + D), Dsel = D;
  unsigned s2 = dk_pass<R, false>(af, bf, cand, Rr, N, D, unused);
  if (!(W == 1 ? s2 == sel : __all_sync(gmask, s2 == sel))) {
    sel = s2;
#pragma unroll 1
    for (int it = 0; it < R * W + 2; ++it) {
#pragma unroll
      for (int o = W >> 1; o > 0; o >>= 1) {
        N += __shfl_xor_sync(gmask, N, o, W);
        D += __shfl_xor_sync(gmask, D, o, W);
      }
      Rr = __fdividef(N, vt0 + D);
      Dsel = D;
      const unsigned s = dk_pass<R, false>(af, bf, cand, Rr, N, D, unused);
      if (W == 1 ? s == sel : __all_sync(gmask, s == sel)) break;
      sel = s;
    }
  }
  if ((gmask & -gmask) == (1u << (threadIdx.x & 31))) *rp = Rr;
  const float q = S.lam32[pos] / (vt0 + Dsel);
  const unsigned uq = __float_as_uint(q);
  const unsigned mq = (uq & 0x7FFFFFu) | 0x800000u;
  const int eq = (int)(uq >> 23);
#pragma unroll
  for (int p = 0; p < R; ++p)
    if ((sel >> p) & 1u) atomicAdd(sums + jv[p], fixed32_q(mq, eq, vf[p], A.fx_bits));
}

template <int W, int R>
__device__ __forceinline__ void rows32_chunk(const F32Args& A, const float* mg, long long e, long long pos,
                                             unsigned gmask, unsigned long long* sums) {
  const SlView& S = A.rx;
  rows32_segment<W, R>(A, mg, S.prod + e, S.v32 + e, S.vt32 + e, S, pos, gmask, sums);
}

template <int W, int R>
__device__ __forceinline__ void rows32_dispatch_r(const F32Args& A, const float* mg, int rows, long long e,
                                                  long long pos, unsigned gmask, unsigned long long* sums) {
  if (rows == R) {
    rows32_chunk<W, R>(A, mg, e, pos, gmask, sums);
  } else if constexpr (R > rows_lo<W>()) {
    rows32_dispatch_r<W, R - 1>(A, mg, rows, e, pos, gmask, sums);
  }
}

template <int SC, int MS>
__global__ void __launch_bounds__(RowsCfg<SC, MS, 1>::threads, RowsCfg<SC, MS, 1>::minb) k_seg_rows32(F32Args A) {
  extern __shared__ unsigned long long acc[];  // SC == 1: [n] fixed-point sums; MS: + [n] binary32 margins
  if (A.st->converged) return;
  const int n = A.n;
  const float* mg = A.marg32;
  if (SC == 1) {
    float* smg = reinterpret_cast<float*>(acc + n);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      acc[j] = 0ull;
      if (MS) smg[j] = A.marg32[j];
    }
    if (MS) mg = smg;
    __syncthreads();
  }
  unsigned long long* sums = SC == 1 ? acc : A.s_fx;
  const SlView& S = A.rx;
  const int wl = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < S.nchunks; c += nw) {
    const long long o = S.off[c];
    const int rows = (int)((S.off[c + 1] - o) >> 5);
    int k = 0;
    while (k < kRowsClasses - 1 && c >= S.cls_c[k + 1]) ++k;  // warp-uniform
    const int W = 16 >> k;
    const long long pos = S.cls_pos[k] + (c - S.cls_c[k]) * (32 / W) + wl / W;
    const long long e = o + wl;
    const unsigned gmask = W == 1 ? (1u << wl) : (((1u << W) - 1u) << (wl & ~(W - 1)));
    switch (W) {
      case 1: rows32_dispatch_r<1, rows_hi<1>()>(A, mg, rows, e, pos, gmask, sums); break;
      case 2: rows32_dispatch_r<2, rows_hi<2>()>(A, mg, rows, e, pos, gmask, sums); break;
      case 4: rows32_dispatch_r<4, rows_hi<4>()>(A, mg, rows, e, pos, gmask, sums); break;
      case 8: rows32_dispatch_r<8, rows_hi<8>()>(A, mg, rows, e, pos, gmask, sums); break;
      default: rows32_dispatch_r<16, rows_hi<16>()>(A, mg, rows, e, pos, gmask, sums); break;
    }
  }
  // the iterate pass forms no segment values: the dual step takes sum_l z_l as sum_j m_j s_j
  if (threadIdx.x == 0) A.zpart[blockIdx.x] = 0.0;
  if (SC == 1) {
    __syncthreads();
    unsigned long long* dst = A.part + (size_t)blockIdx.x * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) dst[j] = acc[j];
  }
}

template <class K>
int rows_blocks(K kernel, int smem, int threads) {
  return kernel_blocks(kernel, threads, smem);
}

}  // namespace

bool rows_plan(int n, int sms, FastPlan* plan) {
  plan->rows_ok = 0;
  plan->rows_redo_grid = sms;
  const long long sums = 8ll * n, ms = 12ll * n;
  // Binary64: shared sums with the binary32 margins read through L1 when two
  // blocks fit per SM (more warps at fewer registers), else shared sums and
  // margins, else shared sums alone, else global sums.
  const int s64 = sums <= kFastMaxSmem ? rows_blocks(k_seg_rows<1, 0>, (int)sums, RowsCfg<1, 0, 0>::threads) : 0;
  const int m64 = ms <= kTmaMaxSmem ? rows_blocks(k_seg_rows<1, 1>, (int)ms, RowsCfg<1, 1, 0>::threads) : 0;
  if (s64 >= 2 || (s64 >= 1 && m64 < 1)) {
    plan->rows_ms = 0, plan->rows_smem = (int)sums, plan->rows_grid = s64 * sms;
  } else if (m64 >= 1) {
    plan->rows_ms = 1, plan->rows_smem = (int)ms, plan->rows_grid = m64 * sms;
  } else {
    const int g64 = rows_blocks(k_seg_rows<2, 0>, 0, RowsCfg<2, 0, 0>::threads);
    if (g64 < 1) return false;
    plan->rows_ms = 0, plan->rows_smem = 0, plan->rows_grid = g64 * sms;
  }
  // Binary32: shared sums and margins, else shared sums, else global sums.
  const int m32 = ms <= kTmaMaxSmem ? rows_blocks(k_seg_rows32<1, 1>, (int)ms, RowsCfg<1, 1, 1>::threads) : 0;
  const int s32 = sums <= kFastMaxSmem ? rows_blocks(k_seg_rows32<1, 0>, (int)sums, RowsCfg<1, 0, 1>::threads) : 0;
  if (m32 >= 1) {
    plan->rows_ms32 = 1, plan->rows_smem32 = (int)ms, plan->rows_grid32 = m32 * sms;
  } else if (s32 >= 1) {
    plan->rows_ms32 = 0, plan->rows_smem32 = (int)sums, plan->rows_grid32 = s32 * sms;
  } else {
    const int g32 = rows_blocks(k_seg_rows32<2, 0>, 0, RowsCfg<2, 0, 1>::threads);
    if (g32 < 1) return false;
    plan->rows_ms32 = 0, plan->rows_smem32 = 0, plan->rows_grid32 = g32 * sms;
  }
  plan->rows_ok = 1;
  return true;
}

cudaError_t launch_seg_rows(const FastArgs& A, const FastPlan& pl, cudaStream_t s) {
  if (pl.rows_ms) k_seg_rows<1, 1><<<pl.rows_grid, RowsCfg<1, 1, 0>::threads, pl.rows_smem, s>>>(A);
  else if (pl.rows_smem > 0) k_seg_rows<1, 0><<<pl.rows_grid, RowsCfg<1, 0, 0>::threads, pl.rows_smem, s>>>(A);
  else k_seg_rows<2, 0><<<pl.rows_grid, RowsCfg<2, 0, 0>::threads, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_seg_rows32(const F32Args& A, const FastPlan& pl, cudaStream_t s) {
  if (pl.rows_ms32) k_seg_rows32<1, 1><<<pl.rows_grid32, RowsCfg<1, 1, 1>::threads, pl.rows_smem32, s>>>(A);
  else if (pl.rows_smem32 > 0) k_seg_rows32<1, 0><<<pl.rows_grid32, RowsCfg<1, 0, 1>::threads, pl.rows_smem32, s>>>(A);
  else k_seg_rows32<2, 0><<<pl.rows_grid32, RowsCfg<2, 0, 1>::threads, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_reduce_redo(const FastArgs& A, const FastPlan& pl, int nparts, const unsigned long long* part,
                               cudaStream_t s) {
  const int n = A.P.n;
  // about 8 partial rows per thread: one round of loads in flight (the fixed-point
  // sums are exact in any order)
  const int chunks = std::max(1, std::min(64, (nparts + 7) / 8));
  dim3 grid(n > 0 ? (n + 255) / 256 : 1, chunks + 1);
  k_reduce_redo<<<grid, 256, 0, s>>>(A, n, nparts, part, chunks);
  return cudaGetLastError();
}

cudaError_t launch_rows_redo(const FastArgs& A, int sms, cudaStream_t s) {
  k_rows_redo<<<sms > 0 ? sms : 1, 256, 0, s>>>(A);
  return cudaGetLastError();
}

}  // namespace spfom
