// Segment kernel for GB300's binary64 budget (binary64 results, binary32 decisions
// with a certificate).
//
// GB300 executes binary64 arithmetic and every binary64 <-> binary32/int
// conversion at about 1/60 of the binary32 rate, so a segment solve that
// sorts and scans in binary64 is bound by that pipe, far from HBM speed. This
// kernel keeps binary64 for the values that feed the dual step and takes the
// discrete decision -- which products the optimal assortment holds -- in
// binary32, with a certificate that the binary32 decision is the exact one.
//
// Decision (Section 4.1 inner problem, GAM form; build letters). With
// a_j = m_j v_j, b_j = vt_j for the products with m_j > 0, the optimal
// assortment is S* = {j : a_j > R* b_j} where R* = N(S*)/D(S*),
// N(S) = sum_S a_j, D(S) = vt_0 + sum_S b_j (the greedy order of Lemma 1:
// item j enters exactly when its key a_j / b_j exceeds the optimal rate).
// Dinkelbach's iteration R <- N(S(R))/D(S(R)), S(R) = {a_j > R b_j}, reaches
// such a fixed point from any start (after one step R <= R*; from there R
// rises and S shrinks), and every fixed point is optimal: for any T,
// N(T) - R D(T) <= N(S) - R D(S) = 0. It runs in binary32 on binary32 images
// of the inputs, started from the segment's ratio of the previous iteration
// (the margins move little between iterations). The decision is certified when
// every candidate clears the threshold by a relative margin
// |a_j - R b_j| > 2^-16 (a_j + R b_j); the binary32 rounding of a_j, b_j, N, D
// and R stays below 5e-6 relative (each sum is a lane's sum of at most 8 slots
// and a shuffle tree of at most 4 levels: depth <= 11 for sets of up to 128
// products), so a certified set is the exact-arithmetic optimum S*. Segments that are not
// certified (a near-tie, or an input outside binary32's normal range) repeat
// the iteration in binary64.
//
// Values, in binary64: D* = vt_0 + sum_{S*} vt_j, q = lambda / D* and the
// sales x_j = q v_j of the chosen products; N* = sum_{S*} m_j v_j and
// z = q N* only where segment values are asked for (evaluation passes, a
// batch's per-segment values): an iterate pass leaves sum_l z_l to the dual
// step, which forms it as sum_j m_j s_j.
//
// Layout: W lanes per segment, P = 8 products per lane (lane r holds products
// r, r + W, r + 2W, ... of the segment's set: contiguous loads from the CSR
// slice, or one 32-entry row per slot in the slot-major copy), and the group's
// binary64 reductions cost log2(W) shuffle steps shared by 32/W segments per
// warp instruction. The margins are read from global memory, or (MS) from a
// copy in shared memory.
//
// Sales aggregate: each block sums x_j per product in shared memory as
// unsigned 64-bit fixed point (x * 2^F rounded; F fixed per instance so that
// the arrival mass fits in 62 bits), which makes the sum exact and
// independent of order, and writes its n partial sums out; k_reduce_products
// folds them into the product sales. Wider instances add into global sums.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "spfom_device.cuh"
#include "spfom_internal.h"

namespace spfom {

namespace {

// Segment order of the plain-load kernels. Each warp takes chunks of 32 / W
// consecutive segments (one per lane group, so a warp's loads stay
// contiguous), chunk c for c = its global warp id, + #warps, ... In a batch the
// union's consecutive segments belong to one instance and share its few
// thousand products, so every SM's fixed-point atomics would hit the same
// addresses at once; there chunk c is remapped to c * perm_a mod #chunks
// (perm_a coprime to #chunks: a bijection) and concurrent warps work on
// segments spread over all instances.
struct SegOrder {
  long long nchunks, nwarps, first, pc, step;
  int g;
  __device__ SegOrder(long long L, int W, long long perm_a, long long perm_d) {
    const long long C = 32 / W;
    nchunks = (L + C - 1) / C;
    nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    first = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    g = (int)((threadIdx.x & 31) / W);
    pc = perm_a ? (first * perm_a) % (nchunks > 0 ? nchunks : 1) : first;
    step = perm_a ? perm_d : nwarps;
    C_ = C;
    perm_ = perm_a != 0;
  }
  // segment of this lane's group in the current chunk; advances to the next chunk
  __device__ long long next() {
    const long long l = pc * C_ + g;
    pc += step;
    if (perm_ && pc >= nchunks) pc -= nchunks;
    return l;
  }
  long long C_;
  bool perm_;
};

// One segment of the certified-decision pass (see the file comment): the
// binary32 Dinkelbach decision with its certificate (binary64 redo when it
// fails), binary64 values, and the fixed-point sales added to sums[j - base]
// (none when sums is null); mg = the margins (global or shared memory).
// Called by all W lanes of the segment's group. The lane's slot p (product
// lane + p W of the set) is sp[p T], vv[p T], vtv[p T] with T = W for the CSR
// layout (slot valid iff lane + p W < lim = K) and T = 32 for the slot-major
// layout (slot valid iff p < lim = the chunk's slot rows and its id >= 0).
// rp: the segment's carried Dinkelbach ratio (or null); zs: where to write its
// value (or null: added to zacc). ZV: form the value at all (see below).
template <int W, int P, bool SL, bool ZV>
__device__ __forceinline__ void seg_solve(const FastArgs& A, const double* __restrict__ mg,
                                          const int* __restrict__ sp, const double* __restrict__ vv,
                                          const double* __restrict__ vtv, int lim, double lam, double vt0, float* rp,
                                          double* zs, int lane, unsigned gmask, unsigned long long* sums, int base,
                                          double& zacc, int& fallbacks) {
  constexpr int T = SL ? 32 : W;
  // Registers hold the binary32 images a = m v, b = vt and the product ids;
  // the binary64 values are read again (L1) for the products chosen.
  int jv[P];
  float af[P], bf[P];
  unsigned cand = 0;
  bool ok = true;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    jv[p] = 0;
    af[p] = bf[p] = 0.f;
    if (SL ? p < lim : lane + p * W < lim) {
      const int j = SL ? __ldcg(sp + p * T) : sp[p * T];  // slot-major: ids are not read again, keep L1 for v, vt
      if (!SL || j >= 0) {
        jv[p] = j;
        const double m = mg[j];
        if (__double_as_longlong(m) > 0) {  // m_j > 0
          cand |= 1u << p;
          af[p] = f32_trunc(m, ok) * f32_trunc(vv[p * T], ok);
          bf[p] = f32_trunc(vtv[p * T], ok);
        }
      }
    }
  }
  const float vt0f = f32_trunc(vt0, ok);
  // Dinkelbach in binary32, started at the segment's ratio of the previous
  // iteration (any start reaches a fixed point, and every fixed point is
  // optimal; the margins move little between iterations, so this one is
  // usually confirmed by the second pass).
  float R = rp ? (SL ? __ldcg(rp) : *rp) : 0.f;
  unsigned sel = 0xffffffffu;  // no previous set
  bool conv = false;
  for (int it = 0; it < P * W + 3; ++it) {
    unsigned s = 0;
    float N = 0.f, D = 0.f;
#pragma unroll
    for (int p = 0; p < P; ++p)
      if (((cand >> p) & 1u) && af[p] > R * bf[p]) {
        s |= 1u << p;
        N += af[p];
        D += bf[p];
      }
    if (__all_sync(gmask, s == sel)) {
      conv = true;
      break;
    }
#pragma unroll
    for (int o = W >> 1; o > 0; o >>= 1) {
      N += __shfl_xor_sync(gmask, N, o, W);
      D += __shfl_xor_sync(gmask, D, o, W);
    }
    R = __fdividef(N, vt0f + D);
    sel = s;
  }
  if (rp && lane == 0 && conv) *rp = R;
  bool good = ok && conv;
#pragma unroll
  for (int p = 0; p < P; ++p)
    if ((cand >> p) & 1u) {
      const float a = af[p], c = R * bf[p];
      if (!(fabsf(a - c) > kCertDelta * (a + c))) good = false;
    }
  unsigned S = sel;
  if (!__all_sync(gmask, good)) {
    // Not certified: the same iteration in binary64.
    if (lane == 0) ++fallbacks;
    double Rd = 0.0;
    unsigned prev = 0xffffffffu;
    for (int it = 0; it < P * W + 2; ++it) {
      unsigned s = 0;
      double N = 0.0, D = 0.0;
#pragma unroll
      for (int p = 0; p < P; ++p)
        if ((cand >> p) & 1u) {
          const double a = mg[jv[p]] * vv[p * T], t = vtv[p * T];
          if (a > Rd * t) {
            s |= 1u << p;
            N += a;
            D += t;
          }
        }
      if (__all_sync(gmask, s == prev)) break;
#pragma unroll
      for (int o = W >> 1; o > 0; o >>= 1) {
        N += __shfl_xor_sync(gmask, N, o, W);
        D += __shfl_xor_sync(gmask, D, o, W);
      }
      Rd = N / (vt0 + D);
      prev = s;
    }
    S = prev;
  }
  // binary64 values of the chosen assortment. The segment's value z = q N* is
  // formed only where it is asked for (evaluation passes, per-segment values of
  // a batch): an iterate pass with product sums leaves sum_l z_l to the dual
  // step, which forms it as sum_j m_j s_j (z_l = sum_j m_j x_lj), and skips N*.
  constexpr bool Z = ZV;  // the launch chose it: no product sums, or per-segment values asked for
  double Nl = 0.0, Dl = 0.0;
#pragma unroll
  for (int p = 0; p < P; ++p)
    if ((S >> p) & 1u) {
      Dl += vtv[p * T];
      if (Z) Nl = fma(mg[jv[p]], vv[p * T], Nl);
    }
#pragma unroll
  for (int o = W >> 1; o > 0; o >>= 1) {
    if (Z) Nl += __shfl_xor_sync(gmask, Nl, o, W);
    Dl += __shfl_xor_sync(gmask, Dl, o, W);
  }
  const double q = quotient(lam, vt0 + Dl);
  if (Z && lane == 0) {
    if (zs) *zs = q * Nl;
    else zacc += q * Nl;
  }
  if (sums) {
#pragma unroll
    for (int p = 0; p < P; ++p)
      if ((S >> p) & 1u) atomicAdd(sums + (jv[p] - base), fixed_product(q, vv[p * T], A.fx_bits));
  }
}

// Walk of a warp over its chunks of the slot-major copy (c = first, first + nw,
// ...): each step returns the chunk's first entry and slot-row count, loads
// the offsets two chunks ahead and asks L2 for the next chunk's slot rows
// (ids, and the values v0, v1), so the rows are on chip when the warp gets to
// them and no offset load stalls the warp.
struct SlWalk {
  const long long* off;
  long long nch, nw, c;
  long long o0, o1, n0, n1;  // offsets of chunk c and of chunk c + nw
  __device__ SlWalk(const long long* off_, long long nch_, long long first, long long nw_)
      : off(off_), nch(nch_), nw(nw_), c(first), o0(0), o1(0), n0(0), n1(0) {
    if (c < nch) {
      o0 = off[c];
      o1 = off[c + 1];
    }
    if (c + nw < nch) {
      n0 = off[c + nw];
      n1 = off[c + nw + 1];
    }
  }
  template <class T0, class T1, class T2>
  __device__ void prefetch_next(const T0* a, const T1* b, const T2* d, int wl) const {
    if (c + nw >= nch) return;
    const int rn = (int)((n1 - n0) >> 5);
    for (int p = 0; p < rn; ++p) {
      const long long e = n0 + wl + 32ll * p;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a + e));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(b + e));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(d + e));
    }
  }
  __device__ void advance() {
    c += nw;
    o0 = n0;
    o1 = n1;
    if (c + nw < nch) {
      n0 = off[c + nw];
      n1 = off[c + nw + 1];
    }
  }
};

// One segment l of the CSR layout.
template <int W, int P, bool ZV = true>
__device__ __forceinline__ void fast_segment(const FastArgs& A, const double* __restrict__ mg, long long l, int lane,
                                             unsigned gmask, unsigned long long* sums, int base, double& zacc,
                                             int& fallbacks) {
  const Problem& Pr = A.P;
  const long long b = Pr.seg_ptr[l];
  const int K = (int)(Pr.seg_ptr[l + 1] - b);
  seg_solve<W, P, false, ZV>(A, mg, Pr.seg_prod + b + lane, Pr.v + b + lane, Pr.vt + b + lane, K, Pr.lam[l], Pr.vt0[l],
                         A.rprev ? A.rprev + l : nullptr, A.z_seg ? A.z_seg + l : nullptr, lane, gmask, sums, base,
                         zacc, fallbacks);
}

// MS = 1 (tilings 2, 3; needs SC == 1): one block of 1024 threads per SM that
// also copies the n binary64 margins into shared memory after the sums, so the
// gather of a segment's margins reads shared memory instead of L2.
// SL = 1 (tiling 3): the slot-major copy, one warp per chunk of 32 / W
// positions, every slot row one contiguous load of the warp.
template <int W, int P, int SC, int MS = 0, int SL = 0, bool ZV = (SC == 0)>
__global__ void __launch_bounds__(MS ? kMsThreads : kFastThreads, MS ? 1 : 2) k_seg_fast(FastArgs A) {
  extern __shared__ unsigned long long acc[];  // [n] product sales (fixed point) when SC == 1; MS: + [n] margins
  __shared__ double sh[32];
  if (A.st && A.st->converged) return;
  const Problem& Pr = A.P;
  const double* mg = A.marg;
  if (SC == 1) {
    double* smg = reinterpret_cast<double*>(acc + Pr.n);
    for (int j = threadIdx.x; j < Pr.n; j += blockDim.x) {
      acc[j] = 0ull;
      if (MS) smg[j] = A.marg[j];
    }
    if (MS) mg = smg;
    __syncthreads();
  }
  const int lane = threadIdx.x & (W - 1);
  const int gbase = (threadIdx.x & 31) & ~(W - 1);
  const unsigned gmask = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << gbase);
  double zacc = 0.0;
  int fallbacks = 0;
  unsigned long long* sums = SC == 0 ? nullptr : (SC == 1 ? acc : A.s_fx);
  if (SL) {
    const int wl = threadIdx.x & 31;
    SlWalk wk(A.sl.off, A.sl.nchunks, (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
              (long long)gridDim.x * (blockDim.x >> 5));
    for (; wk.c < wk.nch; wk.advance()) {
      wk.prefetch_next(A.sl.prod, A.sl.v, A.sl.vt, wl);
      const long long o = wk.o0 + wl;
      const int rows = (int)((wk.o1 - wk.o0) >> 5);
      const long long pos = wk.c * (32 / W) + wl / W;
      seg_solve<W, P, true, ZV>(A, mg, A.sl.prod + o, A.sl.v + o, A.sl.vt + o, rows, __ldcg(A.sl.lam + pos),
                            __ldcg(A.sl.vt0 + pos), A.sl.rprev ? A.sl.rprev + pos : nullptr, nullptr, lane, gmask,
                            sums, 0, zacc, fallbacks);
    }
  } else {
    SegOrder ord(Pr.L, W, A.perm_a, A.perm_d);
    for (long long ch = ord.first; ch < ord.nchunks; ch += ord.nwarps) {
      const long long l = ord.next();
      if (l >= Pr.L) continue;
      if (A.seg_inst && A.inst_conv[A.seg_inst[l]]) continue;  // batch: instance already converged
      fast_segment<W, P, ZV>(A, mg, l, lane, gmask, sums, 0, zacc, fallbacks);
    }
  }
  const double tot = block_sum_d(zacc, sh);
  if (threadIdx.x == 0) A.zpart[blockIdx.x] = tot;
  if (fallbacks && A.fallbacks) atomicAdd(A.fallbacks, (unsigned long long)fallbacks);
  if (SC == 1) {
    __syncthreads();
    unsigned long long* dst = A.part + (size_t)blockIdx.x * Pr.n;
    for (int j = threadIdx.x; j < Pr.n; j += blockDim.x) dst[j] = acc[j];
  }
}

// Instance chunks of a batch (see spfom_segments_bchunk.cu): the same
// segment solves as k_seg_fast, with the fixed-point sales summed in shared
// memory per chunk of one instance's segments and flushed to the global sums
// once per chunk, instead of one global atomic per chosen product.
template <int W, int P>
__global__ void __launch_bounds__(kFastThreads, 2) k_seg_fast_bchunk(FastArgs A) {
  extern __shared__ unsigned long long acc[];  // [kBChunkProducts]
  __shared__ double sh[32];
  if (A.st && A.st->converged) return;
  const int lane = threadIdx.x & (W - 1);
  const int gbase = (threadIdx.x & 31) & ~(W - 1);
  const unsigned gmask = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << gbase);
  const int gpb = blockDim.x / W;
  double zacc = 0.0;
  int fallbacks = 0;
  for (long long c = blockIdx.x; c < A.bc_count; c += gridDim.x) {
    const int bi = A.bc_inst[c];
    if (A.inst_conv[bi]) continue;  // uniform over the block
    const long long l0 = A.bc_seg[c], l1 = A.bc_seg[c + 1];
    const int pb = A.bc_prod_ptr[bi], nb = A.bc_prod_ptr[bi + 1] - pb;
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc[i] = 0ull;
    __syncthreads();
    for (long long l = l0 + threadIdx.x / W; l < l1; l += gpb)
      fast_segment<W, P, false>(A, A.marg, l, lane, gmask, acc, pb, zacc, fallbacks);  // an iterate pass: no values
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
      if (acc[i]) atomicAdd(A.s_fx + pb + i, acc[i]);
  }
  const double tot = block_sum_d(zacc, sh);
  if (threadIdx.x == 0) A.zpart[blockIdx.x] = tot;
  if (fallbacks && A.fallbacks) atomicAdd(A.fallbacks, (unsigned long long)fallbacks);
}

// One segment of the binary32 bulk pass (k_seg_f32): the lane's slot p is
// sp[p T], v32[p T], vt32[p T] with T = W (CSR layout, slot valid iff
// lane + p W < lim = K) or T = 32 (slot-major layout, slot valid iff p < lim =
// the chunk's slot rows and its id >= 0); rp / zs as in seg_solve.
template <int W, int P, int SC, bool SL>
__device__ __forceinline__ void f32_solve(const F32Args& A, const float* __restrict__ mg, const int* __restrict__ sp,
                                          const float* __restrict__ v32, const float* __restrict__ vt32, int lim,
                                          float lam, float vt0, float* rp, double* zs, int lane, unsigned gmask,
                                          unsigned long long* sums, float& zacc) {
  constexpr int T = SL ? 32 : W;
  int jv[P];
  float tv[P], af[P];
  unsigned cand = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    jv[p] = 0;
    tv[p] = af[p] = 0.f;
    if (SL ? p < lim : lane + p * W < lim) {
      jv[p] = sp[p * T];
      af[p] = v32[p * T];
      tv[p] = vt32[p * T];
    }
  }
#pragma unroll
  for (int p = 0; p < P; ++p)
    if (SL ? (p < lim && jv[p] >= 0) : lane + p * W < lim) {
      const float m = mg[jv[p]];
      if (m > 0.f) {
        cand |= 1u << p;
        af[p] = m * af[p];
      } else {
        af[p] = 0.f;
      }
    }
  float R = rp ? *rp : 0.f, Nsel = 0.f, Dsel = 0.f;  // Dinkelbach from the last ratio
  unsigned sel = 0xffffffffu;
  for (int it = 0; it < P * W + 3; ++it) {
    unsigned s = 0;
    float N = 0.f, D = 0.f;
#pragma unroll
    for (int p = 0; p < P; ++p)
      if (((cand >> p) & 1u) && af[p] > R * tv[p]) {
        s |= 1u << p;
        N += af[p];
        D += tv[p];
      }
    if (__all_sync(gmask, s == sel)) break;
#pragma unroll
    for (int o = W >> 1; o > 0; o >>= 1) {
      N += __shfl_xor_sync(gmask, N, o, W);
      D += __shfl_xor_sync(gmask, D, o, W);
    }
    R = __fdividef(N, vt0 + D);
    sel = s;
    Nsel = N;
    Dsel = D;
  }
  if (rp && lane == 0) *rp = R;
  const float q = lam / (vt0 + Dsel);
  if (lane == 0 && zs) *zs = (double)(q * Nsel);  // the sum of z comes from the dual step (sum_j m_j s_j)
  if (SC != 0) {
    for (unsigned msk = sel; msk; msk &= msk - 1) {  // this lane's chosen slots
      const int k = (__ffs(msk) - 1) * T;
      atomicAdd(sums + sp[k], fixed_product32(q, v32[k], A.fx_bits));
    }
  }
}

// Binary32 bulk iteration (the precision-32 mode): the same decision as
// k_seg_fast without certificate, and binary32 values: the final Dinkelbach
// set's N and D give q = lambda / (vt0 + D) and z = q N; the sales are the exact
// products q v rounded once to fixed point. Reads 12 B per nonzero.
// MS = 1 (tilings 7, 8; needs SC == 1): one block of 1024 threads per SM with
// the binary32 margins copied into shared memory after the sums. SL = 1
// (tiling 8): the slot-major copy, one warp per chunk.
template <int W, int P, int SC, int MS = 0, int SL = 0>
__global__ void __launch_bounds__(MS ? kMsThreads : kFastThreads, MS ? 1 : 2) k_seg_f32(F32Args A) {
  extern __shared__ unsigned long long acc[];  // [n] sums when SC == 1; MS: + [n] binary32 margins
  __shared__ double sh[32];
  if (A.st->converged) return;
  const float* mg = A.marg32;
  if (SC == 1) {
    float* smg = reinterpret_cast<float*>(acc + A.n);
    for (int j = threadIdx.x; j < A.n; j += blockDim.x) {
      acc[j] = 0ull;
      if (MS) smg[j] = A.marg32[j];
    }
    if (MS) mg = smg;
    __syncthreads();
  }
  const int lane = threadIdx.x & (W - 1);
  const int gbase = (threadIdx.x & 31) & ~(W - 1);
  const unsigned gmask = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << gbase);
  float zacc = 0.f;
  unsigned long long* sums = SC == 1 ? acc : A.s_fx;
  if (SL && MS) {
    // margins in shared memory: the plain chunk loop (measured faster here than the
    // pipelined walk, whose extra registers cost more than its prefetch gains)
    const int wl = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < A.sl.nchunks; c += nw) {
      const long long o = A.sl.off[c] + wl;
      const int rows = (int)((A.sl.off[c + 1] - A.sl.off[c]) >> 5);
      const long long pos = c * (32 / W) + wl / W;
      f32_solve<W, P, SC, true>(A, mg, A.sl.prod + o, A.sl.v32 + o, A.sl.vt32 + o, rows, A.sl.lam32[pos],
                                A.sl.vt0_32[pos], A.sl.rprev ? A.sl.rprev + pos : nullptr, nullptr, lane, gmask, sums,
                                zacc);
    }
  } else if (SL) {
    // margins from global memory: the pipelined walk with the next chunk's rows prefetched
    const int wl = threadIdx.x & 31;
    SlWalk wk(A.sl.off, A.sl.nchunks, (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
              (long long)gridDim.x * (blockDim.x >> 5));
    for (; wk.c < wk.nch; wk.advance()) {
      wk.prefetch_next(A.sl.prod, A.sl.v32, A.sl.vt32, wl);
      const long long o = wk.o0 + wl;
      const int rows = (int)((wk.o1 - wk.o0) >> 5);
      const long long pos = wk.c * (32 / W) + wl / W;
      f32_solve<W, P, SC, true>(A, mg, A.sl.prod + o, A.sl.v32 + o, A.sl.vt32 + o, rows, A.sl.lam32[pos],
                                A.sl.vt0_32[pos], A.sl.rprev ? A.sl.rprev + pos : nullptr, nullptr, lane, gmask, sums,
                                zacc);
    }
  } else {
    SegOrder ord(A.L, W, A.perm_a, A.perm_d);
    for (long long ch = ord.first; ch < ord.nchunks; ch += ord.nwarps) {
      const long long l = ord.next();
      if (l >= A.L) continue;
      if (A.seg_inst && A.inst_conv[A.seg_inst[l]]) continue;  // batch: instance already converged
      const long long b = A.seg_ptr[l];
      f32_solve<W, P, SC, false>(A, mg, A.seg_prod + b + lane, A.v32 + b + lane, A.vt32 + b + lane,
                                 (int)(A.seg_ptr[l + 1] - b), A.lam32[l], A.vt0_32[l],
                                 A.rprev ? A.rprev + l : nullptr, A.z_seg ? A.z_seg + l : nullptr, lane, gmask, sums,
                                 zacc);
    }
  }
  const double tot = block_sum_d((double)zacc, sh);
  if (threadIdx.x == 0) A.zpart[blockIdx.x] = tot;
  if (SC == 1) {
    __syncthreads();
    unsigned long long* dst = A.part + (size_t)blockIdx.x * A.n;
    for (int j = threadIdx.x; j < A.n; j += blockDim.x) dst[j] = acc[j];
  }
}

// ---------------------------------------------------------------------------
// TMA-staged binary32 kernel. The per-segment work is short and its loads are
// dependent (offsets, then products, then margins), so with the 32 warps per SM
// the registers allow, k_seg_f32 waits on memory. Here the block's next tile of
// segments (<= kTileSegs segments, <= kTileItems products) is copied into shared
// memory by the Tensor Memory Accelerator while the block works on the current
// one: one elected thread issues six 1-D bulk copies (cp.async.bulk) per tile,
// completion is tracked by a transaction-count mbarrier per stage, and two
// stages alternate. Copies start and end on 16-byte boundaries (ranges are
// widened outward; the device arrays carry 4 elements of slack at the end).
// Every wait is bounded: on expiry the block records an error in the device
// state (reported as SPFOM_ETIMEOUT), waits once more, boundedly, for its own
// copies and returns.
constexpr int kTileSegs = 512;
constexpr int kTileItems = 4096;

struct StageLayout {  // byte offsets inside one stage
  static constexpr int segp = 0;                                  // int64 [kTileSegs + 4]
  static constexpr int lam = segp + (kTileSegs + 4) * 8;          // f32 [kTileSegs + 8]
  static constexpr int vt0 = lam + (kTileSegs + 8) * 4;           // f32 [kTileSegs + 8]
  static constexpr int prod = vt0 + (kTileSegs + 8) * 4;          // i32 [kTileItems + 8]
  static constexpr int v = prod + (kTileItems + 8) * 4;           // f32 [kTileItems + 8]
  static constexpr int vt = v + (kTileItems + 8) * 4;             // f32 [kTileItems + 8]
  static constexpr int bytes = vt + (kTileItems + 8) * 4;
};
static_assert(StageLayout::bytes % 16 == 0, "stage size must keep 16-byte alignment");

// Issue the copies of tile t into stage `stage` (called by one thread).
__device__ void issue_tile(const F32Args& A, long long t, unsigned char* stage, unsigned bar) {
  const long long l0 = A.tile_ptr[t], l1 = A.tile_ptr[t + 1];
  const long long b = A.seg_ptr[l0], e = A.seg_ptr[l1];
  const long long sa = l0 & ~1ll, se = (l1 + 2) & ~1ll;  // int64 offsets [l0, l1], widened to 16 B
  const long long fa = l0 & ~3ll, fe = (l1 + 3) & ~3ll;  // f32 per-segment [l0, l1)
  const long long ia = b & ~3ll, ie = (e + 3) & ~3ll;    // 4-byte per-product [b, e)
  const unsigned segb = (unsigned)((se - sa) * 8), fb = (unsigned)((fe - fa) * 4), ib = (unsigned)((ie - ia) * 4);
  // order the block's earlier generic reads of this stage before the async-proxy writes
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(bar, segb + 2 * fb + 3 * ib);
  const unsigned base = smem_addr(stage);
  bulk_g2s(base + StageLayout::segp, A.seg_ptr + sa, segb, bar);
  bulk_g2s(base + StageLayout::lam, A.lam32 + fa, fb, bar);
  bulk_g2s(base + StageLayout::vt0, A.vt0_32 + fa, fb, bar);
  if (ib) {
    bulk_g2s(base + StageLayout::prod, A.seg_prod + ia, ib, bar);
    bulk_g2s(base + StageLayout::v, A.v32 + ia, ib, bar);
    bulk_g2s(base + StageLayout::vt, A.vt32 + ia, ib, bar);
  }
}

template <int W, int P, int SC>
__global__ void __launch_bounds__(kTmaThreads, 1) k_seg_f32_tma(F32Args A) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long bars[2];
  __shared__ double sh[32];
  if (A.st->converged) return;
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem);
  unsigned char* stages = smem + A.acc_bytes;  // acc_bytes is a multiple of 128
  const unsigned bar0 = smem_addr(&bars[0]), bar1 = smem_addr(&bars[1]);
  const long long ntiles = A.ntiles;
  if (threadIdx.x == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (SC == 1)
    for (int j = threadIdx.x; j < A.n; j += blockDim.x) acc[j] = 0ull;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 2; ++k) {
      const long long t = blockIdx.x + (long long)k * gridDim.x;
      if (t < ntiles) issue_tile(A, t, stages + k * StageLayout::bytes, k ? bar1 : bar0);
    }
  }
  const int lane = threadIdx.x & (W - 1);
  const int gbase = (threadIdx.x & 31) & ~(W - 1);
  const unsigned gmask = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << gbase);
  const int gpb = blockDim.x / W, group = threadIdx.x / W;
  float zacc = 0.f;
  bool failed = false;
  int k = 0;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
    const int stg = k & 1;
    unsigned char* S = stages + stg * StageLayout::bytes;
    const bool ok = mbar_wait_bounded(stg ? bar1 : bar0, (unsigned)((k >> 1) & 1), A.wait_limit);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    const long long l0 = A.tile_ptr[t], l1 = A.tile_ptr[t + 1];
    const long long* segp = reinterpret_cast<const long long*>(S + StageLayout::segp) + (l0 & 1);
    const float* lam_s = reinterpret_cast<const float*>(S + StageLayout::lam) + (l0 & 3);
    const float* vt0_s = reinterpret_cast<const float*>(S + StageLayout::vt0) + (l0 & 3);
    const long long ibase = segp[0] & ~3ll;
    const int* prod_s = reinterpret_cast<const int*>(S + StageLayout::prod);
    const float* v_s = reinterpret_cast<const float*>(S + StageLayout::v);
    const float* vt_s = reinterpret_cast<const float*>(S + StageLayout::vt);
    const int nseg = (int)(l1 - l0);
    for (int ls = group; ls < nseg; ls += gpb) {
      if (A.seg_inst && A.inst_conv[A.seg_inst[l0 + ls]]) continue;  // batch: instance converged
      const int b = (int)(segp[ls] - ibase);
      const int K = (int)(segp[ls + 1] - segp[ls]);
      // per slot: a = m v (binary32) for candidates, b = v - w; ids and v are re-read
      // from shared memory by the scatter, so they need no registers here
      float tv[P], af[P];
      unsigned cand = 0;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int kk = lane + p * W;
        tv[p] = af[p] = 0.f;
        if (kk < K) {
          tv[p] = vt_s[b + kk];
          const float m = A.marg32[prod_s[b + kk]];
          if (m > 0.f) {
            cand |= 1u << p;
            af[p] = m * v_s[b + kk];
          }
        }
      }
      const float lam = lam_s[ls], vt0 = vt0_s[ls];
      float R = 0.f, Nsel = 0.f, Dsel = 0.f;
      unsigned sel = 0xffffffffu;
      for (int it = 0; it < P * W + 2; ++it) {
        unsigned s = 0;
        float N = 0.f, D = 0.f;
#pragma unroll
        for (int p = 0; p < P; ++p)
          if (((cand >> p) & 1u) && af[p] > R * tv[p]) {
            s |= 1u << p;
            N += af[p];
            D += tv[p];
          }
        if (__all_sync(gmask, s == sel)) break;
#pragma unroll
        for (int o = W >> 1; o > 0; o >>= 1) {
          N += __shfl_xor_sync(gmask, N, o, W);
          D += __shfl_xor_sync(gmask, D, o, W);
        }
        R = __fdividef(N, vt0 + D);
        sel = s;
        Nsel = N;
        Dsel = D;
      }
      const float q = __fdividef(lam, vt0 + Dsel);
      if (lane == 0) {
        if (A.z_seg) A.z_seg[l0 + ls] = (double)(q * Nsel);
        else zacc += q * Nsel;
      }
      if (SC != 0) {
#pragma unroll
        for (int p = 0; p < P; ++p)
          if ((sel >> p) & 1u) {
            const int kk = b + lane + p * W;
            atomicAdd((SC == 1 ? acc : A.s_fx) + prod_s[kk], fixed_product32(q, v_s[kk], A.fx_bits));
          }
      }
    }
    __syncthreads();  // every thread is done with this stage
    if (threadIdx.x == 0) {
      const long long tn = t + 2ll * gridDim.x;
      if (tn < ntiles) issue_tile(A, tn, S, stg ? bar1 : bar0);
    }
  }
  if (failed) {
    // Record the timeout, give the copies still in flight -- stage k's (the wait
    // that expired) and stage k+1's if that tile was issued -- one more bounded
    // wait each, and leave.
    if (threadIdx.x == 0) {
      atomicExch(&A.st_rw->error, 1);
      const long long t = blockIdx.x + (long long)k * gridDim.x;
      mbar_wait_bounded((k & 1) ? bar1 : bar0, (unsigned)((k >> 1) & 1));
      if (t + gridDim.x < ntiles) mbar_wait_bounded(((k + 1) & 1) ? bar1 : bar0, (unsigned)(((k + 1) >> 1) & 1));
    }
    return;
  }
  const double tot = block_sum_d((double)zacc, sh);
  if (threadIdx.x == 0) A.zpart[blockIdx.x] = tot;
  if (SC == 1) {
    __syncthreads();
    unsigned long long* dst = A.part + (size_t)blockIdx.x * A.n;
    for (int j = threadIdx.x; j < A.n; j += blockDim.x) dst[j] = acc[j];
  }
}

// s_fx[j] += sum of one chunk of the per-block partial sums (grid.y chunks).
__global__ void k_reduce_products(int n, int nparts, const unsigned long long* __restrict__ part,
                                  unsigned long long* __restrict__ s_fx, const DevState* st) {
  if (st->converged) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int per = (nparts + gridDim.y - 1) / gridDim.y;
  const int b0 = blockIdx.y * per, b1 = min(nparts, b0 + per);
  unsigned long long acc = 0ull;
#pragma unroll 4
  for (int b = b0; b < b1; ++b) acc += __ldcg(part + (size_t)b * n + j);
  if (acc) atomicAdd(s_fx + j, acc);
}

// perm_a coprime to the number of chunks, near 0.382 of it; perm_d = #warps * perm_a mod #chunks.
void set_order(long long L, int W, int grid, bool batch, long long* a, long long* d) {
  *a = *d = 0;
  if (!batch || L <= 0) return;
  const long long C = 32 / W, nch = (L + C - 1) / C;
  if (nch < 3) return;
  auto gcd = [](long long x, long long y) {
    while (y) {
      const long long t = x % y;
      x = y;
      y = t;
    }
    return x;
  };
  long long pa = (long long)(0.381966 * (double)nch);
  if (pa < 1) pa = 1;
  while (gcd(pa, nch) != 1) ++pa;
  const long long nwarps = (long long)grid * (kFastThreads / 32);
  *a = pa;
  *d = (long long)((__int128)nwarps * pa % nch);
}

template <int SC, bool ZV>
cudaError_t launch_fast_wz(const FastArgs& A, int W, int grid, int smem, cudaStream_t s) {
  switch (W) {  // 8 products per lane
    case 1: k_seg_fast<1, 8, SC, 0, 0, ZV><<<grid, kFastThreads, smem, s>>>(A); break;
    case 2: k_seg_fast<2, 8, SC, 0, 0, ZV><<<grid, kFastThreads, smem, s>>>(A); break;
    case 4: k_seg_fast<4, 8, SC, 0, 0, ZV><<<grid, kFastThreads, smem, s>>>(A); break;
    case 8: k_seg_fast<8, 8, SC, 0, 0, ZV><<<grid, kFastThreads, smem, s>>>(A); break;    // sets of 33..64
    case 16: k_seg_fast<16, 8, SC, 0, 0, ZV><<<grid, kFastThreads, smem, s>>>(A); break;  // sets of 65..128
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Segment values are formed by evaluation passes and for the per-segment values
// of a batch; an iterate pass of a single instance leaves them to the dual step.
template <int SC>
cudaError_t launch_fast_w(const FastArgs& A0, int W, int grid, int smem, cudaStream_t s) {
  FastArgs A = A0;
  set_order(A0.P.L, W, grid, A0.seg_inst != nullptr, &A.perm_a, &A.perm_d);
  if constexpr (SC == 0) return launch_fast_wz<0, true>(A, W, grid, smem, s);
  else return A.z_seg ? launch_fast_wz<SC, true>(A, W, grid, smem, s) : launch_fast_wz<SC, false>(A, W, grid, smem, s);
}

template <int SC>
cudaError_t launch_f32_w(const F32Args& A0, int W, int grid, int smem, cudaStream_t s) {
  F32Args A = A0;
  set_order(A0.L, W, grid, A0.seg_inst != nullptr, &A.perm_a, &A.perm_d);
  switch (W) {
    case 1: k_seg_f32<1, 4, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    case 2: k_seg_f32<2, 4, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    case 4: k_seg_f32<4, 4, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    case 8: k_seg_f32<8, 4, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    case 16: k_seg_f32<16, 4, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    case 32: k_seg_f32<32, 4, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int SC>
cudaError_t launch_f32_p16(const F32Args& A0, int W16, int grid, int smem, cudaStream_t s) {
  F32Args A = A0;
  set_order(A0.L, W16, grid, A0.seg_inst != nullptr, &A.perm_a, &A.perm_d);
  switch (W16) {  // 16 products per lane
    case 1: k_seg_f32<1, 16, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    case 2: k_seg_f32<2, 16, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int SC>
cudaError_t launch_f32_p8(const F32Args& A0, int W8, int grid, int smem, cudaStream_t s) {
  F32Args A = A0;
  set_order(A0.L, W8, grid, A0.seg_inst != nullptr, &A.perm_a, &A.perm_d);
  switch (W8) {  // 8 products per lane
    case 1: k_seg_f32<1, 8, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    case 2: k_seg_f32<2, 8, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    case 4: k_seg_f32<4, 8, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    case 8: k_seg_f32<8, 8, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    case 16: k_seg_f32<16, 8, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Margins in shared memory (precision-64 tiling 2, precision-32 tiling 7):
// one block of kMsThreads per SM, shared-memory sums only.
template <bool ZV>
cudaError_t launch_fast_msz(const FastArgs& A, int W8, int grid, int smem, cudaStream_t s) {
  switch (W8) {
    case 1: k_seg_fast<1, 8, 1, 1, 0, ZV><<<grid, kMsThreads, smem, s>>>(A); break;
    case 2: k_seg_fast<2, 8, 1, 1, 0, ZV><<<grid, kMsThreads, smem, s>>>(A); break;
    case 4: k_seg_fast<4, 8, 1, 1, 0, ZV><<<grid, kMsThreads, smem, s>>>(A); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_fast_ms(const FastArgs& A, int W8, int grid, int smem, cudaStream_t s) {
  return A.z_seg ? launch_fast_msz<true>(A, W8, grid, smem, s) : launch_fast_msz<false>(A, W8, grid, smem, s);
}

cudaError_t launch_f32_ms(const F32Args& A, int W8, int grid, int smem, cudaStream_t s) {
  switch (W8) {
    case 1: k_seg_f32<1, 8, 1, 1><<<grid, kMsThreads, smem, s>>>(A); break;
    case 2: k_seg_f32<2, 8, 1, 1><<<grid, kMsThreads, smem, s>>>(A); break;
    case 4: k_seg_f32<4, 8, 1, 1><<<grid, kMsThreads, smem, s>>>(A); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Slot-major tilings (precision-64 tiling 3, precision-32 tiling 8): margins
// in shared memory when they fit (ms_ok), else read from global memory.
template <int W>
cudaError_t launch_fast_sl_w(const FastArgs& A, const FastPlan& pl, cudaStream_t s) {
  if (pl.ms_ok) k_seg_fast<W, 8, 1, 1, 1><<<pl.ms_grid, kMsThreads, pl.ms_smem64, s>>>(A);
  else if (pl.scatter == 1) k_seg_fast<W, 8, 1, 0, 1><<<pl.grid, kFastThreads, pl.smem, s>>>(A);
  else k_seg_fast<W, 8, 2, 0, 1><<<pl.grid, kFastThreads, 0, s>>>(A);
  return cudaGetLastError();
}

template <int W>
cudaError_t launch_f32_sl_w(const F32Args& A, const FastPlan& pl, cudaStream_t s) {
  if (pl.ms_ok) k_seg_f32<W, 8, 1, 1, 1><<<pl.ms_grid32, kMsThreads, pl.ms_smem32, s>>>(A);
  else if (pl.scatter == 1) k_seg_f32<W, 8, 1, 0, 1><<<pl.grid32, kFastThreads, pl.smem, s>>>(A);
  else k_seg_f32<W, 8, 2, 0, 1><<<pl.grid32, kFastThreads, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_fast_sl(const FastArgs& A, const FastPlan& pl, cudaStream_t s) {
  switch (pl.W8) {
    case 1: return launch_fast_sl_w<1>(A, pl, s);
    case 2: return launch_fast_sl_w<2>(A, pl, s);
    case 4: return launch_fast_sl_w<4>(A, pl, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_f32_sl(const F32Args& A, const FastPlan& pl, cudaStream_t s) {
  switch (pl.W8) {
    case 1: return launch_f32_sl_w<1>(A, pl, s);
    case 2: return launch_f32_sl_w<2>(A, pl, s);
    case 4: return launch_f32_sl_w<4>(A, pl, s);
    default: return cudaErrorInvalidValue;
  }
}

// Shared-memory limits of the slot-major kernels (W8 lanes), as the plan needs them.
template <int W>
bool sl_attributes(const FastPlan& pl) {
  bool ok = true;
  if (pl.ms_ok) {
    ok &= kernel_smem(k_seg_fast<W, 8, 1, 1, 1>, pl.ms_smem64) == cudaSuccess;
    ok &= kernel_smem(k_seg_f32<W, 8, 1, 1, 1>, pl.ms_smem32) == cudaSuccess;
  }
  if (pl.scatter == 1) {
    ok &= kernel_smem(k_seg_fast<W, 8, 1, 0, 1>, pl.smem) == cudaSuccess;
    ok &= kernel_smem(k_seg_f32<W, 8, 1, 0, 1>, pl.smem) == cudaSuccess;
  }
  return ok;
}

template <int SC>
cudaError_t launch_tma_w(const F32Args& A, int W, int grid, int smem, cudaStream_t s) {
  switch (W) {  // 8 products per lane
    case 1: k_seg_f32_tma<1, 8, SC><<<grid, kTmaThreads, smem, s>>>(A); break;
    case 2: k_seg_f32_tma<2, 8, SC><<<grid, kTmaThreads, smem, s>>>(A); break;
    case 4: k_seg_f32_tma<4, 8, SC><<<grid, kTmaThreads, smem, s>>>(A); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class K>
int blocks_per_sm(K kernel, int smem, int threads = kFastThreads) {
  return kernel_blocks(kernel, threads, smem);
}

// The shared-memory limit of the variants that form segment values (a batch's
// per-segment values), which occupancy() and ms_blocks() do not query.
bool zv_attributes(int W8, int smem, int ms_smem) {
  bool ok = true;
  auto set = [&](auto k, int bytes) {
    if (bytes > 0) ok &= kernel_smem(k, bytes) == cudaSuccess;
  };
  if (W8 == 1) { set(k_seg_fast<1, 8, 1, 0, 0, true>, smem); set(k_seg_fast<1, 8, 1, 1, 0, true>, ms_smem); }
  if (W8 == 2) { set(k_seg_fast<2, 8, 1, 0, 0, true>, smem); set(k_seg_fast<2, 8, 1, 1, 0, true>, ms_smem); }
  if (W8 == 4) { set(k_seg_fast<4, 8, 1, 0, 0, true>, smem); set(k_seg_fast<4, 8, 1, 1, 0, true>, ms_smem); }
  return ok;
}

// Blocks per SM of the margins-in-shared kernels (binary64 or binary32).
int ms_blocks(int W8, int smem, bool f32) {
  if (W8 == 1) return f32 ? blocks_per_sm(k_seg_f32<1, 8, 1, 1>, smem, kMsThreads)
                          : blocks_per_sm(k_seg_fast<1, 8, 1, 1>, smem, kMsThreads);
  if (W8 == 2) return f32 ? blocks_per_sm(k_seg_f32<2, 8, 1, 1>, smem, kMsThreads)
                          : blocks_per_sm(k_seg_fast<2, 8, 1, 1>, smem, kMsThreads);
  if (W8 == 4) return f32 ? blocks_per_sm(k_seg_f32<4, 8, 1, 1>, smem, kMsThreads)
                          : blocks_per_sm(k_seg_fast<4, 8, 1, 1>, smem, kMsThreads);
  return 0;
}

int occupancy(int W, int sc, int smem, bool f32) {
#define SPFOM_OCC32(WW)                                                                        \
  if (f32 && W == WW)                                                                          \
    return sc == 1 ? blocks_per_sm(k_seg_f32<WW, 4, 1>, smem) : blocks_per_sm(k_seg_f32<WW, 4, 2>, 0);
#define SPFOM_OCC64(WW)                                                                        \
  if (!f32 && W == WW)                                                                         \
    return sc == 0 ? blocks_per_sm(k_seg_fast<WW, 8, 0>, 0)                                   \
                   : (sc == 1 ? blocks_per_sm(k_seg_fast<WW, 8, 1>, smem)                     \
                              : blocks_per_sm(k_seg_fast<WW, 8, 2>, 0));
  SPFOM_OCC32(1)
  SPFOM_OCC32(2)
  SPFOM_OCC32(4)
  SPFOM_OCC32(8)
  SPFOM_OCC32(16)
  SPFOM_OCC32(32)
  SPFOM_OCC64(1)
  SPFOM_OCC64(2)
  SPFOM_OCC64(4)
  SPFOM_OCC64(8)
  SPFOM_OCC64(16)
#undef SPFOM_OCC32
#undef SPFOM_OCC64
  return 0;
}

}  // namespace

bool fast_plan(int n, int kmax, int sms, FastPlan* plan) {
  if (kmax > kFastMaxSet) return false;
  int W = 1, W8 = 1;
  while (W * 4 < kmax) W <<= 1;
  while (W8 * 8 < kmax) W8 <<= 1;
  const int smem = n * (int)sizeof(unsigned long long);
  const int sc = smem <= kFastMaxSmem ? 1 : 2;
  const int nb = occupancy(W8, sc, smem, false);
  const int nb32 = occupancy(W, sc, smem, true);
  const int nbe = occupancy(W8, 0, 0, false);
  if (nb <= 0 || nbe <= 0 || nb32 <= 0) return false;
  if (sc == 1) {  // the 8- and 16-products-per-lane binary32 variants share the grid of the 4-per-lane one
    kernel_smem(k_seg_f32<1, 8, 1>, smem);
    kernel_smem(k_seg_f32<2, 8, 1>, smem);
    kernel_smem(k_seg_f32<4, 8, 1>, smem);
    kernel_smem(k_seg_f32<8, 8, 1>, smem);
    kernel_smem(k_seg_f32<16, 8, 1>, smem);
    kernel_smem(k_seg_f32<1, 16, 1>, smem);
    kernel_smem(k_seg_f32<2, 16, 1>, smem);
  }
  // margins in shared memory after the sums: 16 n (binary64) or 12 n (binary32) bytes
  plan->ms_ok = 0;
  if (sc == 1 && W8 <= 4 && 16ll * n <= kTmaMaxSmem) {
    const int b64 = ms_blocks(W8, 16 * n, false), b32 = ms_blocks(W8, 12 * n, true);
    if (b64 >= 1 && b32 >= 1) {
      plan->ms_ok = 1;
      plan->ms_smem64 = 16 * n;
      plan->ms_smem32 = 12 * n;
      plan->ms_grid = b64 * sms;
      plan->ms_grid32 = b32 * sms;
    }
  }
  {  // slot-major kernels: the same grids as their CSR counterparts (equal register and shared-memory needs)
    FastPlan q = *plan;
    q.W8 = W8;
    q.scatter = sc;
    q.smem = sc == 1 ? smem : 0;
    plan->sl_attr = W8 == 1 ? sl_attributes<1>(q) : (W8 == 2 ? sl_attributes<2>(q) : sl_attributes<4>(q));
  }
  if (!zv_attributes(W8, sc == 1 ? smem : 0, plan->ms_ok ? plan->ms_smem64 : 0)) return false;
  plan->W16 = kmax <= 16 ? 1 : 2;
  plan->W = W;
  plan->W8 = W8;
  plan->scatter = sc;
  plan->smem = sc == 1 ? smem : 0;
  plan->grid = nb * sms;
  plan->grid32 = nb32 * sms;
  plan->grid_eval = nbe * sms;
  plan->reduce_chunks = 16;
  return true;
}

cudaError_t launch_seg_fast(const FastArgs& A, const FastPlan& plan, bool scatter, cudaStream_t s) {
  if (scatter && plan.bchunk64_ok && A.bc_count > 0) {
    switch (plan.W8) {
      case 1: k_seg_fast_bchunk<1, 8><<<plan.bchunk64_grid, kFastThreads, plan.bchunk_smem, s>>>(A); break;
      case 2: k_seg_fast_bchunk<2, 8><<<plan.bchunk64_grid, kFastThreads, plan.bchunk_smem, s>>>(A); break;
      case 4: k_seg_fast_bchunk<4, 8><<<plan.bchunk64_grid, kFastThreads, plan.bchunk_smem, s>>>(A); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  if (!scatter) return launch_fast_w<0>(A, plan.W8, plan.grid_eval, 0, s);
  if (plan.fast_sl && A.sl.nchunks > 0) return launch_fast_sl(A, plan, s);
  if (plan.fast_ms && plan.ms_ok) return launch_fast_ms(A, plan.W8, plan.ms_grid, plan.ms_smem64, s);
  return plan.scatter == 1 ? launch_fast_w<1>(A, plan.W8, plan.grid, plan.smem, s)
                           : launch_fast_w<2>(A, plan.W8, plan.grid, 0, s);
}

cudaError_t launch_seg_f32(const F32Args& A, const FastPlan& plan, cudaStream_t s) {
  if (plan.bchunk && A.bc_count > 0) return launch_seg_f32_bchunk(A, plan, s);
  if (plan.coop) return launch_seg_f32_coop(A, plan, s);
  if (plan.tma)
    return plan.scatter == 1 ? launch_tma_w<1>(A, plan.tma_W, plan.tma_grid, plan.tma_smem, s)
                             : launch_tma_w<2>(A, plan.tma_W, plan.tma_grid, plan.tma_smem, s);
  if (plan.f32_sl && A.sl.nchunks > 0) return launch_f32_sl(A, plan, s);
  if (plan.f32_ms && plan.ms_ok) return launch_f32_ms(A, plan.W8, plan.ms_grid32, plan.ms_smem32, s);
  if (plan.f32_p16)
    return plan.scatter == 1 ? launch_f32_p16<1>(A, plan.W16, plan.grid32, plan.smem, s)
                             : launch_f32_p16<2>(A, plan.W16, plan.grid32, 0, s);
  if (plan.f32_p8)
    return plan.scatter == 1 ? launch_f32_p8<1>(A, plan.W8, plan.grid32, plan.smem, s)
                             : launch_f32_p8<2>(A, plan.W8, plan.grid32, 0, s);
  return plan.scatter == 1 ? launch_f32_w<1>(A, plan.W, plan.grid32, plan.smem, s)
                           : launch_f32_w<2>(A, plan.W, plan.grid32, 0, s);
}

bool tma_plan(int n, int kmax, int sms, FastPlan* plan) {
  int W8 = 1;  // lanes per segment with 8 products per lane
  while (W8 * 8 < kmax) W8 <<= 1;
  if (W8 > 4) return false;
  const int acc = plan->scatter == 1 ? ((n * 8 + 127) / 128) * 128 : 0;
  const int smem = acc + 2 * StageLayout::bytes;
  if (smem > kTmaMaxSmem) return false;
  int nb = 0;
#define SPFOM_TMA_OCC(WW)                                                                                   \
  if (W8 == WW) {                                                                                           \
    if (plan->scatter == 1) {                                                                               \
      nb = kernel_blocks(k_seg_f32_tma<WW, 8, 1>, kTmaThreads, smem);                                     \
    } else {                                                                                                \
      nb = kernel_blocks(k_seg_f32_tma<WW, 8, 2>, kTmaThreads, smem);                                     \
    }                                                                                                       \
  }
  SPFOM_TMA_OCC(1)
  SPFOM_TMA_OCC(2)
  SPFOM_TMA_OCC(4)
#undef SPFOM_TMA_OCC
  if (nb < 1) return false;
  plan->tma = 1;
  plan->tma_ok = 1;
  plan->tma_W = W8;
  plan->tma_smem = smem;
  plan->acc_bytes = acc;
  plan->tma_grid = nb * sms;
  return true;
}

// Tiles of consecutive segments with at most kTileSegs segments and kTileItems
// products each (host side; seg_ptr is the caller's host array).
bool bchunk64_plan(int max_inst_products, int sms, FastPlan* plan) {
  if (plan->W8 > 4 || max_inst_products > kBChunkProducts) return false;
  const int smem = kBChunkProducts * (int)sizeof(unsigned long long);
  int nb = 0;
#define SPFOM_BC64(WW)                                                                                   \
  if (plan->W8 == WW) {                                                                                  \
    nb = kernel_blocks(k_seg_fast_bchunk<WW, 8>, kFastThreads, smem);                                    \
  }
  SPFOM_BC64(1)
  SPFOM_BC64(2)
  SPFOM_BC64(4)
#undef SPFOM_BC64
  if (nb < 1) return false;
  plan->bchunk64_ok = 1;
  plan->bchunk_smem = smem;
  plan->bchunk64_grid = nb * sms;
  return true;
}

long long make_tiles(const long long* seg_ptr, long long L, long long* tiles_out) {
  long long nt = 0, l = 0;
  if (tiles_out) tiles_out[0] = 0;
  while (l < L) {
    long long e = l;
    while (e < L && e - l < kTileSegs && seg_ptr[e + 1] - seg_ptr[l] <= kTileItems) ++e;
    if (e == l) e = l + 1;  // a single segment never exceeds kTileItems (sets hold <= 32 products)
    ++nt;
    if (tiles_out) tiles_out[nt] = e;
    l = e;
  }
  return nt;
}

cudaError_t launch_reduce_products(const Problem& P, const FastPlan& plan, int nparts,
                                   const unsigned long long* part, unsigned long long* s_fx, const DevState* st,
                                   cudaStream_t s) {
  if (P.n <= 0 || plan.scatter != 1) return cudaSuccess;
  dim3 grid((P.n + 255) / 256, plan.reduce_chunks);
  k_reduce_products<<<grid, 256, 0, s>>>(P.n, nparts, part, s_fx, st);
  return cudaGetLastError();
}

}  // namespace spfom
