// Precision-64 segment kernel without binary64 arithmetic in the common case:
// binary32 decisions with a certificate (as in k_seg_fast) and the values in
// double-binary32 ("double-float") arithmetic.
//
// GB300 runs binary64 at about 1/60 of the binary32 rate, so in k_seg_fast the
// binary64 sums of the chosen products (N = sum m_j v_j, D = sum vt_j: one add
// and one multiply-add per product slot) and the per-segment quotient keep the
// binary64 pipe busy while HBM idles. Here every binary64 input is stored as
// an unevaluated pair of binary32 numbers (hi = round(x), lo = round(x - hi)),
// written once at load for the attractions, lambda and vt_0, and per iteration
// for the margins, in the same 8 bytes per value. The decision (Dinkelbach on
// the hi parts, certified by the relative margin 2^-16, Section 4.1 inner
// problem with Lemma 1's ordering) is k_seg_fast's; the values are computed
// with error-free transformations (TwoSum, FMA-based TwoProduct) on the pairs:
//   N = sum_{S*} m_j v_j and D = vt_0 + sum_{S*} vt_j  (double-float sums),
//   q = lambda / D  (double-float quotient: binary32 estimate + one correction),
//   z = q N,  x_j = q v_j rounded once to the fixed-point unit 2^-F.
// A pair carries 48 significand bits; each operation adds at most a few units
// of 2^-46 relative error, so values agree with binary64 arithmetic to about
// 1e-13 relative. Uncertified segments (a near-tie, or an input outside
// binary32's normal range, marked by a NaN hi part) repeat the decision and
// the values in binary64 from the binary64 arrays, as k_seg_fast does.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "spfom_device.cuh"
#include "spfom_internal.h"

namespace spfom {

namespace {

// ---- double-float primitives (each result is hi + lo, |lo| <= ulp(hi) / 2) ----

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b|
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ float2 dd_add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  float h, l;
  fast_two_sum(s, e, h, l);
  return make_float2(h, l);
}

__device__ __forceinline__ float2 dd_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  float h, l;
  fast_two_sum(p, e, h, l);
  return make_float2(h, l);
}

// a / b for b > 0: binary32 quotient, its residual in double-float, one correction.
__device__ __forceinline__ float2 dd_div(float2 a, float2 b) {
  const float r = __frcp_rn(b.x);
  const float q1 = __fmul_rn(a.x, r);
  // a - q1 b, with q1 b = p + pe exactly (TwoProduct) plus q1 b.lo
  const float p = __fmul_rn(q1, b.x);
  const float pe = __fmaf_rn(q1, b.x, -p);
  float res = __fsub_rn(a.x, p);  // exact: p is within a few ulps of a.x
  res = __fsub_rn(res, pe);
  res = __fadd_rn(res, a.y);
  res = __fmaf_rn(-q1, b.y, res);
  const float q2 = __fmul_rn(res, r);
  float h, l;
  fast_two_sum(q1, q2, h, l);
  return make_float2(h, l);
}

__device__ __forceinline__ double dd_to_double(float2 a) { return (double)a.x + (double)a.y; }

// round(c * 2^F) for a signed binary32 c whose magnitude is far below 2^(62 - F).
__device__ __forceinline__ long long fixed_signed32(float c, int F) {
  const unsigned u = __float_as_uint(c);
  const int e = (int)((u >> 23) & 0xFFu);
  if (e == 0) return 0;  // zero or subnormal: far below the fixed-point unit
  const long long m = (long long)((u & 0x7FFFFFu) | 0x800000u);
  const int sh = 150 - F - e;  // |c| 2^F = m / 2^sh
  long long v;
  if (sh <= 0) v = m << (-sh);
  else if (sh > 30) v = 0;
  else v = (m + (1ll << (sh - 1))) >> sh;
  return (u >> 31) ? -v : v;
}

// round(q v 2^F) for double-float q, v > 0: the exact product of the hi parts,
// rounded once (fixed_product32), plus the first-order cross terms, rounded.
__device__ __forceinline__ unsigned long long fixed_dd(float2 q, float2 v, int F) {
  const unsigned long long a = fixed_product32(q.x, v.x, F);
  const float c = __fmaf_rn(q.x, v.y, __fmul_rn(q.y, v.x));
  return a + (unsigned long long)fixed_signed32(c, F);
}

template <int W, int P, int SC, int MINB>
__global__ void __launch_bounds__(kFastThreads, MINB) k_seg_dd(DdArgs A) {
  extern __shared__ unsigned long long acc[];  // [n] product sales (fixed point) when SC == 1
  __shared__ double sh[32];
  if (A.st && A.st->converged) return;
  if (SC == 1) {
    for (int j = threadIdx.x; j < A.n; j += blockDim.x) acc[j] = 0ull;
    __syncthreads();
  }
  const int lane = threadIdx.x & (W - 1);
  const int gbase = (threadIdx.x & 31) & ~(W - 1);
  const unsigned gmask = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << gbase);
  const long long gpb = blockDim.x / W;
  const long long ngroups = (long long)gridDim.x * gpb;
  float2 zacc = make_float2(0.f, 0.f);
  int fallbacks = 0;
  long long l = blockIdx.x * gpb + threadIdx.x / W;
  long long nb = 0, ne = 0;  // bounds of the group's next segment, loaded one segment ahead
  if (l < A.L) {
    nb = A.seg_ptr[l];
    ne = A.seg_ptr[l + 1];
  }
  for (; l < A.L; l += ngroups) {
    const long long b = nb;
    const int K = (int)(ne - nb);
    if (l + ngroups < A.L) {
      nb = A.seg_ptr[l + ngroups];
      ne = A.seg_ptr[l + ngroups + 1];
    }
    if (A.seg_inst && A.inst_conv[A.seg_inst[l]]) continue;  // batch: instance already converged
    int jv[P];
    float af[P], bf[P];
    unsigned cand = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int k = lane + p * W;
      jv[p] = 0;
      af[p] = bf[p] = 0.f;
      if (k < K) {
        jv[p] = A.seg_prod[b + k];
        const float mh = A.marg2[jv[p]].x;
        if (!(mh <= 0.f)) {  // m_j > 0, or NaN: a margin the pair cannot hold (certificate fails)
          cand |= 1u << p;
          af[p] = mh * A.v2[b + k].x;
          bf[p] = A.vt2[b + k].x;
        }
      }
    }
    const float4 sg = A.seg4[l];  // lambda (hi, lo), vt_0 (hi, lo)
    // Dinkelbach in binary32 from R = 0 (as in k_seg_fast)
    float R = 0.f;
    unsigned sel = 0xffffffffu;
    bool conv = false;
    for (int it = 0; it < P * W + 2; ++it) {
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
      R = N / (sg.z + D);
      sel = s;
    }
    bool good = conv && (sg.x == sg.x) && (sg.z == sg.z);
#pragma unroll
    for (int p = 0; p < P; ++p)
      if ((cand >> p) & 1u) {
        const float a = af[p], c = R * bf[p];
        if (!(fabsf(a - c) > kCertDelta * (a + c))) good = false;
      }
    if (__all_sync(gmask, good)) {
      // double-float values of the certified assortment
      float2 Nl = make_float2(0.f, 0.f), Dl = make_float2(0.f, 0.f);
#pragma unroll
      for (int p = 0; p < P; ++p)
        if ((sel >> p) & 1u) {
          const int k = lane + p * W;
          Dl = dd_add(Dl, A.vt2[b + k]);
          Nl = dd_add(Nl, dd_mul(A.marg2[jv[p]], A.v2[b + k]));
        }
#pragma unroll
      for (int o = W >> 1; o > 0; o >>= 1) {
        const float2 on = make_float2(__shfl_xor_sync(gmask, Nl.x, o, W), __shfl_xor_sync(gmask, Nl.y, o, W));
        const float2 od = make_float2(__shfl_xor_sync(gmask, Dl.x, o, W), __shfl_xor_sync(gmask, Dl.y, o, W));
        Nl = dd_add(Nl, on);
        Dl = dd_add(Dl, od);
      }
      const float2 q = dd_div(make_float2(sg.x, sg.y), dd_add(make_float2(sg.z, sg.w), Dl));
      const float2 z = dd_mul(q, Nl);
      if (lane == 0) {
        if (A.z_seg) A.z_seg[l] = dd_to_double(z);
        else zacc = dd_add(zacc, z);
      }
      if (SC != 0) {
#pragma unroll
        for (int p = 0; p < P; ++p)
          if ((sel >> p) & 1u)
            atomicAdd((SC == 1 ? acc : A.s_fx) + jv[p], fixed_dd(q, A.v2[b + lane + p * W], A.fx_bits));
      }
    } else {
      // not certified: the decision and the values in binary64 (k_seg_fast's fallback)
      if (lane == 0) ++fallbacks;
      double Rd = 0.0;
      unsigned prev = 0xffffffffu;
      const double vt0 = A.vt0[l], lam = A.lam[l];
      for (int it = 0; it < P * W + 2; ++it) {
        unsigned s = 0;
        double N = 0.0, D = 0.0;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const int k = lane + p * W;
          if (k < K && A.marg[jv[p]] > 0.0) {
            const double a = A.marg[jv[p]] * A.v[b + k], t = A.vt[b + k];
            if (a > Rd * t) {
              s |= 1u << p;
              N += a;
              D += t;
            }
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
      double Nd = 0.0, Dd = 0.0;
#pragma unroll
      for (int p = 0; p < P; ++p)
        if ((prev >> p) & 1u) {
          const int k = lane + p * W;
          Dd += A.vt[b + k];
          Nd = fma(A.marg[jv[p]], A.v[b + k], Nd);
        }
#pragma unroll
      for (int o = W >> 1; o > 0; o >>= 1) {
        Nd += __shfl_xor_sync(gmask, Nd, o, W);
        Dd += __shfl_xor_sync(gmask, Dd, o, W);
      }
      const double q = quotient(lam, vt0 + Dd);
      if (lane == 0) {
        if (A.z_seg) A.z_seg[l] = q * Nd;
        else zacc = dd_add(zacc, make_float2((float)(q * Nd), (float)(q * Nd - (double)(float)(q * Nd))));
      }
      if (SC != 0) {
#pragma unroll
        for (int p = 0; p < P; ++p)
          if ((prev >> p) & 1u)
            atomicAdd((SC == 1 ? acc : A.s_fx) + jv[p], fixed_product(q, A.v[b + lane + p * W], A.fx_bits));
      }
    }
  }
  const double tot = block_sum_d(dd_to_double(zacc), sh);
  if (threadIdx.x == 0) A.zpart[blockIdx.x] = tot;
  if (fallbacks && A.fallbacks) atomicAdd(A.fallbacks, (unsigned long long)fallbacks);
  if (SC == 1) {
    __syncthreads();
    unsigned long long* dst = A.part + (size_t)blockIdx.x * A.n;
    for (int j = threadIdx.x; j < A.n; j += blockDim.x) dst[j] = acc[j];
  }
}

__global__ void k_split_items(long long nnz, const double* __restrict__ v, const double* __restrict__ vt,
                              float2* __restrict__ v2, float2* __restrict__ vt2) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p < nnz) {
    v2[p] = split_pair(v[p]);
    vt2[p] = split_pair(vt[p]);
  }
}

__global__ void k_split_segments(long long L, const double* __restrict__ lam, const double* __restrict__ vt0,
                                 float4* __restrict__ seg4) {
  const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l < L) {
    const float2 a = split_pair(lam[l]), c = split_pair(vt0[l]);
    seg4[l] = make_float4(a.x, a.y, c.x, c.y);
  }
}

// Tilings (spfom_autotune chooses among them): 1 = 8 products per lane at two
// 512-thread blocks per SM (64 registers), 2 = 8 products per lane at three
// blocks per SM (42 registers), 3 = 4 products per lane at three blocks per SM.
template <int SC, int P, int MINB>
cudaError_t launch_dd_t(const DdArgs& A, int W, int grid, int smem, cudaStream_t s) {
  switch (W) {
    case 1: k_seg_dd<1, P, SC, MINB><<<grid, kFastThreads, smem, s>>>(A); break;
    case 2: k_seg_dd<2, P, SC, MINB><<<grid, kFastThreads, smem, s>>>(A); break;
    case 4: k_seg_dd<4, P, SC, MINB><<<grid, kFastThreads, smem, s>>>(A); break;
    case 8:
      if (P == 4) {
        k_seg_dd<8, P, SC, MINB><<<grid, kFastThreads, smem, s>>>(A);
        break;
      }
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int SC>
cudaError_t launch_dd_w(const DdArgs& A, const FastPlan& plan, int grid, int smem, cudaStream_t s) {
  switch (plan.dd_variant) {
    case 2: return launch_dd_t<SC, 8, 3>(A, plan.W8, grid, smem, s);
    case 3: return launch_dd_t<SC, 4, 3>(A, plan.W, grid, smem, s);
    default: return launch_dd_t<SC, 8, 2>(A, plan.W8, grid, smem, s);
  }
}

template <class Kern>
int dd_blocks(Kern k, int smem) {
  return kernel_blocks(k, kFastThreads, smem);
}

// Blocks per SM of tiling v for scatter mode sc (shared memory smem when sc == 1).
template <int P, int MINB>
int dd_occ(int W, int sc, int smem) {
#define SPFOM_DD_OCC(WW)                                                                             \
  if (W == WW)                                                                                       \
    return sc == 0 ? dd_blocks(k_seg_dd<WW, P, 0, MINB>, 0)                                          \
                   : (sc == 1 ? dd_blocks(k_seg_dd<WW, P, 1, MINB>, smem) : dd_blocks(k_seg_dd<WW, P, 2, MINB>, 0));
  SPFOM_DD_OCC(1)
  SPFOM_DD_OCC(2)
  SPFOM_DD_OCC(4)
  if (P == 4) {
    SPFOM_DD_OCC(8)
  }
#undef SPFOM_DD_OCC
  return 0;
}

}  // namespace

cudaError_t launch_dd_prep(const Problem& P, float2* v2, float2* vt2, float4* seg4, cudaStream_t s) {
  if (P.nnz > 0) k_split_items<<<(unsigned)((P.nnz + 255) / 256), 256, 0, s>>>(P.nnz, P.v, P.vt, v2, vt2);
  if (P.L > 0) k_split_segments<<<(unsigned)((P.L + 255) / 256), 256, 0, s>>>(P.L, P.lam, P.vt0, seg4);
  return cudaGetLastError();
}

cudaError_t launch_seg_dd(const DdArgs& A, const FastPlan& plan, bool scatter, cudaStream_t s) {
  const int v = plan.dd_variant >= 1 && plan.dd_variant <= 3 ? plan.dd_variant : 1;
  if (!scatter) return launch_dd_w<0>(A, plan, plan.dd_grid_eval[v], 0, s);
  return plan.scatter == 1 ? launch_dd_w<1>(A, plan, plan.dd_grid[v], plan.smem, s)
                           : launch_dd_w<2>(A, plan, plan.dd_grid[v], 0, s);
}

bool dd_setup(FastPlan* plan, int sms) {
  const int sc = plan->scatter, smem = plan->smem;
  const int occ[4][2] = {{0, 0},
                         {dd_occ<8, 2>(plan->W8, sc, smem), dd_occ<8, 2>(plan->W8, 0, 0)},
                         {dd_occ<8, 3>(plan->W8, sc, smem), dd_occ<8, 3>(plan->W8, 0, 0)},
                         {dd_occ<4, 3>(plan->W, sc, smem), dd_occ<4, 3>(plan->W, 0, 0)}};
  for (int v = 1; v <= 3; ++v) {
    plan->dd_grid[v] = occ[v][0] * sms;
    plan->dd_grid_eval[v] = occ[v][1] * sms;
  }
  plan->dd_grid[0] = plan->dd_grid_eval[0] = 0;
  plan->dd_variant = 1;
  return occ[1][0] > 0 && occ[1][1] > 0;
}

int dd_variant_ok(const FastPlan& plan, int v) {
  return v >= 1 && v <= 3 && plan.dd_grid[v] > 0 && plan.dd_grid_eval[v] > 0;
}

}  // namespace spfom
