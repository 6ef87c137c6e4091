// Device helpers shared by the segment kernels (spfom_segments_fast.cu,
// spfom_segments_tma.cu): binary32 images of binary64 values, fixed-point
// products, the reciprocal-seed quotient, block sums, and the mbarrier /
// bulk-copy primitives of the TMA tile staging.
#pragma once
#include <cuda_runtime.h>

namespace spfom {
namespace {

constexpr unsigned kWaitLimit = 1u << 22;  // try_wait polls before a staged-copy wait gives up

constexpr float kCertDelta = 1.52587890625e-05f;  // 2^-16

// binary32 image of a non-negative binary64, by dropping the low 29 mantissa
// bits and rebiasing the exponent (no conversion instruction; relative error
// below 2^-23). Zero maps to zero; ok is cleared for values outside binary32's
// normal range and for negative values.
__device__ __forceinline__ float f32_trunc(double d, bool& ok) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  if ((hi | lo) == 0u) return 0.f;
  ok &= ((hi >> 20) - 897u) < 254u;
  return __uint_as_float(__funnelshift_l(lo, hi, 3) - 0xC0000000u);
}

// round(a * b * 2^F) for positive normal binary64 a, b with a * b * 2^F < 2^62,
// from the 53-bit significands on the integer unit (one rounding, of the exact
// product). a = ma 2^(ea - 1075), b = mb 2^(eb - 1075) with biased exponents ea, eb.
__device__ __forceinline__ unsigned long long fixed_product(double a, double b, int F) {
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
  const unsigned long long ub = (unsigned long long)__double_as_longlong(b);
  const unsigned long long ma = (ua & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const unsigned long long mb = (ub & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const int sh = 2150 - F - (int)(ua >> 52) - (int)(ub >> 52);  // a b 2^F = ma mb / 2^sh
  if (sh < 43 || sh > 126) return 0ull;  // sh < 43 cannot occur below 2^62; sh > 126 rounds to 0
  unsigned long long lo = ma * mb, hi = __umul64hi(ma, mb);
  if (sh <= 64) {
    const unsigned long long half = 1ull << (sh - 1);
    lo += half;
    hi += (lo < half) ? 1ull : 0ull;
  } else {
    hi += 1ull << (sh - 65);
  }
  return sh < 64 ? (hi << (64 - sh)) | (lo >> sh) : (hi >> (sh - 64));
}

// lam / d for positive normal d: binary32 reciprocal seed (24 bits, from the
// integer image of d), two binary64 Newton steps r <- r + r (1 - d r), then one
// product (a few ulps from the correctly rounded quotient).
__device__ __forceinline__ double quotient(double lam, double d) {
  bool ok = true;
  const float r32 = __frcp_rn(f32_trunc(d, ok));
  const unsigned rb = __float_as_uint(r32);
  // widen the binary32 seed to binary64: rebias the exponent, shift the significand
  double r = __hiloint2double((int)(((rb >> 23) + 896u) << 20 | ((rb & 0x7FFFFFu) >> 3)), (int)(rb << 29));
  if (!ok) r = 1.0 / d;
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  return lam * r;
}

__device__ double block_sum_d(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)((blockDim.x + 31) >> 5); ++k) tot += sh[k];
  return tot;
}

// round(a * b * 2^F) for non-negative binary32 a, b with a * b * 2^F < 2^62: the
// 48-bit product of the significands is exact in 64 bits, so the only
// rounding is the final one. a = ma 2^(ea - 150), b = mb 2^(eb - 150).
__device__ __forceinline__ unsigned long long fixed_product32(float a, float b, int F) {
  const unsigned ua = __float_as_uint(a), ub = __float_as_uint(b);
  const int ea = (int)(ua >> 23), eb = (int)(ub >> 23);
  if (ea == 0 || eb == 0) return 0ull;  // zero or subnormal: far below the fixed-point unit
  const unsigned long long prod =
      (unsigned long long)((ua & 0x7FFFFFu) | 0x800000u) * (unsigned long long)((ub & 0x7FFFFFu) | 0x800000u);
  const int sh = 300 - F - ea - eb;  // a b 2^F = prod / 2^sh
  if (sh <= 0) return prod << (-sh);
  if (sh > 63) return 0ull;
  return (prod + (1ull << (sh - 1))) >> sh;
}

// (hi, lo) pair of a binary64 value: hi = round(x), lo = round(x - hi). A
// nonzero value outside [1e-30, 1e30] in magnitude gets hi = NaN, which makes
// the certificate of the double-float kernel fail (binary64 fallback).
__device__ __forceinline__ float2 split_pair(double x) {
  const double ax = fabs(x);
  if (x != 0.0 && !(ax >= 1e-30 && ax <= 1e30)) return make_float2(__int_as_float(0x7fc00000), 0.f);
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

// Step factor of a restart forced by the epoch-length rule (restart_tau_balance
// = b > 0): clamp(sqrt(pinf / gap), b, 1 / b), 1 when either residual is 0.
__device__ __forceinline__ double balance_factor(double pinf, double gap, double b) {
  double f = (pinf > 0.0 && gap > 0.0) ? sqrt(pinf / gap) : 1.0;
  const double hi = 1.0 / b;
  f = f < b ? b : f;
  return f > hi ? hi : f;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0u;
}
// limit: polls before giving up (kWaitLimit unless a test lowers it; the waits
// that let a failing block's own copies land always use kWaitLimit)
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, unsigned limit = kWaitLimit) {
  for (unsigned it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}


__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

}  // namespace
}  // namespace spfom
