// Binary64 certified-decision segment pass fed by a warp-specialised TMA
// pipeline (precision 64, full batch).
//
// The certified kernel (k_seg_fast) waits on chains of dependent global loads
// (offsets, products, then the binary64 values of the chosen products). Here a
// producer warp streams tiles of consecutive segments (<= kTile64Segs segments,
// <= kTile64Items products) into shared memory with 1-D bulk copies
// (cp.async.bulk, completion counted in bytes on a "full" mbarrier per stage),
// and fifteen consumer warps solve the tile's segments from shared memory. A
// consumer warp releases a stage by arriving on its "empty" mbarrier (one
// arrival per consumer warp); the producer refills a stage once all consumer
// warps have released it. Warps therefore never meet at a block-wide barrier
// inside the loop: a slow segment (a binary64 redo) delays only the refill of
// its own stage, with kStages - 1 tiles of slack.
//
// Copies start and end on 16-byte boundaries (ranges widened outward; the
// device arrays carry zeroed slack at their ends). Every mbarrier wait is
// bounded; on expiry the block records an error in the device state (reported
// as SPFOM_ETIMEOUT), waits boundedly for the copies it issued, and finishes.
//
// The arithmetic per segment is k_seg_fast's: binary32 Dinkelbach decision with
// certificate (binary64 redo when not certified), binary64 values D*, N*,
// q = lambda / D*, z = q N*, fixed-point sales round(q v 2^F).
#include <cuda_runtime.h>
#include <math_constants.h>

#include "spfom_device.cuh"
#include "spfom_internal.h"

namespace spfom {

namespace {

constexpr int kStages = 3;
constexpr int kConsumerWarps = kPipeThreads / 32 - 1;

struct Stage64 {  // byte offsets inside one stage
  static constexpr int segp = 0;                                // int64 [kTile64Segs + 4]
  static constexpr int lam = segp + (kTile64Segs + 4) * 8;      // f64 [kTile64Segs + 4]
  static constexpr int vt0 = lam + (kTile64Segs + 4) * 8;       // f64 [kTile64Segs + 4]
  static constexpr int prod = vt0 + (kTile64Segs + 4) * 8;      // i32 [kTile64Items + 8]
  static constexpr int v = prod + (kTile64Items + 8) * 4;       // f64 [kTile64Items + 4]
  static constexpr int vt = v + (kTile64Items + 4) * 8;         // f64 [kTile64Items + 4]
  static constexpr int bytes = vt + (kTile64Items + 4) * 8;
};
static_assert(Stage64::lam % 16 == 0 && Stage64::vt0 % 16 == 0 && Stage64::prod % 16 == 0 &&
                  Stage64::v % 16 == 0 && Stage64::vt % 16 == 0 && Stage64::bytes % 16 == 0,
              "stage regions must start on 16-byte boundaries");

// Copies of tile t into a stage (one thread). Widened ranges: int64 and f64
// arrays to even indices, 4-byte arrays to multiples of 4.
__device__ void issue_tile64(const FastArgs& A, long long t, unsigned char* stage, unsigned bar) {
  const long long l0 = A.tile_ptr[t], l1 = A.tile_ptr[t + 1];
  const long long b = A.P.seg_ptr[l0], e = A.P.seg_ptr[l1];
  const long long sa = l0 & ~1ll, se = (l1 + 2) & ~1ll;  // seg_ptr [l0, l1]
  const long long la = l0 & ~1ll, le = (l1 + 1) & ~1ll;  // lam, vt0 [l0, l1)
  const long long pa = b & ~3ll, pe = (e + 3) & ~3ll;    // products [b, e)
  const long long da = b & ~1ll, de = (e + 1) & ~1ll;    // v, vt [b, e)
  const unsigned sb = (unsigned)((se - sa) * 8), lb = (unsigned)((le - la) * 8);
  const unsigned pb = (unsigned)((pe - pa) * 4), db = (unsigned)((de - da) * 8);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(bar, sb + 2 * lb + pb + 2 * db);
  const unsigned base = smem_addr(stage);
  bulk_g2s(base + Stage64::segp, A.P.seg_ptr + sa, sb, bar);
  bulk_g2s(base + Stage64::lam, A.P.lam + la, lb, bar);
  bulk_g2s(base + Stage64::vt0, A.P.vt0 + la, lb, bar);
  if (pb) bulk_g2s(base + Stage64::prod, A.P.seg_prod + pa, pb, bar);
  if (db) {
    bulk_g2s(base + Stage64::v, A.P.v + da, db, bar);
    bulk_g2s(base + Stage64::vt, A.P.vt + da, db, bar);
  }
}

template <int W, int P, int SC>
__global__ void __launch_bounds__(kPipeThreads, 1) k_seg_fast_pipe(FastArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long full_bar[kStages], empty_bar[kStages];
  __shared__ double sh[32];
  if (A.st->converged) return;
  const Problem& Pr = A.P;
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem);
  unsigned char* stages = smem + A.acc_bytes;
  const long long ntiles = A.ntiles;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_addr(&full_bar[s]), 1);
      mbar_init(smem_addr(&empty_bar[s]), kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (SC == 1)
    for (int j = threadIdx.x; j < Pr.n; j += blockDim.x) acc[j] = 0ull;
  __syncthreads();
  double zacc = 0.0;
  int fallbacks = 0;
  bool failed = false;
  if (warp == 0) {
    // ---- producer ----
    if (threadIdx.x == 0) {
      long long k = 0;
      for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int s = (int)(k % kStages);
        if (k >= kStages &&
            !mbar_wait_bounded(smem_addr(&empty_bar[s]), (unsigned)(((k / kStages) - 1) & 1))) {
          failed = true;
          break;
        }
        issue_tile64(A, t, stages + s * Stage64::bytes, smem_addr(&full_bar[s]));
      }
      // Before leaving, the copies of the last stages issued must have landed
      // (in the normal course the consumers have waited on them already).
      for (long long j = (k > kStages ? k - kStages : 0); j < k; ++j)
        mbar_wait_bounded(smem_addr(&full_bar[j % kStages]), (unsigned)((j / kStages) & 1));
    }
  } else {
    // ---- consumers ----
    const int ct = threadIdx.x - 32;  // consumer thread index
    const int lane = threadIdx.x & (W - 1);
    const int gbase = (threadIdx.x & 31) & ~(W - 1);
    const unsigned gmask = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << gbase);
    const int groups = (kConsumerWarps * 32) / W, group = ct / W;
    long long k = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
      const int s = (int)(k % kStages);
      if (!mbar_wait_bounded(smem_addr(&full_bar[s]), (unsigned)((k / kStages) & 1))) {
        failed = true;
        break;
      }
      const unsigned char* S = stages + s * Stage64::bytes;
      const long long l0 = A.tile_ptr[t], l1 = A.tile_ptr[t + 1];
      const long long* segp = reinterpret_cast<const long long*>(S + Stage64::segp) + (l0 & 1);
      const double* lam_s = reinterpret_cast<const double*>(S + Stage64::lam) + (l0 & 1);
      const double* vt0_s = reinterpret_cast<const double*>(S + Stage64::vt0) + (l0 & 1);
      const long long b0 = segp[0];
      const int* prod_s = reinterpret_cast<const int*>(S + Stage64::prod) + (b0 & 3);
      const double* v_s = reinterpret_cast<const double*>(S + Stage64::v) + (b0 & 1);
      const double* vt_s = reinterpret_cast<const double*>(S + Stage64::vt) + (b0 & 1);
      const int nseg = (int)(l1 - l0);
      for (int ls = group; ls < nseg; ls += groups) {
        const int b = (int)(segp[ls] - b0);
        const int K = (int)(segp[ls + 1] - segp[ls]);
        float af[P], bf[P];
        unsigned cand = 0;
        bool ok = true;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const int kk = lane + p * W;
          af[p] = bf[p] = 0.f;
          if (kk < K) {
            const double m = A.marg[prod_s[b + kk]];
            if (__double_as_longlong(m) > 0) {
              cand |= 1u << p;
              af[p] = f32_trunc(m, ok) * f32_trunc(v_s[b + kk], ok);
              bf[p] = f32_trunc(vt_s[b + kk], ok);
            }
          }
        }
        const double lam = lam_s[ls], vt0 = vt0_s[ls];
        const float vt0f = f32_trunc(vt0, ok);
        float R = 0.f;
        unsigned sel = 0xffffffffu;
        bool conv = false;
        for (int it = 0; it < P * W + 2; ++it) {
          unsigned sset = 0;
          float N = 0.f, D = 0.f;
#pragma unroll
          for (int p = 0; p < P; ++p)
            if (((cand >> p) & 1u) && af[p] > R * bf[p]) {
              sset |= 1u << p;
              N += af[p];
              D += bf[p];
            }
          if (__all_sync(gmask, sset == sel)) {
            conv = true;
            break;
          }
#pragma unroll
          for (int o = W >> 1; o > 0; o >>= 1) {
            N += __shfl_xor_sync(gmask, N, o, W);
            D += __shfl_xor_sync(gmask, D, o, W);
          }
          R = N / (vt0f + D);
          sel = sset;
        }
        bool good = ok && conv;
#pragma unroll
        for (int p = 0; p < P; ++p)
          if ((cand >> p) & 1u) {
            const float a = af[p], c = R * bf[p];
            if (!(fabsf(a - c) > kCertDelta * (a + c))) good = false;
          }
        unsigned Sset = sel;
        if (!__all_sync(gmask, good)) {
          if (lane == 0) ++fallbacks;
          double Rd = 0.0;
          unsigned prev = 0xffffffffu;
          for (int it = 0; it < P * W + 2; ++it) {
            unsigned sset = 0;
            double N = 0.0, D = 0.0;
#pragma unroll
            for (int p = 0; p < P; ++p)
              if ((cand >> p) & 1u) {
                const int kk = b + lane + p * W;
                const double a = A.marg[prod_s[kk]] * v_s[kk], tt = vt_s[kk];
                if (a > Rd * tt) {
                  sset |= 1u << p;
                  N += a;
                  D += tt;
                }
              }
            if (__all_sync(gmask, sset == prev)) break;
#pragma unroll
            for (int o = W >> 1; o > 0; o >>= 1) {
              N += __shfl_xor_sync(gmask, N, o, W);
              D += __shfl_xor_sync(gmask, D, o, W);
            }
            Rd = N / (vt0 + D);
            prev = sset;
          }
          Sset = prev;
        }
        double Nl = 0.0, Dl = 0.0;
#pragma unroll
        for (int p = 0; p < P; ++p)
          if ((Sset >> p) & 1u) {
            const int kk = b + lane + p * W;
            Dl += vt_s[kk];
            Nl = fma(A.marg[prod_s[kk]], v_s[kk], Nl);
          }
#pragma unroll
        for (int o = W >> 1; o > 0; o >>= 1) {
          Nl += __shfl_xor_sync(gmask, Nl, o, W);
          Dl += __shfl_xor_sync(gmask, Dl, o, W);
        }
        const double q = quotient(lam, vt0 + Dl);
        if (lane == 0) zacc += q * Nl;
        if (SC != 0) {
#pragma unroll
          for (int p = 0; p < P; ++p)
            if ((Sset >> p) & 1u) {
              const int kk = b + lane + p * W;
              atomicAdd((SC == 1 ? acc : A.s_fx) + prod_s[kk], fixed_product(q, v_s[kk], A.fx_bits));
            }
        }
      }
      __syncwarp();
      if ((threadIdx.x & 31) == 0) mbar_arrive(smem_addr(&empty_bar[s]));
    }
  }
  if (__syncthreads_or(failed)) {
    if (threadIdx.x == 0) atomicExch(&A.st_rw->error, 1);
    return;
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

template <int SC>
cudaError_t launch_pipe_w(const FastArgs& A, int W, int grid, int smem, cudaStream_t s) {
  switch (W) {  // 8 products per lane
    case 1: k_seg_fast_pipe<1, 8, SC><<<grid, kPipeThreads, smem, s>>>(A); break;
    case 2: k_seg_fast_pipe<2, 8, SC><<<grid, kPipeThreads, smem, s>>>(A); break;
    case 4: k_seg_fast_pipe<4, 8, SC><<<grid, kPipeThreads, smem, s>>>(A); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class K>
int pipe_blocks(K kernel, int smem) {
  return kernel_blocks(kernel, kPipeThreads, smem);
}

}  // namespace

bool pipe_plan(int n, int sms, FastPlan* plan) {
  const int W = plan->W8;
  if (W > 4) return false;
  const int acc = plan->scatter == 1 ? ((n * 8 + 127) / 128) * 128 : 0;
  const int smem = acc + kStages * Stage64::bytes;
  if (smem > kTmaMaxSmem) return false;
  int nb = 0;
#define SPFOM_PIPE_OCC(WW)                                                                        \
  if (W == WW) nb = plan->scatter == 1 ? pipe_blocks(k_seg_fast_pipe<WW, 8, 1>, smem)             \
                                       : pipe_blocks(k_seg_fast_pipe<WW, 8, 2>, smem);
  SPFOM_PIPE_OCC(1)
  SPFOM_PIPE_OCC(2)
  SPFOM_PIPE_OCC(4)
#undef SPFOM_PIPE_OCC
  if (nb < 1) return false;
  plan->pipe = 1;
  plan->pipe_smem = smem;
  plan->pipe_acc_bytes = acc;
  plan->pipe_grid = nb * sms;
  return true;
}

cudaError_t launch_seg_fast_pipe(const FastArgs& A, const FastPlan& plan, cudaStream_t s) {
  return plan.scatter == 1 ? launch_pipe_w<1>(A, plan.W8, plan.pipe_grid, plan.pipe_smem, s)
                           : launch_pipe_w<2>(A, plan.W8, plan.pipe_grid, plan.pipe_smem, s);
}

long long make_tiles64(const long long* seg_ptr, long long L, long long* tiles_out) {
  long long nt = 0, l = 0;
  if (tiles_out) tiles_out[0] = 0;
  while (l < L) {
    long long e = l;
    while (e < L && e - l < kTile64Segs && seg_ptr[e + 1] - seg_ptr[l] <= kTile64Items) ++e;
    if (e == l) e = l + 1;  // one segment holds at most 32 products
    ++nt;
    if (tiles_out) tiles_out[nt] = e;
    l = e;
  }
  return nt;
}

}  // namespace spfom
