// Cooperatively staged binary32 segment kernel (precision 32, tiling 4).
//
// The plain-load kernels spend most of their time waiting on dependent loads:
// a group reads its segment's bounds, then the product ids, then the margins
// of those products, and with 32 resident warps per SM those round trips are
// not hidden. Here a block works through tiles of consecutive segments (at
// most kCoop* segments and products, cut on the host) in two phases:
//   A. all 512 threads stream the tile's consideration-set slice with
//      coalesced loads -- product ids, v, v - w -- gather each product's
//      margin, and leave in shared memory, per product, a = m v (0 when
//      m <= 0), v - w, v and the id; and per segment its offset, lambda and
//      v_0 + sum w;
//   B. groups of W lanes solve the tile's segments from shared memory
//      (k_seg_f32's binary32 Dinkelbach, same slot layout and summation
//      order, so the results equal that tiling's bit for bit) and add the
//      fixed-point sales.
// Phase A of one block overlaps phase B of the other block on the SM. Every
// product's loads in phase A are independent of each other, so many are in
// flight per thread.
#include <cuda_runtime.h>

#include "spfom_device.cuh"
#include "spfom_internal.h"

namespace spfom {

namespace {

struct CoopLayout {
  int acc, af, bt, v, j, off, lam, vt0, bytes;
};

__host__ __device__ inline CoopLayout coop_layout(int n, int sc, int items, int segs) {
  CoopLayout L{};
  int o = 0;
  L.acc = 0;
  o = sc == 1 ? ((n * 8 + 15) / 16) * 16 : 0;
  L.af = o;
  o += items * 4;
  L.bt = o;
  o += items * 4;
  L.v = o;
  o += items * 4;
  L.j = o;
  o += items * 4;
  L.off = o;
  o += ((segs + 1) * 4 + 15) / 16 * 16;
  L.lam = o;
  o += segs * 4;
  L.vt0 = o;
  o += segs * 4;
  L.bytes = (o + 15) / 16 * 16;
  return L;
}

template <int W, int P, int SC>
__global__ void __launch_bounds__(kFastThreads, 2) k_seg_f32_coop(F32Args A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sh[32];
  if (A.st->converged) return;
  const CoopLayout Lo = coop_layout(A.n, SC, A.coop_items, A.coop_segs);
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem + Lo.acc);
  float* s_af = reinterpret_cast<float*>(smem + Lo.af);
  float* s_bt = reinterpret_cast<float*>(smem + Lo.bt);
  float* s_v = reinterpret_cast<float*>(smem + Lo.v);
  int* s_j = reinterpret_cast<int*>(smem + Lo.j);
  int* s_off = reinterpret_cast<int*>(smem + Lo.off);
  float* s_lam = reinterpret_cast<float*>(smem + Lo.lam);
  float* s_vt0 = reinterpret_cast<float*>(smem + Lo.vt0);
  if (SC == 1) {
    for (int j = threadIdx.x; j < A.n; j += blockDim.x) acc[j] = 0ull;
  }
  const int lane = threadIdx.x & (W - 1);
  const int gbase = (threadIdx.x & 31) & ~(W - 1);
  const unsigned gmask = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << gbase);
  const int gpb = blockDim.x / W;
  float zacc = 0.f;
  for (long long t = blockIdx.x; t < A.coop_ntiles; t += gridDim.x) {
    const long long l0 = A.coop_tile_ptr[t], l1 = A.coop_tile_ptr[t + 1];
    const int nseg = (int)(l1 - l0);
    const long long b0 = A.seg_ptr[l0];
    const int nitem = (int)(A.seg_ptr[l1] - b0);
    __syncthreads();  // the previous tile's phase B is done with the buffers (and the sums are cleared)
    // phase A: stream the tile into shared memory
    for (int i = threadIdx.x; i <= nseg; i += blockDim.x) s_off[i] = (int)(A.seg_ptr[l0 + i] - b0);
    for (int i = threadIdx.x; i < nseg; i += blockDim.x) {
      s_lam[i] = A.lam32[l0 + i];
      s_vt0[i] = A.vt0_32[l0 + i];
    }
    for (int i = threadIdx.x; i < nitem; i += blockDim.x) {
      const int j = A.seg_prod[b0 + i];
      const float v = A.v32[b0 + i];
      const float bt = A.vt32[b0 + i];
      const float m = A.marg32[j];
      s_j[i] = j;
      s_v[i] = v;
      s_bt[i] = bt;
      s_af[i] = m > 0.f ? m * v : -1.f;  // -1 marks a product with m <= 0
    }
    __syncthreads();
    // phase B: one group of W lanes per segment
    for (int ls = threadIdx.x / W; ls < nseg; ls += gpb) {
      const long long l = l0 + ls;
      if (A.seg_inst && A.inst_conv[A.seg_inst[l]]) continue;  // batch: instance already converged
      const int b = s_off[ls], K = s_off[ls + 1] - b;
      float tv[P], af[P];
      unsigned cand = 0;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int k = lane + p * W;
        tv[p] = af[p] = 0.f;
        if (k < K) {
          const float a = s_af[b + k];
          tv[p] = s_bt[b + k];
          if (a >= 0.f) {
            cand |= 1u << p;
            af[p] = a;
          }
        }
      }
      const float lam = s_lam[ls], vt0 = s_vt0[ls];
      float R = A.rprev ? A.rprev[l] : 0.f, Nsel = 0.f, Dsel = 0.f;  // as k_seg_f32
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
      if (A.rprev && lane == 0) A.rprev[l] = R;
      const float q = lam / (vt0 + Dsel);
      if (lane == 0) {
        if (A.z_seg) A.z_seg[l] = (double)(q * Nsel);
        else zacc += q * Nsel;
      }
      if (SC != 0) {
        for (unsigned msk = sel; msk; msk &= msk - 1) {
          const int k = b + lane + (__ffs(msk) - 1) * W;
          atomicAdd((SC == 1 ? acc : A.s_fx) + s_j[k], fixed_product32(q, s_v[k], A.fx_bits));
        }
      }
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

template <int SC, int P>
cudaError_t launch_coop_t(const F32Args& A, int W, int grid, int smem, cudaStream_t s) {
  switch (W) {
    case 1: k_seg_f32_coop<1, P, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    case 2: k_seg_f32_coop<2, P, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    case 4: k_seg_f32_coop<4, P, SC><<<grid, kFastThreads, smem, s>>>(A); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class Kern>
int coop_blocks(Kern k, int smem) {
  return kernel_blocks(k, kFastThreads, smem);
}

}  // namespace

// Plan of the cooperative kernel: 8 products per lane (W8 lanes); tiles of at
// most 1536 products (shared-memory sums, two blocks per SM) or 4096 products
// (global sums), and at most a quarter as many segments.
bool coop_plan(int n, int kmax, int sms, FastPlan* plan) {
  if (kmax > 32 || plan->W8 > 4) return false;
  const int items = plan->scatter == 1 ? 1536 : 4096;
  const int segs = items / 4;
  const CoopLayout Lo = coop_layout(n, plan->scatter, items, segs);
  if (Lo.bytes > kTmaMaxSmem) return false;
  int nb = 0;
#define SPFOM_COOP_OCC(WW)                                                                                   \
  if (plan->W8 == WW) nb = plan->scatter == 1 ? coop_blocks(k_seg_f32_coop<WW, 8, 1>, Lo.bytes)              \
                                              : coop_blocks(k_seg_f32_coop<WW, 8, 2>, Lo.bytes);
  SPFOM_COOP_OCC(1)
  SPFOM_COOP_OCC(2)
  SPFOM_COOP_OCC(4)
#undef SPFOM_COOP_OCC
  if (nb < 1) return false;
  plan->coop_ok = 1;
  plan->coop_items = items;
  plan->coop_segs = segs;
  plan->coop_smem = Lo.bytes;
  plan->coop_grid = nb * sms;
  return true;
}

long long make_tiles_lim(const long long* seg_ptr, long long L, int max_segs, int max_items, long long* tiles_out) {
  long long nt = 0, l = 0;
  if (tiles_out) tiles_out[0] = 0;
  while (l < L) {
    long long e = l;
    while (e < L && e - l < max_segs && seg_ptr[e + 1] - seg_ptr[l] <= max_items) ++e;
    if (e == l) e = l + 1;  // a single segment never exceeds the limit (sets hold <= 32 products)
    ++nt;
    if (tiles_out) tiles_out[nt] = e;
    l = e;
  }
  return nt;
}

cudaError_t launch_seg_f32_coop(const F32Args& A, const FastPlan& plan, cudaStream_t s) {
  return plan.scatter == 1 ? launch_coop_t<1, 8>(A, plan.W8, plan.coop_grid, plan.coop_smem, s)
                           : launch_coop_t<2, 8>(A, plan.W8, plan.coop_grid, plan.coop_smem, s);
}

}  // namespace spfom
