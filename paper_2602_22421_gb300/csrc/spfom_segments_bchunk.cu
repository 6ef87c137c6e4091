// Instance-chunked binary32 segment kernel for batches (precision 32, tiling 6).
//
// A batch is the block-diagonal union of its instances, with far more
// products (hundreds of thousands) than a block's shared memory can hold as
// fixed-point sums, so the plain kernels add every chosen product's sales
// straight into global memory. Instances with few products and many segments
// then receive thousands of atomic additions per product and iteration, and
// those same-address atomics bound the pass (measured: 3.5x the per-nonzero
// cost of a single instance on the 256-instance family).
//
// Here the union's segments are cut on the host into chunks that never cross
// an instance (at most kBChunkSegs segments each). A block takes a chunk,
// clears shared-memory sums for that instance's products only (at most
// kBChunkProducts of them), solves the chunk's segments exactly as k_seg_f32
// does (same slot layout and summation order, so the results equal that
// tiling's bit for bit), and adds the nonzero sums to the global ones: one
// atomic per product per chunk instead of one per chosen product per segment.
// A chunk of a converged instance is skipped as a whole.
#include <cuda_runtime.h>

#include "spfom_device.cuh"
#include "spfom_internal.h"

namespace spfom {

namespace {

template <int W, int P>
__global__ void __launch_bounds__(kFastThreads, 2) k_seg_f32_bchunk(F32Args A) {
  extern __shared__ unsigned long long acc[];  // [kBChunkProducts]
  __shared__ double sh[32];
  if (A.st->converged) return;
  const int lane = threadIdx.x & (W - 1);
  const int gbase = (threadIdx.x & 31) & ~(W - 1);
  const unsigned gmask = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << gbase);
  const int gpb = blockDim.x / W;
  float zacc = 0.f;
  for (long long c = blockIdx.x; c < A.bc_count; c += gridDim.x) {
    const int b = A.bc_inst[c];
    if (A.inst_conv[b]) continue;  // uniform over the block: the chunk's instance has converged
    const long long l0 = A.bc_seg[c], l1 = A.bc_seg[c + 1];
    const int pb = A.bc_prod_ptr[b], nb = A.bc_prod_ptr[b + 1] - pb;
    __syncthreads();  // the previous chunk's flush is done with the sums
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc[i] = 0ull;
    __syncthreads();
    for (long long l = l0 + threadIdx.x / W; l < l1; l += gpb) {
      const long long sb = A.seg_ptr[l];
      const int K = (int)(A.seg_ptr[l + 1] - sb);
      const int* __restrict__ sp = A.seg_prod + sb;
      const float* __restrict__ v32 = A.v32 + sb;
      int jv[P];
      float tv[P], af[P];
      unsigned cand = 0;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int k = lane + p * W;
        jv[p] = 0;
        tv[p] = af[p] = 0.f;
        if (k < K) {
          jv[p] = sp[k];
          af[p] = v32[k];
          tv[p] = A.vt32[sb + k];
        }
      }
#pragma unroll
      for (int p = 0; p < P; ++p)
        if (lane + p * W < K) {
          const float m = A.marg32[jv[p]];
          if (m > 0.f) {
            cand |= 1u << p;
            af[p] = m * af[p];
          } else {
            af[p] = 0.f;
          }
        }
      const float lam = A.lam32[l], vt0 = A.vt0_32[l];
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
      for (unsigned msk = sel; msk; msk &= msk - 1) {
        const int k = lane + (__ffs(msk) - 1) * W;
        atomicAdd(acc + (sp[k] - pb), fixed_product32(q, v32[k], A.fx_bits));
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
      if (acc[i]) atomicAdd(A.s_fx + pb + i, acc[i]);
  }
  const double tot = block_sum_d((double)zacc, sh);
  if (threadIdx.x == 0) A.zpart[blockIdx.x] = tot;
}

template <int P>
cudaError_t launch_bchunk_t(const F32Args& A, int W, int grid, int smem, cudaStream_t s) {
  switch (W) {
    case 1: k_seg_f32_bchunk<1, P><<<grid, kFastThreads, smem, s>>>(A); break;
    case 2: k_seg_f32_bchunk<2, P><<<grid, kFastThreads, smem, s>>>(A); break;
    case 4: k_seg_f32_bchunk<4, P><<<grid, kFastThreads, smem, s>>>(A); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

// Plan: 8 products per lane (W8 lanes), shared sums for kBChunkProducts
// products. Needs every instance of the batch within that many products.
bool bchunk_plan(int max_inst_products, int sms, FastPlan* plan) {
  if (plan->W8 > 4 || max_inst_products > kBChunkProducts) return false;
  const int smem = kBChunkProducts * (int)sizeof(unsigned long long);
  int nb = 0;
  auto occ = [&](auto k) {
    return kernel_blocks(k, kFastThreads, smem);
  };
  if (plan->W8 == 1) nb = occ(k_seg_f32_bchunk<1, 8>);
  if (plan->W8 == 2) nb = occ(k_seg_f32_bchunk<2, 8>);
  if (plan->W8 == 4) nb = occ(k_seg_f32_bchunk<4, 8>);
  if (nb < 1) return false;
  plan->bchunk_ok = 1;
  plan->bchunk_smem = smem;
  plan->bchunk_grid = nb * sms;
  return true;
}

// Chunks of at most max_segs consecutive segments inside one instance:
// seg_out[c] (start; seg_out[count] = L) and inst_out[c]. Returns the count.
long long make_batch_chunks(const std::vector<long long>& seg_off, int max_segs, long long* seg_out,
                            int* inst_out) {
  long long c = 0;
  const int count = (int)seg_off.size() - 1;
  for (int b = 0; b < count; ++b)
    for (long long l = seg_off[b]; l < seg_off[b + 1]; l += max_segs) {
      if (seg_out) seg_out[c] = l;
      if (inst_out) inst_out[c] = b;
      ++c;
    }
  if (seg_out) seg_out[c] = count > 0 ? seg_off[count] : 0;
  return c;
}

cudaError_t launch_seg_f32_bchunk(const F32Args& A, const FastPlan& plan, cudaStream_t s) {
  return launch_bchunk_t<8>(A, plan.W8, plan.bchunk_grid, plan.bchunk_smem, s);
}

}  // namespace spfom
