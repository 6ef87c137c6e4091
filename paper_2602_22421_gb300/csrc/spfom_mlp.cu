// The warm-start perceptron (include/spfom_mlp.h): BF16 tensor-core matrix
// products on tcgen05 with FP32 accumulators in tensor memory, operands staged
// by TMA, and the elementwise parts of the forward pass, the backward pass and
// Adam as plain kernels.
//
// Every product is C[M x N] = A[M x K] . B[N x K]^T with both operands stored
// K-contiguous in BF16 ("TN"), so each operand tile is a TMA box of 64 K
// values (128 bytes) by 128 (A) or BN (B) rows with the 128-byte swizzle,
// which is also the layout the tcgen05 shared-memory descriptor reads. The
// transposes the backward pass needs are written by the epilogue of the
// product that makes the matrix (a transposed BF16 copy), so no separate
// transpose runs.
//
// One CTA computes a 128 x BN tile (BN = 16 or 256); thread 0 issues the TMA
// loads of a ring of 2 (the 256-wide row tiles, two CTAs per SM) or 4 stages
// and the MMAs (K = 16 per instruction), tcgen05.commit releases each stage
// back to the loads, and a final commit signals the epilogue warps, which read
// the accumulator rows of their TMEM lane quarter. The 256-wide row tiles run
// eight warps (two per lane quarter, one per column half) and send their BF16
// outputs through shared memory with tensor stores; their epilogue also forms
// the output layer's dot product (the hidden layer) and one ReLU-mask bit per
// output, which the masked backward products read instead of the outputs.
// Products with a long K (the weight gradients, K = rows) split K over grid.y
// and sum the partial tiles in a fixed order; the output layer's weight
// gradient is a weighted column sum of the row-major hidden activations. Every
// wait is bounded; a wait that gives up sets the network's error flag, and the
// host reports SPFOM_ETIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/spfom_mlp.h"
#include "spfom_device.cuh"

namespace spfom {
namespace mlp {

namespace {

constexpr int kF = SPFOM_MLP_FEATURES;
constexpr int kH = SPFOM_MLP_HIDDEN;
constexpr int kBM = 128, kBK = 64, kThreads = 128;
constexpr int kOutPad = 16;  // the output layer runs as a 16-column product (column 0 used)
constexpr int kKPad = 64;    // products with K = 16 read operands padded to one 64-wide TMA box

// Offsets in the packed parameter vector.
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kF, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH, kParams = kOffB3 + 1;
static_assert(kParams == SPFOM_MLP_PARAMS, "parameter layout");

// ---- tcgen05 / TMA primitives -------------------------------------------------

// Shared-memory matrix descriptor for a K-major operand in the 128-byte swizzle
// layout: rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte
// offset), descriptor version 1, layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused by swizzled K-major layouts)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 32 columns of the warp's 32 lanes and the wait for them, in one statement
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

// barrier 1 or 2 (barrier 0 is __syncthreads) over `threads` threads
__device__ __forceinline__ void named_bar(uint32_t id, uint32_t threads) {
  if (id == 1u) asm volatile("bar.sync 1, %0;" ::"r"(threads) : "memory");
  else asm volatile("bar.sync 2, %0;" ::"r"(threads) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Tensor store from shared memory (bulk-group completion) and its waits.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"((uint64_t)map),
               "r"(src), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// every committed store has read its shared-memory source (the CTA may exit;
// the global writes complete with the grid)
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---- the product kernel ----------------------------------------------------------

struct Epi {
  int M, N;                      // valid rows and columns of C
  int ksplit;                    // K tiles per CTA along grid.y
  const float* bias;             // [N] added to every row, or null
  int relu;                      // max(0, .) after the bias
  const __nv_bfloat16* mask;     // keep C[r][c] only where mask[r][c] > 0 (ReLU backward), or null
  int ldmask;
  float* out32;                  // FP32 row-major (split k: partial tile of grid.y at out32 + y * M * ld32)
  int ld32;
  __nv_bfloat16* out16;          // BF16 row-major, or null
  int ld16;
  __nv_bfloat16* out16t;         // BF16 transposed: out16t[c * ld16t + r], or null
  int ld16t;
  int zpad;                      // rows M..zpad-1 of out16t are written as zeros (K padding of later products)
  int staged;                    // BN = 256: out16 / out16t leave through shared memory by tensor stores
  // staged tiles only: dotout[r * lddot] = dotb[0] + sum_c bf16(C[r][c]) dotw[c] (the next layer
  // when it is one output: its product need not read C back), or null
  const __nv_bfloat16* dotw;
  const float* dotb;
  float* dotout;
  int lddot;
  // staged tiles only (N = 256): outbits[r * 8 + c / 32] bit c % 32 = (BF16 output > 0), the
  // ReLU mask a later product reads in place of the outputs; maskbits: such a mask, used in
  // place of `mask`
  uint32_t* outbits;
  const uint32_t* maskbits;
  int* error;                    // set to 1 when a wait gives up
  unsigned wait_limit;           // polls of the producer's waits before they give up
};

// ST stages in the operand ring. Row tiles of the wide product take 2, so that
// two CTAs (2 x 256 TMEM columns) share an SM and one CTA's epilogue overlaps
// the other's loads and MMAs; the split-K weight gradients (at most one CTA
// per SM, 64 K tiles each) take 4.
template <int BN, int ST>
struct GemmShape {
  static constexpr int kA = kBM * kBK * 2;  // bytes of an A stage (16 KB)
  static constexpr int kB = BN * kBK * 2;   // bytes of a B stage
  static constexpr int kStage = kA + kB;
  static constexpr int kStages = ST;
  static constexpr int kSmem = kStages * kStage + 1024;  // + alignment slack
  static constexpr uint32_t kCols = BN < 32 ? 32 : BN;   // TMEM columns (power of two >= 32)
  static_assert(kStage % 1024 == 0, "stages must keep the 1024-byte swizzle alignment");
};

__device__ __forceinline__ bool bf16_positive(__nv_bfloat16 h) {
  const unsigned short b = __bfloat16_as_ushort(h);
  return b != 0 && (b & 0x8000u) == 0;
}

// bias, ReLU and ReLU-backward mask of one thread's 16 accumulator columns
__device__ __forceinline__ void epi_apply(const Epi& E, int row, int c0, int nc, float (&v)[16]) {
  if (E.bias)
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (i < nc) v[i] += E.bias[c0 + i];
  if (E.relu)
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = v[i] > 0.f ? v[i] : 0.f;
  if (E.mask) {
    const __nv_bfloat16* mp = E.mask + (size_t)row * E.ldmask + c0;
    if (nc == 16 && (E.ldmask & 7) == 0 && ((uintptr_t)mp & 15) == 0) {
      const uint4 a = __ldg(reinterpret_cast<const uint4*>(mp)), b = __ldg(reinterpret_cast<const uint4*>(mp) + 1);
      const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 16; ++i)  // a BF16 is > 0 iff its bits, read as a signed 16-bit integer, are
        if ((short)(uint16_t)(w[i >> 1] >> (16 * (i & 1))) <= 0) v[i] = 0.f;
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (i < nc && !bf16_positive(mp[i])) v[i] = 0.f;
    }
  }
}

// Threads of a CTA: the 256-wide row tiles (2 stages) run eight warps, two per
// TMEM lane quarter, each half of them storing one half of the columns; the
// other instantiations four.
template <int BN, int ST>
__host__ __device__ constexpr int gemm_threads() {
  return BN == 256 && ST == 2 ? 2 * kThreads : kThreads;
}

template <int BN, int ST>
__global__ void __launch_bounds__(gemm_threads<BN, ST>(), gemm_threads<BN, ST>() > kThreads ? 2 : 1)
    k_gemm_tn(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
              const __grid_constant__ CUtensorMap tr, const __grid_constant__ CUtensorMap tt, int K, Epi E) {
  using S = GemmShape<BN, ST>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) unsigned long long full[S::kStages], empty[S::kStages], done;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM;
  const int KT = (K + kBK - 1) / kBK;
  const int kt0 = blockIdx.y * E.ksplit;
  const int nkt = max(0, min(KT, kt0 + E.ksplit) - kt0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S::kStages; ++s) {
      mbar_init(smem_addr(&full[s]), 1);
      mbar_init(smem_addr(&empty[s]), 1);
    }
    mbar_init(smem_addr(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_base, S::kCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  int ok = 1;
  if (threadIdx.x == 0 && nkt > 0) {
    const uint32_t idesc = idesc_bf16(kBM, BN);
    auto load = [&](int i) {
      const int s = i % S::kStages;
      const uint32_t a = smem_addr(base + s * S::kStage), fb = smem_addr(&full[s]);
      mbar_expect_tx(fb, S::kStage);
      tma_load_2d(a, &ta, (kt0 + i) * kBK, m0, fb);
      tma_load_2d(a + S::kA, &tb, (kt0 + i) * kBK, 0, fb);
    };
    const int pre = nkt < S::kStages ? nkt : S::kStages;
    for (int i = 0; i < pre; ++i) load(i);
    int issued = pre, consumed = 0;
    for (int i = 0; i < nkt; ++i) {
      const int s = i % S::kStages;
      if (!mbar_wait_bounded(smem_addr(&full[s]), (unsigned)(i / S::kStages) & 1u, E.wait_limit)) {
        ok = 0;
        break;
      }
      consumed = i + 1;
      tc_fence_after();
      const int kleft = K - (kt0 + i) * kBK;
      const int ksteps = ((kleft < kBK ? kleft : kBK) + 15) / 16;
      const uint32_t a = smem_addr(base + s * S::kStage), b = a + S::kA;
      for (int kk = 0; kk < ksteps; ++kk)
        umma_bf16(tmem, sdesc_sw128(a + kk * 32), sdesc_sw128(b + kk * 32), idesc, (i > 0 || kk > 0) ? 1u : 0u);
      umma_commit(smem_addr(&empty[s]));
      // refill the stage of the previous tile once its MMAs have read it
      if (i >= 1 && i - 1 + S::kStages < nkt) {
        const int p = i - 1;
        if (!mbar_wait_bounded(smem_addr(&empty[p % S::kStages]), (unsigned)(p / S::kStages) & 1u, E.wait_limit)) {
          ok = 0;
          break;
        }
        load(p + S::kStages);
        ++issued;
      }
    }
    umma_commit(smem_addr(&done));
    if (!ok) {
      // let the copies still in flight land before the CTA can exit
      for (int i = consumed; i < issued; ++i) mbar_wait_bounded(smem_addr(&full[i % S::kStages]), (unsigned)(i / S::kStages) & 1u);
      atomicExch(E.error, 1);
    }
  }
  __syncwarp();
  int have = nkt > 0;
  if (have && !mbar_wait_bounded(smem_addr(&done), 0u)) ok = 0;
  const int any_fail = __syncthreads_or(!ok);
  if (any_fail) {
    if (threadIdx.x == 0) atomicExch(E.error, 1);
    have = 0;
  }
  tc_fence_after();

  constexpr int kHalves = gemm_threads<BN, ST>() / kThreads;  // column halves of the epilogue
  const int quarter = warp & 3, half = warp >> 2;  // TMEM lanes 32 quarter.. (tile rows), columns
  const int rl = quarter * 32 + lane;
  const int row = m0 + rl;
  const bool row_ok = row < E.M;
  const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
  static_assert(BN != 256 || S::kStages * S::kStage >= 65536, "the staged epilogue needs 64 KB of the ring");
  if (BN == 256 && E.staged) {
    // Staged epilogue: 64 columns at a time into a shared-memory buffer (the
    // ring's, free once the MMAs are done): the row-major BF16 tile [128][64] in
    // the 128-byte swizzle of the row-major tensor map, the transposed tile
    // [64][128] plain (rows M..zpad-1 zero); one thread per column half issues
    // the tensor stores, which clip rows and columns outside the maps. With one
    // half the groups alternate between two buffers; with two halves each half
    // has its own buffer.
    constexpr int kGroups = BN / 64 / kHalves;
    const int lead = half * kThreads;
    __shared__ float dot_half[kThreads];  // the second column half's part of the row's dot product
    float dot = 0.f;
    const uint32_t bar = 1u + (uint32_t)half;
#pragma unroll 1
    for (int gi = 0; gi < kGroups; ++gi) {
      const int g = half * kGroups + gi;
      unsigned char* sr = base + (kHalves == 1 ? (gi & 1) : half) * 32768;
      unsigned char* st = sr + 16384;
      if (kHalves == 1 ? gi >= 2 : gi >= 1) {
        if (threadIdx.x == lead) {  // the stores that last read this buffer are done with it
          if (kHalves == 1) bulk_wait_read1();
          else bulk_wait_read0();
        }
        named_bar(bar, kThreads);
      }
#pragma unroll
      for (int sub = 0; sub < 2; ++sub) {
        const int cs = g * 64 + sub * 32;
        // the mask's 32 columns in flight with the accumulator load
        uint4 mk[4];
        const bool mbits = E.maskbits != nullptr && row_ok;
        const bool masked = !mbits && E.mask != nullptr && row_ok;
        const uint32_t mword = mbits ? __ldg(E.maskbits + (size_t)row * 8 + (cs >> 5)) : 0u;
        uint32_t oword = 0u;
        if (masked) {
          const uint4* mp = reinterpret_cast<const uint4*>(E.mask + (size_t)row * E.ldmask + cs);
#pragma unroll
          for (int u = 0; u < 4; ++u) mk[u] = __ldg(mp + u);
        }
        uint32_t r[32];
        if (have) {
          tmem_ld32(trow + (uint32_t)cs, r);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) r[i] = 0u;
        }
#pragma unroll
        for (int qq = 0; qq < 2; ++qq) {
          const int q = sub * 2 + qq;  // 16-column chunk of the group
          const int c0 = g * 64 + q * 16;
          float v[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = row_ok ? __uint_as_float(r[qq * 16 + i]) : 0.f;
          if (row_ok) {
            if (E.bias) {
              const float4* b4 = reinterpret_cast<const float4*>(E.bias + c0);
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const float4 b = __ldg(b4 + u);
                v[4 * u] += b.x;
                v[4 * u + 1] += b.y;
                v[4 * u + 2] += b.z;
                v[4 * u + 3] += b.w;
              }
            }
            if (E.relu)
#pragma unroll
              for (int i = 0; i < 16; ++i) v[i] = v[i] > 0.f ? v[i] : 0.f;
            if (masked) {
              const uint32_t w[8] = {mk[2 * qq].x, mk[2 * qq].y, mk[2 * qq].z, mk[2 * qq].w,
                                     mk[2 * qq + 1].x, mk[2 * qq + 1].y, mk[2 * qq + 1].z, mk[2 * qq + 1].w};
#pragma unroll
              for (int i = 0; i < 16; ++i)  // BF16 > 0 iff its bits as a signed 16-bit integer are
                if ((short)(uint16_t)(w[i >> 1] >> (16 * (i & 1))) <= 0) v[i] = 0.f;
            }
            if (mbits) {
#pragma unroll
              for (int i = 0; i < 16; ++i)
                if (!((mword >> (qq * 16 + i)) & 1u)) v[i] = 0.f;
            }
          }
          uint32_t h[8];  // BF16 pairs (column 2i in the low half)
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const __nv_bfloat162 p2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            h[i] = *reinterpret_cast<const uint32_t*>(&p2);
          }
          if (E.outbits) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              oword |= (uint32_t)((short)(uint16_t)(h[i] & 0xFFFFu) > 0) << (qq * 16 + 2 * i);
              oword |= (uint32_t)((short)(uint16_t)(h[i] >> 16) > 0) << (qq * 16 + 2 * i + 1);
            }
          }
          if (E.dotout) {  // the rounded outputs against the next layer's BF16 weights
            const uint4* wp = reinterpret_cast<const uint4*>(E.dotw + c0);
            const uint4 wa = __ldg(wp), wb = __ldg(wp + 1);
            const uint32_t w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              dot = fmaf(__uint_as_float(h[i] << 16), __uint_as_float(w[i] << 16), dot);
              dot = fmaf(__uint_as_float(h[i] & 0xFFFF0000u), __uint_as_float(w[i] & 0xFFFF0000u), dot);
            }
          }
          if (E.out16) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int j = 2 * q + u;  // 16-byte chunk of the tile row's 128 bytes
              *reinterpret_cast<uint4*>(sr + rl * 128 + ((j ^ (rl & 7)) << 4)) =
                  make_uint4(h[4 * u], h[4 * u + 1], h[4 * u + 2], h[4 * u + 3]);
            }
          }
          if (E.out16t) {
            uint16_t* t = reinterpret_cast<uint16_t*>(st) + q * 16 * kBM + rl;
#pragma unroll
            for (int i = 0; i < 16; ++i) t[i * kBM] = (uint16_t)(h[i >> 1] >> (16 * (i & 1)));
          }
        }
        if (E.outbits && row_ok) E.outbits[(size_t)row * 8 + (cs >> 5)] = oword;
      }
      fence_async_smem();
      named_bar(bar, kThreads);
      if (threadIdx.x == lead) {
        if (E.out16) tma_store_2d(&tr, smem_addr(sr), g * 64, m0);
        if (E.out16t) tma_store_2d(&tt, smem_addr(st), m0, g * 64);
        bulk_commit();
      }
    }
    if (threadIdx.x == lead) bulk_wait_read0();
    if (E.dotout && kHalves == 2 && half == 1) dot_half[rl] = dot;
    tc_fence_before();
    __syncthreads();
    if (E.dotout && half == 0 && row_ok)
      E.dotout[(size_t)row * E.lddot] = (dot + (kHalves == 2 ? dot_half[rl] : 0.f)) + E.dotb[0];
    if (warp == 0) {
      tc_fence_after();
      tmem_dealloc(tmem, S::kCols);
    }
    return;
  }
  // plain epilogue: the half's columns [c_lo, c_hi)
  const int c_lo = half * (BN / kHalves), c_hi = c_lo + BN / kHalves;
  if (E.out16t && !row_ok && row < E.zpad)
    for (int c = c_lo; c < c_hi && c < E.N; ++c) E.out16t[(size_t)c * E.ld16t + row] = __float2bfloat16_rn(0.f);
  float* out32 = E.out32 ? E.out32 + (size_t)blockIdx.y * (size_t)E.M * (size_t)E.ld32 : nullptr;
#pragma unroll 1
  for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
    uint32_t r[16];
    if (have) tmem_ld16(trow + (uint32_t)c0, r);
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = have ? __uint_as_float(r[i]) : 0.f;
    if (!row_ok || c0 >= E.N) continue;
    const int nc = E.N - c0 < 16 ? E.N - c0 : 16;
    epi_apply(E, row, c0, nc, v);
    if (out32) {
      float* o = out32 + (size_t)row * E.ld32 + c0;
      if (nc == 16 && (E.ld32 & 3) == 0 && ((uintptr_t)o & 15) == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) reinterpret_cast<float4*>(o)[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (i < nc) o[i] = v[i];
      }
    }
    if (E.out16) {
      if (nc == 16 && (E.ld16 & 7) == 0) {
        uint32_t h[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const __nv_bfloat162 p2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
          h[i] = *reinterpret_cast<const uint32_t*>(&p2);
        }
        uint4* dst = reinterpret_cast<uint4*>(E.out16 + (size_t)row * E.ld16 + c0);
        dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
        dst[1] = make_uint4(h[4], h[5], h[6], h[7]);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (i < nc) E.out16[(size_t)row * E.ld16 + c0 + i] = __float2bfloat16_rn(v[i]);
      }
    }
    if (E.out16t)
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (i < nc) E.out16t[(size_t)(c0 + i) * E.ld16t + row] = __float2bfloat16_rn(v[i]);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, S::kCols);
  }
}

// ---- elementwise kernels -------------------------------------------------------

constexpr int kEw = 256;

// x (FP32 [rows][16]) -> BF16 row-major copy [rows][64] (columns 0..15; the
// K padding 16..63 stays zero from the allocation) and BF16 transposed copy
// [16][ldt] (columns rows..zpad-1 zero); one thread per row.
__global__ void k_inputs(const float* __restrict__ x, long long rows, long long zpad, __nv_bfloat16* __restrict__ xb,
                         __nv_bfloat16* __restrict__ xt, long long ldt) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= zpad) return;
  uint32_t h[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  if (r < rows) {
    const float* xr = x + r * kF;
    const bool vec = ((uintptr_t)x & 15) == 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4 f = vec ? __ldg(reinterpret_cast<const float4*>(xr) + u)
                           : make_float4(xr[4 * u], xr[4 * u + 1], xr[4 * u + 2], xr[4 * u + 3]);
      const __nv_bfloat162 a = __floats2bfloat162_rn(f.x, f.y), b = __floats2bfloat162_rn(f.z, f.w);
      h[2 * u] = *reinterpret_cast<const uint32_t*>(&a);
      h[2 * u + 1] = *reinterpret_cast<const uint32_t*>(&b);
    }
    uint4* dst = reinterpret_cast<uint4*>(xb + r * kKPad);
    dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
    dst[1] = make_uint4(h[4], h[5], h[6], h[7]);
  }
  if (xt) {
    uint16_t* t = reinterpret_cast<uint16_t*>(xt) + r;
#pragma unroll
    for (int c = 0; c < kF; ++c) t[(size_t)c * ldt] = (uint16_t)(h[c >> 1] >> (16 * (c & 1)));
  }
}

// Master FP32 parameters -> BF16 operands: W1 [256][64] (columns 16..63 zero),
// W2 [256][256], its transpose W2t [256][256], the output row padded to 16 rows
// (W3p [16][256], row 0 = w3), W3pt [256][64] (column 0 = w3, the rest zero),
// and the padded output bias b3p [16].
__global__ void k_weights(const float* __restrict__ p, __nv_bfloat16* __restrict__ w1, __nv_bfloat16* __restrict__ w2,
                          __nv_bfloat16* __restrict__ w2t, __nv_bfloat16* __restrict__ w3p,
                          __nv_bfloat16* __restrict__ w3pt, float* __restrict__ b3p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kH * kKPad) {
    const int o = i / kKPad, c = i % kKPad;
    w1[i] = c < kF ? __float2bfloat16_rn(p[kOffW1 + o * kF + c]) : __float2bfloat16_rn(0.f);
    w3pt[i] = c == 0 ? __float2bfloat16_rn(p[kOffW3 + o]) : __float2bfloat16_rn(0.f);
  }
  if (i < kH * kH) {
    const int o = i / kH, c = i % kH;
    const __nv_bfloat16 h = __float2bfloat16_rn(p[kOffW2 + i]);
    w2[i] = h;
    w2t[(size_t)c * kH + o] = h;
  }
  if (i < kOutPad * kH) {
    const int rr = i / kH, c = i % kH;
    w3p[i] = rr == 0 ? __float2bfloat16_rn(p[kOffW3 + c]) : __float2bfloat16_rn(0.f);
  }
  if (i < kOutPad) b3p[i] = i == 0 ? p[kOffB3] : 0.f;
}

// Output column 0 of the padded output product -> out[rows].
__global__ void k_take_output(const float* __restrict__ o16, long long rows, float* __restrict__ out) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < rows) out[r] = o16[(size_t)r * kOutPad];
}

// Loss terms and the output gradient dO_r = 2 (o_r - t_r) / R (BF16, padded to
// 16 columns, row-major and transposed); per-block sums of (o - t)^2.
__global__ void k_loss(const float* __restrict__ o16, const float* __restrict__ t, long long rows, long long zpad,
                       __nv_bfloat16* __restrict__ d16, __nv_bfloat16* __restrict__ d16t, long long ldt,
                       double* __restrict__ partial) {
  __shared__ double sh[32];
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double e2 = 0.0;
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
  if (r < rows) {
    const float e = o16[(size_t)r * kOutPad] - t[r];
    e2 = (double)e * (double)e;
    const __nv_bfloat16 g = __float2bfloat16_rn(2.f * e / (float)rows);
    d16[(size_t)r * kKPad] = g;  // columns 1..63 stay zero from the allocation
    for (int c = 0; c < kOutPad; ++c) d16t[(size_t)c * ldt + r] = c == 0 ? g : z;
  } else if (r < zpad) {
    for (int c = 0; c < kOutPad; ++c) d16t[(size_t)c * ldt + r] = z;
  }
  const double tot = block_sum_d(e2, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void k_loss_finish(const double* __restrict__ partial, int nb, long long rows, double* __restrict__ loss) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[b];
  s = block_sum_d(s, sh);
  if (threadIdx.x == 0) loss[0] = rows > 0 ? s / (double)rows : 0.0;
}

// Bias gradient g[c] = sum_r d[c][r] over the transposed BF16 gradient [C][ldt]
// in two fixed-order passes. First: block (s, c) sums the rows
// [s per, (s + 1) per) of column c (per and rows8 multiples of 8; the rows
// between the valid ones and rows8 hold zeros) with 16-byte loads, FP32 within
// a thread, binary64 across the block, into part[c * S + s].
__global__ void k_bias_partial(const __nv_bfloat16* __restrict__ dt, long long ldt, long long rows8, long long per,
                               float* __restrict__ part) {
  __shared__ double sh[32];
  const int c = blockIdx.y, S = gridDim.x;
  const long long r0 = (long long)blockIdx.x * per, r1 = min(rows8, r0 + per);
  const uint4* src = reinterpret_cast<const uint4*>(dt + (size_t)c * ldt);
  float acc = 0.f;
  for (long long k = r0 / 8 + threadIdx.x; k < r1 / 8; k += blockDim.x) {
    const uint4 u = __ldg(src + k);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
    float t = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[i]));
      t += f.x + f.y;
    }
    acc += t;
  }
  const double tot = block_sum_d((double)acc, sh);
  if (threadIdx.x == 0) part[(size_t)c * S + blockIdx.x] = (float)tot;
}

// Output-weight gradient from the row-major activations: block b sums the
// rows [b per, (b + 1) per) of h [rows][256] (BF16, leading dimension ldh),
// each weighted by d[r * ldd] (the BF16 output gradient), into
// part[c * S + b]. A thread holds 8 columns of one row in 8 (FP32, in row
// order), the block's 8 row groups are added in order in binary64.
__global__ void __launch_bounds__(256) k_col_wsum(const __nv_bfloat16* __restrict__ h, long long ldh,
                                                  const __nv_bfloat16* __restrict__ d, long long ldd, long long rows,
                                                  long long per, float* __restrict__ part) {
  __shared__ float sh[8][256];
  const int cg = threadIdx.x & 31, rg = threadIdx.x >> 5;
  const long long r0 = (long long)blockIdx.x * per, r1 = min(rows, r0 + per);
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (long long r = r0 + rg; r < r1; r += 8) {
    const float dr = __uint_as_float((uint32_t)__bfloat16_as_ushort(d[r * ldd]) << 16);
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(h + r * ldh) + cg);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc[2 * k] = fmaf(__uint_as_float(w[k] << 16), dr, acc[2 * k]);
      acc[2 * k + 1] = fmaf(__uint_as_float(w[k] & 0xFFFF0000u), dr, acc[2 * k + 1]);
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) sh[rg][cg * 8 + k] = acc[k];
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int g = 0; g < 8; ++g) s += (double)sh[g][threadIdx.x];
  part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = (float)s;
}

// Second: g[c] = the column's S partial sums, one warp per column (lane k
// adds the partials k, k + 32, ... in order, then a fixed shuffle tree).
__global__ void k_bias_finish(const float* __restrict__ part, int S, int C, float* __restrict__ g) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (c >= C) return;
  double s = 0.0;
  for (int k = lane; k < S; k += 32) s += (double)part[(size_t)c * S + k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) g[c] = (float)s;
}

// Split-K partial tiles [splits][M][N] -> g [M][N].
__global__ void k_splitk_sum(const float* __restrict__ part, int splits, int M, int N, float* __restrict__ g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * N) return;
  const int r = i / N, c = i % N;
  float s = 0.f;
#pragma unroll 8
  for (int k = 0; k < splits; ++k) s += __ldg(part + (size_t)k * M * N + (size_t)r * N + c);
  g[i] = s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, int n, float lr, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = 0.9f * m1[i] + 0.1f * gi;
  const float b = 0.999f * m2[i] + 0.001f * gi * gi;
  m1[i] = a;
  m2[i] = b;
  p[i] -= lr * (a / bc1) / (sqrtf(b / bc2) + 1e-8f);
}

int blocks(long long n) { return (int)((n + kEw - 1) / kEw); }

// ---- host side -------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map of a BF16 row-major matrix [rows][cols] with leading dimension ld
// (elements), boxes of 64 columns by box_rows rows, 128-byte swizzle.
bool make_map(CUtensorMap* map, const __nv_bfloat16* ptr, long long rows, long long cols, long long ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn || ((uintptr_t)ptr & 15) || (ld * 2) % 16) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of the transposed BF16 output [rows][cols] (ld elements), boxes
// of 128 columns by 64 rows, no swizzle (the staged epilogue's [64][128] tile).
bool make_map_t(CUtensorMap* map, const __nv_bfloat16* ptr, long long rows, long long cols, long long ld) {
  auto fn = encode_fn();
  if (!fn || ((uintptr_t)ptr & 15) || (ld * 2) % 16) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)kBM, 64u};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

long long round64(long long x) { return (x + 63) / 64 * 64; }

}  // namespace

// C[M][N] = A[M][K] . B[N][K]^T (BF16 operands, K-contiguous, leading
// dimensions lda, ldb), epilogue E (E.M, E.N set here). The operands must hold
// zeros in columns K..round64(K)-1 (so every TMA box lies inside them: lda,
// ldb >= round64(K)) and A must have max(M, 128) readable rows and B exactly
// 16 (N <= 16) or 256 rows. splits > 1 splits K; the partial tiles then go to
// E.out32 as [splits][M][ld32] and *splits_used (or NULL) gets their count.
cudaError_t gemm_tn(const __nv_bfloat16* A, long long lda, const __nv_bfloat16* B, long long ldb, int M, int N, int K,
                    int splits, Epi E, cudaStream_t s, int* splits_used = nullptr, int* staged_out = nullptr) {
  CUtensorMap ta, tb;
  const int bn = N <= 16 ? 16 : 256;
  const long long kcols = round64(K);
  if (N > 256 || M <= 0 || K <= 0 || lda < kcols || ldb < kcols) return cudaErrorInvalidValue;
  if (!make_map(&ta, A, M > kBM ? M : kBM, kcols, lda, kBM) || !make_map(&tb, B, bn, kcols, ldb, bn))
    return cudaErrorInvalidValue;
  const int KT = (K + kBK - 1) / kBK;
  if (splits < 1) splits = 1;
  if (splits > KT) splits = KT;
  E.ksplit = (KT + splits - 1) / splits;
  splits = (KT + E.ksplit - 1) / E.ksplit;
  if (splits_used) *splits_used = splits;
  E.M = M;
  E.N = N;
  // 256-wide tiles with BF16 outputs and no FP32 one: the staged epilogue
  // (the tensor maps check the outputs' alignment; without them the plain one)
  CUtensorMap tr = ta, tt = ta;
  E.staged = 0;
  if (bn == 256 && N == 256 && splits == 1 && !E.out32 && (E.out16 || E.out16t) && E.ld16t >= 0) {
    const long long zp = E.out16t ? (E.zpad > M ? E.zpad : M) : 0;
    bool ok = true;
    if (E.out16) ok = make_map(&tr, E.out16, M, N, E.ld16, kBM);
    if (ok && E.out16t) ok = zp <= E.ld16t && make_map_t(&tt, E.out16t, N, zp, E.ld16t);
    if (ok && E.mask) ok = (E.ldmask & 7) == 0 && ((uintptr_t)E.mask & 15) == 0;
    if (ok && E.bias) ok = ((uintptr_t)E.bias & 15) == 0;
    if (ok && E.dotout) ok = ((uintptr_t)E.dotw & 15) == 0;
    E.staged = ok ? 1 : 0;
  }
  if (!E.staged) {  // only the staged epilogue forms the dot product and the bit masks
    E.dotout = nullptr;
    E.outbits = nullptr;
    E.maskbits = nullptr;
  }
  if (staged_out) *staged_out = E.staged;
  dim3 grid((M + kBM - 1) / kBM, splits);
  if (bn == 16) {
    k_gemm_tn<16, 4><<<grid, gemm_threads<16, 4>(), GemmShape<16, 4>::kSmem, s>>>(ta, tb, tr, tt, K, E);
  } else if (splits > 1) {
    k_gemm_tn<256, 4><<<grid, gemm_threads<256, 4>(), GemmShape<256, 4>::kSmem, s>>>(ta, tb, tr, tt, K, E);
  } else {
    k_gemm_tn<256, 2><<<grid, gemm_threads<256, 2>(), GemmShape<256, 2>::kSmem, s>>>(ta, tb, tr, tt, K, E);
  }
  return cudaGetLastError();
}

cudaError_t gemm_setup() {
  cudaError_t e =
      cudaFuncSetAttribute(k_gemm_tn<16, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, GemmShape<16, 4>::kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gemm_tn<256, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, GemmShape<256, 2>::kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gemm_tn<256, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, GemmShape<256, 4>::kSmem);
  return e;
}

}  // namespace mlp
}  // namespace spfom

// ---- the network object and its C ABI ---------------------------------------------

using spfom::mlp::Epi;

struct spfom_mlp {
  int device = 0;
  int* d_error = nullptr;
  unsigned wait_limit = spfom::kWaitLimit;  // polls of the GEMM producer's waits (spfom_mlp_set_wait_limit)
  float* p = nullptr;   // master parameters
  float* g = nullptr;   // gradients
  float* m1 = nullptr;  // Adam moments
  float* m2 = nullptr;
  long long adam_t = 0;
  // BF16 operands
  __nv_bfloat16 *w1 = nullptr, *w2 = nullptr, *w2t = nullptr, *w3p = nullptr, *w3pt = nullptr;
  float* b3p = nullptr;
  bool weights_stale = true;
  // workspaces for `cap` rows
  long long cap = 0;
  std::vector<void*> ws;
  __nv_bfloat16 *xb = nullptr, *xt = nullptr, *h1 = nullptr, *h1t = nullptr, *h2 = nullptr,
                *d16 = nullptr, *d16t = nullptr, *dh2 = nullptr, *dh2t = nullptr, *dh1t = nullptr;
  uint32_t *h1bits = nullptr, *h2bits = nullptr;  // ReLU masks of h1, h2 (8 words per row)
  bool bits_ok = false;                           // the last forward pass with keep wrote them
  float* o16 = nullptr;
  float* part = nullptr;  // split-K partial tiles
  double* lpart = nullptr;
  double* d_loss = nullptr;
};

namespace {

constexpr int kMaxSplits = 76;  // 2 x 76 = 152 CTAs for the 256-row weight gradients: one per SM

void free_ws(spfom_mlp* n) {
  for (void* q : n->ws) cudaFree(q);
  n->ws.clear();
  n->cap = 0;
}

template <typename T>
cudaError_t wsalloc(spfom_mlp* n, T** out, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 256);
  if (e != cudaSuccess) return e;
  n->ws.push_back(q);
  *out = static_cast<T*>(q);
  return cudaSuccess;
}

cudaError_t ensure_rows(spfom_mlp* n, long long rows) {
  if (rows <= n->cap) return cudaSuccess;
  free_ws(n);
  // capacity: a multiple of 64 (the transposed copies are K operands, padded
  // with zeros to whole 64-wide boxes) and at least one 128-row tile
  const long long R = spfom::mlp::round64(rows < 1024 ? 1024 : rows + rows / 4);
  const int H = SPFOM_MLP_HIDDEN, KP = spfom::mlp::kKPad;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t c) {
    if (e == cudaSuccess) e = wsalloc(n, p, c);
  };
  A(&n->xb, (size_t)R * KP);
  A(&n->xt, (size_t)R * 16);
  A(&n->h1, (size_t)R * H);
  A(&n->h1t, (size_t)R * H);
  A(&n->h1bits, (size_t)R * 8);
  A(&n->h2bits, (size_t)R * 8);
  A(&n->h2, (size_t)R * H);
  A(&n->d16, (size_t)R * KP);
  A(&n->d16t, (size_t)R * 16);
  A(&n->dh2, (size_t)R * H);
  A(&n->dh2t, (size_t)R * H);
  A(&n->dh1t, (size_t)R * H);
  A(&n->o16, (size_t)R * 16);
  A(&n->part, (size_t)kMaxSplits * H * H);
  A(&n->lpart, (size_t)(R / 256 + 2));
  A(&n->d_loss, 1);
  // rows beyond the ones a call writes are read by the 128-row tiles (and
  // discarded); start them at zero
  for (size_t k = 0; k < n->ws.size() && e == cudaSuccess; ++k) e = cudaMemset(n->ws[k], 0, 256);
  if (e == cudaSuccess) e = cudaMemset(n->xb, 0, (size_t)R * KP * 2);
  if (e == cudaSuccess) e = cudaMemset(n->d16, 0, (size_t)R * KP * 2);
  if (e == cudaSuccess) e = cudaMemset(n->h1, 0, (size_t)R * H * 2);
  if (e == cudaSuccess) e = cudaMemset(n->h2, 0, (size_t)R * H * 2);
  if (e == cudaSuccess) e = cudaMemset(n->dh2, 0, (size_t)R * H * 2);
  if (e != cudaSuccess) {
    free_ws(n);
    return e;
  }
  n->cap = R;
  return cudaSuccess;
}

spfom_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return SPFOM_OK;
  return e == cudaErrorMemoryAllocation ? SPFOM_ENOMEM : (e == cudaErrorInvalidValue ? SPFOM_EINVAL : SPFOM_ECUDA);
}

#define MLP_TRY(call)                            \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return from_cuda(e_); \
  } while (0)

Epi epi(spfom_mlp* n) {
  Epi E{};
  E.error = n->d_error;
  E.wait_limit = n->wait_limit;
  return E;
}

cudaError_t refresh_weights(spfom_mlp* n, cudaStream_t s) {
  if (!n->weights_stale) return cudaSuccess;
  const int H = SPFOM_MLP_HIDDEN;
  spfom::mlp::k_weights<<<(H * H + 255) / 256, 256, 0, s>>>(n->p, n->w1, n->w2, n->w2t, n->w3p, n->w3pt, n->b3p);
  n->weights_stale = false;
  return cudaGetLastError();
}

// Forward pass over `rows` rows already in n->xb; with keep the transposed
// activations for the backward pass are written too.
cudaError_t forward_rows(spfom_mlp* n, long long rows, bool keep, cudaStream_t s) {
  using spfom::mlp::gemm_tn;
  const int H = SPFOM_MLP_HIDDEN, KP = spfom::mlp::kKPad;
  const long long ldt = n->cap;
  Epi E = epi(n);
  E.bias = n->p + spfom::mlp::kOffB1;
  E.relu = 1;
  E.out16 = n->h1;
  E.ld16 = H;
  E.out16t = keep ? n->h1t : nullptr;
  E.ld16t = (int)ldt;
  E.zpad = (int)spfom::mlp::round64(rows);
  E.outbits = keep ? n->h1bits : nullptr;
  int staged1 = 0;
  cudaError_t e = gemm_tn(n->xb, KP, n->w1, KP, (int)rows, H, SPFOM_MLP_FEATURES, 1, E, s, nullptr, &staged1);
  if (e != cudaSuccess) return e;
  E.bias = n->p + spfom::mlp::kOffB2;
  E.out16 = n->h2;
  E.out16t = nullptr;  // the output-weight gradient reads h2 row-major
  E.outbits = keep ? n->h2bits : nullptr;
  // the output layer (one unit) as the hidden product's epilogue: o = b3 + bf16(h2) . bf16(w3)
  E.dotw = n->w3p;  // row 0 of the padded output weights
  E.dotb = n->b3p;
  E.dotout = n->o16;
  E.lddot = 16;
  int staged = 0;
  e = gemm_tn(n->h1, H, n->w2, H, (int)rows, H, H, 1, E, s, nullptr, &staged);
  n->bits_ok = keep && staged1 && staged;
  if (e != cudaSuccess || staged) return e;
  Epi O = epi(n);
  O.bias = n->b3p;
  O.out32 = n->o16;
  O.ld32 = 16;
  return gemm_tn(n->h2, H, n->w3p, H, (int)rows, 16, H, 1, O, s);
}

int splits_for(long long rows, int mtiles) {
  const long long kt = (rows + 63) / 64;
  long long sp = 304 / mtiles;
  if (sp > kt / 4) sp = kt / 4;
  if (sp < 1) sp = 1;
  if (sp > kMaxSplits) sp = kMaxSplits;
  return (int)sp;
}

spfom_status check_error(spfom_mlp* n, cudaStream_t s) {
  int err = 0;
  MLP_TRY(cudaMemcpyAsync(&err, n->d_error, sizeof(int), cudaMemcpyDeviceToHost, s));
  MLP_TRY(cudaStreamSynchronize(s));
  return err ? SPFOM_ETIMEOUT : SPFOM_OK;
}

// Weight gradient g = (d^T a) for d^T [256][ldt], a^T [N][ldt] over `rows`
// rows (split K, fixed-order sum).
cudaError_t weight_grad(spfom_mlp* n, const __nv_bfloat16* dt, const __nv_bfloat16* at, int N, long long rows,
                        float* g, cudaStream_t s) {
  const int H = SPFOM_MLP_HIDDEN;
  Epi E = epi(n);
  E.out32 = n->part;
  E.ld32 = N;
  int used = 1;
  cudaError_t e = spfom::mlp::gemm_tn(dt, n->cap, at, n->cap, H, N, (int)rows, splits_for(rows, 2), E, s, &used);
  if (e != cudaSuccess) return e;
  spfom::mlp::k_splitk_sum<<<(H * N + 255) / 256, 256, 0, s>>>(n->part, used, H, N, g);
  return cudaGetLastError();
}

// Bias gradient of C columns of the transposed gradient dt [C][ldt] over
// `rows` rows (zeros up to round64(rows)) into g[C]; the partial sums use
// n->part, after the weight gradient that shares it.
cudaError_t bias_grad(spfom_mlp* n, const __nv_bfloat16* dt, int C, long long rows, float* g, cudaStream_t s) {
  const long long rows8 = (rows + 7) / 8 * 8;
  long long S = (4 * 152 + C - 1) / C;            // about four blocks per SM over all columns
  const long long smax = (rows8 + 2047) / 2048;   // at least 2048 rows (one 16-byte load per thread) each
  if (S > smax) S = smax;
  if (S < 1) S = 1;
  const long long per = ((rows8 + S - 1) / S + 7) / 8 * 8;
  S = (rows8 + per - 1) / per;
  spfom::mlp::k_bias_partial<<<dim3((unsigned)S, (unsigned)C), 256, 0, s>>>(dt, n->cap, rows8, per, n->part);
  spfom::mlp::k_bias_finish<<<(C * 32 + 255) / 256, 256, 0, s>>>(n->part, (int)S, C, g);
  return cudaGetLastError();
}

// dw3 = h2^T dO over `rows` rows from the row-major h2 and the output gradient
// (column 0 of d16): partial sums per block, then one warp per column.
cudaError_t out_weight_grad(spfom_mlp* n, long long rows, float* g, cudaStream_t s) {
  const int H = SPFOM_MLP_HIDDEN;
  long long S = (rows + 255) / 256;
  if (S > 4 * 152) S = 4 * 152;
  if (S < 1) S = 1;
  const long long per = (rows + S - 1) / S;
  S = (rows + per - 1) / per;
  spfom::mlp::k_col_wsum<<<(unsigned)S, 256, 0, s>>>(n->h2, H, n->d16, spfom::mlp::kKPad, rows, per, n->part);
  spfom::mlp::k_bias_finish<<<(H * 32 + 255) / 256, 256, 0, s>>>(n->part, (int)S, H, g);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

spfom_status spfom_mlp_create(int32_t device, uint64_t seed, spfom_mlp** out) {
  if (!out) return SPFOM_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return SPFOM_ECUDA;
  if (!spfom::mlp::encode_fn()) return SPFOM_ENOTSUP;
  if (spfom::mlp::gemm_setup() != cudaSuccess) return SPFOM_ECUDA;
  spfom_mlp* n = new spfom_mlp();
  n->device = device;
  const int P = SPFOM_MLP_PARAMS, H = SPFOM_MLP_HIDDEN;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t c) {
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(p), c * sizeof(**p));
  };
  A(&n->d_error, 1);
  A(&n->p, P);
  A(&n->g, P);
  A(&n->m1, P);
  A(&n->m2, P);
  A(&n->w1, (size_t)H * 64);
  A(&n->w2, (size_t)H * H);
  A(&n->w2t, (size_t)H * H);
  A(&n->w3p, (size_t)16 * H);
  A(&n->w3pt, (size_t)H * 64);
  A(&n->b3p, 16);
  if (e == cudaSuccess) e = cudaMemset(n->d_error, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(n->g, 0, sizeof(float) * P);
  if (e != cudaSuccess) {
    spfom_mlp_destroy(n);
    return from_cuda(e);
  }
  // seeded Glorot-uniform initialisation (splitmix64 stream)
  std::vector<float> h(P, 0.f);
  uint64_t st = seed;
  auto uni = [&]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  };
  const double a1 = std::sqrt(6.0 / (16 + H)), a2 = std::sqrt(6.0 / (H + H)), a3 = std::sqrt(6.0 / (H + 1));
  for (int i = 0; i < H * 16; ++i) h[spfom::mlp::kOffW1 + i] = (float)(a1 * uni());
  for (int i = 0; i < H * H; ++i) h[spfom::mlp::kOffW2 + i] = (float)(a2 * uni());
  for (int i = 0; i < H; ++i) h[spfom::mlp::kOffW3 + i] = (float)(a3 * uni());
  spfom_status s = spfom_mlp_set_params(n, h.data());
  if (s != SPFOM_OK) {
    spfom_mlp_destroy(n);
    return s;
  }
  *out = n;
  return SPFOM_OK;
}

void spfom_mlp_destroy(spfom_mlp* n) {
  if (!n) return;
  cudaSetDevice(n->device);
  free_ws(n);
  void* ptrs[] = {n->d_error, n->p, n->g, n->m1, n->m2, n->w1, n->w2, n->w2t, n->w3p, n->w3pt, n->b3p};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete n;
}

spfom_status spfom_mlp_set_wait_limit(spfom_mlp* n, uint32_t polls) {
  if (!n) return SPFOM_EINVAL;
  n->wait_limit = polls;
  return SPFOM_OK;
}

spfom_status spfom_mlp_set_params(spfom_mlp* n, const float* params) {
  if (!n || !params) return SPFOM_EINVAL;
  for (int i = 0; i < SPFOM_MLP_PARAMS; ++i)
    if (!std::isfinite(params[i])) return SPFOM_EINVAL;
  MLP_TRY(cudaSetDevice(n->device));
  MLP_TRY(cudaMemcpy(n->p, params, sizeof(float) * SPFOM_MLP_PARAMS, cudaMemcpyHostToDevice));
  MLP_TRY(cudaMemset(n->m1, 0, sizeof(float) * SPFOM_MLP_PARAMS));
  MLP_TRY(cudaMemset(n->m2, 0, sizeof(float) * SPFOM_MLP_PARAMS));
  n->adam_t = 0;
  n->weights_stale = true;
  return SPFOM_OK;
}

spfom_status spfom_mlp_get_params(spfom_mlp* n, float* params) {
  if (!n || !params) return SPFOM_EINVAL;
  MLP_TRY(cudaSetDevice(n->device));
  MLP_TRY(cudaMemcpy(params, n->p, sizeof(float) * SPFOM_MLP_PARAMS, cudaMemcpyDeviceToHost));
  return SPFOM_OK;
}

spfom_status spfom_mlp_get_grads(spfom_mlp* n, float* grads) {
  if (!n || !grads) return SPFOM_EINVAL;
  MLP_TRY(cudaSetDevice(n->device));
  MLP_TRY(cudaMemcpy(grads, n->g, sizeof(float) * SPFOM_MLP_PARAMS, cudaMemcpyDeviceToHost));
  return SPFOM_OK;
}

spfom_status spfom_mlp_forward(spfom_mlp* n, const float* x, int64_t rows, float* out, void* stream) {
  if (!n || rows < 0 || (rows > 0 && (!x || !out)) || rows > (1ll << 28)) return SPFOM_EINVAL;
  if (rows == 0) return SPFOM_OK;
  MLP_TRY(cudaSetDevice(n->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MLP_TRY(ensure_rows(n, rows));
  MLP_TRY(refresh_weights(n, s));
  const long long zp = spfom::mlp::round64(rows);
  spfom::mlp::k_inputs<<<spfom::mlp::blocks(zp), spfom::mlp::kEw, 0, s>>>(x, rows, zp, n->xb, nullptr, n->cap);
  MLP_TRY(cudaGetLastError());
  MLP_TRY(forward_rows(n, rows, false, s));
  spfom::mlp::k_take_output<<<spfom::mlp::blocks(rows), spfom::mlp::kEw, 0, s>>>(n->o16, rows, out);
  MLP_TRY(cudaGetLastError());
  return check_error(n, s);
}

spfom_status spfom_mlp_loss_grad(spfom_mlp* n, const float* x, const float* t, int64_t rows, double* loss,
                                 void* stream) {
  using spfom::mlp::gemm_tn;
  if (!n || rows <= 0 || !x || !t || rows > (1ll << 28)) return SPFOM_EINVAL;
  MLP_TRY(cudaSetDevice(n->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int H = SPFOM_MLP_HIDDEN, KP = spfom::mlp::kKPad;
  MLP_TRY(ensure_rows(n, rows));
  MLP_TRY(refresh_weights(n, s));
  const long long ldt = n->cap, zp = spfom::mlp::round64(rows);
  spfom::mlp::k_inputs<<<spfom::mlp::blocks(zp), spfom::mlp::kEw, 0, s>>>(x, rows, zp, n->xb, n->xt, ldt);
  MLP_TRY(cudaGetLastError());
  MLP_TRY(forward_rows(n, rows, true, s));
  const int lb = spfom::mlp::blocks(zp);
  spfom::mlp::k_loss<<<lb, spfom::mlp::kEw, 0, s>>>(n->o16, t, rows, zp, n->d16, n->d16t, ldt, n->lpart);
  spfom::mlp::k_loss_finish<<<1, 256, 0, s>>>(n->lpart, lb, rows, n->d_loss);
  MLP_TRY(cudaGetLastError());
  float* g = n->g;
  // output layer: dw3 = h2^T dO (a weighted column sum of h2), db3 = sum dO
  MLP_TRY(out_weight_grad(n, rows, g + spfom::mlp::kOffW3, s));
  MLP_TRY(bias_grad(n, n->d16t, 1, rows, g + spfom::mlp::kOffB3, s));
  // dH2 = (dO w3^T) masked by h2 > 0
  {
    Epi E = epi(n);
    E.mask = n->h2;
    E.maskbits = n->bits_ok ? n->h2bits : nullptr;
    E.ldmask = H;
    E.out16 = n->dh2;
    E.ld16 = H;
    E.out16t = n->dh2t;
    E.ld16t = (int)ldt;
    E.zpad = (int)zp;
    MLP_TRY(gemm_tn(n->d16, KP, n->w3pt, KP, (int)rows, H, 16, 1, E, s));
  }
  // dW2 = dH2^T h1, db2 = sum dH2
  MLP_TRY(weight_grad(n, n->dh2t, n->h1t, H, rows, g + spfom::mlp::kOffW2, s));
  MLP_TRY(bias_grad(n, n->dh2t, H, rows, g + spfom::mlp::kOffB2, s));
  // dH1 = (dH2 W2) masked by h1 > 0 (transposed copy only)
  {
    Epi E = epi(n);
    E.mask = n->h1;
    E.maskbits = n->bits_ok ? n->h1bits : nullptr;
    E.ldmask = H;
    E.out16t = n->dh1t;
    E.ld16t = (int)ldt;
    E.zpad = (int)zp;
    MLP_TRY(gemm_tn(n->dh2, H, n->w2t, H, (int)rows, H, H, 1, E, s));
  }
  // dW1 = dH1^T x, db1 = sum dH1
  MLP_TRY(weight_grad(n, n->dh1t, n->xt, 16, rows, g + spfom::mlp::kOffW1, s));
  MLP_TRY(bias_grad(n, n->dh1t, H, rows, g + spfom::mlp::kOffB1, s));
  MLP_TRY(cudaGetLastError());
  if (loss) MLP_TRY(cudaMemcpyAsync(loss, n->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  return check_error(n, s);
}

spfom_status spfom_mlp_adam(spfom_mlp* n, float lr, void* stream) {
  if (!n || !(lr > 0.f) || !std::isfinite(lr)) return SPFOM_EINVAL;
  MLP_TRY(cudaSetDevice(n->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  n->adam_t += 1;
  const float bc1 = 1.f - (float)std::pow(0.9, (double)n->adam_t);
  const float bc2 = 1.f - (float)std::pow(0.999, (double)n->adam_t);
  spfom::mlp::k_adam<<<spfom::mlp::blocks(SPFOM_MLP_PARAMS), spfom::mlp::kEw, 0, s>>>(
      n->p, n->g, n->m1, n->m2, SPFOM_MLP_PARAMS, lr, bc1, bc2);
  n->weights_stale = true;
  MLP_TRY(cudaGetLastError());
  return SPFOM_OK;
}

spfom_status spfom_mlp_train_step(spfom_mlp* n, const float* x, const float* t, int64_t rows, float lr, double* loss,
                                  void* stream) {
  spfom_status st = spfom_mlp_loss_grad(n, x, t, rows, loss, stream);
  if (st != SPFOM_OK) return st;
  return spfom_mlp_adam(n, lr, stream);
}

}  // extern "C"
