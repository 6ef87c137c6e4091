// SPFOM iteration kernels for sm_103a (binary64).
//
// One iteration (Algorithm 2 with every segment in the batch, or a Bernoulli
// sample of them) is three launches on the ctx stream:
//   k_margins    a1  m_j = r_j - sum_i a_ij y_i, clears the sales vector
//   k_segments   a2  every segment's exact inner solution (Section 4.1, Lemma 1),
//                a3  scatter of the sales into s (global atomics), sum_l z_l
//   k_dual_step  a3  g = A s over the resource-major incidence, r^T s,
//                a4  y <- max(0, (1 - tau mu) y - tau (c - g)) (eq. stronglycvxupdate),
//                a5  epoch sums; the last block to finish folds the per-block
//                    partial sums into the device scalars (no grid barrier)
// and, every eval_every iterations, three more for the KKT residual and the
// restart test (a6): margins at the epoch average, an evaluation-only segment
// pass, and a one-block finish kernel.
//
// Inner problem of segment l at margins m (build letters; the paper's
// customer i / product j / eta_j / w_ij / v_ij are l / j / y / v / w here):
// vt_j = v_j - w_j and vt_0 = v_0 + sum_{C_l} w_j make the GAM denominator of
// Section 3 read vt_0 + sum_{k in S} vt_k; the optimum over assortments S is a
// prefix of the positive-margin products sorted by m v / vt (Lemma 1's greedy
// order), namely the prefix maximising N/D with N = sum m v, D = vt_0 + sum vt
// (the first one on ties). Sales are x_j = lambda v_j / D on that prefix.
//
// Layout: a sub-warp of W lanes (W a power of two >= the largest consideration
// set) owns one segment at a time and each lane one product of it, so the
// segment's CSR slice is read with contiguous loads. Keys are sorted as their
// int64 bit images (all candidate keys are positive doubles, others are -1),
// keeping the comparisons off the binary64 pipe, which on GB300 runs at about
// 1/60 of the binary32 rate.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include <map>
#include <mutex>
#include <tuple>

#include "spfom_device.cuh"
#include "spfom_internal.h"

namespace spfom {

namespace {

typedef CUresult (*CtxCurrentFn)(CUcontext*);

// cuCtxGetCurrent through the runtime's driver entry-point query
CtxCurrentFn ctx_current_fn() {
  static std::once_flag once;
  static CtxCurrentFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxCurrentFn>(p);
  });
  return fn;
}

// the current context (null when it cannot be told: nothing is remembered then)
CUcontext current_context() {
  CUcontext c = nullptr;
  CtxCurrentFn fn = ctx_current_fn();
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

std::mutex g_kattr_mutex;
std::map<std::pair<CUcontext, const void*>, int> g_kattr_smem;                   // limit set per kernel
std::map<std::tuple<CUcontext, const void*, int, int>, int> g_kattr_blocks;      // occupancy answers

}  // namespace

cudaError_t kernel_smem(const void* kernel, int bytes) {
  if (bytes <= 0) return cudaSuccess;
  const CUcontext c = current_context();
  std::lock_guard<std::mutex> lock(g_kattr_mutex);
  if (c) {
    auto it = g_kattr_smem.find({c, kernel});
    if (it != g_kattr_smem.end() && it->second >= bytes) return cudaSuccess;
  }
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && c) g_kattr_smem[{c, kernel}] = bytes;
  return e;
}

int kernel_blocks(const void* kernel, int threads, int bytes) {
  if (kernel_smem(kernel, bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const CUcontext c = current_context();
  if (c) {
    std::lock_guard<std::mutex> lock(g_kattr_mutex);
    auto it = g_kattr_blocks.find(std::make_tuple(c, kernel, threads, bytes));
    if (it != g_kattr_blocks.end()) return it->second;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (c) {
    std::lock_guard<std::mutex> lock(g_kattr_mutex);
    g_kattr_blocks[std::make_tuple(c, kernel, threads, bytes)] = nb;
  }
  return nb;
}

namespace {

constexpr int kSegThreads = 256;
constexpr int kVecThreads = 256;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long key) {
  // SplitMix64 output function (Steele, Lea, Flood 2014) on key + golden gamma.
  unsigned long long z = key + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Sums of three doubles per thread over the block, each in block_sum's order;
// the three trees run side by side (one pass of barriers). sh holds 3 x 32.
__device__ void block_sum3(double& a, double& b, double& c, double* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) {
    sh[w] = a;
    sh[32 + w] = b;
    sh[64 + w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    a = b = c = 0.0;
    for (int k = 0; k < nw; ++k) {
      a += sh[k];
      b += sh[32 + k];
      c += sh[64 + k];
    }
  }
}

// Sum of one double per thread over the block, in a fixed order.
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < nw; ++k) tot += sh[k];
  }
  return tot;  // valid in thread 0
}

// ------------------------------------------------------------------ prep --
__global__ void k_prep_items(long long nnz, const double* __restrict__ v, const double* __restrict__ w,
                             double* __restrict__ vt) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p < nnz) vt[p] = w ? __dsub_rn(v[p], w[p]) : v[p];
}

// vt0 = v0 + sum of the segment's w in CSR order (one thread per segment).
__global__ void k_prep_segments(long long L, const long long* __restrict__ seg_ptr, const double* __restrict__ v0,
                                const double* __restrict__ w, double* __restrict__ vt0) {
  long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l >= L) return;
  double acc = v0[l];
  if (w)
    for (long long p = seg_ptr[l]; p < seg_ptr[l + 1]; ++p) acc = __dadd_rn(acc, w[p]);
  vt0[l] = acc;
}

// ------------------------------------------------------------------- a1 --
// Margins m_j = r_j - sum_i a_ij y_i over the product's resources in stored
// order. avg != 0 uses the epoch average sum_y / count as y. Clears s when
// given (full-batch iterations rebuild the sales from zero).
__global__ void k_margins(Problem P, const double* __restrict__ y, const double* __restrict__ sum_y, int avg,
                          double* __restrict__ marg, double* __restrict__ s_clear,
                          unsigned long long* __restrict__ sfx_clear, const DevState* st,
                          float* __restrict__ marg32 = nullptr, float2* __restrict__ marg2 = nullptr,
                          float* __restrict__ marg32c = nullptr) {
  if (st && st->converged) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P.n) return;
  const double cnt = avg ? (double)st->count : 1.0;
  double acc = 0.0;
  for (int q = P.a_ptr[j]; q < P.a_ptr[j + 1]; ++q) {
    const int i = P.a_idx[q];
    const double a = P.a_val ? P.a_val[q] : 1.0;
    const double yi = avg ? __ddiv_rn(sum_y[i], cnt) : y[i];
    acc = __dadd_rn(acc, __dmul_rn(a, yi));
  }
  const double m = __dsub_rn(P.r[j], acc);
  marg[j] = m;
  if (marg32) marg32[j] = __double2float_rn(m);
  // images for the row-exact kernel's certified decision: a positive margin
  // outside binary32's normal range becomes NaN (that segment is redone in binary64)
  if (marg32c) {
    const float f = __double2float_rn(m);
    marg32c[j] = m > 0.0 ? ((f >= 1.17549435e-38f && f <= 3.40282347e38f) ? f : __int_as_float(0x7fc00000)) : 0.f;
  }
  // pairs for the double-float kernel: only positive margins enter its decision
  if (marg2) marg2[j] = m > 0.0 ? split_pair(m) : make_float2(m < 0.0 ? -1.f : 0.f, 0.f);
  if (s_clear) s_clear[j] = 0.0;
  if (sfx_clear) sfx_clear[j] = 0ull;
}

// ------------------------------------------------------------------- a2 --
enum SegMode { kIterate = 0, kEvalSum = 1, kEvalSeg = 2 };

template <int W, int MODE, bool SAMPLED>
__global__ void __launch_bounds__(kSegThreads) k_segments(Problem P, const double* __restrict__ marg,
                                                          double* __restrict__ s, double* __restrict__ x_cur,
                                                          double* __restrict__ z_seg, double* __restrict__ zpart,
                                                          const DevState* st, unsigned long long seed,
                                                          unsigned long long thr, double* __restrict__ xsum) {
  if (st && MODE != kEvalSeg && st->converged) return;
  __shared__ double sh[32];
  const int lane = threadIdx.x & (W - 1);
  const int gbase = (threadIdx.x & 31) & ~(W - 1);
  const unsigned mask = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << gbase);
  const long long groups_per_block = kSegThreads / W;
  const long long ngroups = (long long)gridDim.x * groups_per_block;
  const long long t_next = SAMPLED ? st->t + 1 : 0;
  double zacc = 0.0;
  for (long long l = blockIdx.x * groups_per_block + threadIdx.x / W; l < P.L; l += ngroups) {
    if (SAMPLED && splitmix64(seed ^ ((unsigned long long)t_next << 32) ^ (unsigned long long)l) >= thr) continue;
    const long long b = P.seg_ptr[l];
    const int K = (int)(P.seg_ptr[l + 1] - b);
    const double lam = P.lam[l], vt0 = P.vt0[l];
    int j = 0;
    double v = 0.0, vt = 0.0, mv = 0.0;
    long long key = -1;  // int64 image of the sort key; -1 = not a candidate
    if (lane < K) {
      j = P.seg_prod[b + lane];
      v = P.v[b + lane];
      vt = P.vt[b + lane];
      const double mj = marg[j];
      if (mj > 0.0) {
        mv = __dmul_rn(mj, v);
        key = __double_as_longlong(vt == 0.0 ? CUDART_INF : __ddiv_rn(mv, vt));
      }
    }
    // Bitonic sort over the group: descending key, ties by lower CSR position.
    int idx = lane;
#pragma unroll
    for (int k = 2; k <= W; k <<= 1) {
#pragma unroll
      for (int d = k >> 1; d > 0; d >>= 1) {
        const long long ok = __shfl_xor_sync(mask, key, d, W);
        const int oi = __shfl_xor_sync(mask, idx, d, W);
        const bool other_first = (ok > key) || (ok == key && oi < idx);
        const bool lower = (lane & d) == 0;
        const bool desc = (lane & k) == 0;
        if (desc == lower ? other_first : !other_first) {
          key = ok;
          idx = oi;
        }
      }
    }
    // Lane r now holds the rank-r product (original lane idx).
    const int nc = __popc(__ballot_sync(mask, key >= 0) & mask);
    const double mv_r = __shfl_sync(mask, mv, idx, W);
    const double vt_r = __shfl_sync(mask, vt, idx, W);
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
    const double D = vt0 + Dp;
    const double R = lane < nc ? __ddiv_rn(N, D) : 0.0;
    long long best = __double_as_longlong(R);  // R >= 0: the bit image orders like the value
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
    const double bestD = __shfl_sync(mask, D, bl, W);
    const double z = lam * __longlong_as_double(best);
    if (MODE == kIterate) {
      const double x = lane < kstar ? __ddiv_rn(__dmul_rn(lam, v_r), bestD) : 0.0;
      if (SAMPLED) {
        if (idx < K) {
          const long long p = b + idx;
          const double xo = x_cur[p];
          if (x != xo) atomicAdd(s + j_r, x - xo);
          x_cur[p] = x;
        }
      } else if (lane < kstar) {
        atomicAdd(s + j_r, x);
      }
      if (!SAMPLED && xsum && lane < K) {
        // epoch sums of the responses (x-bar); the first iteration of an epoch starts them afresh
        const long long p = b + idx;
        xsum[p] = st->count == 0 ? x : __dadd_rn(xsum[p], x);
      }
    }
    if (lane == 0) {
      zacc += z;
      if (MODE == kEvalSeg) z_seg[l] = z;
    }
  }
  const double tot = block_sum(zacc, sh);
  if (threadIdx.x == 0) zpart[blockIdx.x] = tot;
}

// -------------------------------------------------------------- a3 .. a5 --
__global__ void __launch_bounds__(kVecThreads) k_dual_step(Problem P, Work Wk, RunConfig cfg, int full,
                                                              int zparts) {
  DevState* st = Wk.st;
  if (st->converged) return;
  __shared__ double sh[96];
  __shared__ bool last;
  const double tau = st->tau, shrink = __dsub_rn(1.0, __dmul_rn(st->tau, st->mu));
  double cy = 0.0, pr = 0.0, zm = 0.0;
  const bool fx = Wk.fast && full;
  // The first blocks take one resource per warp: the lanes fetch the
  // resource's products and their sales together (one round of dependent
  // loads per 32 products). With unit incidence and fixed-point sales the
  // warp adds the integer sales exactly; otherwise lane 0 adds the binary64
  // terms in ascending product order. The remaining blocks convert the
  // product sales, one product per thread.
  constexpr int kWarps = kVecThreads / 32;
  const int rblocks = (P.m + kWarps - 1) / kWarps;
  if ((int)blockIdx.x < rblocks) {
    const int i = blockIdx.x * kWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i < P.m) {
      const double yo = Wk.y[i], c = P.c[i], sy = Wk.sum_y[i], sg = Wk.sum_g[i];
      const int q0 = P.at_ptr[i], q1 = P.at_ptr[i + 1];
      double g = 0.0;
      if (fx && !P.at_val) {
        // unit incidence: g_i = 2^-F sum_j s_fx[j], summed exactly in fixed point
        // (the total stays below 2^62), then rounded once
        unsigned long long acc = 0ull;
        for (int q = q0 + lane; q < q1; q += 32) acc += Wk.s_fx[P.at_idx[q]];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        g = __dmul_rn(__ull2double_rn(acc), Wk.inv_fx_scale);
      }
      for (int qb = q0; qb < q1 && !(fx && !P.at_val); qb += 32) {
        const int q = qb + lane;
        double term = 0.0;
        if (q < q1) {
          const int j = P.at_idx[q];
          const double sv = fx ? __dmul_rn(__ull2double_rn(Wk.s_fx[j]), Wk.inv_fx_scale) : Wk.s[j];
          term = __dmul_rn(P.at_val ? P.at_val[q] : 1.0, sv);
        }
        const int cnt = q1 - qb < 32 ? q1 - qb : 32;
        for (int k = 0; k < cnt; ++k) {
          const double t = __shfl_sync(0xffffffffu, term, k);
          if (lane == 0) g = __dadd_rn(g, t);
        }
      }
      if (lane == 0) {
        const double yn = __dsub_rn(__dmul_rn(shrink, yo), __dmul_rn(tau, __dsub_rn(c, g)));
        Wk.y[i] = yn > 0.0 ? yn : 0.0;
        Wk.g[i] = g;
        Wk.sum_y[i] = __dadd_rn(sy, yo);
        Wk.sum_g[i] = __dadd_rn(sg, g);
        if (yo != 0.0) cy = __dmul_rn(c, yo);
      }
    }
  } else {
    const int j = (blockIdx.x - rblocks) * blockDim.x + threadIdx.x;
    if (j < P.n) {
      double sj = Wk.s[j];
      if (fx) {
        sj = __dmul_rn(__ull2double_rn(Wk.s_fx[j]), Wk.inv_fx_scale);
        Wk.s[j] = sj;
        zm = __dmul_rn(Wk.marg[j], sj);  // sum_l z_l = sum_j m_j s_j (z_l = sum_j m_j x_lj)
      }
      pr = __dmul_rn(P.r[j], sj);
    }
  }
  block_sum3(cy, pr, zm, sh);
  if (threadIdx.x == 0) {
    Wk.cypart[blockIdx.x] = cy;
    Wk.Ppart[blockIdx.x] = pr;
    Wk.zmpart[blockIdx.x] = zm;
    __threadfence();
    const unsigned prev = atomicAdd(&st->ticket, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  // Last block: fold the partial sums (strided over the block, then a tree).
  __threadfence();
  double zs = 0.0, cys = 0.0, Ps = 0.0;
  if (fx) {  // the segment kernel left z to this step
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) zs += __ldcg(Wk.zmpart + b);
  } else {
    for (int b = threadIdx.x; b < zparts; b += blockDim.x) zs += __ldcg(Wk.zpart + b);
  }
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    cys += __ldcg(Wk.cypart + b);
    Ps += __ldcg(Wk.Ppart + b);
  }
  block_sum3(zs, cys, Ps, sh);
  if (threadIdx.x != 0) return;
  st->z_sum = full ? zs : CUDART_NAN;
  st->dual_iter = full ? cys + zs : CUDART_NAN;
  st->P = Ps;
  st->sum_P += Ps;
  st->count += 1;
  st->t += 1;
  st->ticket = 0;
}

// ------------------------------------------------------------------- a6 --
// KKT residual of the epoch averages and the restart test (solver addition;
// the paper's Remark in Section 4.2 notes SPFOM forms no residuals).
__global__ void __launch_bounds__(1024) k_eval_finish(Problem P, Work Wk, RunConfig cfg, int zparts) {
  DevState* st = Wk.st;
  if (st->converged) return;
  __shared__ double sh[32];
  __shared__ int restart, progress;
  const double cnt = (double)st->count;
  double cy = 0.0, over2 = 0.0, c2 = 0.0;
  for (int i = threadIdx.x; i < P.m; i += blockDim.x) {
    const double yb = __ddiv_rn(Wk.sum_y[i], cnt), gb = __ddiv_rn(Wk.sum_g[i], cnt), c = P.c[i];
    if (yb != 0.0) cy += __dmul_rn(c, yb);
    const double o = __dsub_rn(gb, c);
    if (o > 0.0) over2 += __dmul_rn(o, o);
    c2 += __dmul_rn(c, c);
  }
  double zs = 0.0;
  for (int b = threadIdx.x; b < zparts; b += blockDim.x) zs += Wk.zpart_eval[b];
  zs = block_sum(zs, sh);
  const double tcy = block_sum(cy, sh);
  const double tover = block_sum(over2, sh);
  const double tc2 = block_sum(c2, sh);
  if (threadIdx.x == 0) {
    const double Pbar = st->sum_P / cnt;
    const double D = tcy + zs;
    const double pinf = sqrt(tover) / (1.0 + sqrt(tc2));
    const double gap = fabs(D - Pbar) / (1.0 + fabs(D) + fabs(Pbar));
    const double kkt = pinf > gap ? pinf : gap;
    st->pinf = pinf;
    st->gap = gap;
    st->kkt = kkt;
    st->dual_avg = D;
    st->primal_avg = Pbar;
    st->evals += 1;
    st->converged = kkt <= cfg.kkt_tol;
    progress = kkt <= cfg.restart_beta * st->kkt_anchor;
    restart = !st->converged && (progress || (double)st->count >= cfg.restart_artificial * (double)st->t);
  }
  __syncthreads();
  if (!restart) return;
  for (int i = threadIdx.x; i < P.m; i += blockDim.x) {
    Wk.y[i] = __ddiv_rn(Wk.sum_y[i], cnt);
    Wk.sum_y[i] = 0.0;
    Wk.sum_g[i] = 0.0;
  }
  if (threadIdx.x == 0) {
    st->sum_P = 0.0;
    st->count = 0;
    st->kkt_anchor = st->kkt;
    if (st->mu > 0.0) st->mu *= 0.5;
    st->tau *= cfg.restart_tau_decay;
    if (!progress && cfg.restart_tau_balance > 0.0)
      st->tau *= balance_factor(st->pinf, st->gap, cfg.restart_tau_balance);
    st->restarts += 1;
  }
}

// Dual(y) = c^T y + sum_l z_l(y) for spfom_evaluate.
__global__ void __launch_bounds__(1024) k_evaluate_finish(Problem P, Work Wk) {
  __shared__ double sh[32];
  double cy = 0.0;
  for (int i = threadIdx.x; i < P.m; i += blockDim.x)
    if (Wk.y_eval[i] != 0.0) cy += __dmul_rn(P.c[i], Wk.y_eval[i]);
  const double tcy = block_sum(cy, sh);
  double zs = 0.0;
  for (int b = threadIdx.x; b < Wk.seg_blocks; b += blockDim.x) zs += Wk.zpart_eval[b];
  zs = block_sum(zs, sh);
  if (threadIdx.x == 0) Wk.st->eval_out = tcy + zs;
}

template <int MODE, bool SAMPLED>
cudaError_t launch_segments_w(const Problem& P, const Work& Wk, const double* marg, double* zpart,
                              const DevState* st, const RunConfig& cfg, cudaStream_t s, double* xsum = nullptr) {
  const int g = Wk.seg_blocks;
  switch (Wk.W) {
#define SPFOM_SEG_CASE(WW)                                                                              \
  case WW:                                                                                              \
    k_segments<WW, MODE, SAMPLED><<<g, kSegThreads, 0, s>>>(P, marg, Wk.s, Wk.x_cur, Wk.z_seg, zpart, st, \
                                                            cfg.seed, cfg.sample_thr, xsum);           \
    break;
    SPFOM_SEG_CASE(1)
    SPFOM_SEG_CASE(2)
    SPFOM_SEG_CASE(4)
    SPFOM_SEG_CASE(8)
    SPFOM_SEG_CASE(16)
    SPFOM_SEG_CASE(32)
#undef SPFOM_SEG_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// k_dual_step: one warp per resource, then one thread per product.
int vec_grid(const Problem& P) {
  const int g = (P.m + kVecThreads / 32 - 1) / (kVecThreads / 32) + (P.n + kVecThreads - 1) / kVecThreads;
  return g > 0 ? g : 1;
}

}  // namespace

namespace {

// One thread per segment: its offsets, lambda, v0, then its nonzeros in
// order (id in range, not repeated earlier in the segment, v finite and > 0,
// w in [0, v]); with f32, v and v - w (and lambda, v0) normal binary32 numbers
// (v - w and lambda may be 0). The first failure of a segment ends its checks.
// Nonzeros are read only inside [0, nnz) and only for the first kFastMaxSet of
// a set (a larger set is rejected by its size).
__device__ __forceinline__ bool in_f32(double x, bool zero_ok) {
  return (zero_ok && x == 0.0) || (x >= 1.1754943508222875e-38 && x <= 3.4028234663852886e+38);
}

__global__ void k_validate_items(const Problem P, const double* __restrict__ w, const double* __restrict__ v0,
                                 int f32, unsigned long long* __restrict__ keys) {
  unsigned kmax = 0u;  // the largest set this thread saw (one atomic per warp at the end)
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < P.L;
       l += (long long)gridDim.x * blockDim.x) {
    const unsigned long long seg = (unsigned long long)l << kCheckSegShift;
    const long long b = P.seg_ptr[l], e = P.seg_ptr[l + 1];
    if (e < b) {
      atomicMin(keys, seg | kSegOrder);
      continue;
    }
    if (b < 0 || e > P.nnz) continue;  // a decrease elsewhere reports it
    const long long K = e - b;
    kmax = max(kmax, (unsigned)(K < 0x7fffffffll ? K : 0x7fffffffll));
    const double lam = P.lam[l], v0l = v0[l];
    if (!(lam >= 0.0 && isfinite(lam))) {
      atomicMin(keys, seg | kSegLam);
      continue;
    }
    if (!(v0l > 0.0 && isfinite(v0l))) {
      atomicMin(keys, seg | kSegV0);
      continue;
    }
    if (f32 && (!in_f32(lam, true) || !in_f32(v0l, false))) atomicMin(keys + 1, (unsigned long long)(P.nnz + l));
    for (long long p = b; p < e && p < b + kFastMaxSet; ++p) {
      const int j = P.seg_prod[p];
      int code = 0;
      if (j < 0 || j >= P.n) {
        code = kBadId;
      } else {
        for (long long q = b; q < p; ++q)
          if (P.seg_prod[q] == j) code = kRepeated;
      }
      const double v = P.v[p];
      if (!code && !(v > 0.0 && isfinite(v))) code = kBadV;
      const double wp = w ? w[p] : 0.0;
      if (!code && w && !(wp >= 0.0 && wp <= v)) code = kBadW;
      if (code) {
        atomicMin(keys, seg | (unsigned long long)(kSegItems + 8 * (p - b) + code));
        break;
      }
      if (f32 && (!in_f32(v, false) || !in_f32(w ? __dsub_rn(v, wp) : v, true)))
        atomicMin(keys + 1, (unsigned long long)p);
    }
  }
  kmax = __reduce_max_sync(0xffffffffu, kmax);
  if ((threadIdx.x & 31) == 0 && kmax) atomicMax(keys + 2, (unsigned long long)kmax);
}

}  // namespace

cudaError_t launch_validate_items(const Problem& P, const double* w, const double* v0, bool f32,
                                  unsigned long long* keys, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(keys, 0xff, 2 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(keys + 2, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess || P.L <= 0) return e;
  const long long blocks = (P.L + 255) / 256;
  k_validate_items<<<(unsigned)(blocks < 65535ll * 16 ? blocks : 65535ll * 16), 256, 0, s>>>(P, w, v0, f32 ? 1 : 0,
                                                                                               keys);
  return cudaGetLastError();
}

cudaError_t launch_prep(const Problem& P, const double* w, const double* v0, double* vt, double* vt0,
                        cudaStream_t s) {
  if (P.nnz > 0) k_prep_items<<<(unsigned)((P.nnz + 255) / 256), 256, 0, s>>>(P.nnz, P.v, w, vt);
  if (P.L > 0) k_prep_segments<<<(unsigned)((P.L + 255) / 256), 256, 0, s>>>(P.L, P.seg_ptr, v0, w, vt0);
  return cudaGetLastError();
}

// The iterate pass of a single instance runs the row-exact kernel (precision-64 tiling 4).
bool rows_active(const Work& Wk, const RunConfig& cfg, bool sampled) {
  return Wk.fast && !sampled && !cfg.f32 && !Wk.batch && Wk.plan.fast_rows && Wk.rx.nchunks > 0 && Wk.marg32c;
}

cudaError_t launch_segment_pass(const Problem& P, const Work& Wk, const RunConfig& cfg, const double* marg,
                                bool iterate, cudaStream_t s, int* zparts_out) {
  const int* seg_inst = Wk.batch ? Wk.bm.seg_inst : nullptr;
  const int* conv = Wk.batch ? Wk.bm.conv : nullptr;
  // per-segment values: evaluation passes of a batch (an iterate pass takes the
  // sum of z per instance from the products, sum_j m_j s_j)
  double* z_seg = (Wk.batch && !iterate) ? Wk.bm.z_seg : nullptr;
  if (Wk.v2 && (!iterate || !(cfg.f32 && Wk.v32))) {
    // double-float precision-64 kernel (also the evaluation pass of precision 32)
    const bool it = iterate;
    DdArgs A{P.seg_ptr, P.seg_prod, Wk.v2, Wk.vt2, Wk.seg4, it ? Wk.marg2 : Wk.marg2_eval, marg, P.v, P.vt, P.lam,
             P.vt0, P.L, P.n, Wk.fx_bits, it ? Wk.part : nullptr, it ? Wk.s_fx : nullptr,
             it ? Wk.zpart : Wk.zpart_eval, Wk.st, Wk.fallbacks, seg_inst, conv, z_seg};
    const int v = Wk.plan.dd_variant >= 1 && Wk.plan.dd_variant <= 3 ? Wk.plan.dd_variant : 1;
    *zparts_out = it ? Wk.plan.dd_grid[v] : Wk.plan.dd_grid_eval[v];
    return launch_seg_dd(A, Wk.plan, it, s);
  }
  if (!iterate) {
    FastArgs A{P, marg, nullptr, Wk.zpart_eval, Wk.st, Wk.fx_scale, Wk.fallbacks, Wk.fx_bits, nullptr,
               nullptr, 0, 0, Wk.st, seg_inst, conv, z_seg};
    *zparts_out = Wk.plan.grid_eval;
    return launch_seg_fast(A, Wk.plan, false, s);
  }
  if (cfg.f32 && Wk.v32) {
    F32Args A{P.seg_ptr, P.seg_prod, Wk.v32, Wk.vt32, Wk.lam32, Wk.vt0_32, P.L, P.n, Wk.fx_bits, Wk.marg32,
              Wk.part, Wk.s_fx, Wk.zpart, Wk.st, Wk.tile_ptr, Wk.ntiles, Wk.plan.acc_bytes, Wk.st,
              seg_inst, conv, z_seg, Wk.coop_tile_ptr, Wk.coop_ntiles, Wk.plan.coop_items, Wk.plan.coop_segs,
              Wk.rprev, 0, 0, Wk.batch ? Wk.bc_count : 0, Wk.bc_seg, Wk.bc_inst,
              Wk.batch ? Wk.bm.prod_ptr : nullptr, Wk.sl};
    A.wait_limit = Wk.wait_limit;
    const bool bchunk = Wk.plan.bchunk && Wk.batch && Wk.bc_count > 0;
    const FastPlan& pl = Wk.plan;
    if (!bchunk && !Wk.batch && pl.f32_rows && Wk.rx.nchunks > 0 && Wk.rx.v32) {
      A.rx = Wk.rx;
      *zparts_out = pl.rows_grid32;
      return launch_seg_rows32(A, pl, s);
    }
    if (!bchunk && pl.f32_sl && Wk.sl.nchunks > 0) {
      *zparts_out = pl.ms_ok ? pl.ms_grid32 : pl.grid32;
      return launch_seg_f32(A, pl, s);
    }
    *zparts_out = bchunk ? pl.bchunk_grid
                         : (pl.coop ? pl.coop_grid
                                    : (pl.tma ? pl.tma_grid
                                              : (pl.f32_p16 ? pl.grid32 : (pl.f32_ms && pl.ms_ok ? pl.ms_grid32 : pl.grid32))));
    return launch_seg_f32(A, Wk.plan, s);
  }
  FastArgs A{P, marg, Wk.part, Wk.zpart, Wk.st, Wk.fx_scale, Wk.fallbacks, Wk.fx_bits, Wk.s_fx,
             Wk.tile64_ptr, Wk.ntiles64, Wk.plan.pipe_acc_bytes, Wk.st, seg_inst, conv, z_seg, Wk.rprev, 0, 0,
             Wk.batch ? Wk.bc_count : 0, Wk.bc_seg, Wk.bc_inst, Wk.batch ? Wk.bm.prod_ptr : nullptr, Wk.sl};
  if (Wk.plan.pipe && !Wk.batch) {
    *zparts_out = Wk.plan.pipe_grid;
    return launch_seg_fast_pipe(A, Wk.plan, s);
  }
  if (iterate && rows_active(Wk, cfg, false)) {
    A.marg32c = Wk.marg32c;
    A.rx = Wk.rx;
    *zparts_out = Wk.plan.rows_grid;
    return launch_seg_rows(A, Wk.plan, s);
  }
  if (Wk.plan.bchunk64_ok && A.bc_count > 0) *zparts_out = Wk.plan.bchunk64_grid;
  else if ((Wk.plan.fast_sl && Wk.sl.nchunks > 0) || Wk.plan.fast_ms) *zparts_out = Wk.plan.ms_ok ? Wk.plan.ms_grid : Wk.plan.grid;
  else *zparts_out = Wk.plan.grid;
  return launch_seg_fast(A, Wk.plan, true, s);
}

cudaError_t launch_iteration(const Problem& P, const Work& Wk, const RunConfig& cfg, cudaStream_t s,
                             cudaEvent_t seg_begin, cudaEvent_t seg_end) {
  if (Wk.batch) return launch_batch_iteration(P, Wk, cfg, s, seg_begin, seg_end);
  const bool sampled = cfg.batch_frac < 1.0;
  const bool fast = Wk.fast && !sampled;
  const bool f32 = fast && cfg.f32 && Wk.v32;
  const int gv = vec_grid(P);
  const int gn = (P.n + kVecThreads - 1) / kVecThreads > 0 ? (P.n + kVecThreads - 1) / kVecThreads : 1;
  k_margins<<<gn, kVecThreads, 0, s>>>(P, Wk.y, nullptr, 0, Wk.marg, (sampled || fast) ? nullptr : Wk.s,
                                       fast ? Wk.s_fx : nullptr, Wk.st, f32 ? Wk.marg32 : nullptr,
                                       (fast && !f32) ? Wk.marg2 : nullptr,
                                       (fast && !f32 && Wk.plan.fast_rows) ? Wk.marg32c : nullptr);
  if (seg_begin) cudaEventRecord(seg_begin, s);
  cudaError_t e;
  int zparts = Wk.seg_blocks;
  if (fast) {
    e = launch_segment_pass(P, Wk, cfg, Wk.marg, true, s, &zparts);
  } else {
    e = sampled ? launch_segments_w<kIterate, true>(P, Wk, Wk.marg, Wk.zpart, Wk.st, cfg, s)
                : launch_segments_w<kIterate, false>(P, Wk, Wk.marg, Wk.zpart, Wk.st, cfg, s, Wk.xsum);
  }
  if (seg_end) cudaEventRecord(seg_end, s);
  if (e != cudaSuccess) return e;
  const bool rows = rows_active(Wk, cfg, sampled);  // segments the row-exact kernel left for binary64
  FastArgs R{P, Wk.marg, nullptr, nullptr, Wk.st, Wk.fx_scale, Wk.fallbacks, Wk.fx_bits, Wk.s_fx};
  R.rx = Wk.rx;
  // the row-exact kernel keeps per-block sums exactly when it has shared memory for them (rows_smem)
  if (rows) {
    e = Wk.plan.rows_smem > 0 ? launch_reduce_redo(R, Wk.plan, zparts, Wk.part, s)
                              : launch_rows_redo(R, Wk.plan.rows_redo_grid, s);
    if (e != cudaSuccess) return e;
  } else if (fast) {
    e = launch_reduce_products(P, Wk.plan, zparts, Wk.part, Wk.s_fx, Wk.st, s);
    if (e != cudaSuccess) return e;
  }
  k_dual_step<<<gv, kVecThreads, 0, s>>>(P, Wk, cfg, sampled ? 0 : 1, zparts);
  return cudaGetLastError();
}

cudaError_t launch_eval(const Problem& P, const Work& Wk, const RunConfig& cfg, cudaStream_t s) {
  if (Wk.batch) return launch_batch_eval(P, Wk, cfg, s);
  const int gn = (P.n + kVecThreads - 1) / kVecThreads > 0 ? (P.n + kVecThreads - 1) / kVecThreads : 1;
  k_margins<<<gn, kVecThreads, 0, s>>>(P, nullptr, Wk.sum_y, 1, Wk.marg_eval, nullptr, nullptr, Wk.st, nullptr,
                                       Wk.fast ? Wk.marg2_eval : nullptr);
  cudaError_t e;
  int zparts = Wk.seg_blocks;
  if (Wk.fast) {
    e = launch_segment_pass(P, Wk, cfg, Wk.marg_eval, false, s, &zparts);
  } else {
    e = launch_segments_w<kEvalSum, false>(P, Wk, Wk.marg_eval, Wk.zpart_eval, Wk.st, cfg, s);
  }
  if (e != cudaSuccess) return e;
  k_eval_finish<<<1, 1024, 0, s>>>(P, Wk, cfg, zparts);
  return cudaGetLastError();
}

// Product sales of every segment's best response at the duals in Wk.y_eval
// (the expected sales of bid-price control at those prices), into Wk.s.
cudaError_t launch_sales_at(const Problem& P, const Work& Wk, cudaStream_t s) {
  RunConfig cfg{};
  const int gn = (P.n + kVecThreads - 1) / kVecThreads > 0 ? (P.n + kVecThreads - 1) / kVecThreads : 1;
  k_margins<<<gn, kVecThreads, 0, s>>>(P, Wk.y_eval, nullptr, 0, Wk.marg_eval, Wk.s, nullptr, nullptr);
  return launch_segments_w<kIterate, false>(P, Wk, Wk.marg_eval, Wk.zpart_eval, nullptr, cfg, s);
}

cudaError_t launch_evaluate_at(const Problem& P, const Work& Wk, bool want_seg, cudaStream_t s) {
  RunConfig cfg{};
  k_margins<<<(P.n + kVecThreads - 1) / kVecThreads > 0 ? (P.n + kVecThreads - 1) / kVecThreads : 1, kVecThreads,
              0, s>>>(P, Wk.y_eval, nullptr, 0, Wk.marg_eval, nullptr, nullptr, nullptr);
  cudaError_t e = want_seg ? launch_segments_w<kEvalSeg, false>(P, Wk, Wk.marg_eval, Wk.zpart_eval, nullptr, cfg, s)
                           : launch_segments_w<kEvalSum, false>(P, Wk, Wk.marg_eval, Wk.zpart_eval, nullptr, cfg, s);
  if (e != cudaSuccess) return e;
  k_evaluate_finish<<<1, 1024, 0, s>>>(P, Wk);
  return cudaGetLastError();
}

namespace {

__global__ void k_xbar(long long nnz, const double* __restrict__ xsum, const DevState* st, double* __restrict__ out) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  const double cnt = (double)st->count;
  out[p] = st->count > 0 ? __ddiv_rn(xsum[p], cnt) : CUDART_NAN;
}

// Lemma recover, one group of W lanes per segment: ranks by u = x / v
// (bitonic sort on the binary64 values, ties by lower CSR position), the
// balance row gives x_0, and alpha_r = (u_(r) - u_(r+1)) D_r / lam with D_r the
// prefix of vt over the ranking started at vt_0.
template <int W>
__global__ void __launch_bounds__(kSegThreads) k_recover(Problem P, const double* __restrict__ x,
                                                         double* __restrict__ alpha, int* __restrict__ order) {
  const int lane = threadIdx.x & (W - 1);
  const int gbase = (threadIdx.x & 31) & ~(W - 1);
  const unsigned mask = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << gbase);
  const long long gpb = kSegThreads / W, ngroups = (long long)gridDim.x * gpb;
  for (long long l = blockIdx.x * gpb + threadIdx.x / W; l < P.L; l += ngroups) {
    const long long b = P.seg_ptr[l];
    const int K = (int)(P.seg_ptr[l + 1] - b);
    const double lam = P.lam[l], vt0 = P.vt0[l];
    double u = -CUDART_INF, vt = 0.0, bal = 0.0;
    if (lane < K) {
      const double v = P.v[b + lane], xv = x[b + lane];
      vt = P.vt[b + lane];
      u = __ddiv_rn(xv, v);
      bal = __dmul_rn(__ddiv_rn(vt, v), xv);
    }
#pragma unroll
    for (int o = W >> 1; o > 0; o >>= 1) bal = __dadd_rn(bal, __shfl_xor_sync(mask, bal, o, W));
    int idx = lane;
#pragma unroll
    for (int k = 2; k <= W; k <<= 1)
#pragma unroll
      for (int d = k >> 1; d > 0; d >>= 1) {
        const double ou = __shfl_xor_sync(mask, u, d, W);
        const int oi = __shfl_xor_sync(mask, idx, d, W);
        const bool other_first = (ou > u) || (ou == u && oi < idx);
        if (((lane & k) == 0) == ((lane & d) == 0) ? other_first : !other_first) {
          u = ou;
          idx = oi;
        }
      }
    const double vt_r = __shfl_sync(mask, vt, idx, W);
    double D = lane < K ? vt_r : 0.0;
#pragma unroll
    for (int d = 1; d < W; d <<= 1) {
      const double t = __shfl_up_sync(mask, D, d, W);
      if (lane >= d) D = __dadd_rn(D, t);
    }
    D = __dadd_rn(vt0, D);
    const double nxt = __shfl_down_sync(mask, u, 1, W);
    const double u1 = __shfl_sync(mask, u, 0, W);
    double* al = alpha + b + l;
    if (!(lam > 0.0)) {
      if (lane == 0) al[0] = 1.0;
      if (lane < K) al[lane + 1] = 0.0;
    } else {
      if (lane == 0) {
        const double u0 = __ddiv_rn(__dsub_rn(lam, bal), vt0);
        al[0] = __ddiv_rn(__dmul_rn(__dsub_rn(u0, K > 0 ? u1 : 0.0), vt0), lam);
      }
      if (lane < K) {
        const double next = lane + 1 < K ? nxt : 0.0;
        al[lane + 1] = __ddiv_rn(__dmul_rn(__dsub_rn(u, next), D), lam);
      }
    }
    if (order && lane < K) order[b + lane] = idx;
  }
}

}  // namespace

cudaError_t launch_xbar(const Problem& P, const Work& Wk, double* out, cudaStream_t s) {
  if (!Wk.xsum) return cudaErrorInvalidValue;
  if (P.nnz > 0) k_xbar<<<(unsigned)((P.nnz + 255) / 256), 256, 0, s>>>(P.nnz, Wk.xsum, Wk.st, out);
  return cudaGetLastError();
}

cudaError_t launch_recover(const Problem& P, const Work& Wk, const double* x, double* alpha, int* order,
                           cudaStream_t s) {
  const int g = Wk.seg_blocks;
  switch (Wk.W) {
    case 1: k_recover<1><<<g, kSegThreads, 0, s>>>(P, x, alpha, order); break;
    case 2: k_recover<2><<<g, kSegThreads, 0, s>>>(P, x, alpha, order); break;
    case 4: k_recover<4><<<g, kSegThreads, 0, s>>>(P, x, alpha, order); break;
    case 8: k_recover<8><<<g, kSegThreads, 0, s>>>(P, x, alpha, order); break;
    case 16: k_recover<16><<<g, kSegThreads, 0, s>>>(P, x, alpha, order); break;
    case 32: k_recover<32><<<g, kSegThreads, 0, s>>>(P, x, alpha, order); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int kernel_launches_per_iteration(const Work& Wk, const RunConfig& cfg) {
  if (Wk.batch) return batch_launches_per_iteration(Wk);
  if (!(Wk.fast && cfg.batch_frac >= 1.0)) return 3;
  if (rows_active(Wk, cfg, false)) return 4;  // margins, row-exact pass, fold + redo (or redo), dual step
  return Wk.plan.scatter == 1 ? 4 : 3;
}

namespace {
__global__ void k_prep_f32_items(long long nnz, const double* __restrict__ v, const double* __restrict__ vt,
                                 float* __restrict__ v32, float* __restrict__ vt32) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p < nnz) {
    v32[p] = __double2float_rn(v[p]);
    vt32[p] = __double2float_rn(vt[p]);
  }
}
__global__ void k_prep_f32_segments(long long L, const double* __restrict__ lam, const double* __restrict__ vt0,
                                    float* __restrict__ lam32, float* __restrict__ vt0_32) {
  const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l < L) {
    lam32[l] = __double2float_rn(lam[l]);
    vt0_32[l] = __double2float_rn(vt0[l]);
  }
}
}  // namespace

cudaError_t launch_prep_f32(const Problem& P, Work& Wk, cudaStream_t s) {
  if (P.nnz > 0) k_prep_f32_items<<<(unsigned)((P.nnz + 255) / 256), 256, 0, s>>>(P.nnz, P.v, P.vt, Wk.v32, Wk.vt32);
  if (P.L > 0) k_prep_f32_segments<<<(unsigned)((P.L + 255) / 256), 256, 0, s>>>(P.L, P.lam, P.vt0, Wk.lam32, Wk.vt0_32);
  return cudaGetLastError();
}
int kernel_launches_per_eval() { return 3; }  // single instance and batch alike

namespace {
// End of one evaluation period inside the device loop: count the period, and
// keep looping unless the iteration has converged (every member of a batch),
// the phase's cap is reached, or a binary32 batch is down to its last 5 % of
// members (the host then switches to binary64 iterations).
__global__ void k_loop_test(const Work Wk, DevLoop* lp, cudaGraphConditionalHandle h, int E) {
  __shared__ int active;
  if (threadIdx.x == 0) active = 0;
  __syncthreads();
  int conv = 0;
  if (Wk.batch) {
    int a = 0;
    for (int b = threadIdx.x; b < Wk.bm.count; b += blockDim.x) a += Wk.bm.conv[b] ? 0 : 1;
    atomicAdd(&active, a);
    __syncthreads();
    conv = active == 0;
  } else {
    conv = Wk.st->converged;
  }
  if (threadIdx.x != 0) return;
  const long long t = Wk.batch ? lp->t + E : Wk.st->t;
  lp->t = t;
  int ended = conv ? 1 : (t + E > lp->t_end ? 2 : 0);
  if (!ended && lp->batch_switch && (long long)active * 20 <= (long long)Wk.bm.count) ended = 3;
  lp->ended = ended;
  cudaGraphSetConditional(h, ended ? 0u : 1u);
}
}  // namespace

cudaError_t launch_loop_test(const Work& Wk, DevLoop* lp, cudaGraphConditionalHandle h, int E, cudaStream_t s) {
  k_loop_test<<<1, 256, 0, s>>>(Wk, lp, h, E);
  return cudaGetLastError();
}

}  // namespace spfom
