// Batched re-solves (spfom_load_batch): many choice-based LPs in one set of
// launches.
//
// Instances share no product, resource or segment, so a batch is the
// block-diagonal union of its instances: the margins, the segment pass and the
// sales reduction run over the union unchanged, one launch each for the whole
// batch. What differs per instance is the scalar side of the iteration, kept in
// an InstState per instance: the step size tau_b = tau0 mean(r_b)/mean(c_b), the
// regulariser, the epoch sums, the KKT residual, the restart test and the
// convergence flag. A converged instance is frozen: the segment kernels skip
// its segments and the dual step leaves its duals alone, so the batch's cost
// falls as instances converge. Per-instance sums (sum z_l, c^T y, r^T s, the
// KKT terms) are taken by one block per instance over the instance's contiguous
// segment, resource and product ranges, in a fixed order.
//
// This serves Section 5.1's multi-period setting: each period re-solves every
// base instance with its remaining capacities (spfom_batch_update) warm-started
// from the previous period's duals, which are the bid prices of the period.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "spfom_device.cuh"
#include "spfom_internal.h"

namespace spfom {

namespace {

constexpr int kThreads = 256;

__device__ double bsum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
  return t;  // thread 0
}

// Margins m_j = r_j - sum_i a_ij y_i (avg: y = sum_y / count of the product's
// instance); clears the fixed-point sales and fills the binary32 copy if asked.
__global__ void k_b_margins(Problem P, BatchMaps B, const double* __restrict__ y, const double* __restrict__ sum_y,
                            int avg, double* __restrict__ marg, float* __restrict__ marg32,
                            unsigned long long* __restrict__ sfx_clear, float2* __restrict__ marg2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P.n) return;
  const InstState& I = B.inst[B.prod_inst[j]];
  if (I.converged) return;
  const double cnt = avg ? (double)I.count : 1.0;
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
  if (marg2) marg2[j] = m > 0.0 ? split_pair(m) : make_float2(m < 0.0 ? -1.f : 0.f, 0.f);
  if (sfx_clear) sfx_clear[j] = 0ull;
}

// Dual step of every resource with its instance's tau and mu; epoch sums;
// product sales in binary64 for the reductions.
__global__ void k_b_dual(Problem P, Work Wk) {
  const BatchMaps& B = Wk.bm;
  // First blocks: one warp per resource (the lanes fetch its products' sales
  // together; unit incidence: the exact fixed-point sum, rounded once; else
  // lane 0 adds the binary64 terms in ascending product order). Then one
  // thread per product.
  constexpr int kWarps = kThreads / 32;
  const int rblocks = (P.m + kWarps - 1) / kWarps;
  if ((int)blockIdx.x < rblocks) {
    const int i = blockIdx.x * kWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= P.m) return;
    const InstState& I = B.inst[B.res_inst[i]];
    if (I.converged) return;  // uniform over the warp
    const int q0 = P.at_ptr[i], q1 = P.at_ptr[i + 1];
    double g = 0.0;
    if (!P.at_val) {
      unsigned long long acc = 0ull;
      for (int q = q0 + lane; q < q1; q += 32) acc += Wk.s_fx[P.at_idx[q]];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      g = __dmul_rn(__ull2double_rn(acc), Wk.inv_fx_scale);
    } else {
      for (int qb = q0; qb < q1; qb += 32) {
        const int q = qb + lane;
        const double term = q < q1 ? __dmul_rn(P.at_val[q], __dmul_rn(__ull2double_rn(Wk.s_fx[P.at_idx[q]]),
                                                                       Wk.inv_fx_scale))
                                   : 0.0;
        const int cnt = q1 - qb < 32 ? q1 - qb : 32;
        for (int k = 0; k < cnt; ++k) {
          const double t = __shfl_sync(0xffffffffu, term, k);
          if (lane == 0) g = __dadd_rn(g, t);
        }
      }
    }
    if (lane != 0) return;
    const double shrink = __dsub_rn(1.0, __dmul_rn(I.tau, I.mu));
    const double yo = Wk.y[i], c = P.c[i];
    const double yn = __dsub_rn(__dmul_rn(shrink, yo), __dmul_rn(I.tau, __dsub_rn(c, g)));
    Wk.y[i] = yn > 0.0 ? yn : 0.0;
    Wk.g[i] = g;
    Wk.sum_y[i] = __dadd_rn(Wk.sum_y[i], yo);
    Wk.sum_g[i] = __dadd_rn(Wk.sum_g[i], g);
    B.cy_res[i] = yo != 0.0 ? __dmul_rn(c, yo) : 0.0;
    return;
  }
  const int j = (blockIdx.x - rblocks) * blockDim.x + threadIdx.x;
  if (j < P.n && !B.inst[B.prod_inst[j]].converged)
    Wk.s[j] = __dmul_rn(__ull2double_rn(Wk.s_fx[j]), Wk.inv_fx_scale);
}

// One block per instance: sum z_l (= sum_j m_j s_j), c^T y, r^T s of the
// iteration; counters.
constexpr int kFinThreads = 1024;

// sum of z_seg over [l0, l1) by the block: four interleaved accumulators per
// thread (a fixed order), so the dependent binary64 adds are a quarter as deep
__device__ double seg_sum(const double* __restrict__ z, long long l0, long long l1) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  const long long st = blockDim.x;
  long long l = l0 + threadIdx.x;
  for (; l + 3 * st < l1; l += 4 * st) {
    a0 += z[l];
    a1 += z[l + st];
    a2 += z[l + 2 * st];
    a3 += z[l + 3 * st];
  }
  for (; l < l1; l += st) a0 += z[l];
  return (a0 + a1) + (a2 + a3);
}

__global__ void __launch_bounds__(kFinThreads) k_b_finish(Problem P, Work Wk) {
  __shared__ double sh[32];
  const BatchMaps& B = Wk.bm;
  const int b = blockIdx.x;
  InstState& I = B.inst[b];
  if (I.converged) return;
  double zs = 0.0, cys = 0.0, Ps = 0.0;
  for (int i = B.res_ptr[b] + threadIdx.x; i < B.res_ptr[b + 1]; i += blockDim.x) cys += B.cy_res[i];
  for (int j = B.prod_ptr[b] + threadIdx.x; j < B.prod_ptr[b + 1]; j += blockDim.x) {
    Ps += __dmul_rn(P.r[j], Wk.s[j]);
    zs += __dmul_rn(Wk.marg[j], Wk.s[j]);  // sum_l z_l = sum_j m_j s_j over the instance
  }
  zs = bsum(zs, sh);
  cys = bsum(cys, sh);
  Ps = bsum(Ps, sh);
  if (threadIdx.x == 0) {
    I.z_sum = zs;
    I.dual_iter = cys + zs;
    I.P = Ps;
    I.sum_P += Ps;
    I.count += 1;
    I.t += 1;
  }
}

// One block per instance: KKT residual of the epoch averages and the restart
// test, as for a single instance.
__global__ void __launch_bounds__(kFinThreads) k_b_eval_finish(Problem P, Work Wk, RunConfig cfg) {
  __shared__ double sh[32];
  __shared__ int restart, progress;
  const BatchMaps& B = Wk.bm;
  const int b = blockIdx.x;
  InstState& I = B.inst[b];
  if (I.converged) return;
  const double cnt = (double)I.count;
  const int i0 = B.res_ptr[b], i1 = B.res_ptr[b + 1];
  double cy = 0.0, over2 = 0.0, c2 = 0.0, zs = 0.0;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double yb = __ddiv_rn(Wk.sum_y[i], cnt), gb = __ddiv_rn(Wk.sum_g[i], cnt), c = P.c[i];
    if (yb != 0.0) cy += __dmul_rn(c, yb);
    const double o = __dsub_rn(gb, c);
    if (o > 0.0) over2 += __dmul_rn(o, o);
    c2 += __dmul_rn(c, c);
  }
  zs = seg_sum(B.z_seg, B.seg_off[b], B.seg_off[b + 1]);
  cy = bsum(cy, sh);
  over2 = bsum(over2, sh);
  c2 = bsum(c2, sh);
  zs = bsum(zs, sh);
  if (threadIdx.x == 0) {
    const double Pbar = I.sum_P / cnt;
    const double D = cy + zs;
    const double pinf = sqrt(over2) / (1.0 + sqrt(c2));
    const double gap = fabs(D - Pbar) / (1.0 + fabs(D) + fabs(Pbar));
    const double kkt = pinf > gap ? pinf : gap;
    I.pinf = pinf;
    I.gap = gap;
    I.kkt = kkt;
    I.dual_avg = D;
    I.primal_avg = Pbar;
    I.evals += 1;
    I.converged = kkt <= cfg.kkt_tol;
    B.conv[b] = I.converged;
    progress = kkt <= cfg.restart_beta * I.kkt_anchor;
    restart = !I.converged && (progress || (double)I.count >= cfg.restart_artificial * (double)I.t);
  }
  __syncthreads();
  if (!restart) return;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    Wk.y[i] = __ddiv_rn(Wk.sum_y[i], cnt);
    Wk.sum_y[i] = 0.0;
    Wk.sum_g[i] = 0.0;
  }
  if (threadIdx.x == 0) {
    I.sum_P = 0.0;
    I.count = 0;
    I.kkt_anchor = I.kkt;
    if (I.mu > 0.0) I.mu *= 0.5;
    I.tau *= cfg.restart_tau_decay;
    if (!progress && cfg.restart_tau_balance > 0.0) I.tau *= balance_factor(I.pinf, I.gap, cfg.restart_tau_balance);
    I.restarts += 1;
  }
}

int blocks_for(int n) { return n > 0 ? (n + kThreads - 1) / kThreads : 1; }

}  // namespace

cudaError_t launch_batch_iteration(const Problem& P, const Work& Wk, const RunConfig& cfg, cudaStream_t s,
                                   cudaEvent_t seg_begin, cudaEvent_t seg_end) {
  const bool f32 = cfg.f32 && Wk.v32;
  k_b_margins<<<blocks_for(P.n), kThreads, 0, s>>>(P, Wk.bm, Wk.y, nullptr, 0, Wk.marg, f32 ? Wk.marg32 : nullptr,
                                                    Wk.s_fx, f32 ? nullptr : Wk.marg2);
  int zparts = 0;
  if (seg_begin) cudaEventRecord(seg_begin, s);
  cudaError_t e = launch_segment_pass(P, Wk, cfg, Wk.marg, true, s, &zparts);
  if (seg_end) cudaEventRecord(seg_end, s);
  if (e != cudaSuccess) return e;
  e = launch_reduce_products(P, Wk.plan, zparts, Wk.part, Wk.s_fx, Wk.st, s);
  if (e != cudaSuccess) return e;
  k_b_dual<<<(P.m + kThreads / 32 - 1) / (kThreads / 32) + blocks_for(P.n), kThreads, 0, s>>>(P, Wk);
  k_b_finish<<<Wk.bm.count, kFinThreads, 0, s>>>(P, Wk);
  return cudaGetLastError();
}

cudaError_t launch_batch_eval(const Problem& P, const Work& Wk, const RunConfig& cfg, cudaStream_t s) {
  k_b_margins<<<blocks_for(P.n), kThreads, 0, s>>>(P, Wk.bm, nullptr, Wk.sum_y, 1, Wk.marg_eval, nullptr, nullptr,
                                                    Wk.marg2_eval);
  int zparts = 0;
  cudaError_t e = launch_segment_pass(P, Wk, cfg, Wk.marg_eval, false, s, &zparts);
  if (e != cudaSuccess) return e;
  k_b_eval_finish<<<Wk.bm.count, kFinThreads, 0, s>>>(P, Wk, cfg);
  return cudaGetLastError();
}

int batch_launches_per_iteration(const Work& Wk) { return Wk.plan.scatter == 1 ? 5 : 4; }
int batch_launches_per_eval() { return 3; }

}  // namespace spfom
