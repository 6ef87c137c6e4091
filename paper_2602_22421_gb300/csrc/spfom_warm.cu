// Per-resource features of the learned warm start (spfom_features in
// include/spfom_mlp.h) and the scaling of the network's output to duals.
//
// The features describe each resource at zero prices: the expected sales
// s_j(0) of every segment's best assortment when nothing is priced (the segment
// pass at y = 0, Section 4.1 inner problem), the demand d_i = sum_j a_ij s_j(0)
// that would fall on the resource, its capacity, and the prices of the
// products that use it, weighted by the demand they bring (a_ij s_j(0)). The
// duals of the capacity rows are the bid prices of Section 5.1, measured in
// revenue units, so revenue features are divided by mean(r) and capacity
// features by mean(c); the network predicts y_i / mean(r).
#include <cuda_runtime.h>

#include "../../include/spfom_mlp.h"
#include "spfom_device.cuh"
#include "spfom_internal.h"

namespace spfom {

namespace {

constexpr int kT = 256;
constexpr double kRhoCap = 8.0;

// totals[0] = sum r, totals[1] = sum c, totals[2] = sum d (one block, fixed order).
__global__ void k_warm_totals(Problem P, const double* __restrict__ d, double* __restrict__ totals) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int j = threadIdx.x; j < P.n; j += blockDim.x) a += P.r[j];
  for (int i = threadIdx.x; i < P.m; i += blockDim.x) {
    b += P.c[i];
    c += d[i];
  }
  a = block_sum_d(a, sh);
  b = block_sum_d(b, sh);
  c = block_sum_d(c, sh);
  if (threadIdx.x == 0) {
    totals[0] = a;
    totals[1] = b;
    totals[2] = c;
  }
}

// d_i = sum_j a_ij s_j(0) over the resource's products.
__global__ void k_warm_demand(Problem P, const double* __restrict__ s0, double* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.m) return;
  double acc = 0.0;
  for (int q = P.at_ptr[i]; q < P.at_ptr[i + 1]; ++q) acc += (P.at_val ? P.at_val[q] : 1.0) * s0[P.at_idx[q]];
  d[i] = acc;
}

__device__ __forceinline__ double load_ratio(double d, double c) {
  if (d <= 0.0) return 0.0;
  if (c <= 0.0) return kRhoCap;
  const double r = d / c;
  return r < kRhoCap ? r : kRhoCap;
}

// rho_j = the largest min(d_k / c_k, 8) over the resources k of product j.
__global__ void k_warm_prod(Problem P, const double* __restrict__ d, double* __restrict__ rho) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P.n) return;
  double best = 0.0;
  for (int q = P.a_ptr[j]; q < P.a_ptr[j + 1]; ++q) {
    const int k = P.a_idx[q];
    const double r = load_ratio(d[k], P.c[k]);
    best = r > best ? r : best;
  }
  rho[j] = best;
}

__global__ void k_warm_features(Problem P, const double* __restrict__ s0, const double* __restrict__ d,
                                const double* __restrict__ rho, const double* __restrict__ totals,
                                float* __restrict__ f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.m) return;
  const double mean_r = P.n ? totals[0] / P.n : 1.0, mean_c = P.m ? totals[1] / P.m : 1.0;
  const double rs = mean_r > 0.0 ? 1.0 / mean_r : 0.0, cs = mean_c > 0.0 ? 1.0 / mean_c : 0.0;
  const double nnz_per_res = P.m ? (double)P.a_ptr[P.n] / P.m : 1.0;
  double w = 0.0, wr = 0.0, wr2 = 0.0, wshare = 0.0, wrho = 0.0, rmax = 0.0;
  const int q0 = P.at_ptr[i], q1 = P.at_ptr[i + 1];
  for (int q = q0; q < q1; ++q) {
    const int j = P.at_idx[q];
    const double a = (P.at_val ? P.at_val[q] : 1.0) * s0[j], r = P.r[j];
    const int nres = P.a_ptr[j + 1] - P.a_ptr[j];
    w += a;
    wr += a * r;
    wr2 += a * r * r;
    wshare += a * r / (nres > 0 ? nres : 1);
    wrho += a * rho[j];
    rmax = r > rmax ? r : rmax;
  }
  const double c = P.c[i], di = d[i];
  const double mean = w > 0.0 ? wr / w : 0.0;
  const double var = w > 0.0 ? wr2 / w - mean * mean : 0.0;
  double lr = (di > 0.0 && c > 0.0) ? log(di / c) : (di > 0.0 ? 6.0 : -6.0);
  lr = lr < -6.0 ? -6.0 : (lr > 6.0 ? 6.0 : lr);
  const double ratio = di > 0.0 ? (c / di < 4.0 ? c / di : 4.0) : 4.0;
  float* o = f + (size_t)i * SPFOM_MLP_FEATURES;
  o[0] = (float)(c * cs);
  o[1] = (float)(di * cs);
  o[2] = (float)ratio;
  o[3] = (float)lr;
  o[4] = (float)(mean * rs);
  o[5] = (float)(rmax * rs);
  o[6] = (float)(sqrt(var > 0.0 ? var : 0.0) * rs);
  o[7] = (float)(w > 0.0 ? wshare / w * rs : 0.0);
  o[8] = (float)((q1 - q0) / (nnz_per_res > 0.0 ? nnz_per_res : 1.0));
  o[9] = (float)(totals[2] > 0.0 ? totals[1] / totals[2] : 4.0);
  o[10] = (float)(w > 0.0 ? wrho / w : 0.0);
  o[11] = 1.f;
  o[12] = di > c ? 1.f : 0.f;
  o[13] = o[14] = o[15] = 0.f;
}

// y0_i = max(0, o_i) mean(r) (binary64), from the network outputs o.
__global__ void k_warm_duals(int m, const float* __restrict__ o, const double* __restrict__ totals, int n,
                             double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double mean_r = n ? totals[0] / n : 1.0;
  const double v = (double)o[i];
  y[i] = v > 0.0 ? v * mean_r : 0.0;
}

int nb(long long n) { return n > 0 ? (int)((n + kT - 1) / kT) : 1; }

}  // namespace

// Features of the loaded single instance: s0 [n] (the sales at y = 0, already
// computed into it), scratch d [m], rho [n], totals [3]; f [m][16].
cudaError_t launch_features(const Problem& P, const double* s0, double* d, double* rho, double* totals, float* f,
                            cudaStream_t s) {
  k_warm_demand<<<nb(P.m), kT, 0, s>>>(P, s0, d);
  k_warm_totals<<<1, 1024, 0, s>>>(P, d, totals);
  k_warm_prod<<<nb(P.n), kT, 0, s>>>(P, d, rho);
  k_warm_features<<<nb(P.m), kT, 0, s>>>(P, s0, d, rho, totals, f);
  return cudaGetLastError();
}

cudaError_t launch_warm_duals(int m, int n, const float* o, const double* totals, double* y, cudaStream_t s) {
  k_warm_duals<<<nb(m), kT, 0, s>>>(m, o, totals, n, y);
  return cudaGetLastError();
}

}  // namespace spfom
