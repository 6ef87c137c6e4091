// C ABI of the SPFOM library (declared in include/spfom.h): validation and
// upload of an instance, the ctx's device buffers, and the host-side order of
// kernel launches. Every decision inside a run of iterations (convergence,
// restart, step size) is taken on the device, so spfom_step enqueues its
// launches without reading anything back until the end of the call.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/spfom.h"
#include "spfom_internal.h"

using spfom::DevState;
using spfom::Problem;
using spfom::RunConfig;
using spfom::Work;

struct spfom_ctx {
  spfom_params p{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  bool loaded = false;
  Problem P{};
  Work W{};
  RunConfig cfg{};
  double tau_init = 0.0;
  long long host_t = 0;
  std::vector<void*> bufs;  // device allocations of the loaded instance
  DevState* d_state = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> prof_ev;  // event pairs of profiled segment launches
  int sms = 0;
  unsigned long long fallback_host = 0;
  bool polishing = false;  // precision 32: binary64 iterations after the first converged evaluation
  cudaGraphExec_t period[2] = {nullptr, nullptr};  // one evaluation period, [binary64, binary32 pass]
  bool period_failed = false;                      // capture unavailable on this stream
};

namespace {

spfom_status fail(spfom_ctx* ctx, spfom_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  return s;
}

spfom_status cuda_fail(spfom_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, SPFOM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SPFOM_CUDA(ctx, call)                                       \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);     \
  } while (0)

void drop_graphs(spfom_ctx* ctx) {
  for (auto& g : ctx->period)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  ctx->period_failed = false;
}

void free_instance(spfom_ctx* ctx) {
  drop_graphs(ctx);
  for (void* b : ctx->bufs) cudaFreeAsync(b, ctx->stream);
  ctx->bufs.clear();
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  ctx->loaded = false;
  ctx->P = Problem{};
  Work w{};
  w.st = ctx->W.st;
  ctx->W = w;
}

template <class T>
spfom_status dalloc(spfom_ctx* ctx, T** out, size_t count) {
  *out = nullptr;
  if (count == 0) count = 1;
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, count * sizeof(T), ctx->stream);
  if (e != cudaSuccess) return fail(ctx, SPFOM_ENOMEM, "device allocation of %zu bytes: %s", count * sizeof(T),
                                    cudaGetErrorString(e));
  ctx->bufs.push_back(p);
  *out = static_cast<T*>(p);
  return SPFOM_OK;
}

// Copy count elements; `slack` more elements are allocated after them and
// zeroed (bulk copies widened to 16-byte boundaries may read them).
template <class T>
spfom_status upload(spfom_ctx* ctx, T** out, const T* src, size_t count, size_t slack = 0) {
  spfom_status s = dalloc(ctx, out, count + slack);
  if (s != SPFOM_OK) return s;
  if (count) SPFOM_CUDA(ctx, cudaMemcpyAsync(*out, src, count * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  if (slack) SPFOM_CUDA(ctx, cudaMemsetAsync(*out + count, 0, slack * sizeof(T), ctx->stream));
  return SPFOM_OK;
}

constexpr size_t kSlack = 4;  // elements of zeroed slack after arrays that bulk copies read

bool is_finite(double x) { return std::isfinite(x); }

spfom_status validate(spfom_ctx* ctx, const spfom_instance* I, int* kmax_out) {
  if (!I) return fail(ctx, SPFOM_EINVAL, "instance is NULL");
  if (I->n < 0 || I->m < 0 || I->L < 0) return fail(ctx, SPFOM_EINVAL, "negative size");
  if ((I->n > 0 && (!I->r || !I->a_ptr)) || (I->m > 0 && !I->c) || !I->seg_ptr || (I->L > 0 && (!I->lam || !I->v0)))
    return fail(ctx, SPFOM_EINVAL, "missing array");
  for (int j = 0; j < I->n; ++j)
    if (!is_finite(I->r[j])) return fail(ctx, SPFOM_EINVAL, "r[%d] is not finite", j);
  for (int i = 0; i < I->m; ++i)
    if (!(I->c[i] >= 0.0) || !is_finite(I->c[i])) return fail(ctx, SPFOM_EINVAL, "c[%d] must be finite and >= 0", i);
  if (I->n > 0 && I->a_ptr[0] != 0) return fail(ctx, SPFOM_EINVAL, "a_ptr[0] != 0");
  std::vector<int> stamp((size_t)(I->m > I->n ? I->m : I->n) + 1, -1);
  for (int j = 0; j < I->n; ++j) {
    if (I->a_ptr[j + 1] < I->a_ptr[j]) return fail(ctx, SPFOM_EINVAL, "a_ptr not monotone at %d", j);
    for (int q = I->a_ptr[j]; q < I->a_ptr[j + 1]; ++q) {
      int i = I->a_idx[q];
      if (i < 0 || i >= I->m) return fail(ctx, SPFOM_EINVAL, "a_idx[%d] = %d out of range", q, i);
      if (stamp[i] == j) return fail(ctx, SPFOM_EINVAL, "resource %d repeated for product %d", i, j);
      stamp[i] = j;
      if (I->a_val && !(I->a_val[q] > 0.0 && is_finite(I->a_val[q])))
        return fail(ctx, SPFOM_EINVAL, "a_val[%d] must be finite and > 0", q);
    }
  }
  if (I->seg_ptr[0] != 0) return fail(ctx, SPFOM_EINVAL, "seg_ptr[0] != 0");
  std::fill(stamp.begin(), stamp.end(), -1);
  std::vector<long long> stampl((size_t)I->n + 1, -1);
  int kmax = 0;
  for (long long l = 0; l < I->L; ++l) {
    long long b = I->seg_ptr[l], e = I->seg_ptr[l + 1];
    if (e < b) return fail(ctx, SPFOM_EINVAL, "seg_ptr not monotone at %lld", l);
    if (e - b > kmax) kmax = (int)(e - b > 1 << 30 ? 1 << 30 : e - b);
    if (!(I->lam[l] >= 0.0) || !is_finite(I->lam[l])) return fail(ctx, SPFOM_EINVAL, "lam[%lld] must be >= 0", l);
    if (!(I->v0[l] > 0.0) || !is_finite(I->v0[l])) return fail(ctx, SPFOM_EINVAL, "v0[%lld] must be > 0", l);
    for (long long p = b; p < e; ++p) {
      int j = I->seg_prod[p];
      if (j < 0 || j >= I->n) return fail(ctx, SPFOM_EINVAL, "seg_prod[%lld] = %d out of range", p, j);
      if (stampl[j] == l) return fail(ctx, SPFOM_EINVAL, "product %d repeated in segment %lld", j, l);
      stampl[j] = l;
      double v = I->v[p];
      if (!(v > 0.0) || !is_finite(v)) return fail(ctx, SPFOM_EINVAL, "v[%lld] must be finite and > 0", p);
      if (I->w) {
        double w = I->w[p];
        if (!(w >= 0.0) || !(w <= v)) return fail(ctx, SPFOM_EINVAL, "w[%lld] must lie in [0, v]", p);
      }
    }
  }
  if (I->L > 0 && (I->seg_ptr[I->L] > 0) && (!I->seg_prod || !I->v))
    return fail(ctx, SPFOM_EINVAL, "missing segment arrays");
  *kmax_out = kmax;
  return SPFOM_OK;
}

spfom_status init_state(spfom_ctx* ctx, const double* y0) {
  Work& W = ctx->W;
  const Problem& P = ctx->P;
  if (y0) {
    for (int i = 0; i < P.m; ++i)
      if (!(y0[i] >= 0.0) || !is_finite(y0[i])) return fail(ctx, SPFOM_EINVAL, "y0[%d] must be finite and >= 0", i);
    SPFOM_CUDA(ctx, cudaMemcpyAsync(W.y, y0, sizeof(double) * P.m, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    SPFOM_CUDA(ctx, cudaMemsetAsync(W.y, 0, sizeof(double) * (P.m ? P.m : 1), ctx->stream));
  }
  SPFOM_CUDA(ctx, cudaMemsetAsync(W.sum_y, 0, sizeof(double) * (P.m ? P.m : 1), ctx->stream));
  SPFOM_CUDA(ctx, cudaMemsetAsync(W.sum_g, 0, sizeof(double) * (P.m ? P.m : 1), ctx->stream));
  SPFOM_CUDA(ctx, cudaMemsetAsync(W.g, 0, sizeof(double) * (P.m ? P.m : 1), ctx->stream));
  SPFOM_CUDA(ctx, cudaMemsetAsync(W.s, 0, sizeof(double) * (P.n ? P.n : 1), ctx->stream));
  SPFOM_CUDA(ctx, cudaMemsetAsync(W.marg, 0, sizeof(double) * (P.n ? P.n : 1), ctx->stream));
  if (W.x_cur) SPFOM_CUDA(ctx, cudaMemsetAsync(W.x_cur, 0, sizeof(double) * (P.nnz ? P.nnz : 1), ctx->stream));
  if (W.s_fx) SPFOM_CUDA(ctx, cudaMemsetAsync(W.s_fx, 0, sizeof(unsigned long long) * (P.n ? P.n : 1), ctx->stream));
  if (W.fallbacks) SPFOM_CUDA(ctx, cudaMemsetAsync(W.fallbacks, 0, sizeof(unsigned long long), ctx->stream));
  ctx->fallback_host = 0;
  DevState st{};
  st.tau = ctx->tau_init;
  st.mu = ctx->p.mu;
  st.z_sum = st.P = st.dual_iter = NAN;
  st.kkt = st.pinf = st.gap = st.dual_avg = st.primal_avg = NAN;
  st.kkt_anchor = INFINITY;
  SPFOM_CUDA(ctx, cudaMemcpyAsync(W.st, &st, sizeof st, cudaMemcpyHostToDevice, ctx->stream));
  SPFOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->host_t = 0;
  ctx->polishing = false;
  ctx->cfg.f32 = ctx->p.precision == 32 ? 1 : 0;
  return SPFOM_OK;
}

void fill_stats(const spfom_ctx* ctx, const DevState& st, double secs, spfom_stats* out) {
  if (!out) return;
  spfom_stats s{};
  s.fallback_segments = (long long)ctx->fallback_host;
  s.fast_path = (ctx->W.fast && ctx->cfg.batch_frac >= 1.0) ? 1 : 0;
  s.iter_precision = (s.fast_path && ctx->cfg.f32) ? 32 : 64;
  s.iters = st.t;
  s.restarts = st.restarts;
  s.evals = st.evals;
  s.epoch_iters = st.count;
  s.converged = st.converged;
  s.kkt = st.kkt;
  s.pinf = st.pinf;
  s.gap = st.gap;
  s.dual_avg = st.dual_avg;
  s.primal_avg = st.primal_avg;
  s.dual_iter = st.dual_iter;
  s.z_sum = st.z_sum;
  s.revenue = st.P;
  s.sum_revenue = st.sum_P;
  s.tau = st.tau;
  s.mu = st.mu;
  s.seconds = secs;
  *out = s;
}

spfom_status read_state(spfom_ctx* ctx, DevState* st) {
  SPFOM_CUDA(ctx, cudaMemcpyAsync(st, ctx->W.st, sizeof *st, cudaMemcpyDeviceToHost, ctx->stream));
  if (ctx->W.fallbacks)
    SPFOM_CUDA(ctx, cudaMemcpyAsync(&ctx->fallback_host, ctx->W.fallbacks, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, ctx->stream));
  SPFOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SPFOM_OK;
}

}  // namespace

extern "C" {

void spfom_default_params(spfom_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->precision = 64;
  p->tau = 0.0;
  p->tau0 = 0.1;
  p->mu = 0.0;
  p->batch_frac = 1.0;
  p->seed = 0;
  p->eval_every = 64;
  p->restart_beta = 0.2;
  p->restart_artificial = 0.36;
  p->restart_tau_decay = 1.0;
  p->kkt_tol = 1e-4;
  p->max_iters = 100000;
  p->device = 0;
  p->polish = 1;
  p->graphs = 1;
  p->pipeline = 0;
  p->stream = nullptr;
}

const char* spfom_status_string(spfom_status s) {
  switch (s) {
    case SPFOM_OK: return "SPFOM_OK";
    case SPFOM_EINVAL: return "SPFOM_EINVAL";
    case SPFOM_ENOMEM: return "SPFOM_ENOMEM";
    case SPFOM_ECUDA: return "SPFOM_ECUDA";
    case SPFOM_ESTATE: return "SPFOM_ESTATE";
    case SPFOM_ETIMEOUT: return "SPFOM_ETIMEOUT";
    case SPFOM_ENOTCONV: return "SPFOM_ENOTCONV";
    case SPFOM_ENOTSUP: return "SPFOM_ENOTSUP";
  }
  return "SPFOM_(unknown)";
}

const char* spfom_last_error(const spfom_ctx* ctx) { return ctx ? ctx->err.c_str() : "ctx is NULL"; }

spfom_status spfom_create(const spfom_params* p, spfom_ctx** out) {
  if (!out) return SPFOM_EINVAL;
  *out = nullptr;
  spfom_params prm;
  if (p) prm = *p; else spfom_default_params(&prm);
  if (prm.precision != 64 && prm.precision != 32) return SPFOM_ENOTSUP;
  if (!(prm.batch_frac > 0.0) || !(prm.restart_beta >= 0.0) || !(prm.kkt_tol >= 0.0) || prm.tau0 < 0 ||
      prm.mu < 0 || !(prm.restart_tau_decay > 0.0))
    return SPFOM_EINVAL;
  spfom_ctx* ctx = new (std::nothrow) spfom_ctx;
  if (!ctx) return SPFOM_ENOMEM;
  ctx->p = prm;
  cudaError_t e = cudaSetDevice(prm.device);
  if (e == cudaSuccess && prm.stream) {
    ctx->stream = static_cast<cudaStream_t>(prm.stream);
  } else if (e == cudaSuccess) {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    ctx->own_stream = (e == cudaSuccess);
  }
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, prm.device);
  if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_state, sizeof(DevState));
  if (e != cudaSuccess) {
    spfom_destroy(ctx);
    return SPFOM_ECUDA;
  }
  ctx->W.st = ctx->d_state;
  *out = ctx;
  return SPFOM_OK;
}

void spfom_destroy(spfom_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->p.device);
  free_instance(ctx);
  if (ctx->d_state) cudaFree(ctx->d_state);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

spfom_status spfom_load_instance(spfom_ctx* ctx, const spfom_instance* I) {
  if (!ctx) return SPFOM_EINVAL;
  int kmax = 0;
  spfom_status s = validate(ctx, I, &kmax);
  if (s != SPFOM_OK) return s;
  if (kmax > 32) return fail(ctx, SPFOM_ENOTSUP, "consideration set of %d products (at most 32 supported)", kmax);
  if (ctx->p.precision == 32) {
    // binary32 copies must stay normal numbers (zero allowed for v - w and lambda)
    auto in32 = [](double x, bool zero_ok) { return (zero_ok && x == 0.0) || (x >= 1.1754943508222875e-38 && x <= 3.4028234663852886e+38); };
    for (long long p = 0; p < I->seg_ptr[I->L]; ++p) {
      const double vt = I->w ? I->v[p] - I->w[p] : I->v[p];
      if (!in32(I->v[p], false) || !in32(vt, true))
        return fail(ctx, SPFOM_ENOTSUP, "precision 32: attraction at %lld outside binary32's normal range", p);
    }
    for (long long l = 0; l < I->L; ++l)
      if (!in32(I->lam[l], true) || !in32(I->v0[l], false))
        return fail(ctx, SPFOM_ENOTSUP, "precision 32: lambda or v0 of segment %lld outside binary32's range", l);
  }
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  free_instance(ctx);
  const int n = I->n, m = I->m;
  const long long L = I->L, nnz = I->seg_ptr[L];
  const int nnzA = n > 0 ? I->a_ptr[n] : 0;
  // resource-major copy of the incidence, products ascending within a resource
  std::vector<int> at_ptr((size_t)m + 1, 0), at_idx((size_t)nnzA);
  std::vector<double> at_val(I->a_val ? (size_t)nnzA : 0);
  for (int q = 0; q < nnzA; ++q) at_ptr[(size_t)I->a_idx[q] + 1]++;
  for (int i = 0; i < m; ++i) at_ptr[i + 1] += at_ptr[i];
  {
    std::vector<int> fillp(at_ptr.begin(), at_ptr.end() - 1);
    for (int j = 0; j < n; ++j)
      for (int q = I->a_ptr[j]; q < I->a_ptr[j + 1]; ++q) {
        int i = I->a_idx[q];
        int dst = fillp[i]++;
        at_idx[dst] = j;
        if (I->a_val) at_val[dst] = I->a_val[q];
      }
  }
  Problem P{};
  P.n = n; P.m = m; P.nnzA = nnzA; P.L = L; P.nnz = nnz;
  double *d_r, *d_c, *d_aval = nullptr, *d_atval = nullptr, *d_v, *d_w = nullptr, *d_lam, *d_v0, *d_vt, *d_vt0;
  int *d_aptr, *d_aidx, *d_atptr, *d_atidx, *d_prod;
  long long* d_segptr;
#define SPFOM_TRY(x) do { spfom_status s_ = (x); if (s_ != SPFOM_OK) { free_instance(ctx); return s_; } } while (0)
  SPFOM_TRY(upload(ctx, &d_r, I->r, (size_t)n));
  SPFOM_TRY(upload(ctx, &d_c, I->c, (size_t)m));
  SPFOM_TRY(upload(ctx, &d_aptr, I->a_ptr, (size_t)n + 1));
  SPFOM_TRY(upload(ctx, &d_aidx, I->a_idx, (size_t)nnzA));
  if (I->a_val) SPFOM_TRY(upload(ctx, &d_aval, I->a_val, (size_t)nnzA));
  SPFOM_TRY(upload(ctx, &d_atptr, at_ptr.data(), (size_t)m + 1));
  SPFOM_TRY(upload(ctx, &d_atidx, at_idx.data(), (size_t)nnzA));
  if (I->a_val) SPFOM_TRY(upload(ctx, &d_atval, at_val.data(), (size_t)nnzA));
  static_assert(sizeof(long long) == sizeof(int64_t), "int64");
  SPFOM_TRY(upload(ctx, &d_segptr, reinterpret_cast<const long long*>(I->seg_ptr), (size_t)L + 1, kSlack));
  SPFOM_TRY(upload(ctx, &d_prod, I->seg_prod, (size_t)nnz, kSlack));
  SPFOM_TRY(upload(ctx, &d_v, I->v, (size_t)nnz, kSlack));
  if (I->w) SPFOM_TRY(upload(ctx, &d_w, I->w, (size_t)nnz));
  SPFOM_TRY(upload(ctx, &d_lam, I->lam, (size_t)L, kSlack));
  SPFOM_TRY(upload(ctx, &d_v0, I->v0, (size_t)L));
  SPFOM_TRY(dalloc(ctx, &d_vt, (size_t)nnz + kSlack));
  SPFOM_TRY(dalloc(ctx, &d_vt0, (size_t)L + kSlack));
  SPFOM_CUDA(ctx, cudaMemsetAsync(d_vt + nnz, 0, kSlack * sizeof(double), ctx->stream));
  SPFOM_CUDA(ctx, cudaMemsetAsync(d_vt0 + L, 0, kSlack * sizeof(double), ctx->stream));
  P.r = d_r; P.c = d_c; P.a_ptr = d_aptr; P.a_idx = d_aidx; P.a_val = d_aval;
  P.at_ptr = d_atptr; P.at_idx = d_atidx; P.at_val = d_atval;
  P.seg_ptr = d_segptr; P.seg_prod = d_prod; P.v = d_v; P.vt = d_vt; P.lam = d_lam; P.vt0 = d_vt0;
  cudaError_t e = spfom::launch_prep(P, d_w, d_v0, d_vt, d_vt0, ctx->stream);
  if (e != cudaSuccess) { free_instance(ctx); return cuda_fail(ctx, e, "preprocessing launch"); }
  // work buffers
  Work& W = ctx->W;
  int Wl = 1;
  while (Wl < kmax) Wl <<= 1;
  W.W = Wl;
  const long long groups = (L * Wl + 255) / 256;
  long long sb = groups < (long long)ctx->sms * 8 ? groups : (long long)ctx->sms * 8;
  W.seg_blocks = (int)(sb > 0 ? sb : 1);
  const int nv = n > m ? n : m;
  W.vec_blocks = (nv + 255) / 256 > 0 ? (nv + 255) / 256 : 1;
  SPFOM_TRY(dalloc(ctx, &W.y, (size_t)m));
  SPFOM_TRY(dalloc(ctx, &W.sum_y, (size_t)m));
  SPFOM_TRY(dalloc(ctx, &W.sum_g, (size_t)m));
  SPFOM_TRY(dalloc(ctx, &W.g, (size_t)m));
  SPFOM_TRY(dalloc(ctx, &W.y_eval, (size_t)m));
  SPFOM_TRY(dalloc(ctx, &W.s, (size_t)n));
  SPFOM_TRY(dalloc(ctx, &W.marg, (size_t)n));
  SPFOM_TRY(dalloc(ctx, &W.marg_eval, (size_t)n));
  SPFOM_TRY(dalloc(ctx, &W.z_seg, (size_t)L));
  // certified-decision kernel: plan, fixed-point scale 2^F with sum(lambda) * 2^F < 2^61
  W.fast = false;
  W.zparts_iter = W.zparts_eval = W.seg_blocks;
  {
    double mass = 0.0;
    for (long long l = 0; l < L; ++l) mass += I->lam[l];
    int e2 = 0;
    std::frexp(mass > 1.0 ? mass : 1.0, &e2);  // mass < 2^e2
    const int F = 61 - e2;
    spfom::FastPlan plan{};
    if (ctx->p.path == 0 && F >= 30 && spfom::fast_plan(n, kmax, ctx->sms, &plan)) {
      W.fast = true;
      if (ctx->p.pipeline && spfom::pipe_plan(n, ctx->sms, &plan)) {
        // tiles of consecutive segments for the binary64 pipeline
        const long long nt = spfom::make_tiles64(reinterpret_cast<const long long*>(I->seg_ptr), L, nullptr);
        std::vector<long long> tiles((size_t)nt + 1);
        spfom::make_tiles64(reinterpret_cast<const long long*>(I->seg_ptr), L, tiles.data());
        SPFOM_TRY(upload(ctx, &W.tile64_ptr, tiles.data(), tiles.size()));
        W.ntiles64 = nt;
      }
      if (ctx->p.precision == 32 && spfom::tma_plan(n, kmax, ctx->sms, &plan)) {
        // tiles of consecutive segments for the bulk-copy staging of the binary32 pass
        const long long nt = spfom::make_tiles(reinterpret_cast<const long long*>(I->seg_ptr), L, nullptr);
        std::vector<long long> tiles((size_t)nt + 1);
        spfom::make_tiles(reinterpret_cast<const long long*>(I->seg_ptr), L, tiles.data());
        SPFOM_TRY(upload(ctx, &W.tile_ptr, tiles.data(), tiles.size()));
        W.ntiles = nt;
      }
      W.plan = plan;
      W.fx_scale = std::ldexp(1.0, F);
      W.fx_bits = F;
      W.inv_fx_scale = std::ldexp(1.0, -F);
      W.zparts_iter = std::max(std::max(plan.grid, plan.grid32), plan.pipe ? plan.pipe_grid : 0);
      W.zparts_eval = plan.grid_eval;
      if (plan.scatter == 1)
        SPFOM_TRY(dalloc(ctx, &W.part, (size_t)std::max(plan.grid, plan.grid32) * (size_t)(n > 0 ? n : 1)));
      SPFOM_TRY(dalloc(ctx, &W.s_fx, (size_t)n));
    }
    if (ctx->p.precision == 32) {
      if (!W.fast) {
        free_instance(ctx);
        return fail(ctx, SPFOM_ENOTSUP, "precision 32 needs the certified-decision kernel (path 0)");
      }
      SPFOM_TRY(dalloc(ctx, &W.v32, (size_t)nnz + kSlack));
      SPFOM_TRY(dalloc(ctx, &W.vt32, (size_t)nnz + kSlack));
      SPFOM_TRY(dalloc(ctx, &W.lam32, (size_t)L + kSlack));
      SPFOM_TRY(dalloc(ctx, &W.vt0_32, (size_t)L + kSlack));
      SPFOM_CUDA(ctx, cudaMemsetAsync(W.v32 + nnz, 0, kSlack * sizeof(float), ctx->stream));
      SPFOM_CUDA(ctx, cudaMemsetAsync(W.vt32 + nnz, 0, kSlack * sizeof(float), ctx->stream));
      SPFOM_CUDA(ctx, cudaMemsetAsync(W.lam32 + L, 0, kSlack * sizeof(float), ctx->stream));
      SPFOM_CUDA(ctx, cudaMemsetAsync(W.vt0_32 + L, 0, kSlack * sizeof(float), ctx->stream));
      SPFOM_TRY(dalloc(ctx, &W.marg32, (size_t)n));
    }
    SPFOM_TRY(dalloc(ctx, &W.fallbacks, 1));
  }
  SPFOM_TRY(dalloc(ctx, &W.zpart, (size_t)std::max(W.seg_blocks, W.zparts_iter)));
  SPFOM_TRY(dalloc(ctx, &W.zpart_eval, (size_t)std::max(W.seg_blocks, W.zparts_eval)));
  SPFOM_TRY(dalloc(ctx, &W.cypart, (size_t)W.vec_blocks));
  SPFOM_TRY(dalloc(ctx, &W.Ppart, (size_t)W.vec_blocks));
  W.x_cur = nullptr;
  if (ctx->p.batch_frac < 1.0) SPFOM_TRY(dalloc(ctx, &W.x_cur, (size_t)nnz));
#undef SPFOM_TRY
  ctx->P = P;
  if (W.v32) {
    e = spfom::launch_prep_f32(P, W, ctx->stream);
    if (e != cudaSuccess) { free_instance(ctx); return cuda_fail(ctx, e, "binary32 copies"); }
  }
  // step size: tau, or tau0 * mean(r) / mean(c) (sums in index order)
  double sr = 0.0, sc = 0.0;
  for (int j = 0; j < n; ++j) sr += I->r[j];
  for (int i = 0; i < m; ++i) sc += I->c[i];
  const double mr = n > 0 ? sr / n : 0.0, mc = m > 0 ? sc / m : 0.0;
  ctx->tau_init = ctx->p.tau > 0.0 ? ctx->p.tau : ((mc > 0.0 && mr > 0.0) ? ctx->p.tau0 * mr / mc : ctx->p.tau0);
  RunConfig& cfg = ctx->cfg;
  cfg.batch_frac = ctx->p.batch_frac;
  cfg.seed = ctx->p.seed;
  cfg.sample_thr = ctx->p.batch_frac >= 1.0 ? ~0ULL : (unsigned long long)std::ldexp(ctx->p.batch_frac, 64);
  cfg.restart_beta = ctx->p.restart_beta;
  cfg.restart_artificial = ctx->p.restart_artificial;
  cfg.restart_tau_decay = ctx->p.restart_tau_decay;
  cfg.kkt_tol = ctx->p.kkt_tol;
  cfg.f32 = ctx->p.precision == 32 ? 1 : 0;
  ctx->loaded = true;
  s = init_state(ctx, nullptr);
  if (s != SPFOM_OK) {
    free_instance(ctx);
    return s;
  }
  return SPFOM_OK;
}

spfom_status spfom_reset(spfom_ctx* ctx, const double* y0) {
  if (!ctx) return SPFOM_EINVAL;
  if (!ctx->loaded) return fail(ctx, SPFOM_ESTATE, "no instance loaded");
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  return init_state(ctx, y0);
}

namespace {

// Capture one evaluation period (eval_every iterations, then the evaluation)
// on the ctx stream into an executable graph. Returns null when the stream
// cannot be captured (the caller then launches directly).
cudaGraphExec_t capture_period(spfom_ctx* ctx) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  bool ok = true;
  for (long long k = 0; k < ctx->p.eval_every && ok; ++k)
    ok = spfom::launch_iteration(ctx->P, ctx->W, ctx->cfg, ctx->stream) == cudaSuccess;
  if (ok) ok = spfom::launch_eval(ctx->P, ctx->W, ctx->cfg, ctx->stream) == cudaSuccess;
  if (cudaStreamEndCapture(ctx->stream, &g) != cudaSuccess || !ok) ok = false;
  if (ok && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    ok = false;
    ex = nullptr;
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  return ok ? ex : nullptr;
}

}  // namespace

spfom_status spfom_step(spfom_ctx* ctx, int64_t iters, spfom_stats* out) {
  if (!ctx) return SPFOM_EINVAL;
  if (!ctx->loaded) return fail(ctx, SPFOM_ESTATE, "no instance loaded");
  if (iters < 0) return fail(ctx, SPFOM_EINVAL, "iters < 0");
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  const long long E = ctx->p.eval_every;
  const bool prof = ctx->p.profile != 0;
  if (prof) {
    while ((long long)ctx->prof_ev.size() < 2 * iters) {
      cudaEvent_t e;
      SPFOM_CUDA(ctx, cudaEventCreate(&e));
      ctx->prof_ev.push_back(e);
    }
  }
  const bool graphs = ctx->p.graphs != 0 && !prof && E > 0;
  const long long per_iter = spfom::kernel_launches_per_iteration(ctx->W, ctx->cfg);
  SPFOM_CUDA(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
  long long t = ctx->host_t, launches = 0;
  for (int64_t k = 0; k < iters;) {
    if (graphs && t % E == 0 && iters - k >= E && !ctx->period_failed) {
      cudaGraphExec_t& ex = ctx->period[ctx->cfg.f32 ? 1 : 0];
      if (!ex) ex = capture_period(ctx);
      if (ex) {
        SPFOM_CUDA(ctx, cudaGraphLaunch(ex, ctx->stream));
        launches += E * per_iter + spfom::kernel_launches_per_eval();
        k += E;
        t += E;
        continue;
      }
      ctx->period_failed = true;
    }
    cudaError_t e = spfom::launch_iteration(ctx->P, ctx->W, ctx->cfg, ctx->stream,
                                            prof ? ctx->prof_ev[2 * k] : nullptr,
                                            prof ? ctx->prof_ev[2 * k + 1] : nullptr);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "iteration launch");
    launches += per_iter;
    ++t;
    ++k;
    if (E > 0 && t % E == 0) {
      e = spfom::launch_eval(ctx->P, ctx->W, ctx->cfg, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "evaluation launch");
      launches += spfom::kernel_launches_per_eval();
    }
  }
  SPFOM_CUDA(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
  DevState st;
  spfom_status s = read_state(ctx, &st);
  if (s != SPFOM_OK) return s;
  float ms = 0.f;
  SPFOM_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  double seg = 0.0;
  if (prof)
    for (int64_t k = 0; k < iters; ++k) {
      float sm = 0.f;
      SPFOM_CUDA(ctx, cudaEventElapsedTime(&sm, ctx->prof_ev[2 * k], ctx->prof_ev[2 * k + 1]));
      seg += sm * 1e-3;
    }
  ctx->host_t = st.t;
  fill_stats(ctx, st, ms * 1e-3, out);
  if (st.error) {
    if (out) {
      out->seg_kernel_seconds = seg;
      out->kernel_launches = launches;
    }
    return fail(ctx, SPFOM_ETIMEOUT, "a bounded device wait (bulk-copy staging) gave up; results are invalid");
  }
  if (out) {
    out->seg_kernel_seconds = seg;
    out->seg_kernel_launches = prof ? iters : 0;
    out->kernel_launches = launches;
  }
  return SPFOM_OK;
}

spfom_status spfom_solve(spfom_ctx* ctx, const double* y0, spfom_stats* out) {
  spfom_status s = spfom_reset(ctx, y0);
  if (s != SPFOM_OK) return s;
  const long long E = ctx->p.eval_every > 0 ? ctx->p.eval_every : 1024;
  spfom_stats st{};
  double secs = 0.0, seg = 0.0;
  long long segl = 0, launches = 0;
  for (;;) {
    long long left = ctx->p.max_iters - ctx->host_t;
    if (left <= 0) break;
    s = spfom_step(ctx, left < E ? left : E, &st);
    if (s != SPFOM_OK) return s;
    secs += st.seconds;
    seg += st.seg_kernel_seconds;
    segl += st.seg_kernel_launches;
    launches += st.kernel_launches;
    if (st.converged && ctx->cfg.f32 && ctx->p.polish) {
      // binary64 polish: clear the flag and iterate in binary64 until the next evaluation
      ctx->cfg.f32 = 0;
      ctx->polishing = true;
      const int zero = 0;
      SPFOM_CUDA(ctx, cudaMemcpyAsync(&ctx->W.st->converged, &zero, sizeof zero, cudaMemcpyHostToDevice,
                                      ctx->stream));
      continue;
    }
    if (st.converged) break;
  }
  st.seconds = secs;
  st.seg_kernel_seconds = seg;
  st.seg_kernel_launches = segl;
  st.kernel_launches = launches;
  if (out) *out = st;
  return st.converged ? SPFOM_OK : fail(ctx, SPFOM_ENOTCONV, "KKT %.3e above %.1e after %lld iterations", st.kkt,
                                         ctx->p.kkt_tol, (long long)st.iters);
}

spfom_status spfom_get_stats(spfom_ctx* ctx, spfom_stats* out) {
  if (!ctx || !out) return SPFOM_EINVAL;
  if (!ctx->loaded) return fail(ctx, SPFOM_ESTATE, "no instance loaded");
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  DevState st;
  spfom_status s = read_state(ctx, &st);
  if (s != SPFOM_OK) return s;
  fill_stats(ctx, st, 0.0, out);
  return SPFOM_OK;
}

spfom_status spfom_vector(spfom_ctx* ctx, spfom_vector_id which, double* out) {
  if (!ctx || !out) return SPFOM_EINVAL;
  if (!ctx->loaded) return fail(ctx, SPFOM_ESTATE, "no instance loaded");
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  const Work& W = ctx->W;
  const int m = ctx->P.m, n = ctx->P.n;
  const double* src = nullptr;
  size_t cnt = 0;
  switch (which) {
    case SPFOM_VEC_Y: src = W.y; cnt = m; break;
    case SPFOM_VEC_SUM_Y: src = W.sum_y; cnt = m; break;
    case SPFOM_VEC_SUM_G: src = W.sum_g; cnt = m; break;
    case SPFOM_VEC_G: src = W.g; cnt = m; break;
    case SPFOM_VEC_S: src = W.s; cnt = n; break;
    case SPFOM_VEC_MARGINS: src = W.marg; cnt = n; break;
    case SPFOM_VEC_YBAR: {
      DevState st;
      spfom_status s = read_state(ctx, &st);
      if (s != SPFOM_OK) return s;
      if (st.count == 0) { src = W.y; cnt = m; break; }
      if (m) SPFOM_CUDA(ctx, cudaMemcpyAsync(out, W.sum_y, sizeof(double) * m, cudaMemcpyDeviceToHost, ctx->stream));
      SPFOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      const double c = (double)st.count;
      for (int i = 0; i < m; ++i) out[i] = out[i] / c;
      return SPFOM_OK;
    }
    default:
      return fail(ctx, SPFOM_EINVAL, "unknown vector id %d", (int)which);
  }
  if (cnt) SPFOM_CUDA(ctx, cudaMemcpyAsync(out, src, sizeof(double) * cnt, cudaMemcpyDeviceToHost, ctx->stream));
  SPFOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SPFOM_OK;
}

spfom_status spfom_duals(spfom_ctx* ctx, int32_t averaged, double* y_out) {
  return spfom_vector(ctx, averaged ? SPFOM_VEC_YBAR : SPFOM_VEC_Y, y_out);
}

spfom_status spfom_evaluate(spfom_ctx* ctx, const double* y, double* z_out, double* dual_out) {
  if (!ctx || !y) return SPFOM_EINVAL;
  if (!ctx->loaded) return fail(ctx, SPFOM_ESTATE, "no instance loaded");
  const Problem& P = ctx->P;
  for (int i = 0; i < P.m; ++i)
    if (!(y[i] >= 0.0) || !is_finite(y[i])) return fail(ctx, SPFOM_EINVAL, "y[%d] must be finite and >= 0", i);
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  if (P.m) SPFOM_CUDA(ctx, cudaMemcpyAsync(ctx->W.y_eval, y, sizeof(double) * P.m, cudaMemcpyHostToDevice, ctx->stream));
  cudaError_t e = spfom::launch_evaluate_at(P, ctx->W, z_out != nullptr, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "evaluation launch");
  if (z_out && P.L)
    SPFOM_CUDA(ctx, cudaMemcpyAsync(z_out, ctx->W.z_seg, sizeof(double) * P.L, cudaMemcpyDeviceToHost, ctx->stream));
  DevState st;
  spfom_status s = read_state(ctx, &st);
  if (s != SPFOM_OK) return s;
  if (dual_out) *dual_out = st.eval_out;
  return SPFOM_OK;
}

}  // extern "C"
