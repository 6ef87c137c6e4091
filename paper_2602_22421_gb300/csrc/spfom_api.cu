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
#include <chrono>
#include <new>
#include <string>
#include <vector>

#include "../../include/spfom.h"
#include "../../include/spfom_mlp.h"
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
  cudaMemPool_t pool = nullptr;  // their stream-ordered pool: keeps its memory across loads (null: the default pool)
  DevState* d_state = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> prof_ev;  // event pairs of profiled segment launches
  int sms = 0;
  unsigned wait_limit = 1u << 22;  // polls of a bounded device wait (spfom_set_wait_limit; the kernels' default)
  unsigned long long fallback_host = 0;
  bool polishing = false;  // precision 32: binary64 iterations after the first converged evaluation
  cudaGraphExec_t period[2] = {nullptr, nullptr};  // one evaluation period, [binary64, binary32 pass]
  bool period_stale[2] = {false, false};           // its launches may name buffers or values that changed
  Problem period_P[2]{};                           // the problem, work and configuration it was captured
  Work period_W[2]{};                              // with: identical ones (a reload of the same instance
  RunConfig period_cfg[2]{};                       // into the same pool blocks) make it valid again as it is
  long long period_E[2] = {0, 0};
  bool period_failed = false;                      // capture unavailable on this stream
  cudaGraphExec_t loop[2] = {nullptr, nullptr};    // device loop over periods (params.device_loop)
  spfom::DevLoop* d_loop = nullptr;                // its state (device, per loaded instance)
  // batch (spfom_load_batch)
  struct BatchSpec {
    int count;
    std::vector<int> res_ptr, prod_ptr;
    std::vector<long long> seg_off;
  };
  const BatchSpec* loading_batch = nullptr;  // set while spfom_load_batch loads the union
  BatchSpec batch;
  std::vector<double> inst_tau;              // per-instance initial step sizes
  std::vector<double> inst_mean_r;           // per-instance mean price (step size after spfom_update)
  std::vector<spfom::InstState> h_inst;      // last state read back
  // learned warm start: device scratch (features, outputs, demand, duals)
  void* warm_buf = nullptr;
  size_t warm_bytes = 0;
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

// The period graphs are kept but marked stale: the next capture updates them
// in place (cheaper than a new instantiation when the kernels are the same,
// as after a reload of an instance of the same shape); the loop graphs go.
void drop_graphs(spfom_ctx* ctx) {
  for (int k = 0; k < 2; ++k)
    if (ctx->period[k]) ctx->period_stale[k] = true;
  for (auto& g : ctx->loop)
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
  ctx->d_loop = nullptr;  // freed with the instance's buffers
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
  cudaError_t e = ctx->pool ? cudaMallocFromPoolAsync(&p, count * sizeof(T), ctx->pool, ctx->stream)
                            : cudaMallocAsync(&p, count * sizeof(T), ctx->stream);
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

// Host checks of an instance. items = false leaves the per-segment and
// per-nonzero checks (offsets, lambda, v0, ids, repeats, v, w) and the largest
// set to the device pass of spfom_load_instance (*kmax_out is then not set).
spfom_status validate(spfom_ctx* ctx, const spfom_instance* I, int* kmax_out, bool items = true) {
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
  for (long long l = 0; l < (items ? I->L : 0); ++l) {
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

// The slot-major copy of the loaded single instance (tilings 3 and 8), built
// on first use: positions and chunk offsets on the host from the segment
// offsets, then the items and per-position values gathered on the device.
spfom_status build_sliced(spfom_ctx* ctx) {
  Work& W = ctx->W;
  if (W.sl.nchunks > 0 || !W.fast || !W.plan.sl_ok) return SPFOM_OK;
  const Problem& P = ctx->P;
  std::vector<long long> seg_ptr((size_t)P.L + 1);
  SPFOM_CUDA(ctx, cudaMemcpyAsync(seg_ptr.data(), P.seg_ptr, sizeof(long long) * seg_ptr.size(),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  SPFOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::vector<long long> perm, off;
  const long long nch = spfom::sliced_layout(seg_ptr.data(), P.L, W.plan.W8, &perm, &off);
  const size_t entries = (size_t)std::max(off[(size_t)nch], 1ll), npos = perm.size();
  spfom::SlView sl{};
  long long* d_perm = nullptr;
#define SPFOM_TRYS(x) do { spfom_status s_ = (x); if (s_ != SPFOM_OK) return s_; } while (0)
  SPFOM_TRYS(upload(ctx, &sl.off, off.data(), off.size()));
  SPFOM_TRYS(upload(ctx, &d_perm, perm.data(), npos));
  SPFOM_TRYS(dalloc(ctx, &sl.prod, entries));
  if (W.v32) {
    SPFOM_TRYS(dalloc(ctx, &sl.v32, entries));
    SPFOM_TRYS(dalloc(ctx, &sl.vt32, entries));
    SPFOM_TRYS(dalloc(ctx, &sl.lam32, npos));
    SPFOM_TRYS(dalloc(ctx, &sl.vt0_32, npos));
  } else {
    SPFOM_TRYS(dalloc(ctx, &sl.v, entries));
    SPFOM_TRYS(dalloc(ctx, &sl.vt, entries));
    SPFOM_TRYS(dalloc(ctx, &sl.lam, npos));
    SPFOM_TRYS(dalloc(ctx, &sl.vt0, npos));
  }
  SPFOM_TRYS(dalloc(ctx, &sl.rprev, npos));
#undef SPFOM_TRYS
  SPFOM_CUDA(ctx, cudaMemsetAsync(sl.rprev, 0, sizeof(float) * npos, ctx->stream));
  sl.nchunks = nch;
  W.sl = sl;
  W.sl_perm = d_perm;
  cudaError_t e = spfom::launch_slice_items(P, W, W.plan.W8, ctx->stream);
  if (e == cudaSuccess) e = spfom::launch_slice_segments(P, W, W.plan.W8, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // the host vectors go out of scope
  if (e != cudaSuccess) {
    W.sl = spfom::SlView{};
    W.sl_perm = nullptr;
    return cuda_fail(ctx, e, "slot-major copy");
  }
  return SPFOM_OK;
}

// The row-exact copy of the loaded single instance (precision-64 tiling 4:
// binary64 v, vt, lambda, vt_0; precision-32 tiling 9: their binary32 copies),
// built on first use like the slot-major copy: positions, chunk offsets and
// classes on the host, the items and per-position values gathered on the device.
spfom_status build_rows(spfom_ctx* ctx) {
  Work& W = ctx->W;
  if (W.rx.nchunks > 0 || !W.fast || !W.plan.rows_ok) return SPFOM_OK;
  const Problem& P = ctx->P;
#define SPFOM_TRYS(x) do { spfom_status s_ = (x); if (s_ != SPFOM_OK) return s_; } while (0)
  // the layout needs only the histogram of set sizes; the segments are placed
  // on the device
  constexpr int KN = spfom::kFastMaxSet + 1;
  unsigned long long* d_cnt = nullptr;  // [KN] histogram, [KN] the scatter's cursors
  SPFOM_TRYS(dalloc(ctx, &d_cnt, 2 * KN));
  SPFOM_CUDA(ctx, cudaMemsetAsync(d_cnt, 0, 2 * KN * sizeof(unsigned long long), ctx->stream));
  SPFOM_CUDA(ctx, spfom::launch_rows_hist(P, d_cnt, ctx->stream));
  std::vector<unsigned long long> cnt(KN);
  SPFOM_CUDA(ctx, cudaMemcpyAsync(cnt.data(), d_cnt, KN * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                  ctx->stream));
  SPFOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::vector<long long> off, pos_start(KN, 0);
  spfom::SlView rx{};
  const long long nch = spfom::rows_layout_counts(cnt.data(), &off, rx.cls_c, rx.cls_pos, pos_start.data());
  const long long npos_l = rx.cls_pos[spfom::kRowsClasses];
  const size_t entries = (size_t)std::max(off[(size_t)nch], 1ll), npos = (size_t)std::max(npos_l, 1ll);
  long long* d_perm = nullptr;
  long long* d_pos_start = nullptr;
  SPFOM_TRYS(upload(ctx, &rx.off, off.data(), off.size()));
  SPFOM_TRYS(upload(ctx, &d_pos_start, pos_start.data(), pos_start.size()));
  SPFOM_TRYS(dalloc(ctx, &d_perm, npos));
  SPFOM_CUDA(ctx, cudaMemsetAsync(d_perm, 0xFF, npos * sizeof(long long), ctx->stream));  // -1: padding
  SPFOM_CUDA(ctx, spfom::launch_rows_scatter(P, d_pos_start, d_cnt + KN, d_perm, ctx->stream));
  SPFOM_TRYS(dalloc(ctx, &rx.prod, entries));
  if (W.v32) {
    SPFOM_TRYS(dalloc(ctx, &rx.v32, entries));
    SPFOM_TRYS(dalloc(ctx, &rx.vt32, entries));
    SPFOM_TRYS(dalloc(ctx, &rx.lam32, npos));
    SPFOM_TRYS(dalloc(ctx, &rx.vt0_32, npos));
  } else {
    SPFOM_TRYS(dalloc(ctx, &rx.v, entries));
    SPFOM_TRYS(dalloc(ctx, &rx.vt, entries));
    SPFOM_TRYS(dalloc(ctx, &rx.lam, npos));
    SPFOM_TRYS(dalloc(ctx, &rx.vt0, npos));
  }
  SPFOM_TRYS(dalloc(ctx, &rx.rprev, npos));
  SPFOM_TRYS(dalloc(ctx, &rx.redo, npos));
  SPFOM_TRYS(dalloc(ctx, &rx.redo_ctl, 2));
#undef SPFOM_TRYS
  SPFOM_CUDA(ctx, cudaMemsetAsync(rx.rprev, 0, sizeof(float) * npos, ctx->stream));
  SPFOM_CUDA(ctx, cudaMemsetAsync(rx.redo_ctl, 0, 2 * sizeof(unsigned), ctx->stream));
  rx.mixed = 1;
  rx.nchunks = nch;
  W.rx = rx;
  W.rx_perm = d_perm;
  cudaError_t e = spfom::launch_rows_items(P, W.rx, W.rx_perm, W.v32, W.vt32, ctx->stream);
  if (e == cudaSuccess) e = spfom::launch_rows_segments(P, W.rx, W.rx_perm, W.lam32, W.vt0_32, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // the host vectors go out of scope
  if (e != cudaSuccess) {
    W.rx = spfom::SlView{};
    W.rx_perm = nullptr;
    return cuda_fail(ctx, e, "row-exact copy");
  }
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
  if (W.batch) {
    const int cnt = W.bm.count;
    ctx->h_inst.assign((size_t)cnt, spfom::InstState{});
    for (int b = 0; b < cnt; ++b) {
      spfom::InstState& I = ctx->h_inst[b];
      I.tau = ctx->inst_tau[b];
      I.mu = ctx->p.mu;
      I.z_sum = I.P = I.dual_iter = NAN;
      I.kkt = I.pinf = I.gap = I.dual_avg = I.primal_avg = NAN;
      I.kkt_anchor = INFINITY;
    }
    SPFOM_CUDA(ctx, cudaMemcpyAsync(W.bm.inst, ctx->h_inst.data(), sizeof(spfom::InstState) * cnt,
                                    cudaMemcpyHostToDevice, ctx->stream));
    SPFOM_CUDA(ctx, cudaMemsetAsync(W.bm.conv, 0, sizeof(int) * cnt, ctx->stream));
    SPFOM_CUDA(ctx, cudaMemsetAsync(W.bm.z_seg, 0, sizeof(double) * (P.L ? P.L : 1), ctx->stream));
    SPFOM_CUDA(ctx, cudaMemsetAsync(W.bm.cy_res, 0, sizeof(double) * (P.m ? P.m : 1), ctx->stream));
  }
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
  if (ctx->W.batch && !ctx->h_inst.empty()) {
    // the batch: iterations and evaluations of the longest-running instance, sums of the
    // objectives and counts, the largest residuals; converged when every instance is
    long long it = 0, ev = 0, rs = 0, ep = 0;
    double kkt = 0, pinf = 0, gap = 0, da = 0, pa = 0, di = 0, zs = 0, rv = 0, srv = 0;
    int conv = 1;
    for (const auto& I : ctx->h_inst) {
      it = std::max(it, I.t);
      ev = std::max(ev, I.evals);
      ep = std::max(ep, I.count);
      rs += I.restarts;
      kkt = std::max(kkt, std::isnan(I.kkt) ? INFINITY : I.kkt);
      pinf = std::max(pinf, std::isnan(I.pinf) ? INFINITY : I.pinf);
      gap = std::max(gap, std::isnan(I.gap) ? INFINITY : I.gap);
      da += I.dual_avg; pa += I.primal_avg; di += I.dual_iter; zs += I.z_sum; rv += I.P; srv += I.sum_P;
      conv &= I.converged;
    }
    s.iters = it; s.evals = ev; s.restarts = rs; s.epoch_iters = ep; s.converged = conv;
    s.kkt = kkt; s.pinf = pinf; s.gap = gap; s.dual_avg = da; s.primal_avg = pa; s.dual_iter = di;
    s.z_sum = zs; s.revenue = rv; s.sum_revenue = srv;
    s.tau = ctx->h_inst[0].tau; s.mu = ctx->h_inst[0].mu;
  }
  *out = s;
}

void inst_stats(const spfom_ctx* ctx, const spfom::InstState& I, spfom_stats* out) {
  spfom_stats s{};
  s.iters = I.t; s.restarts = I.restarts; s.evals = I.evals; s.epoch_iters = I.count; s.converged = I.converged;
  s.kkt = I.kkt; s.pinf = I.pinf; s.gap = I.gap; s.dual_avg = I.dual_avg; s.primal_avg = I.primal_avg;
  s.dual_iter = I.dual_iter; s.z_sum = I.z_sum; s.revenue = I.P; s.sum_revenue = I.sum_P; s.tau = I.tau; s.mu = I.mu;
  s.fast_path = 1;
  s.iter_precision = ctx->cfg.f32 ? 32 : 64;
  *out = s;
}

spfom_status read_state(spfom_ctx* ctx, DevState* st) {
  SPFOM_CUDA(ctx, cudaMemcpyAsync(st, ctx->W.st, sizeof *st, cudaMemcpyDeviceToHost, ctx->stream));
  if (ctx->W.batch)
    SPFOM_CUDA(ctx, cudaMemcpyAsync(ctx->h_inst.data(), ctx->W.bm.inst, sizeof(spfom::InstState) * ctx->W.bm.count,
                                    cudaMemcpyDeviceToHost, ctx->stream));
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
      prm.mu < 0 || !(prm.restart_tau_decay > 0.0) ||
      !(prm.restart_tau_balance >= 0.0 && prm.restart_tau_balance <= 1.0) || prm.tiling < 0 || prm.tiling > 9)
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
  if (e == cudaSuccess) {
    // a private pool whose freed memory stays reserved (release threshold: all of it), so
    // that reloading an instance of the same size maps no new memory
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = prm.device;
    if (cudaMemPoolCreate(&ctx->pool, &props) == cudaSuccess) {
      uint64_t keep = ~0ull;
      if (cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
        cudaMemPoolDestroy(ctx->pool);
        ctx->pool = nullptr;
      }
    } else {
      ctx->pool = nullptr;
    }
    (void)cudaGetLastError();  // a refused pool leaves the default one in use
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
  for (auto& g : ctx->period)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);  // its allocations are freed and the stream synchronized
  if (ctx->warm_buf) cudaFree(ctx->warm_buf);
  if (ctx->d_state) cudaFree(ctx->d_state);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

spfom_status spfom_load_instance(spfom_ctx* ctx, const spfom_instance* I) {
  if (!ctx) return SPFOM_EINVAL;
  int kmax = 0;  // from the device pass below
  spfom_status s = validate(ctx, I, &kmax, false);  // the per-segment and per-nonzero checks run on the device
  if (s != SPFOM_OK) return s;
  if (I->L > 0 && (I->seg_ptr[I->L] > 0) && (!I->seg_prod || !I->v))
    return fail(ctx, SPFOM_EINVAL, "missing segment arrays");
  if (I->L > 0 && I->seg_ptr[I->L] < 0) return fail(ctx, SPFOM_EINVAL, "seg_ptr not monotone at %lld", I->L - 1);
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
  {
    // per-segment and per-nonzero checks on the device: the first failure in
    // the order of a host loop over segments, and the largest set
    unsigned long long* d_keys = nullptr;
    SPFOM_TRY(dalloc(ctx, &d_keys, 3));
    unsigned long long keys[3];
    cudaError_t ev = spfom::launch_validate_items(P, d_w, d_v0, ctx->p.precision == 32, d_keys, ctx->stream);
    if (ev == cudaSuccess) ev = cudaMemcpyAsync(keys, d_keys, sizeof keys, cudaMemcpyDeviceToHost, ctx->stream);
    if (ev == cudaSuccess) ev = cudaStreamSynchronize(ctx->stream);
    if (ev != cudaSuccess) { free_instance(ctx); return cuda_fail(ctx, ev, "instance check"); }
    if (keys[0] != ~0ull) {
      const long long l = (long long)(keys[0] >> spfom::kCheckSegShift);
      const int sub = (int)(keys[0] & ((1ull << spfom::kCheckSegShift) - 1));
      free_instance(ctx);
      if (sub == spfom::kSegOrder) return fail(ctx, SPFOM_EINVAL, "seg_ptr not monotone at %lld", l);
      if (sub == spfom::kSegLam) return fail(ctx, SPFOM_EINVAL, "lam[%lld] must be >= 0", l);
      if (sub == spfom::kSegV0) return fail(ctx, SPFOM_EINVAL, "v0[%lld] must be > 0", l);
      const long long p = I->seg_ptr[l] + ((sub - spfom::kSegItems) >> 3);
      const int code = (sub - spfom::kSegItems) & 7, j = I->seg_prod[p];
      if (code == spfom::kBadId) return fail(ctx, SPFOM_EINVAL, "seg_prod[%lld] = %d out of range", p, j);
      if (code == spfom::kRepeated) return fail(ctx, SPFOM_EINVAL, "product %d repeated in segment %lld", j, l);
      if (code == spfom::kBadV) return fail(ctx, SPFOM_EINVAL, "v[%lld] must be finite and > 0", p);
      return fail(ctx, SPFOM_EINVAL, "w[%lld] must lie in [0, v]", p);
    }
    kmax = (int)keys[2];
    if (kmax > spfom::kFastMaxSet) {
      free_instance(ctx);
      return fail(ctx, SPFOM_ENOTSUP, "consideration set of %d products (at most %d supported)", kmax,
                  spfom::kFastMaxSet);
    }
    if (kmax > 32 && (ctx->p.path != 0 || ctx->p.track_xbar || ctx->p.batch_frac < 1.0 || ctx->loading_batch)) {
      free_instance(ctx);
      return fail(ctx, SPFOM_ENOTSUP,
                  "consideration set of %d products: sets of more than 32 need the certified-decision path "
                  "(path 0, batch_frac 1, a single instance, no track_xbar)", kmax);
    }
    if (keys[1] != ~0ull) {  // precision 32: attractions first (in nonzero order), then the segments
      const long long pos = (long long)keys[1];
      free_instance(ctx);
      if (pos < nnz) return fail(ctx, SPFOM_ENOTSUP, "precision 32: attraction at %lld outside binary32's normal range", pos);
      return fail(ctx, SPFOM_ENOTSUP, "precision 32: lambda or v0 of segment %lld outside binary32's range",
                  pos - nnz);
    }
  }
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
  W.vec_blocks = (m + 7) / 8 + (n + 255) / 256 > 0 ? (m + 7) / 8 + (n + 255) / 256 : 1;  // k_dual_step's grid
  SPFOM_TRY(dalloc(ctx, &W.y, (size_t)m));
  SPFOM_TRY(dalloc(ctx, &W.sum_y, (size_t)m));
  SPFOM_TRY(dalloc(ctx, &W.sum_g, (size_t)m));
  SPFOM_TRY(dalloc(ctx, &W.g, (size_t)m));
  SPFOM_TRY(dalloc(ctx, &W.y_eval, (size_t)m));
  SPFOM_TRY(dalloc(ctx, &W.s_eval, (size_t)n));
  SPFOM_TRY(dalloc(ctx, &W.s, (size_t)n));
  SPFOM_TRY(dalloc(ctx, &W.marg, (size_t)n));
  SPFOM_TRY(dalloc(ctx, &W.marg_eval, (size_t)n));
  SPFOM_TRY(dalloc(ctx, &W.z_seg, (size_t)L));
  // certified-decision kernel: plan, fixed-point scale 2^F with sum(lambda) * 2^F < 2^61
  W.fast = false;
  W.zparts_iter = W.zparts_eval = W.seg_blocks;
  {
    // only the exponent of the arrival mass matters: four interleaved sums
    double m4[4] = {0.0, 0.0, 0.0, 0.0};
    long long l = 0;
    for (; l + 3 < L; l += 4)
      for (int k = 0; k < 4; ++k) m4[k] += I->lam[l + k];
    for (; l < L; ++l) m4[0] += I->lam[l];
    const double mass = (m4[0] + m4[1]) + (m4[2] + m4[3]);
    int e2 = 0;
    std::frexp(mass > 1.0 ? mass : 1.0, &e2);  // mass < 2^e2
    const int F = 61 - e2;
    spfom::FastPlan plan{};
    if (ctx->p.path != 1 && !ctx->p.track_xbar && F >= 30 && spfom::fast_plan(n, kmax, ctx->sms, &plan)) {
      W.fast = true;
      if (ctx->p.pipeline && !ctx->loading_batch && spfom::pipe_plan(n, ctx->sms, &plan)) {
        // tiles of consecutive segments for the binary64 pipeline
        const long long nt = spfom::make_tiles64(reinterpret_cast<const long long*>(I->seg_ptr), L, nullptr);
        std::vector<long long> tiles((size_t)nt + 1);
        spfom::make_tiles64(reinterpret_cast<const long long*>(I->seg_ptr), L, tiles.data());
        SPFOM_TRY(upload(ctx, &W.tile64_ptr, tiles.data(), tiles.size()));
        W.ntiles64 = nt;
      }
      if (ctx->loading_batch && plan.scatter == 2) {
        // instance chunks of the batch for the chunked kernels (shared sums per instance)
        const auto& B = *ctx->loading_batch;
        int maxn = 0;
        for (int b = 0; b < B.count; ++b) maxn = std::max(maxn, B.prod_ptr[b + 1] - B.prod_ptr[b]);
        const bool c32 = ctx->p.precision == 32 && spfom::bchunk_plan(maxn, ctx->sms, &plan);
        const bool c64 = spfom::bchunk64_plan(maxn, ctx->sms, &plan);
        if (c32 || c64) {
          const long long nc = spfom::make_batch_chunks(B.seg_off, spfom::kBChunkSegs, nullptr, nullptr);
          std::vector<long long> cseg((size_t)nc + 1);
          std::vector<int> cinst((size_t)(nc > 0 ? nc : 1));
          spfom::make_batch_chunks(B.seg_off, spfom::kBChunkSegs, cseg.data(), cinst.data());
          SPFOM_TRY(upload(ctx, &W.bc_seg, cseg.data(), cseg.size()));
          SPFOM_TRY(upload(ctx, &W.bc_inst, cinst.data(), cinst.size()));
          W.bc_count = nc;
        }
      }
      if (ctx->p.precision == 32 && spfom::coop_plan(n, kmax, ctx->sms, &plan)) {
        // tiles of consecutive segments for the cooperatively staged binary32 kernel
        const auto* sp = reinterpret_cast<const long long*>(I->seg_ptr);
        const long long nt = spfom::make_tiles_lim(sp, L, plan.coop_segs, plan.coop_items, nullptr);
        std::vector<long long> tiles((size_t)nt + 1);
        spfom::make_tiles_lim(sp, L, plan.coop_segs, plan.coop_items, tiles.data());
        SPFOM_TRY(upload(ctx, &W.coop_tile_ptr, tiles.data(), tiles.size()));
        W.coop_ntiles = nt;
      }
      if (ctx->p.precision == 32 && spfom::tma_plan(n, kmax, ctx->sms, &plan)) {
        // tiles of consecutive segments for the bulk-copy staging of the binary32 pass
        const long long nt = spfom::make_tiles(reinterpret_cast<const long long*>(I->seg_ptr), L, nullptr);
        std::vector<long long> tiles((size_t)nt + 1);
        spfom::make_tiles(reinterpret_cast<const long long*>(I->seg_ptr), L, tiles.data());
        SPFOM_TRY(upload(ctx, &W.tile_ptr, tiles.data(), tiles.size()));
        W.ntiles = nt;
      }
      const bool dd = ctx->p.path == 2 && spfom::dd_setup(&plan, ctx->sms);
      // row-exact copy for the precision-64 tiling 4 (single instances, path 0)
      if (!(ctx->p.path == 0 && !ctx->loading_batch && L > 0 && spfom::rows_plan(n, ctx->sms, &plan)))
        plan.rows_ok = 0;
      W.plan = plan;
      W.fx_scale = std::ldexp(1.0, F);
      W.fx_bits = F;
      W.inv_fx_scale = std::ldexp(1.0, -F);
      W.zparts_iter = std::max(std::max(plan.grid, plan.grid32), std::max(plan.pipe ? plan.pipe_grid : 0,
                                                                          plan.tma_ok ? plan.tma_grid : 0));
      if (plan.coop_ok) W.zparts_iter = std::max(W.zparts_iter, plan.coop_grid);
      if (plan.bchunk_ok) W.zparts_iter = std::max(W.zparts_iter, plan.bchunk_grid);
      if (plan.bchunk64_ok) W.zparts_iter = std::max(W.zparts_iter, plan.bchunk64_grid);
      if (plan.ms_ok) W.zparts_iter = std::max(W.zparts_iter, std::max(plan.ms_grid, plan.ms_grid32));
      if (plan.rows_ok) W.zparts_iter = std::max(W.zparts_iter, std::max(plan.rows_grid, plan.rows_grid32));
      W.zparts_eval = plan.grid_eval;
      if (dd)
        for (int v = 1; v <= 3; ++v) {
          W.zparts_iter = std::max(W.zparts_iter, plan.dd_grid[v]);
          W.zparts_eval = std::max(W.zparts_eval, plan.dd_grid_eval[v]);
        }
      W.dd_ok = dd;
      // slot-major copy for the sliced tilings (single instances, path 0)
      W.plan.sl_ok = ctx->p.path == 0 && !ctx->loading_batch && L > 0 && plan.sl_attr && plan.W8 <= 4 ? 1 : 0;
      if (ctx->p.tiling > 0) {  // a requested tiling of the active segment pass
        const int t = ctx->p.tiling;
        bool ok = t <= 9;
        if (ok && ctx->p.precision == 32) {
          ok = (t != 2 || W.plan.tma_ok) && (t != 4 || W.plan.coop_ok) && (t != 6 || W.plan.bchunk_ok) &&
               (t != 7 || W.plan.ms_ok) && (t != 8 || W.plan.sl_ok) && (t != 5 || kmax <= 32) &&
               (t != 9 || W.plan.rows_ok);
          W.plan.f32_rows = t == 9 ? 1 : 0;
          W.plan.bchunk = t == 6 ? 1 : 0;
          W.plan.tma = t == 2 ? 1 : 0;
          W.plan.f32_p8 = t == 3 ? 1 : 0;
          W.plan.coop = t == 4 ? 1 : 0;
          W.plan.f32_p16 = t == 5 ? 1 : 0;
          W.plan.f32_ms = t == 7 ? 1 : 0;
          W.plan.f32_sl = t == 8 ? 1 : 0;
        } else if (ok) {
          // double-float kernel: its tilings 1..3; binary64-sum kernel: 1 = margins read
          // from global memory, 2 = margins in shared memory, 3 = slot-major copy
          ok = t <= 8 && (dd ? spfom::dd_variant_ok(W.plan, t) != 0
                             : (t == 1 || (t == 2 && W.plan.ms_ok) || (t == 3 && W.plan.sl_ok) ||
                                (t == 4 && W.plan.rows_ok)));
          if (dd) {
            W.plan.dd_variant = t;
          } else {
            W.plan.fast_ms = t == 2 ? 1 : 0;
            W.plan.fast_sl = t == 3 ? 1 : 0;
            W.plan.fast_rows = t == 4 ? 1 : 0;
          }
        }
        if (!ok) {
          free_instance(ctx);
          return fail(ctx, SPFOM_ENOTSUP, "tiling %d is not available for this instance", t);
        }
      }
      if (plan.scatter == 1)
        SPFOM_TRY(dalloc(ctx, &W.part, (size_t)W.zparts_iter * (size_t)(n > 0 ? n : 1)));
      SPFOM_TRY(dalloc(ctx, &W.s_fx, (size_t)n));
      if (W.plan.rows_ok && ctx->p.precision == 64) SPFOM_TRY(dalloc(ctx, &W.marg32c, (size_t)(n > 0 ? n : 1)));
      SPFOM_TRY(dalloc(ctx, &W.rprev, (size_t)(L > 0 ? L : 1)));
      SPFOM_CUDA(ctx, cudaMemsetAsync(W.rprev, 0, sizeof(float) * (size_t)(L > 0 ? L : 1), ctx->stream));
    }
    if (W.fast && W.dd_ok) {
      // double-float images for k_seg_dd (the precision-64 iteration and every evaluation pass)
      SPFOM_TRY(dalloc(ctx, &W.v2, (size_t)(nnz > 0 ? nnz : 1)));
      SPFOM_TRY(dalloc(ctx, &W.vt2, (size_t)(nnz > 0 ? nnz : 1)));
      SPFOM_TRY(dalloc(ctx, &W.seg4, (size_t)(L > 0 ? L : 1)));
      SPFOM_TRY(dalloc(ctx, &W.marg2, (size_t)(n > 0 ? n : 1)));
      SPFOM_TRY(dalloc(ctx, &W.marg2_eval, (size_t)(n > 0 ? n : 1)));
    }
    if (kmax > 32 && !W.fast) {
      free_instance(ctx);
      return fail(ctx, SPFOM_ENOTSUP, "sets of more than 32 products need the certified-decision kernel");
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
  SPFOM_TRY(dalloc(ctx, &W.zmpart, (size_t)W.vec_blocks));
  W.x_cur = nullptr;
  if (ctx->p.batch_frac < 1.0) SPFOM_TRY(dalloc(ctx, &W.x_cur, (size_t)nnz));
  W.xsum = nullptr;
  if (ctx->p.track_xbar) {
    if (ctx->p.precision != 64 || ctx->p.batch_frac < 1.0 || ctx->loading_batch || kmax > 32) {
      free_instance(ctx);
      return fail(ctx, SPFOM_ENOTSUP, "track_xbar needs precision 64, batch_frac 1, a single instance and sets "
                                      "of <= 32 products");
    }
    SPFOM_TRY(dalloc(ctx, &W.xsum, (size_t)(nnz > 0 ? nnz : 1)));
    SPFOM_CUDA(ctx, cudaMemsetAsync(W.xsum, 0, sizeof(double) * (size_t)(nnz > 0 ? nnz : 1), ctx->stream));
  }
  W.sl = spfom::SlView{};
  W.sl_perm = nullptr;
  W.rx = spfom::SlView{};
  W.rx_perm = nullptr;
#undef SPFOM_TRY
  ctx->P = P;
  if (W.v2) {
    e = spfom::launch_dd_prep(P, W.v2, W.vt2, W.seg4, ctx->stream);
    if (e != cudaSuccess) { free_instance(ctx); return cuda_fail(ctx, e, "double-float images"); }
  }
  if (W.v32) {
    e = spfom::launch_prep_f32(P, W, ctx->stream);
    if (e != cudaSuccess) { free_instance(ctx); return cuda_fail(ctx, e, "binary32 copies"); }
  }
  if (W.fast && (W.plan.fast_sl || W.plan.f32_sl)) {  // a requested slot-major tiling
    const spfom_status st = build_sliced(ctx);
    if (st != SPFOM_OK) { free_instance(ctx); return st; }
  }
  if (W.fast && (W.plan.fast_rows || W.plan.f32_rows)) {  // the requested row-exact tiling
    const spfom_status st = build_rows(ctx);
    if (st != SPFOM_OK) { free_instance(ctx); return st; }
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
  cfg.restart_tau_balance = ctx->p.restart_tau_balance;
  cfg.kkt_tol = ctx->p.kkt_tol;
  cfg.f32 = ctx->p.precision == 32 ? 1 : 0;
  ctx->W.wait_limit = ctx->wait_limit;
  ctx->loaded = true;
  W.batch = false;
  if (ctx->loading_batch) {
    const auto& B = *ctx->loading_batch;
    if (!W.fast) {
      free_instance(ctx);
      return fail(ctx, SPFOM_ENOTSUP, "a batch needs the certified-decision kernel (sets of <= 32 products, path 0)");
    }
    ctx->batch = B;
    std::vector<int> res_inst((size_t)m), prod_inst((size_t)n), seg_inst((size_t)L);
    ctx->inst_tau.assign((size_t)B.count, 0.0);
    ctx->inst_mean_r.assign((size_t)B.count, 0.0);
    for (int b = 0; b < B.count; ++b) {
      for (int i = B.res_ptr[b]; i < B.res_ptr[b + 1]; ++i) res_inst[i] = b;
      for (int j = B.prod_ptr[b]; j < B.prod_ptr[b + 1]; ++j) prod_inst[j] = b;
      for (long long l = B.seg_off[b]; l < B.seg_off[b + 1]; ++l) seg_inst[l] = b;
      double sr = 0.0, sc = 0.0;
      const int nb = B.prod_ptr[b + 1] - B.prod_ptr[b], mb = B.res_ptr[b + 1] - B.res_ptr[b];
      for (int j = B.prod_ptr[b]; j < B.prod_ptr[b + 1]; ++j) sr += I->r[j];
      for (int i = B.res_ptr[b]; i < B.res_ptr[b + 1]; ++i) sc += I->c[i];
      const double mr = nb > 0 ? sr / nb : 0.0, mc = mb > 0 ? sc / mb : 0.0;
      ctx->inst_mean_r[b] = mr;
      ctx->inst_tau[b] = ctx->p.tau > 0.0 ? ctx->p.tau : ((mc > 0.0 && mr > 0.0) ? ctx->p.tau0 * mr / mc : ctx->p.tau0);
    }
    spfom::BatchMaps& M = W.bm;
    M.count = B.count;
    int *d_ri, *d_pi, *d_si, *d_rp, *d_pp, *d_conv;
    long long* d_so;
    spfom::InstState* d_inst;
#define SPFOM_TRYB(x) do { spfom_status s_ = (x); if (s_ != SPFOM_OK) { free_instance(ctx); return s_; } } while (0)
    SPFOM_TRYB(upload(ctx, &d_ri, res_inst.data(), res_inst.size()));
    SPFOM_TRYB(upload(ctx, &d_pi, prod_inst.data(), prod_inst.size()));
    SPFOM_TRYB(upload(ctx, &d_si, seg_inst.data(), seg_inst.size()));
    SPFOM_TRYB(upload(ctx, &d_rp, B.res_ptr.data(), B.res_ptr.size()));
    SPFOM_TRYB(upload(ctx, &d_pp, B.prod_ptr.data(), B.prod_ptr.size()));
    SPFOM_TRYB(upload(ctx, &d_so, B.seg_off.data(), B.seg_off.size()));
    SPFOM_TRYB(dalloc(ctx, &d_inst, (size_t)B.count));
    SPFOM_TRYB(dalloc(ctx, &d_conv, (size_t)B.count));
    SPFOM_TRYB(dalloc(ctx, &M.z_seg, (size_t)L));
    SPFOM_TRYB(dalloc(ctx, &M.cy_res, (size_t)m));
#undef SPFOM_TRYB
    M.res_inst = d_ri; M.prod_inst = d_pi; M.seg_inst = d_si; M.res_ptr = d_rp; M.prod_ptr = d_pp;
    M.seg_off = d_so; M.inst = d_inst; M.conv = d_conv;
    W.batch = true;
  }
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
// `old` (a stale executable graph of an earlier capture, or null) is updated
// in place from the new capture when the update is possible, else destroyed.
cudaGraphExec_t capture_period(spfom_ctx* ctx, cudaGraphExec_t old) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    if (old) cudaGraphExecDestroy(old);
    return nullptr;
  }
  bool ok = true;
  for (long long k = 0; k < ctx->p.eval_every && ok; ++k)
    ok = spfom::launch_iteration(ctx->P, ctx->W, ctx->cfg, ctx->stream) == cudaSuccess;
  if (ok) ok = spfom::launch_eval(ctx->P, ctx->W, ctx->cfg, ctx->stream) == cudaSuccess;
  if (cudaStreamEndCapture(ctx->stream, &g) != cudaSuccess || !ok) ok = false;
  if (ok && old) {
    cudaGraphExecUpdateResultInfo info{};
    if (cudaGraphExecUpdate(old, g, &info) == cudaSuccess) {
      ex = old;
      old = nullptr;
    }
    cudaGetLastError();
  }
  if (ok && !ex && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    ok = false;
    ex = nullptr;
  }
  if (old) cudaGraphExecDestroy(old);
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  return ok ? ex : nullptr;
}

// One graph whose conditional WHILE node replays the evaluation period (the
// iterations and the evaluation of capture_period) followed by the test
// kernel, which sets the node's condition on the device: a whole phase of
// spfom_solve runs without a host round trip.
cudaGraphExec_t capture_loop(spfom_ctx* ctx) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return nullptr;
  bool ok = true;
  cudaGraphConditionalHandle h{};
  ok = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node{};
  if (ok) ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
  if (ok) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
         cudaSuccess;
    if (ok) {
      for (long long k = 0; k < ctx->p.eval_every && ok; ++k)
        ok = spfom::launch_iteration(ctx->P, ctx->W, ctx->cfg, ctx->stream) == cudaSuccess;
      if (ok) ok = spfom::launch_eval(ctx->P, ctx->W, ctx->cfg, ctx->stream) == cudaSuccess;
      if (ok) ok = spfom::launch_loop_test(ctx->W, ctx->d_loop, h, (int)ctx->p.eval_every, ctx->stream) == cudaSuccess;
      cudaGraph_t cap = nullptr;
      if (cudaStreamEndCapture(ctx->stream, &cap) != cudaSuccess) ok = false;
    }
  }
  if (ok && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    ok = false;
    ex = nullptr;
  }
  cudaGraphDestroy(g);
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
      const int pk = ctx->cfg.f32 ? 1 : 0;
      cudaGraphExec_t& ex = ctx->period[pk];
      if (ex && ctx->period_stale[pk] && ctx->period_E[pk] == E &&
          std::memcmp(&ctx->period_P[pk], &ctx->P, sizeof(Problem)) == 0 &&
          std::memcmp(&ctx->period_W[pk], &ctx->W, sizeof(Work)) == 0 &&
          std::memcmp(&ctx->period_cfg[pk], &ctx->cfg, sizeof(RunConfig)) == 0)
        ctx->period_stale[pk] = false;  // every captured launch would be the same
      if (!ex || ctx->period_stale[pk]) {
        ex = capture_period(ctx, ex);
        ctx->period_stale[pk] = false;
        if (ex) {
          std::memcpy(&ctx->period_P[pk], &ctx->P, sizeof(Problem));
          std::memcpy(&ctx->period_W[pk], &ctx->W, sizeof(Work));
          std::memcpy(&ctx->period_cfg[pk], &ctx->cfg, sizeof(RunConfig));
          ctx->period_E[pk] = E;
        }
      }
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
  if (ctx->W.batch) {
    // the host counts batch iterations itself (instances stop counting when they converge)
    ctx->host_t = t;
  }
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

namespace {

// One phase of spfom_solve as a single launch of the device-loop graph
// (params.device_loop): evaluation periods until the device-side test ends the
// phase. *used stays false (and nothing runs) when the loop does not apply:
// device_loop off, graphs off or unavailable, profiling, less than one period
// left, or the iteration count between periods.
spfom_status run_loop(spfom_ctx* ctx, long long left, spfom_stats* out, bool* used) {
  *used = false;
  const long long E = ctx->p.eval_every;
  if (!ctx->p.device_loop || !ctx->p.graphs || E <= 0 || ctx->p.profile || left < E || ctx->host_t % E != 0 ||
      ctx->period_failed)
    return SPFOM_OK;
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  if (!ctx->d_loop) {
    spfom_status a = dalloc(ctx, &ctx->d_loop, 1);
    if (a != SPFOM_OK) return a;
  }
  spfom::DevLoop L{};
  L.t = ctx->host_t;
  L.t_end = ctx->host_t + left;
  L.batch_switch = (ctx->W.batch && ctx->cfg.f32) ? 1 : 0;
  SPFOM_CUDA(ctx, cudaMemcpyAsync(ctx->d_loop, &L, sizeof L, cudaMemcpyHostToDevice, ctx->stream));
  cudaGraphExec_t& ex = ctx->loop[ctx->cfg.f32 ? 1 : 0];
  if (!ex) ex = capture_loop(ctx);
  if (!ex) return SPFOM_OK;  // conditional graphs unavailable: the caller steps period by period
  SPFOM_CUDA(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
  SPFOM_CUDA(ctx, cudaGraphLaunch(ex, ctx->stream));
  SPFOM_CUDA(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
  SPFOM_CUDA(ctx, cudaMemcpyAsync(&L, ctx->d_loop, sizeof L, cudaMemcpyDeviceToHost, ctx->stream));
  DevState st;
  spfom_status s = read_state(ctx, &st);  // synchronises the stream
  if (s != SPFOM_OK) return s;
  float ms = 0.f;
  SPFOM_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  const long long periods = (L.t - ctx->host_t) / E;
  ctx->host_t = ctx->W.batch ? L.t : st.t;
  fill_stats(ctx, st, ms * 1e-3, out);
  *used = true;
  if (st.error)
    return fail(ctx, SPFOM_ETIMEOUT, "a bounded device wait (bulk-copy staging) gave up; results are invalid");
  if (out) {
    out->kernel_launches =
        periods * (E * spfom::kernel_launches_per_iteration(ctx->W, ctx->cfg) + spfom::kernel_launches_per_eval() + 1);
    out->seg_kernel_seconds = 0.0;
    out->seg_kernel_launches = 0;
  }
  return SPFOM_OK;
}

}  // namespace

spfom_status spfom_solve(spfom_ctx* ctx, const double* y0, spfom_stats* out) {
  spfom_status s = spfom_reset(ctx, y0);
  if (s != SPFOM_OK) return s;
  const long long E = ctx->p.eval_every > 0 ? ctx->p.eval_every : 1024;
  spfom_stats st{};
  double secs = 0.0, seg = 0.0;
  long long segl = 0, launches = 0;
  // the paper's stagnation rule, logged: iterations since the evaluated dual objective last improved
  double best_dual = INFINITY;
  long long last_improved = 0;
  const long long stall_limit = std::max(1LL, (long long)(ctx->P.L / 100));
  bool polished = false;  // precision 32: the binary64 confirmation period has run
  for (;;) {
    long long left = ctx->p.max_iters - ctx->host_t;
    if (left <= 0) break;
    bool looped = false;
    s = run_loop(ctx, left, &st, &looped);
    if (s != SPFOM_OK) return s;
    if (!looped) {
      s = spfom_step(ctx, left < E ? left : E, &st);
      if (s != SPFOM_OK) return s;
    }
    if (st.evals > 0 && std::isfinite(st.dual_avg)) {
      if (!(st.dual_avg >= best_dual - 1e-9 * std::fabs(best_dual))) {
        best_dual = st.dual_avg;
        last_improved = st.iters;
      }
    }
    st.stall_iters = st.iters - last_improved;
    st.stagnated = st.stall_iters >= stall_limit ? 1 : 0;
    secs += st.seconds;
    seg += st.seg_kernel_seconds;
    segl += st.seg_kernel_launches;
    launches += st.kernel_launches;
    if (ctx->W.batch && ctx->cfg.f32 && !st.converged && !ctx->h_inst.empty()) {
      // a few members left: finish them with binary64 iterations (a binary32 run can stall
      // above the tolerance near ties, and the frozen members cost little either way), and
      // confirm the members that converged in binary32 now, with binary64 iterations that
      // run beside the last members' instead of after them
      long long active = 0;
      for (const auto& I : ctx->h_inst) active += I.converged ? 0 : 1;
      if (active * 20 <= (long long)ctx->h_inst.size()) {
        ctx->cfg.f32 = 0;  // the binary64 period graph is kept apart from the binary32 one
        ctx->polishing = true;
        if (ctx->p.polish && !polished) {
          polished = true;
          for (auto& I : ctx->h_inst) I.converged = 0;
          SPFOM_CUDA(ctx, cudaMemcpyAsync(ctx->W.bm.inst, ctx->h_inst.data(),
                                          sizeof(spfom::InstState) * ctx->W.bm.count, cudaMemcpyHostToDevice,
                                          ctx->stream));
          SPFOM_CUDA(ctx, cudaMemsetAsync(ctx->W.bm.conv, 0, sizeof(int) * ctx->W.bm.count, ctx->stream));
        }
      }
    }
    if (st.converged && ctx->p.precision == 32 && ctx->p.polish && !polished) {
      polished = true;
      // binary64 polish: clear the flag(s) and iterate in binary64 until the next evaluation
      ctx->cfg.f32 = 0;
      ctx->polishing = true;
      const int zero = 0;
      SPFOM_CUDA(ctx, cudaMemcpyAsync(&ctx->W.st->converged, &zero, sizeof zero, cudaMemcpyHostToDevice,
                                      ctx->stream));
      if (ctx->W.batch) {
        for (auto& I : ctx->h_inst) I.converged = 0;
        SPFOM_CUDA(ctx, cudaMemcpyAsync(ctx->W.bm.inst, ctx->h_inst.data(),
                                        sizeof(spfom::InstState) * ctx->W.bm.count, cudaMemcpyHostToDevice,
                                        ctx->stream));
        SPFOM_CUDA(ctx, cudaMemsetAsync(ctx->W.bm.conv, 0, sizeof(int) * ctx->W.bm.count, ctx->stream));
      }
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
  if (ctx->W.W > 32) return fail(ctx, SPFOM_ENOTSUP, "spfom_evaluate needs sets of <= 32 products (the sorting kernel)");
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

extern "C" {

spfom_status spfom_load_batch(spfom_ctx* ctx, const spfom_instance* insts, int32_t count) {
  if (!ctx) return SPFOM_EINVAL;
  if (!insts || count <= 0) return fail(ctx, SPFOM_EINVAL, "a batch needs at least one instance");
  // validate each instance, then concatenate them into the block-diagonal union
  long long n = 0, m = 0, L = 0, nnz = 0, nnzA = 0;
  bool any_w = false, any_aval = false;
  for (int b = 0; b < count; ++b) {
    int kmax = 0;
    spfom_status s = validate(ctx, &insts[b], &kmax);
    if (s != SPFOM_OK) {
      ctx->err = "instance " + std::to_string(b) + ": " + ctx->err;
      return s;
    }
    n += insts[b].n;
    m += insts[b].m;
    L += insts[b].L;
    nnz += insts[b].seg_ptr[insts[b].L];
    nnzA += insts[b].n > 0 ? insts[b].a_ptr[insts[b].n] : 0;
    any_w |= insts[b].w != nullptr;
    any_aval |= insts[b].a_val != nullptr;
  }
  if (n > INT32_MAX || m > INT32_MAX || nnzA > INT32_MAX) return fail(ctx, SPFOM_EINVAL, "batch too large");
  std::vector<double> r((size_t)n), c((size_t)m), aval(any_aval ? (size_t)nnzA : 0), v((size_t)nnz),
      w(any_w ? (size_t)nnz : 0), lam((size_t)L), v0((size_t)L);
  std::vector<int32_t> a_ptr((size_t)n + 1, 0), a_idx((size_t)nnzA), prod((size_t)nnz);
  std::vector<int64_t> seg_ptr((size_t)L + 1, 0);
  spfom_ctx::BatchSpec B;
  B.count = count;
  B.res_ptr.assign((size_t)count + 1, 0);
  B.prod_ptr.assign((size_t)count + 1, 0);
  B.seg_off.assign((size_t)count + 1, 0);
  long long jo = 0, io = 0, lo = 0, po = 0, qo = 0;
  for (int b = 0; b < count; ++b) {
    const spfom_instance& I = insts[b];
    const long long Kb = I.seg_ptr[I.L], Ab = I.n > 0 ? I.a_ptr[I.n] : 0;
    for (int j = 0; j < I.n; ++j) {
      r[jo + j] = I.r[j];
      a_ptr[jo + j + 1] = (int32_t)(qo + I.a_ptr[j + 1]);
    }
    for (long long q = 0; q < Ab; ++q) {
      a_idx[qo + q] = (int32_t)(io + I.a_idx[q]);
      if (any_aval) aval[qo + q] = I.a_val ? I.a_val[q] : 1.0;
    }
    for (int i = 0; i < I.m; ++i) c[io + i] = I.c[i];
    for (long long l = 0; l < I.L; ++l) {
      seg_ptr[lo + l + 1] = po + I.seg_ptr[l + 1];
      lam[lo + l] = I.lam[l];
      v0[lo + l] = I.v0[l];
    }
    for (long long p = 0; p < Kb; ++p) {
      prod[po + p] = (int32_t)(jo + I.seg_prod[p]);
      v[po + p] = I.v[p];
      if (any_w) w[po + p] = I.w ? I.w[p] : 0.0;
    }
    jo += I.n;
    io += I.m;
    lo += I.L;
    po += Kb;
    qo += Ab;
    B.res_ptr[b + 1] = (int)io;
    B.prod_ptr[b + 1] = (int)jo;
    B.seg_off[b + 1] = lo;
  }
  spfom_instance U{};
  U.n = (int32_t)n;
  U.m = (int32_t)m;
  U.L = L;
  U.r = r.data();
  U.c = c.data();
  U.a_ptr = a_ptr.data();
  U.a_idx = a_idx.data();
  U.a_val = any_aval ? aval.data() : nullptr;
  U.seg_ptr = seg_ptr.data();
  U.seg_prod = prod.data();
  U.v = v.data();
  U.w = any_w ? w.data() : nullptr;
  U.lam = lam.data();
  U.v0 = v0.data();
  ctx->loading_batch = &B;
  spfom_status s = spfom_load_instance(ctx, &U);
  ctx->loading_batch = nullptr;
  return s;
}

spfom_status spfom_batch_stats(spfom_ctx* ctx, spfom_stats* out) {
  if (!ctx || !out) return SPFOM_EINVAL;
  if (!ctx->loaded || !ctx->W.batch) return fail(ctx, SPFOM_ESTATE, "no batch loaded");
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  DevState st;
  spfom_status s = read_state(ctx, &st);
  if (s != SPFOM_OK) return s;
  for (int b = 0; b < ctx->W.bm.count; ++b) inst_stats(ctx, ctx->h_inst[b], &out[b]);
  return SPFOM_OK;
}

spfom_status spfom_update(spfom_ctx* ctx, const double* c, const double* lam) {
  if (!ctx) return SPFOM_EINVAL;
  if (!ctx->loaded) return fail(ctx, SPFOM_ESTATE, "no instance loaded");
  const Problem& P = ctx->P;
  if (c)
    for (int i = 0; i < P.m; ++i)
      if (!(c[i] >= 0.0) || !is_finite(c[i])) return fail(ctx, SPFOM_EINVAL, "c[%d] must be finite and >= 0", i);
  double mass = 0.0;
  if (lam) {
    for (long long l = 0; l < P.L; ++l) {
      if (!(lam[l] >= 0.0) || !is_finite(lam[l])) return fail(ctx, SPFOM_EINVAL, "lam[%lld] must be >= 0", l);
      mass += lam[l];
    }
    int e2 = 0;
    std::frexp(mass > 1.0 ? mass : 1.0, &e2);
    const int F = 61 - e2;
    if (ctx->W.fast && F < 30) return fail(ctx, SPFOM_ENOTSUP, "arrival mass too large for the fixed-point sales");
    if (ctx->W.fast) {
      ctx->W.fx_bits = F;
      ctx->W.fx_scale = std::ldexp(1.0, F);
      ctx->W.inv_fx_scale = std::ldexp(1.0, -F);
    }
  }
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  drop_graphs(ctx);  // captured launches carry the fixed-point scale
  if (c) SPFOM_CUDA(ctx, cudaMemcpyAsync(const_cast<double*>(P.c), c, sizeof(double) * P.m, cudaMemcpyHostToDevice,
                                         ctx->stream));
  if (lam) {
    SPFOM_CUDA(ctx, cudaMemcpyAsync(const_cast<double*>(P.lam), lam, sizeof(double) * P.L, cudaMemcpyHostToDevice,
                                    ctx->stream));
    if (ctx->W.v32) {
      cudaError_t e = spfom::launch_prep_f32(P, ctx->W, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "binary32 copies");
    }
    if (ctx->W.v2) {  // the double-float images of lambda
      cudaError_t e = spfom::launch_dd_prep(P, ctx->W.v2, ctx->W.vt2, ctx->W.seg4, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "double-float images");
    }
    if (ctx->W.sl.nchunks > 0) {  // lambda of the slot-major copy
      cudaError_t e = spfom::launch_slice_segments(P, ctx->W, ctx->W.plan.W8, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "slot-major copy");
    }
    if (ctx->W.rx.nchunks > 0) {  // lambda of the row-exact copy
      cudaError_t e = spfom::launch_rows_segments(P, ctx->W.rx, ctx->W.rx_perm, ctx->W.lam32, ctx->W.vt0_32,
                                                  ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "row-exact copy");
    }
  }
  // step sizes follow the new capacities: tau0 * mean(r) / mean(c), per instance in a batch
  if (c && !(ctx->p.tau > 0.0)) {
    auto tau_of = [&](double mr, double mc) { return (mc > 0.0 && mr > 0.0) ? ctx->p.tau0 * mr / mc : ctx->p.tau0; };
    if (ctx->W.batch) {
      for (int b = 0; b < ctx->batch.count; ++b) {
        double sc = 0.0;
        const int i0 = ctx->batch.res_ptr[b], i1 = ctx->batch.res_ptr[b + 1];
        for (int i = i0; i < i1; ++i) sc += c[i];
        ctx->inst_tau[b] = tau_of(ctx->inst_mean_r[b], i1 > i0 ? sc / (i1 - i0) : 0.0);
      }
    } else {
      std::vector<double> r((size_t)P.n);
      SPFOM_CUDA(ctx, cudaMemcpyAsync(r.data(), P.r, sizeof(double) * P.n, cudaMemcpyDeviceToHost, ctx->stream));
      SPFOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      double sr = 0.0, sc = 0.0;
      for (int j = 0; j < P.n; ++j) sr += r[j];
      for (int i = 0; i < P.m; ++i) sc += c[i];
      ctx->tau_init = tau_of(P.n > 0 ? sr / P.n : 0.0, P.m > 0 ? sc / P.m : 0.0);
    }
  }
  SPFOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SPFOM_OK;
}

spfom_status spfom_set_wait_limit(spfom_ctx* ctx, uint32_t polls) {
  if (!ctx) return SPFOM_EINVAL;
  ctx->wait_limit = polls;
  ctx->W.wait_limit = polls;
  drop_graphs(ctx);  // captured launches carry the old limit
  return SPFOM_OK;
}

spfom_status spfom_sales_at(spfom_ctx* ctx, const double* y, double* s_out) {
  if (!ctx || !y || !s_out) return SPFOM_EINVAL;
  if (!ctx->loaded) return fail(ctx, SPFOM_ESTATE, "no instance loaded");
  if (ctx->W.W > 32) return fail(ctx, SPFOM_ENOTSUP, "spfom_sales_at needs sets of <= 32 products (the sorting kernel)");
  const Problem& P = ctx->P;
  for (int i = 0; i < P.m; ++i)
    if (!(y[i] >= 0.0) || !is_finite(y[i])) return fail(ctx, SPFOM_EINVAL, "y[%d] must be finite and >= 0", i);
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  if (P.m) SPFOM_CUDA(ctx, cudaMemcpyAsync(ctx->W.y_eval, y, sizeof(double) * P.m, cudaMemcpyHostToDevice, ctx->stream));
  Work w = ctx->W;
  w.s = ctx->W.s_eval;  // scatter into the evaluation buffer: the iteration state stays as it is
  cudaError_t e = spfom::launch_sales_at(P, w, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sales launch");
  if (P.n) SPFOM_CUDA(ctx, cudaMemcpyAsync(s_out, w.s, sizeof(double) * P.n, cudaMemcpyDeviceToHost, ctx->stream));
  SPFOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SPFOM_OK;
}

}  // extern "C"

extern "C" spfom_status spfom_autotune(spfom_ctx* ctx, int32_t iters, int32_t* choice_out) {
  if (!ctx) return SPFOM_EINVAL;
  if (!ctx->loaded) return fail(ctx, SPFOM_ESTATE, "no instance loaded");
  if (iters <= 0) return fail(ctx, SPFOM_EINVAL, "iters must be > 0");
  spfom::FastPlan& plan = ctx->W.plan;
  // binary32 pass: the tilings 1..7 of include/spfom.h; double-float binary64 pass: the
  // tilings of k_seg_dd (1..3); binary64-sum pass: 1, and 2 (margins in shared memory).
  const bool f32 = ctx->W.fast && ctx->W.v32 && ctx->cfg.f32;
  const bool dd = ctx->W.fast && ctx->W.v2 && !ctx->cfg.f32;
  const bool f64 = ctx->W.fast && !ctx->cfg.f32 && !dd;
  auto current = [&]() {
    return f32 ? (plan.f32_rows ? 9 : plan.f32_sl ? 8 : plan.f32_ms ? 7
                              : (plan.bchunk ? 6
                                             : (plan.f32_p16 ? 5
                                                             : (plan.coop ? 4 : (plan.tma ? 2 : (plan.f32_p8 ? 3 : 1))))))
               : (dd ? plan.dd_variant : (plan.fast_rows ? 4 : (plan.fast_sl ? 3 : (plan.fast_ms ? 2 : 1))));
  };
  // The staged kernels (2, 4) load whole tiles even when a batch has frozen
  // (converged) members, which the plain-load kernels skip; their early timing
  // would not hold over a batched solve, so batches choose among the plain-load
  // tilings.
  auto available = [&](int c) {
    if (f32 && c == 7) return plan.ms_ok != 0;
    if (f32 && c == 8) return ctx->W.sl.nchunks > 0;
    if (f32 && c == 9) return ctx->W.rx.nchunks > 0;
    if (f64)
      return c == 1 || (c == 2 && plan.ms_ok != 0) || (c == 3 && ctx->W.sl.nchunks > 0) ||
             (c == 4 && ctx->W.rx.nchunks > 0);
    if (f32 && c == 6) return plan.bchunk_ok != 0 && ctx->W.batch && ctx->W.bc_count > 0;
    if (f32 && c == 5) return ctx->W.W <= 32;  // 16 products per lane and at most two lanes
    if (f32) return c == 4 ? (plan.coop_ok != 0 && !ctx->W.batch) : (c != 2 || (plan.tma_ok && !ctx->W.batch));
    return c <= 3 && dd && spfom::dd_variant_ok(plan, c);
  };
  auto select = [&](int c) {
    if (f32) {
      plan.tma = c == 2 ? 1 : 0;
      plan.f32_p8 = c == 3 ? 1 : 0;
      plan.coop = c == 4 ? 1 : 0;
      plan.f32_p16 = c == 5 ? 1 : 0;
      plan.bchunk = c == 6 ? 1 : 0;
      plan.f32_ms = c == 7 ? 1 : 0;
      plan.f32_sl = c == 8 ? 1 : 0;
      plan.f32_rows = c == 9 ? 1 : 0;
    } else if (dd) {
      plan.dd_variant = c;
    } else {
      plan.fast_ms = c == 2 ? 1 : 0;
      plan.fast_sl = c == 3 ? 1 : 0;
      plan.fast_rows = c == 4 ? 1 : 0;
    }
  };
  if (!f32 && !dd && !(f64 && (plan.ms_ok || plan.sl_ok || plan.rows_ok))) {
    if (choice_out) *choice_out = 1;
    return SPFOM_OK;
  }
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  if ((f32 || f64) && plan.sl_ok) {  // the slot-major candidates need their copy
    const spfom_status sb = build_sliced(ctx);
    if (sb != SPFOM_OK) return sb;
  }
  if ((f32 || f64) && plan.rows_ok && !ctx->W.batch) {  // and the row-exact candidate its own
    const spfom_status sb = build_rows(ctx);
    if (sb != SPFOM_OK) return sb;
  }
  std::vector<double> y0((size_t)ctx->P.m);
  if (ctx->P.m)
    SPFOM_CUDA(ctx, cudaMemcpyAsync(y0.data(), ctx->W.y, sizeof(double) * ctx->P.m, cudaMemcpyDeviceToHost,
                                    ctx->stream));
  SPFOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const double saved_tol = ctx->cfg.kkt_tol;
  ctx->cfg.kkt_tol = -1.0;  // no instance may converge (and stop working) while being timed
  double best = INFINITY;
  int choice = current();
  for (int cand = 1; cand <= 9; ++cand) {
    if (!available(cand)) continue;
    select(cand);
    drop_graphs(ctx);
    spfom_status s = init_state(ctx, y0.data());
    spfom_stats st{};
    if (s == SPFOM_OK) s = spfom_step(ctx, iters, &st);   // warm-up
    if (s == SPFOM_OK) s = spfom_step(ctx, iters, &st);
    if (s != SPFOM_OK) {
      ctx->cfg.kkt_tol = saved_tol;
      return s;
    }
    if (st.seconds < best) {
      best = st.seconds;
      choice = cand;
    }
  }
  ctx->cfg.kkt_tol = saved_tol;
  select(choice);
  drop_graphs(ctx);
  spfom_status s = init_state(ctx, y0.data());
  if (s != SPFOM_OK) return s;
  if (choice_out) *choice_out = choice;
  return SPFOM_OK;
}

// ---- learned warm start (include/spfom_mlp.h) ------------------------------------

namespace {

struct WarmScratch {
  float* feat;     // [m][16]
  float* out;      // [m]
  double* d;       // [m]
  double* y;       // [m]
  double* rho;     // [n]
  double* totals;  // [4]
};

spfom_status warm_scratch(spfom_ctx* ctx, WarmScratch* w) {
  const size_t m = (size_t)std::max(ctx->P.m, 1), n = (size_t)std::max(ctx->P.n, 1);
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t need = up(m * 16 * 4) + up(m * 4) + up(m * 8) * 2 + up(n * 8) + up(4 * 8);
  if (need > ctx->warm_bytes) {
    if (ctx->warm_buf) cudaFree(ctx->warm_buf);
    ctx->warm_buf = nullptr;
    ctx->warm_bytes = 0;
    SPFOM_CUDA(ctx, cudaMalloc(&ctx->warm_buf, need));
    ctx->warm_bytes = need;
  }
  char* p = static_cast<char*>(ctx->warm_buf);
  w->feat = reinterpret_cast<float*>(p);
  p += up(m * 16 * 4);
  w->out = reinterpret_cast<float*>(p);
  p += up(m * 4);
  w->d = reinterpret_cast<double*>(p);
  p += up(m * 8);
  w->y = reinterpret_cast<double*>(p);
  p += up(m * 8);
  w->rho = reinterpret_cast<double*>(p);
  p += up(n * 8);
  w->totals = reinterpret_cast<double*>(p);
  return SPFOM_OK;
}

// Features into `feat` (device [m][16]) on the ctx stream, with w's scratch.
spfom_status features_into(spfom_ctx* ctx, const WarmScratch& w, float* feat) {
  const Problem& P = ctx->P;
  if (P.m) SPFOM_CUDA(ctx, cudaMemsetAsync(ctx->W.y_eval, 0, sizeof(double) * P.m, ctx->stream));
  Work wk = ctx->W;
  wk.s = ctx->W.s_eval;
  cudaError_t e = spfom::launch_sales_at(P, wk, ctx->stream);
  if (e == cudaSuccess) e = spfom::launch_features(P, wk.s, w.d, w.rho, w.totals, feat, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "feature launch");
  return SPFOM_OK;
}

}  // namespace

extern "C" spfom_status spfom_features(spfom_ctx* ctx, float* features) {
  if (!ctx || !features) return SPFOM_EINVAL;
  if (!ctx->loaded) return fail(ctx, SPFOM_ESTATE, "no instance loaded");
  if (ctx->W.W > 32) return fail(ctx, SPFOM_ENOTSUP, "spfom_features needs sets of <= 32 products (the sorting kernel)");
  if (ctx->W.batch) return fail(ctx, SPFOM_ENOTSUP, "features are per instance; load a single instance");
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  WarmScratch w{};
  spfom_status s = warm_scratch(ctx, &w);
  if (s == SPFOM_OK) s = features_into(ctx, w, features);
  if (s != SPFOM_OK) return s;
  SPFOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return SPFOM_OK;
}

extern "C" spfom_status spfom_solve_warm(spfom_ctx* ctx, spfom_mlp* net, int64_t warm_iters, spfom_stats* out,
                                         int32_t* mode_out) {
  if (!ctx || !net) return SPFOM_EINVAL;
  if (!ctx->loaded) return fail(ctx, SPFOM_ESTATE, "no instance loaded");
  if (ctx->W.W > 32) return fail(ctx, SPFOM_ENOTSUP, "spfom_solve_warm needs sets of <= 32 products (the sorting kernel)");
  if (ctx->W.batch) return fail(ctx, SPFOM_ENOTSUP, "the warm start is per instance; load a single instance");
  const auto t0 = std::chrono::steady_clock::now();
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  const Problem& P = ctx->P;
  WarmScratch w{};
  spfom_status s = warm_scratch(ctx, &w);
  if (s == SPFOM_OK) s = features_into(ctx, w, w.feat);
  if (s != SPFOM_OK) return s;
  s = spfom_mlp_forward(net, w.feat, P.m, w.out, ctx->stream);
  if (s != SPFOM_OK) return fail(ctx, s, "warm-start forward pass: %s", spfom_status_string(s));
  cudaError_t e = spfom::launch_warm_duals(P.m, P.n, w.out, w.totals, w.y, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "warm-start duals");
  std::vector<double> y0((size_t)P.m), zero((size_t)P.m, 0.0);
  if (P.m) SPFOM_CUDA(ctx, cudaMemcpyAsync(y0.data(), w.y, sizeof(double) * P.m, cudaMemcpyDeviceToHost, ctx->stream));
  SPFOM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  // judge the prediction by the dual objective (an upper bound on the optimum: lower is better)
  double dual_warm = 0.0, dual_cold = 0.0;
  s = spfom_evaluate(ctx, y0.data(), nullptr, &dual_warm);
  if (s == SPFOM_OK) s = spfom_evaluate(ctx, zero.data(), nullptr, &dual_cold);
  if (s != SPFOM_OK) return s;
  int mode = 0;
  if (dual_warm < dual_cold) {
    const long long cap = ctx->p.max_iters;
    if (warm_iters > 0 && warm_iters < cap) ctx->p.max_iters = warm_iters;
    s = spfom_solve(ctx, y0.data(), out);
    ctx->p.max_iters = cap;
    mode = 1;
    if (s == SPFOM_ENOTCONV) {
      mode = 2;
      s = spfom_solve(ctx, nullptr, out);
    }
  } else {
    s = spfom_solve(ctx, nullptr, out);
  }
  if (mode_out) *mode_out = mode;
  if (out) out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return s;
}

// ---- assortment recovery (Section 4.4) ------------------------------------------

extern "C" spfom_status spfom_xbar(spfom_ctx* ctx, double* out) {
  if (!ctx || !out) return SPFOM_EINVAL;
  if (!ctx->loaded) return fail(ctx, SPFOM_ESTATE, "no instance loaded");
  if (!ctx->W.xsum) return fail(ctx, SPFOM_ESTATE, "x-bar is kept only when the ctx is created with track_xbar = 1");
  if (ctx->host_t <= 0) return fail(ctx, SPFOM_ESTATE, "no iteration since the last reset");
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  const long long nnz = ctx->P.nnz;
  if (nnz == 0) return SPFOM_OK;
  double* d = nullptr;
  SPFOM_CUDA(ctx, cudaMalloc(&d, sizeof(double) * (size_t)nnz));
  cudaError_t e = spfom::launch_xbar(ctx->P, ctx->W, d, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(double) * (size_t)nnz, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "x-bar");
  return SPFOM_OK;
}

extern "C" spfom_status spfom_recover(spfom_ctx* ctx, const double* x, double* alpha, int32_t* order) {
  if (!ctx || !alpha) return SPFOM_EINVAL;
  if (!ctx->loaded) return fail(ctx, SPFOM_ESTATE, "no instance loaded");
  if (ctx->W.W > 32) return fail(ctx, SPFOM_ENOTSUP, "recovery needs sets of <= 32 products");
  if (!x && (!ctx->W.xsum || ctx->host_t <= 0))
    return fail(ctx, SPFOM_ESTATE, "no x given and no x-bar kept (track_xbar = 1 and at least one iteration)");
  SPFOM_CUDA(ctx, cudaSetDevice(ctx->p.device));
  const Problem& P = ctx->P;
  const size_t nnz = (size_t)P.nnz, L = (size_t)P.L;
  if (x)
    for (size_t p = 0; p < nnz; ++p)
      if (!is_finite(x[p])) return fail(ctx, SPFOM_EINVAL, "x[%zu] is not finite", p);
  char* buf = nullptr;
  const size_t bx = ((nnz * 8 + 255) / 256) * 256, ba = (((nnz + L) * 8 + 255) / 256) * 256;
  SPFOM_CUDA(ctx, cudaMalloc(&buf, bx + ba + nnz * 4 + 256));
  double* dx = reinterpret_cast<double*>(buf);
  double* da = reinterpret_cast<double*>(buf + bx);
  int* dord = reinterpret_cast<int*>(buf + bx + ba);
  cudaError_t e = cudaSuccess;
  if (x) {
    if (nnz) e = cudaMemcpyAsync(dx, x, sizeof(double) * nnz, cudaMemcpyHostToDevice, ctx->stream);
  } else {
    e = spfom::launch_xbar(P, ctx->W, dx, ctx->stream);
  }
  if (e == cudaSuccess) e = spfom::launch_recover(P, ctx->W, dx, da, dord, ctx->stream);
  if (e == cudaSuccess && nnz + L)
    e = cudaMemcpyAsync(alpha, da, sizeof(double) * (nnz + L), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess && order && nnz)
    e = cudaMemcpyAsync(order, dord, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "recovery");
  return SPFOM_OK;
}
