// Internal types shared by the kernels (spfom_kernels.cu) and the C ABI
// (spfom_api.cu). Not installed; the public interface is include/spfom.h.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace spfom {

// Scalars of the iteration, resident in device memory so that every decision
// (convergence, restart, step-size changes) is taken on the device and a run
// of iterations needs no host round trip.
struct DevState {
  double tau, mu;
  double sum_P;
  double z_sum, P, dual_iter;
  double kkt, pinf, gap, dual_avg, primal_avg, kkt_anchor;
  long long t, count, restarts, evals;
  int converged, error;
  unsigned int ticket;  // arrival counter of the last-block reduction
  unsigned int pad;
  double eval_out;      // Dual(y) of spfom_evaluate
};

// Instance in device memory (all pointers device pointers).
struct Problem {
  int n, m, nnzA;
  long long L, nnz;
  const double* r;
  const double* c;
  const int* a_ptr;      // [n+1] product -> resources
  const int* a_idx;
  const double* a_val;   // may be null (all ones)
  const int* at_ptr;     // [m+1] resource -> products (ascending product id)
  const int* at_idx;
  const double* at_val;  // may be null
  const long long* seg_ptr;  // [L+1]
  const int* seg_prod;   // [nnz]
  const double* v;       // [nnz] nominal attraction
  const double* vt;      // [nnz] v - w
  const double* lam;     // [L]
  const double* vt0;     // [L] v0 + sum_{C_l} w
};

// Work buffers of one ctx.
struct Work {
  double* y;
  double* sum_y;
  double* sum_g;
  double* g;
  double* s;
  double* marg;
  double* marg_eval;
  double* y_eval;      // dual point handed to spfom_evaluate
  double* z_seg;       // [L] per-segment values of spfom_evaluate
  double* zpart;       // [seg_blocks]
  double* zpart_eval;  // [seg_blocks]
  double* cypart;      // [vec_blocks]
  double* Ppart;       // [vec_blocks]
  double* x_cur;       // [nnz] current responses (sampling only)
  DevState* st;
  int seg_blocks;
  int vec_blocks;
  int W;               // lanes per segment (power of two >= max |C_l|)
};

struct RunConfig {
  double batch_frac;
  unsigned long long seed;
  unsigned long long sample_thr;  // segment l is solved at t iff hash < sample_thr
  double restart_beta, restart_artificial, restart_tau_decay, kkt_tol;
};

// Launchers (spfom_kernels.cu). Each returns the launch status.
cudaError_t launch_prep(const Problem& P, const double* w, const double* v0, double* vt, double* vt0,
                        cudaStream_t s);
// seg_begin / seg_end (may be null) are recorded around the segment kernel.
cudaError_t launch_iteration(const Problem& P, const Work& Wk, const RunConfig& cfg, cudaStream_t s,
                             cudaEvent_t seg_begin = nullptr, cudaEvent_t seg_end = nullptr);
cudaError_t launch_eval(const Problem& P, const Work& Wk, const RunConfig& cfg, cudaStream_t s);
cudaError_t launch_evaluate_at(const Problem& P, const Work& Wk, bool want_seg, cudaStream_t s);
int kernel_launches_per_iteration();
int kernel_launches_per_eval();

}  // namespace spfom
