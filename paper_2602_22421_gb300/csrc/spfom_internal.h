// Internal types shared by the kernels (spfom_kernels.cu,
// spfom_segments_fast.cu) and the C ABI (spfom_api.cu). Not installed; the
// public interface is include/spfom.h.
#pragma once
#include <cuda_runtime.h>

#include <vector>
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

// Per-instance scalars of a batch (spfom_load_batch): the batch is the
// block-diagonal union of its instances, and every instance keeps its own step
// size, regulariser, epoch sums, KKT residual, restart and convergence state.
struct InstState {
  double tau, mu;
  double sum_P;
  double z_sum, P, dual_iter;
  double kkt, pinf, gap, dual_avg, primal_avg, kkt_anchor;
  long long t, count, restarts, evals;
  int converged, pad;
};

// Batch maps in device memory.
struct BatchMaps {
  int count;                  // instances
  const int* res_inst;        // [m] instance of each resource
  const int* prod_inst;       // [n] instance of each product
  const int* seg_inst;        // [L] instance of each segment
  const int* res_ptr;         // [count+1] resource offsets
  const int* prod_ptr;        // [count+1] product offsets
  const long long* seg_off;   // [count+1] segment offsets
  InstState* inst;            // [count]
  int* conv;                  // [count] converged flags (read by the segment kernels)
  double* z_seg;              // [L] segment values of the last pass
  double* cy_res;             // [m] c_i y_i of the dual point of the last iteration
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

constexpr int kFastThreads = 512;
// Largest consideration set of the certified-decision path: 16 lanes x 8 slots
// (binary64), 32 lanes x 4 slots (binary32 tiling 1); the other paths and
// kernels (sorting kernel, double-float, staged, batched) take sets of <= 32.
constexpr int kFastMaxSet = 128;
constexpr int kFastMaxSmem = 200 * 1024;
#ifndef SPFOM_ROWS_MAX
#define SPFOM_ROWS_MAX 8
#endif
constexpr int kRowsMax = SPFOM_ROWS_MAX;  // slot rows per lane of the row-exact tiling (sets of <= kRowsMax on one lane)
constexpr int kRowsClasses = 5;  // its lane classes: 16, 8, 4, 2, 1 lanes per segment
constexpr int kTmaThreads = 1024;
constexpr int kMsThreads = 1024;  // block of the margins-in-shared segment kernels (one per SM)
constexpr int kTmaMaxSmem = 226 * 1024;
constexpr int kPipeThreads = 512;    // binary64 pipeline: 1 producer warp + 15 consumer warps
constexpr int kTile64Segs = 256;     // binary64 pipeline tile: segments
constexpr int kTile64Items = 2048;   // binary64 pipeline tile: products

// Launch plan of the certified-decision segment kernel.
struct FastPlan {
  int W;              // lanes per segment of k_seg_f32 (4 products per lane)
  int W8;             // lanes per segment of k_seg_fast (8 products per lane)
  int scatter;        // 1: shared-memory sums + per-block partials; 2: global atomics
  int smem;           // bytes of the per-block product accumulator (scatter 1)
  int grid;           // blocks of the binary64 iterate launch (= number of partial sums)
  int grid32;         // blocks of the binary32 iterate launch
  int grid_eval;      // blocks of the evaluation launch
  int reduce_chunks;  // grid.y of k_reduce_products
  int tma;            // 1: the binary32 pass runs k_seg_f32_tma (tile staging by bulk copies)
  int tma_W;          // its lanes per segment (8 products per lane)
  int tma_grid;       // its blocks
  int tma_ok;         // 1 when the staged kernel is available (spfom_autotune may switch tma)
  int f32_p8;         // 1: the plain-load binary32 kernel runs 8 products per lane (W8 lanes)
  int f32_p16;        // 1: it runs 16 products per lane (W16 lanes: one lane per set of <= 16)
  int W16;            // lanes per segment with 16 products per lane (1 or 2)
  int bchunk;         // 1: the binary32 pass of a batch runs the instance-chunked kernel (tiling 6)
  int bchunk_ok, bchunk_smem, bchunk_grid;
  int bchunk64_ok, bchunk64_grid;  // the binary64 pass of a batch (k_seg_fast_bchunk), used whenever planned
  int coop;           // 1: the binary32 pass runs the cooperatively staged kernel (tiling 4)
  int coop_ok, coop_items, coop_segs, coop_smem, coop_grid;
  int dd_variant;     // tiling of k_seg_dd (1..3, see spfom_segments_dd.cu)
  int dd_grid[4];     // its grid per tiling (iterate), 0 = unavailable
  int dd_grid_eval[4];  // and for the evaluation pass
  int tma_smem;       // its dynamic shared memory: product sums + two stages
  int acc_bytes;      // bytes of the product sums at the start of that memory
  int ms_ok;          // 1 when the margins-in-shared kernels fit (scatter 1, 16 n bytes of shared memory)
  int ms_smem64, ms_smem32, ms_grid, ms_grid32;
  int fast_ms;        // 1: the binary64 pass runs k_seg_fast with the margins in shared memory (tiling 2)
  int f32_ms;         // 1: the binary32 pass runs k_seg_f32 with the margins in shared memory (tiling 7)
  int fast_sl;        // 1: the binary64 pass reads the slot-major copy (tiling 3; margins shared when ms_ok)
  int f32_sl;         // 1: the binary32 pass reads the slot-major copy (tiling 8; margins shared when ms_ok)
  int sl_attr;        // 1 when the slot-major kernels accept the plan's shared memory
  int sl_ok;          // 1 when the load builds the slot-major copy (single instance, path 0)
  int pipe;           // 1: the binary64 pass runs k_seg_fast_pipe (warp-specialised TMA pipeline)
  int pipe_smem, pipe_acc_bytes, pipe_grid;
  int fast_rows;      // 1: the binary64 pass runs k_seg_rows on the row-exact copy (tiling 4)
  int rows_ok;        // 1 when tiling 4 is available (single instance, path 0)
  int rows_ms;        // 1: k_seg_rows keeps the binary32 margin images in shared memory (12 n bytes)
  int rows_grid, rows_smem;  // its grid and shared memory (0: global sums)
  int rows_ms32, rows_grid32, rows_smem32;  // the same for the binary32 row-exact kernel
  int rows_redo_grid;  // blocks of k_rows_redo (the SM count)
  int f32_rows;        // 1: the binary32 pass runs k_seg_rows32 on the row-exact copy (tiling 9)
};

// Slot-major copy of the consideration sets (the sliced tilings): positions
// = the segments sorted by set size, descending (ties: segment order), cut into
// chunks of C = 32 / W8 positions, one warp per chunk. Chunk c stores its slot
// rows p = 0 .. rows_c - 1 (rows_c = ceil(largest set of the chunk / W8)), 32
// entries each, at off[c] + 32 p: entry g W8 + r of row p is product r + p W8
// of the chunk's g-th segment (id -1, v = vt = 0 past the set's end or for a
// position past L). Each slot row of a warp is then one contiguous line.
struct SlView {
  long long* off;   // [nchunks + 1] first entry of each chunk (multiples of 32)
  int* prod;        // [off[nchunks]]
  double* v;        // [off[nchunks]] binary64 v and v - w (precision 64), else null
  double* vt;
  float* v32;       // binary32 images (precision 32), else null
  float* vt32;
  double* lam;      // [nchunks * C] per position; lam = 0, vt0 = 1 past L
  double* vt0;
  float* lam32;
  float* vt0_32;
  float* rprev;     // [nchunks * C] carried Dinkelbach ratio per position
  long long nchunks;
  // Row-exact copy (precision-64 tiling 4, spfom_segments_rows.cu): the lanes
  // per segment follow the set size (W = the smallest power of two with
  // W kRowsMax >= the set size), so the chunks fall into kRowsClasses classes
  // in order of decreasing size: class k (W = 16 >> k) holds chunks cls_c[k] ..
  // cls_c[k+1] - 1 of 32 / W positions each, its positions start at
  // cls_pos[k], and every chunk has exactly ceil(largest set / W) slot rows.
  int mixed;
  long long cls_c[6];
  long long cls_pos[6];
  long long* redo;     // [cls_pos[kRowsClasses]] positions whose binary32 decision was not certified
  unsigned* redo_ctl;  // [0] entries in redo, [1] blocks done (k_rows_redo's last block clears both)
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
  double* y_eval;      // dual point handed to spfom_evaluate / spfom_sales_at
  double* s_eval;      // [n] product sales of spfom_sales_at
  double* xsum;        // [nnz] epoch sums of every segment's response (track_xbar), or null
  // double-float images for the precision-64 kernel k_seg_dd (null when it is not used)
  float2* v2;          // [nnz] (hi, lo) of v
  float2* vt2;         // [nnz] (hi, lo) of v - w
  float4* seg4;        // [L] (hi, lo) of lambda and of vt_0
  float2* marg2;       // [n] (hi, lo) of the margins (iterate)
  float2* marg2_eval;  // [n] (hi, lo) of the margins (evaluation)
  float* rprev;        // [L] last binary32 Dinkelbach ratio of every segment (start of the next solve)
  long long* bc_seg;   // instance chunks of a batch (k_seg_f32_bchunk)
  int* bc_inst;
  long long bc_count;
  long long* coop_tile_ptr;  // [coop_ntiles + 1] tiles of k_seg_f32_coop
  long long coop_ntiles;
  bool dd_ok;          // k_seg_dd planned (path 0)
  double* z_seg;       // [L] per-segment values of spfom_evaluate
  double* zpart;       // per-block partial sums of z (iterate)
  double* zpart_eval;  // per-block partial sums of z (evaluation)
  double* cypart;      // [vec_blocks]
  double* Ppart;       // [vec_blocks]
  double* zmpart;      // [vec_blocks] partial sums of m_j s_j (the iterate's sum of z, fast path)
  double* x_cur;       // [nnz] current responses (sampling only)
  DevState* st;
  int seg_blocks;      // blocks of the general segment kernel
  int vec_blocks;
  int W;               // lanes per segment of the general kernel (power of two >= max |C_l|)
  int zparts_iter, zparts_eval;  // valid entries of zpart / zpart_eval
  // certified-decision path (spfom_segments_fast.cu)
  bool fast;
  FastPlan plan;
  unsigned long long* part;       // [plan.grid][n] per-block fixed-point product sales
  unsigned long long* s_fx;       // [n] fixed-point product sales
  unsigned long long* fallbacks;  // running count of segments decided in binary64
  double fx_scale, inv_fx_scale;  // 2^F and 2^-F
  int fx_bits;                    // F
  // binary32 copies for the precision-32 mode (null otherwise)
  float* v32;
  float* vt32;
  float* lam32;
  float* vt0_32;
  float* marg32;
  long long* tile_ptr;  // [ntiles+1] (binary32 tile staging)
  long long ntiles;
  long long* tile64_ptr;  // [ntiles64+1] (binary64 pipeline tiles)
  long long ntiles64;
  bool batch;             // instances of a batch (spfom_load_batch)
  BatchMaps bm;
  SlView sl;              // slot-major copy (sliced tilings), nchunks = 0 when absent
  long long* sl_perm;     // [nchunks * C] segment at each position, -1 past L
  SlView rx;              // row-exact copy (precision-64 tiling 4), nchunks = 0 when absent
  long long* rx_perm;     // [rx.cls_pos[kRowsClasses]] segment at each position, -1 past L
  float* marg32c;         // [n] binary32 margin images for tiling 4 (NaN: positive, outside binary32's range)
  unsigned wait_limit;    // polls of a bounded device wait (spfom_set_wait_limit; default 1 << 22)
};

struct FastArgs {
  Problem P;
  const double* marg;
  unsigned long long* part;
  double* zpart;
  const DevState* st;
  double fx_scale;
  unsigned long long* fallbacks;
  int fx_bits;  // F of the fixed-point scale 2^F
  unsigned long long* s_fx;  // product sums when the plan scatters with global atomics
  // pipeline staging (k_seg_fast_pipe)
  const long long* tile_ptr;
  long long ntiles;
  int acc_bytes;
  DevState* st_rw;
  // batch mode: skip converged instances, write per-segment values
  const int* seg_inst;
  const int* inst_conv;
  double* z_seg;
  float* rprev;  // [L] each segment's last Dinkelbach ratio (iterate passes), or null: start at 0
  long long perm_a, perm_d;  // batch: warps visit their segment chunks in the order chunk * perm_a mod #chunks
  // instance chunks of a batch (k_seg_fast_bchunk)
  long long bc_count;
  const long long* bc_seg;
  const int* bc_inst;
  const int* bc_prod_ptr;
  SlView sl;  // slot-major copy (sliced tilings)
  // row-exact tiling (k_seg_rows)
  const float* marg32c;  // [n] binary32 margin images (NaN: positive, outside binary32's normal range)
  SlView rx;             // row-exact copy
};

// Arguments of k_seg_dd (spfom_segments_dd.cu): double-float images, and the
// binary64 arrays for the segments whose decision is not certified.
struct DdArgs {
  const long long* seg_ptr;
  const int* seg_prod;
  const float2* v2;
  const float2* vt2;
  const float4* seg4;
  const float2* marg2;
  const double* marg;
  const double* v;
  const double* vt;
  const double* lam;
  const double* vt0;
  long long L;
  int n;
  int fx_bits;
  unsigned long long* part;
  unsigned long long* s_fx;
  double* zpart;
  const DevState* st;
  unsigned long long* fallbacks;
  const int* seg_inst;
  const int* inst_conv;
  double* z_seg;
};

struct F32Args {
  const long long* seg_ptr;
  const int* seg_prod;
  const float* v32;
  const float* vt32;
  const float* lam32;
  const float* vt0_32;
  long long L;
  int n;
  int fx_bits;
  const float* marg32;
  unsigned long long* part;
  unsigned long long* s_fx;
  double* zpart;
  const DevState* st;
  // tile staging (k_seg_f32_tma)
  const long long* tile_ptr;  // [ntiles+1] segment offsets of the tiles
  long long ntiles;
  int acc_bytes;
  DevState* st_rw;            // for the timeout flag
  // batch mode: skip converged instances, write per-segment values
  const int* seg_inst;
  const int* inst_conv;
  double* z_seg;
  // cooperative staging (k_seg_f32_coop)
  const long long* coop_tile_ptr;
  long long coop_ntiles;
  int coop_items, coop_segs;
  float* rprev;  // [L] each segment's last Dinkelbach ratio, or null: start at 0
  long long perm_a, perm_d;  // batch: warps visit their segment chunks in the order chunk * perm_a mod #chunks
  // instance chunks of a batch (k_seg_f32_bchunk)
  long long bc_count;
  const long long* bc_seg;   // [bc_count + 1] first segment of each chunk
  const int* bc_inst;        // [bc_count] instance of each chunk
  const int* bc_prod_ptr;    // [instances + 1] product offsets
  SlView sl;                 // slot-major copy (sliced tilings)
  unsigned wait_limit;       // polls of a staged-copy wait before it gives up (k_seg_f32_tma)
  SlView rx;                 // row-exact copy (precision-32 tiling 9, binary32 images)
};

struct RunConfig {
  double batch_frac;
  unsigned long long seed;
  unsigned long long sample_thr;  // segment l is solved at t iff hash < sample_thr
  double restart_beta, restart_artificial, restart_tau_decay, kkt_tol;
  double restart_tau_balance;
  int f32;  // run the iterations' segment pass in binary32
};

// Launchers (spfom_kernels.cu). Each returns the launch status.
// Device checks of a loaded instance (spfom_load_instance), one thread per
// segment. keys[0] = the smallest (l << kCheckSegShift | sub) over failed
// checks, sub = kSegOrder (offsets decrease), kSegLam, kSegV0, or
// kSegItems + 8 (p - seg_ptr[l]) + ItemCheck for the nonzero p: the order of
// a host loop over segments and their nonzeros. keys[1] (f32 only) = the
// smallest binary32-range failure: p for an attraction, nnz + l for lambda or
// v0 of segment l. keys[2] = the largest set. ~0 when none failed.
enum ItemCheck { kBadId = 1, kRepeated = 2, kBadV = 3, kBadW = 4 };
enum SegCheck { kSegOrder = 0, kSegLam = 1, kSegV0 = 2, kSegItems = 3 };
constexpr int kCheckSegShift = 36;
// A kernel's dynamic shared-memory limit and occupancy (spfom_kernels.cu),
// remembered per CUDA context. kernel_smem raises the limit to `bytes` when it
// is lower and never lowers it: a plan of another ctx in the same process may
// launch the kernel with more. kernel_blocks returns the resident blocks per
// SM at `threads` threads and `bytes` bytes of dynamic shared memory, raising
// the limit first (0 when either call fails).
cudaError_t kernel_smem(const void* kernel, int bytes);
int kernel_blocks(const void* kernel, int threads, int bytes);
template <class K>
cudaError_t kernel_smem(K* kernel, int bytes) {
  return kernel_smem(reinterpret_cast<const void*>(kernel), bytes);
}
template <class K>
int kernel_blocks(K* kernel, int threads, int bytes) {
  return kernel_blocks(reinterpret_cast<const void*>(kernel), threads, bytes);
}
cudaError_t launch_validate_items(const Problem& P, const double* w, const double* v0, bool f32,
                                  unsigned long long* keys, cudaStream_t s);
cudaError_t launch_prep(const Problem& P, const double* w, const double* v0, double* vt, double* vt0,
                        cudaStream_t s);
// seg_begin / seg_end (may be null) are recorded around the segment kernel.
cudaError_t launch_iteration(const Problem& P, const Work& Wk, const RunConfig& cfg, cudaStream_t s,
                             cudaEvent_t seg_begin = nullptr, cudaEvent_t seg_end = nullptr);
cudaError_t launch_eval(const Problem& P, const Work& Wk, const RunConfig& cfg, cudaStream_t s);
cudaError_t launch_evaluate_at(const Problem& P, const Work& Wk, bool want_seg, cudaStream_t s);
cudaError_t launch_sales_at(const Problem& P, const Work& Wk, cudaStream_t s);
// assortment recovery (spfom_kernels.cu): x-bar = xsum / count into out [nnz];
// alpha [nnz + L] and order [nnz] from sales x [nnz] (Lemma recover)
cudaError_t launch_xbar(const Problem& P, const Work& Wk, double* out, cudaStream_t s);
cudaError_t launch_recover(const Problem& P, const Work& Wk, const double* x, double* alpha, int* order,
                           cudaStream_t s);
// learned warm start (spfom_warm.cu)
cudaError_t launch_features(const Problem& P, const double* s0, double* d, double* rho, double* totals, float* f,
                            cudaStream_t s);
cudaError_t launch_warm_duals(int m, int n, const float* o, const double* totals, double* y, cudaStream_t s);
int kernel_launches_per_iteration(const Work& Wk, const RunConfig& cfg);
int kernel_launches_per_eval();
// Device-side loop of spfom_solve (params.device_loop): state of one phase and
// the test that ends it, launched by the body of a conditional WHILE graph node.
struct DevLoop {
  long long t, t_end;  // iterations done, and the phase's cap (batches: counted here)
  int batch_switch;    // binary32 batch: end the phase when at most 5 % of the members are active
  int ended;           // why the phase ended: 1 converged, 2 cap, 3 switch
};
cudaError_t launch_loop_test(const Work& Wk, DevLoop* lp, cudaGraphConditionalHandle h, int E, cudaStream_t s);

// spfom_segments_fast.cu
bool fast_plan(int n, int kmax, int sms, FastPlan* plan);
cudaError_t launch_seg_fast(const FastArgs& A, const FastPlan& plan, bool scatter, cudaStream_t s);
// double-float precision-64 kernel (spfom_segments_dd.cu)
cudaError_t launch_seg_dd(const DdArgs& A, const FastPlan& plan, bool scatter, cudaStream_t s);
cudaError_t launch_dd_prep(const Problem& P, float2* v2, float2* vt2, float4* seg4, cudaStream_t s);
bool dd_setup(FastPlan* plan, int sms);
// instance-chunked binary32 kernel for batches (spfom_segments_bchunk.cu)
constexpr int kBChunkProducts = 8192;  // shared-memory sums per block (64 KB)
constexpr int kBChunkSegs = 2048;      // segments per chunk
bool bchunk_plan(int max_inst_products, int sms, FastPlan* plan);
bool bchunk64_plan(int max_inst_products, int sms, FastPlan* plan);
long long make_batch_chunks(const std::vector<long long>& seg_off, int max_segs, long long* seg_out, int* inst_out);
cudaError_t launch_seg_f32_bchunk(const F32Args& A, const FastPlan& plan, cudaStream_t s);
// cooperatively staged binary32 kernel (spfom_segments_coop.cu)
bool coop_plan(int n, int kmax, int sms, FastPlan* plan);
long long make_tiles_lim(const long long* seg_ptr, long long L, int max_segs, int max_items, long long* tiles_out);
cudaError_t launch_seg_f32_coop(const F32Args& A, const FastPlan& plan, cudaStream_t s);
int dd_variant_ok(const FastPlan& plan, int v);
cudaError_t launch_seg_f32(const F32Args& A, const FastPlan& plan, cudaStream_t s);
bool tma_plan(int n, int kmax, int sms, FastPlan* plan);
// spfom_batch.cu
cudaError_t launch_batch_iteration(const Problem& P, const Work& Wk, const RunConfig& cfg, cudaStream_t s,
                                   cudaEvent_t seg_begin = nullptr, cudaEvent_t seg_end = nullptr);
cudaError_t launch_batch_eval(const Problem& P, const Work& Wk, const RunConfig& cfg, cudaStream_t s);
int batch_launches_per_iteration(const Work& Wk);
int batch_launches_per_eval();
// the segment pass of one iteration (shared with the single-instance path)
cudaError_t launch_segment_pass(const Problem& P, const Work& Wk, const RunConfig& cfg, const double* marg,
                                bool iterate, cudaStream_t s, int* zparts_out);
// spfom_segments_tma.cu
bool pipe_plan(int n, int sms, FastPlan* plan);
cudaError_t launch_seg_fast_pipe(const FastArgs& A, const FastPlan& plan, cudaStream_t s);
long long make_tiles64(const long long* seg_ptr, long long L, long long* tiles_out);
long long make_tiles(const long long* seg_ptr, long long L, long long* tiles_out);
cudaError_t launch_reduce_products(const Problem& P, const FastPlan& plan, int nparts,
                                   const unsigned long long* part, unsigned long long* s_fx, const DevState* st,
                                   cudaStream_t s);
// binary32 copies of v, vt, lambda, vt0 for the precision-32 mode
cudaError_t launch_prep_f32(const Problem& P, Work& Wk, cudaStream_t s);
// slot-major copy (spfom_sliced.cu): host layout (positions, chunk offsets;
// returns the chunk count), the gather of the items, and of lambda / vt_0
long long sliced_layout(const long long* seg_ptr, long long L, int W8, std::vector<long long>* perm,
                        std::vector<long long>* off);
cudaError_t launch_slice_items(const Problem& P, const Work& Wk, int W8, cudaStream_t s);
cudaError_t launch_slice_segments(const Problem& P, const Work& Wk, int W8, cudaStream_t s);
// row-exact copy (spfom_sliced.cu): the histogram of set sizes (hist[kFastMaxSet
// + 1], zeroed by the caller), the host layout from it (chunk offsets, classes,
// each size's first position; returns the chunk count), the scatter of the
// segments to their positions (perm preset to -1, cursor[kFastMaxSet + 1]
// zeroed), the gather of the items and of lambda / vt_0
cudaError_t launch_rows_hist(const Problem& P, unsigned long long* hist, cudaStream_t s);
long long rows_layout_counts(const unsigned long long* cnt, std::vector<long long>* off, long long cls_c[6],
                             long long cls_pos[6], long long* pos_start);
cudaError_t launch_rows_scatter(const Problem& P, const long long* pos_start, unsigned long long* cursor,
                                long long* perm, cudaStream_t s);
cudaError_t launch_rows_items(const Problem& P, const SlView& S, const long long* perm, const float* v32,
                              const float* vt32, cudaStream_t s);
cudaError_t launch_rows_segments(const Problem& P, const SlView& S, const long long* perm, const float* lam32,
                                 const float* vt0_32, cudaStream_t s);
// row-exact segment kernel (spfom_segments_rows.cu)
bool rows_plan(int n, int sms, FastPlan* plan);
cudaError_t launch_seg_rows(const FastArgs& A, const FastPlan& plan, cudaStream_t s);
// the binary64 redo of the segments the row-exact kernel did not certify (after it, into s_fx)
cudaError_t launch_rows_redo(const FastArgs& A, int sms, cudaStream_t s);
// with per-block sums: the fold of the partial sums and the redo in one launch
cudaError_t launch_reduce_redo(const FastArgs& A, const FastPlan& plan, int nparts, const unsigned long long* part,
                               cudaStream_t s);
// the row-exact binary32 pass (precision-32 tiling 9)
cudaError_t launch_seg_rows32(const F32Args& A, const FastPlan& plan, cudaStream_t s);

}  // namespace spfom
