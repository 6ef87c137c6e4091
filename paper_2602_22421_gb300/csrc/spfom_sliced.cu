// Slot-major copy of the consideration sets for the sliced segment tilings
// (precision-64 tiling 3, precision-32 tiling 8).
//
// In the CSR layout a group of W lanes reads its segment's slice with W-wide
// strided loads, so one load instruction of a warp touches the slices of 32 / W
// segments scattered over a few hundred bytes. Here the segments are sorted by
// set size (so the sets of one chunk are about as long as each other and little
// padding is needed) and each chunk of 32 / W positions stores its slots as
// rows of 32 entries: a warp's slot row is one contiguous 128-byte (binary32,
// ids) or 256-byte (binary64) line. Lane g W + r of the chunk's warp holds
// products r, r + W, ... of the chunk's g-th segment, as in the CSR kernels, so
// the two layouts give the same per-lane sums and the same results.
#include <cuda_runtime.h>

#include <vector>

#include "spfom_internal.h"

namespace spfom {

namespace {

// One warp per chunk: entry 32 p + wl of chunk c is slot p of lane wl.
__global__ void k_slice_items(const Problem P, const float* __restrict__ v32, const float* __restrict__ vt32,
                              SlView S, const long long* __restrict__ perm, int W) {
  const int wl = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  const int C = 32 / W;
  for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < S.nchunks; c += nw) {
    const long long o = S.off[c];
    const int rows = (int)((S.off[c + 1] - o) >> 5);
    const long long l = perm[c * C + wl / W];  // -1 past L
    long long b = 0;
    int K = 0;
    if (l >= 0) {
      b = P.seg_ptr[l];
      K = (int)(P.seg_ptr[l + 1] - b);
    }
    const int r = wl & (W - 1);
    for (int p = 0; p < rows; ++p) {
      const int k = r + p * W;
      const long long e = o + 32ll * p + wl;
      const bool in = k < K;
      S.prod[e] = in ? P.seg_prod[b + k] : -1;
      if (S.v) {
        S.v[e] = in ? P.v[b + k] : 0.0;
        S.vt[e] = in ? P.vt[b + k] : 0.0;
      }
      if (S.v32) {
        S.v32[e] = in ? v32[b + k] : 0.f;
        S.vt32[e] = in ? vt32[b + k] : 0.f;
      }
    }
  }
}

// Per position: lambda and vt_0 of its segment (0 and 1 past L, so that a
// padding position has q = 0).
__global__ void k_slice_segments(const Problem P, const float* __restrict__ lam32, const float* __restrict__ vt0_32,
                                 SlView S, const long long* __restrict__ perm, long long npos) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npos;
       i += (long long)gridDim.x * blockDim.x) {
    const long long l = perm[i];
    if (S.lam) {
      S.lam[i] = l >= 0 ? P.lam[l] : 0.0;
      S.vt0[i] = l >= 0 ? P.vt0[l] : 1.0;
    }
    if (S.lam32) {
      S.lam32[i] = l >= 0 ? lam32[l] : 0.f;
      S.vt0_32[i] = l >= 0 ? vt0_32[l] : 1.f;
    }
  }
}

// Row-exact copy: one warp per chunk, the chunk's lanes per segment W from
// its class; entry 32 p + wl of chunk c is product (wl mod W) + p W of the
// chunk's (wl / W)-th segment.
__device__ __forceinline__ int rows_class(const SlView& S, long long c) {
  int k = 0;
  while (k < kRowsClasses - 1 && c >= S.cls_c[k + 1]) ++k;
  return k;
}

__global__ void k_rows_items(const Problem P, SlView S, const long long* __restrict__ perm,
                             const float* __restrict__ v32, const float* __restrict__ vt32) {
  const int wl = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < S.nchunks; c += nw) {
    const int k = rows_class(S, c), W = 16 >> k;
    const long long o = S.off[c];
    const int rows = (int)((S.off[c + 1] - o) >> 5);
    const long long l = perm[S.cls_pos[k] + (c - S.cls_c[k]) * (32 / W) + wl / W];  // -1 past L
    long long b = 0;
    int K = 0;
    if (l >= 0) {
      b = P.seg_ptr[l];
      K = (int)(P.seg_ptr[l + 1] - b);
    }
    const int r = wl & (W - 1);
    for (int p = 0; p < rows; ++p) {
      const int kk = r + p * W;
      const long long e = o + 32ll * p + wl;
      const bool in = kk < K;
      S.prod[e] = in ? P.seg_prod[b + kk] : -1;
      if (S.v) {
        S.v[e] = in ? P.v[b + kk] : 0.0;
        S.vt[e] = in ? P.vt[b + kk] : 0.0;
      }
      if (S.v32) {
        S.v32[e] = in ? v32[b + kk] : 0.f;
        S.vt32[e] = in ? vt32[b + kk] : 0.f;
      }
    }
  }
}


// Histogram of the set sizes (0..kFastMaxSet): shared-memory counts per block,
// one global add per size and block; lanes with equal sizes add once.
__global__ void k_rows_hist(const long long* __restrict__ seg_ptr, long long L, unsigned long long* __restrict__ hist) {
  __shared__ unsigned int h[kFastMaxSet + 1];
  for (int i = threadIdx.x; i <= kFastMaxSet; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < L; base += stride) {  // uniform over the block
    const long long l = base + threadIdx.x;
    long long K = -1;
    if (l < L) {
      K = seg_ptr[l + 1] - seg_ptr[l];
      K = K < kFastMaxSet ? K : kFastMaxSet;  // the fast path's sets are no larger
    }
    const unsigned peers = __match_any_sync(0xffffffffu, K);
    if (K >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h[K], (unsigned)__popc(peers));
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= kFastMaxSet; i += blockDim.x)
    if (h[i]) atomicAdd(hist + i, (unsigned long long)h[i]);
}

// Each segment to a position of its size's run: pos_start[K] + a rank drawn
// from cursor[K] (lanes with equal sizes draw together). The order within a
// run is the arrival order; every segment's solve is independent of its
// position and the sums are exact, so results do not depend on it.
__global__ void k_rows_scatter(const long long* __restrict__ seg_ptr, long long L,
                               const long long* __restrict__ pos_start, unsigned long long* __restrict__ cursor,
                               long long* __restrict__ perm) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < L; base += stride) {  // uniform over the block
    const long long l = base + threadIdx.x;
    long long K = -1;
    if (l < L) {
      K = seg_ptr[l + 1] - seg_ptr[l];
      K = K < kFastMaxSet ? K : kFastMaxSet;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, K);
    const int leader = __ffs(peers) - 1;
    unsigned long long b = 0ull;
    if (K >= 0 && lane == leader) b = atomicAdd(cursor + K, (unsigned long long)__popc(peers));
    b = __shfl_sync(0xffffffffu, b, leader);
    if (K >= 0) perm[pos_start[K] + (long long)b + __popc(peers & ((1u << lane) - 1u))] = l;
  }
}

}  // namespace

long long rows_layout_counts(const unsigned long long* cnt, std::vector<long long>* off, long long cls_c[6],
                             long long cls_pos[6], long long* pos_start) {
  // the segments in order of decreasing set size, split into the lane classes
  // W = 16, 8, 4, 2, 1; a class's chunks take 32 / W positions each (the last
  // one padded) and as many slot rows as their first (largest) set needs
  auto lanes = [](long long K) {
    int W = 1;
    while (W * kRowsMax < K) W <<= 1;
    return W;
  };
  off->assign(1, 0);
  long long nch = 0, npos = 0;
  int K = kFastMaxSet;
  for (int k = 0; k < kRowsClasses; ++k) {
    const int W = 16 >> k, C = 32 / W;
    cls_c[k] = nch;
    cls_pos[k] = npos;
    const int Ktop = K;
    long long in_class = 0;
    while (K >= 0 && lanes(K) == W) {
      pos_start[K] = npos + in_class;
      in_class += (long long)cnt[K];
      --K;
    }
    const long long chunks = (in_class + C - 1) / C;
    long long seen = 0;
    int Ks = Ktop;
    for (long long c = 0; c < chunks; ++c) {
      const long long first = c * C;  // the chunk's first (largest) segment within the class
      while (seen + (long long)cnt[Ks] <= first) seen += (long long)cnt[Ks--];
      off->push_back(off->back() + 32 * ((Ks + W - 1) / W));
    }
    nch += chunks;
    npos += chunks * C;
  }
  cls_c[kRowsClasses] = nch;
  cls_pos[kRowsClasses] = npos;
  return nch;
}

long long sliced_layout(const long long* seg_ptr, long long L, int W8, std::vector<long long>* perm,
                        std::vector<long long>* off) {
  const int C = 32 / W8;
  const long long nch = (L + C - 1) / C, npos = nch * C;
  // counting sort by set size, descending; equal sizes keep segment order
  std::vector<long long> start(34, 0);
  for (long long l = 0; l < L; ++l) ++start[(size_t)(32 - (seg_ptr[l + 1] - seg_ptr[l])) + 1];
  for (int k = 1; k < 34; ++k) start[k] += start[k - 1];
  perm->assign((size_t)npos, -1);
  for (long long l = 0; l < L; ++l) (*perm)[(size_t)start[(size_t)(32 - (seg_ptr[l + 1] - seg_ptr[l]))]++] = l;
  off->assign((size_t)nch + 1, 0);
  for (long long c = 0; c < nch; ++c) {
    const long long l = (*perm)[(size_t)(c * C)];  // the chunk's largest set
    const long long K = l >= 0 ? seg_ptr[l + 1] - seg_ptr[l] : 0;
    (*off)[(size_t)c + 1] = (*off)[(size_t)c] + 32 * ((K + W8 - 1) / W8);
  }
  return nch;
}

cudaError_t launch_slice_items(const Problem& P, const Work& Wk, int W8, cudaStream_t s) {
  if (Wk.sl.nchunks <= 0) return cudaSuccess;
  const long long blocks = (Wk.sl.nchunks + 7) / 8;  // 8 warps per block
  k_slice_items<<<(unsigned)(blocks < 65535 * 16 ? blocks : 65535 * 16), 256, 0, s>>>(P, Wk.v32, Wk.vt32, Wk.sl,
                                                                                        Wk.sl_perm, W8);
  return cudaGetLastError();
}

cudaError_t launch_slice_segments(const Problem& P, const Work& Wk, int W8, cudaStream_t s) {
  if (Wk.sl.nchunks <= 0) return cudaSuccess;
  const long long npos = Wk.sl.nchunks * (32 / W8);
  const long long blocks = (npos + 255) / 256;
  k_slice_segments<<<(unsigned)(blocks < 65535 * 16 ? blocks : 65535 * 16), 256, 0, s>>>(P, Wk.lam32, Wk.vt0_32,
                                                                                           Wk.sl, Wk.sl_perm, npos);
  return cudaGetLastError();
}

cudaError_t launch_rows_items(const Problem& P, const SlView& S, const long long* perm, const float* v32,
                              const float* vt32, cudaStream_t s) {
  if (S.nchunks <= 0) return cudaSuccess;
  const long long blocks = (S.nchunks + 7) / 8;  // 8 warps per block
  k_rows_items<<<(unsigned)(blocks < 65535 * 16 ? blocks : 65535 * 16), 256, 0, s>>>(P, S, perm, v32, vt32);
  return cudaGetLastError();
}

cudaError_t launch_rows_hist(const Problem& P, unsigned long long* hist, cudaStream_t s) {
  if (P.L <= 0) return cudaSuccess;
  const long long blocks = (P.L + 255) / 256;
  k_rows_hist<<<(unsigned)(blocks < 1216 ? blocks : 1216), 256, 0, s>>>(P.seg_ptr, P.L, hist);
  return cudaGetLastError();
}

cudaError_t launch_rows_scatter(const Problem& P, const long long* pos_start, unsigned long long* cursor,
                                long long* perm, cudaStream_t s) {
  if (P.L <= 0) return cudaSuccess;
  const long long blocks = (P.L + 255) / 256;
  k_rows_scatter<<<(unsigned)(blocks < 1216 ? blocks : 1216), 256, 0, s>>>(P.seg_ptr, P.L, pos_start, cursor, perm);
  return cudaGetLastError();
}

cudaError_t launch_rows_segments(const Problem& P, const SlView& S, const long long* perm, const float* lam32,
                                 const float* vt0_32, cudaStream_t s) {
  const long long npos = S.cls_pos[kRowsClasses];
  if (S.nchunks <= 0 || npos <= 0) return cudaSuccess;
  const long long blocks = (npos + 255) / 256;
  k_slice_segments<<<(unsigned)(blocks < 65535 * 16 ? blocks : 65535 * 16), 256, 0, s>>>(P, lam32, vt0_32, S,
                                                                                           perm, npos);
  return cudaGetLastError();
}

}  // namespace spfom
