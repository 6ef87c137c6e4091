// GB300 throughput microbenchmark: binary64 / binary32 arithmetic, binary64
// conversions, 64-bit integer work, global and shared-memory atomics, and
// read-only HBM streaming. These rates decide the segment kernels' design
// (see the binary64 budget in spfom_segments_fast.cu). A standalone program:
// build it with paper_2602_22421_gb300.build.build_probe() and run it.
// Every index is bounded; nothing waits on another thread.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

template <int OP>
__global__ void k_fp64(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    if (OP == 0) {  // dfma
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    } else if (OP == 1) {  // dadd
      x0 = x0 + b; x1 = x1 + b; x2 = x2 + b; x3 = x3 + b; x4 = x4 + b; x5 = x5 + b; x6 = x6 + b; x7 = x7 + b;
    } else if (OP == 2) {  // ddiv
      x0 = a / x0; x1 = a / x1; x2 = a / x2; x3 = a / x3; x4 = a / x4; x5 = a / x5; x6 = a / x6; x7 = a / x7;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void k_fp32(float* out, int iters, float a, float b) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3f + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_i64cmp(long long* out, int iters, long long a) {
  long long x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 977 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) { long long y = x[k] ^ a; x[k] = (y > x[k]) ? y : x[k] + 1; }
  }
  long long s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16; return x;
}

__global__ void k_atomic_f64(double* dst, int nslots, long long total) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += stride) {
    uint32_t s = hash32((uint32_t)i) % (uint32_t)nslots;
    atomicAdd(dst + s, 0.5);
  }
}
__global__ void k_atomic_f32(float* dst, int nslots, long long total) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += stride) {
    uint32_t s = hash32((uint32_t)i) % (uint32_t)nslots;
    atomicAdd(dst + s, 0.5f);
  }
}
__global__ void k_atomic_u64(unsigned long long* dst, int nslots, long long total) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += stride) {
    uint32_t s = hash32((uint32_t)i) % (uint32_t)nslots;
    atomicAdd(dst + s, 12345ULL);
  }
}
// shared-memory FP64 / FP32 atomics, nslots <= 8192 doubles
__global__ void k_satomic_f64(double* dst, int nslots, int per_thread) {
  extern __shared__ double sm[];
  for (int i = threadIdx.x; i < nslots; i += blockDim.x) sm[i] = 0;
  __syncthreads();
  uint32_t base = blockIdx.x * blockDim.x + threadIdx.x;
  for (int k = 0; k < per_thread; ++k) {
    uint32_t s = hash32(base * 131u + k) % (uint32_t)nslots;
    atomicAdd(sm + s, 0.5);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nslots; i += blockDim.x) atomicAdd(dst + i, sm[i]);
}
__global__ void k_satomic_f32(float* dst, int nslots, int per_thread) {
  extern __shared__ float smf[];
  for (int i = threadIdx.x; i < nslots; i += blockDim.x) smf[i] = 0;
  __syncthreads();
  uint32_t base = blockIdx.x * blockDim.x + threadIdx.x;
  for (int k = 0; k < per_thread; ++k) {
    uint32_t s = hash32(base * 131u + k) % (uint32_t)nslots;
    atomicAdd(smf + s, 0.5f);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nslots; i += blockDim.x) atomicAdd(dst + i, smf[i]);
}

__global__ void k_stream_read(const int4* __restrict__ src, long long n16, unsigned long long* sink) {
  long long stride = (long long)gridDim.x * blockDim.x;
  int acc = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n16; i += stride) {
    int4 v = __ldcs(src + i);
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (acc == 0x7fffffff) atomicAdd(sink, 1ULL);
}

// f64 -> f32 -> f64 round trips that cannot be folded: the f64 value changes each step.
__global__ void k_cvt_d2f(double* out, int iters, double a) {
  double x[8]; float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k + 0.1234567890123;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) { float f = __double2float_rn(x[k]); acc += f; x[k] = __longlong_as_double(__double_as_longlong(x[k]) + 1); }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc + x[0];
}
__global__ void k_cvt_f2d(double* out, int iters) {
  float f[8]; long long acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) f[k] = threadIdx.x * 1e-3f + k + 0.123f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) { double d = (double)f[k]; acc += __double_as_longlong(d); f[k] = __int_as_float(__float_as_int(f[k]) + 1); }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = (double)acc;
}
__global__ void k_cvt_d2ll(double* out, int iters) {
  double x[8]; long long acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e3 + k + 0.5;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) { acc += __double2ll_rn(x[k]); x[k] = __longlong_as_double(__double_as_longlong(x[k]) + 1); }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = (double)acc;
}
__global__ void k_cvt_ll2d(double* out, int iters) {
  long long v[8]; long long acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = threadIdx.x * 977LL + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) { acc += __double_as_longlong(__ll2double_rn(v[k])); v[k] += 3; }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = (double)acc;
}
__global__ void k_frcp(float* out, int iters) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3f + k + 1.f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = __frcp_rn(x[k]) + 1.0f;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[7];
}
__global__ void k_fdiv(float* out, int iters, float a) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3f + k + 1.f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = a / x[k] + 1.0f;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[7];
}
__global__ void k_mul64(unsigned long long* out, int iters) {
  unsigned long long x[8], acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 0x9E3779B97F4A7C15ULL + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) { acc += __umul64hi(x[k], 0xBF58476D1CE4E5B9ULL); x[k] += acc; }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}
__global__ void k_satomic_u64(unsigned long long* dst, int nslots, int per_thread) {
  extern __shared__ unsigned long long su[];
  for (int i = threadIdx.x; i < nslots; i += blockDim.x) su[i] = 0;
  __syncthreads();
  uint32_t base = blockIdx.x * blockDim.x + threadIdx.x;
  for (int k = 0; k < per_thread; ++k) {
    uint32_t s = hash32(base * 131u + k) % (uint32_t)nslots;
    atomicAdd(su + s, 12345ULL);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nslots; i += blockDim.x) atomicAdd(dst + i, su[i]);
}
__global__ void k_satomic_u32(unsigned* dst, int nslots, int per_thread) {
  extern __shared__ unsigned s32[];
  for (int i = threadIdx.x; i < nslots; i += blockDim.x) s32[i] = 0;
  __syncthreads();
  uint32_t base = blockIdx.x * blockDim.x + threadIdx.x;
  for (int k = 0; k < per_thread; ++k) {
    uint32_t s = hash32(base * 131u + k) % (uint32_t)nslots;
    atomicAdd(s32 + s, 123u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nslots; i += blockDim.x) atomicAdd(dst + i, s32[i]);
}
// plain hashing loop without atomics, to subtract the overhead
__global__ void k_hash_only(unsigned* dst, int nslots, int per_thread) {
  uint32_t base = blockIdx.x * blockDim.x + threadIdx.x, acc = 0;
  for (int k = 0; k < per_thread; ++k) acc += hash32(base * 131u + k) % (uint32_t)nslots;
  dst[base % 1024] = acc;
}

int main() {
  int dev = 0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, dev));
  printf("device %s sms %d cc %d.%d smem/block optin %zu l2 %d\n", p.name, p.multiProcessorCount, p.major, p.minor,
         p.sharedMemPerBlockOptin, p.l2CacheSize);
  int sms = p.multiProcessorCount;
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  const int TPB = 256, BPS = 8; int grid = sms * BPS; long long threads = (long long)grid * TPB;
  double* dout; CK(cudaMalloc(&dout, threads * 8));
  float* fout; CK(cudaMalloc(&fout, threads * 4));
  long long* iout; CK(cudaMalloc(&iout, threads * 8));
  // warm
  k_fp64<0><<<grid, TPB>>>(dout, 100, 0.999, 1e-3); CK(cudaDeviceSynchronize());
  {
    int it = 2000;
    cudaEventRecord(e0); k_fp64<0><<<grid, TPB>>>(dout, it, 0.999, 1e-3); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    double ops = (double)threads * it * 8;
    printf("DFMA: %.3f ms  %.3e instr/s  = %.3f TFLOP/s (fma=2)\n", ms, ops / (ms * 1e-3), 2 * ops / (ms * 1e-3) / 1e12);
    cudaEventRecord(e0); k_fp64<1><<<grid, TPB>>>(dout, it, 0.999, 1e-3); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    printf("DADD: %.3f ms  %.3e instr/s\n", ms, ops / (ms * 1e-3));
    int itd = 200; double opsd = (double)threads * itd * 8;
    cudaEventRecord(e0); k_fp64<2><<<grid, TPB>>>(dout, itd, 0.999, 1e-3); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    printf("DDIV: %.3f ms  %.3e div/s\n", ms, opsd / (ms * 1e-3));
  }
  {
    int it = 20000;
    k_fp32<<<grid, TPB>>>(fout, 100, 0.999f, 1e-3f); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_fp32<<<grid, TPB>>>(fout, it, 0.999f, 1e-3f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    double ops = (double)threads * it * 8;
    printf("FFMA: %.3f ms  %.3e instr/s = %.2f TFLOP/s\n", ms, ops / (ms * 1e-3), 2 * ops / (ms * 1e-3) / 1e12);
  }
  {
    int it = 5000;
    cudaEventRecord(e0); k_i64cmp<<<grid, TPB>>>(iout, it, 0x1234567LL); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    double ops = (double)threads * it * 8;
    printf("I64 xor+cmp+sel: %.3f ms  %.3e iters/s\n", ms, ops / (ms * 1e-3));
  }
  // atomics
  {
    long long total = 10000000LL;
    int slots[4] = {2000, 10000, 100000, 20000};
    double* ad; CK(cudaMalloc(&ad, 100000 * 8)); CK(cudaMemset(ad, 0, 100000 * 8));
    float* af; CK(cudaMalloc(&af, 100000 * 4)); CK(cudaMemset(af, 0, 100000 * 4));
    unsigned long long* au; CK(cudaMalloc(&au, 100000 * 8)); CK(cudaMemset(au, 0, 100000 * 8));
    for (int si = 0; si < 4; ++si) {
      int ns = slots[si];
      k_atomic_f64<<<grid, TPB>>>(ad, ns, total); CK(cudaDeviceSynchronize());
      cudaEventRecord(e0); k_atomic_f64<<<grid, TPB>>>(ad, ns, total); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
      cudaEventElapsedTime(&ms, e0, e1);
      printf("atomicAdd f64 global: %lld into %d slots: %.3f ms  %.3e atom/s\n", total, ns, ms, total / (ms * 1e-3));
      cudaEventRecord(e0); k_atomic_f32<<<grid, TPB>>>(af, ns, total); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
      cudaEventElapsedTime(&ms, e0, e1);
      printf("atomicAdd f32 global: %lld into %d slots: %.3f ms  %.3e atom/s\n", total, ns, ms, total / (ms * 1e-3));
      cudaEventRecord(e0); k_atomic_u64<<<grid, TPB>>>(au, ns, total); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
      cudaEventElapsedTime(&ms, e0, e1);
      printf("atomicAdd u64 global: %lld into %d slots: %.3f ms  %.3e atom/s\n", total, ns, ms, total / (ms * 1e-3));
    }
    int nsl = 8192, per = 64;  // 64 KB of doubles
    CK(cudaFuncSetAttribute(k_satomic_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, nsl * 8));
    k_satomic_f64<<<grid, TPB, nsl * 8>>>(ad, nsl, per); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_satomic_f64<<<grid, TPB, nsl * 8>>>(ad, nsl, per); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    printf("atomicAdd f64 shared: %lld atoms (%d slots/block): %.3f ms  %.3e atom/s\n", threads * per, nsl, ms, threads * per / (ms * 1e-3));
    k_satomic_f32<<<grid, TPB, nsl * 4>>>(af, nsl, per); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_satomic_f32<<<grid, TPB, nsl * 4>>>(af, nsl, per); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    printf("atomicAdd f32 shared: %lld atoms (%d slots/block): %.3f ms  %.3e atom/s\n", threads * per, nsl, ms, threads * per / (ms * 1e-3));
    cudaFree(ad); cudaFree(af); cudaFree(au);
  }
  // streaming read bandwidth, 4 GiB buffer
  {
    long long bytes = 4LL << 30; long long n16 = bytes / 16;
    int4* buf; CK(cudaMalloc(&buf, bytes)); CK(cudaMemset(buf, 1, bytes));
    unsigned long long* sink; CK(cudaMalloc(&sink, 8));
    for (int bps = 4; bps <= 16; bps *= 2) {
      int g = sms * bps;
      k_stream_read<<<g, 512>>>(buf, n16, sink); CK(cudaDeviceSynchronize());
      float best = 1e30f;
      for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0); k_stream_read<<<g, 512>>>(buf, n16, sink); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
        cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms;
      }
      printf("stream read int4 4GiB grid %d x 512: %.3f ms  %.1f GB/s\n", g, best, bytes / (best * 1e-3) / 1e9);
    }
    cudaFree(buf); cudaFree(sink);
  }
  {
    unsigned long long* uout; CK(cudaMalloc(&uout, threads * 8));
#define TIME(name, ops, launch) do { launch; CK(cudaDeviceSynchronize()); cudaEventRecord(e0); launch; cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms, e0, e1); printf("%-28s %8.3f ms  %.3e ops/s\n", name, ms, (double)(ops) / (ms * 1e-3)); } while (0)
    int it = 2000;
    TIME("cvt f64->f32 (+int inc)", threads * it * 8, (k_cvt_d2f<<<grid, TPB>>>(dout, it, 1.0)));
    TIME("cvt f32->f64 (+int inc)", threads * it * 8, (k_cvt_f2d<<<grid, TPB>>>(dout, it)));
    TIME("cvt f64->s64", threads * it * 8, (k_cvt_d2ll<<<grid, TPB>>>(dout, it)));
    TIME("cvt s64->f64", threads * it * 8, (k_cvt_ll2d<<<grid, TPB>>>(dout, it)));
    int itf = 20000;
    TIME("frcp_rn + fadd", threads * itf * 8, (k_frcp<<<grid, TPB>>>(fout, itf)));
    TIME("fdiv (ieee) + fadd", threads * it * 8, (k_fdiv<<<grid, TPB>>>(fout, it, 3.f)));
    TIME("umul64hi + add", threads * it * 8, (k_mul64<<<grid, TPB>>>(uout, it)));
    {
      unsigned long long* au; CK(cudaMalloc(&au, 16384 * 8)); CK(cudaMemset(au, 0, 16384 * 8));
      unsigned* a32; CK(cudaMalloc(&a32, 16384 * 4)); CK(cudaMemset(a32, 0, 16384 * 4));
      for (int nsl : {2048, 8192}) {
        int per = 64;
        CK(cudaFuncSetAttribute(k_satomic_u64, cudaFuncAttributeMaxDynamicSharedMemorySize, nsl * 8));
        char nm[64];
        snprintf(nm, 64, "smem atom u64 %d slots", nsl);
        TIME(nm, threads * per, (k_satomic_u64<<<grid, TPB, nsl * 8>>>(au, nsl, per)));
        snprintf(nm, 64, "smem atom u32 %d slots", nsl);
        TIME(nm, threads * per, (k_satomic_u32<<<grid, TPB, nsl * 4>>>(a32, nsl, per)));
        snprintf(nm, 64, "hash only %d", nsl);
        TIME(nm, threads * per, (k_hash_only<<<grid, TPB>>>(a32, nsl, per)));
      }
      cudaFree(au); cudaFree(a32);
    }
  
  }
  CK(cudaGetLastError());
  printf("done\n");
  return 0;
}
