// peak_probe.cu -- throughput microbenchmarks of the pipes the hot path runs
// on, for the roofline denominators: FP64 fused multiply-adds (the md
// algorithms' TwoProd/TwoSum), 32-bit integer multiply-adds (IMAD, the
// products of the integer-limb extended floats), three-input logic (LOP3,
// the carries, shifts and selects) and an even mix of the two integer kinds.
//
// Every thread runs CHAINS independent dependency chains of `iters`
// operations, so each warp always has independent instructions to issue;
// the grid fills every SM (blocks_per_sm blocks of 256 threads).  Block 0
// also reads the SM clock counter and the global nanosecond timer around its
// loop, so the host gets the SM clock of the run.  The result of every chain
// is stored, so nothing is optimised away.  No thread waits on another.
#include <cuda_runtime.h>
#include <stdint.h>

#define CHAINS 8

__global__ void dfma_kernel(double* out, long long* clk, int iters, double seed) {
  double a[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
  const double m = 0.999999999, k = 1e-12;
  long long c0 = 0, t0 = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c0 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) a[c] = __fma_rn(a[c], m, k);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    long long c1 = clock64(), t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    clk[0] = c1 - c0;
    clk[1] = t1 - t0;
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// kind 0: IMAD chains a = a * m + k; 1: LOP3 chains a = lop3(a, b, k, 0x96);
// 2: half of each
__global__ void int_kernel(unsigned* out, long long* clk, int iters, unsigned seed, int kind) {
  unsigned a[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) a[c] = seed + 7u * (threadIdx.x + c);
  const unsigned m = 0x9E3779B1u + seed, k = 0x7F4A7C15u ^ seed, b = 0x85EBCA6Bu + seed;
  long long c0 = 0, t0 = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c0 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  }
  if (kind == 0) {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[c]) : "r"(m), "r"(k));
    }
  } else if (kind == 1) {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c)
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[c]) : "r"(b), "r"(k));
    }
  } else {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < CHAINS; c += 2) {
        asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[c]) : "r"(m), "r"(k));
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[c + 1]) : "r"(b), "r"(k));
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    long long c1 = clock64(), t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    clk[0] = c1 - c0;
    clk[1] = t1 - t0;
  }
  unsigned s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s ^= a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Runs one probe: kind 0 DFMA, 1 IMAD, 2 LOP3, 3 IMAD+LOP3.  Grid:
// num_sms * blocks_per_sm blocks of 256 threads, each thread CHAINS * iters
// operations.  res[0] = elapsed ms (CUDA events), res[1] = SM cycles of
// block 0's loop, res[2] = its nanoseconds, res[3] = thread operations.
// Allocates its own small buffers.  Returns 0 or a CUDA error code.
extern "C" int peak_probe(int kind, int num_sms, int blocks_per_sm, int iters, double* res) {
  const int threads = 256;
  const long long blocks = (long long)num_sms * blocks_per_sm;
  if (kind < 0 || kind > 3 || num_sms < 1 || blocks_per_sm < 1 || iters < 1 || blocks > (1 << 20)) return 1;
  void* out = nullptr;
  long long* clk = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(double) * blocks * threads);
  if (e == cudaSuccess) e = cudaMalloc((void**)&clk, 2 * sizeof(long long));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
    cudaEventRecord(e0);
    if (kind == 0) dfma_kernel<<<(unsigned)blocks, threads>>>((double*)out, clk, iters, 1.0 + rep);
    else int_kernel<<<(unsigned)blocks, threads>>>((unsigned*)out, clk, iters, 12345u + rep, kind - 1);
    cudaEventRecord(e1);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  }
  float ms = 0.f;
  long long c[2] = {0, 0};
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaMemcpy(c, clk, sizeof c, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    res[0] = ms;
    res[1] = (double)c[0];
    res[2] = (double)c[1];
    res[3] = (double)blocks * threads * CHAINS * (double)iters;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  cudaFree(clk);
  return (int)e;
}
