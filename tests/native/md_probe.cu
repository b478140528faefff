// md_probe.cu -- TEST-ONLY device probe: runs the library's multiple double
// primitives (md.cuh) and its integer-limb extended floats (xf.cuh, with the
// inline-PTX carry chains of the device build) elementwise on the GPU, so
// that the GPU tests can check each operation against exact rationals.  Not
// part of the library; built by tests/test_gpu_md.py.
#include <cuda_runtime.h>

#include "md.cuh"
#include "xf.cuh"

using namespace mdn;

// ops on md values (K limbs out):  0 add  1 sub  2 mul  3 fma (a + a*b)
// 4 div  5 recip(a)  6 sqrt(a)  7 rsqrt(a)  8 complex mul (pairs: re, im)
// ops on xf values (2K limbs out, enough for the whole xf mantissa):
// 10 add  11 sub  12 mul  13 recip(a)  14 rsqrt(a)  15 md -> xf -> md
template <int K>
__global__ void probe_kernel(int op, int N, const double* a, const double* b, double* r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double x[K], y[K], z[K];
#pragma unroll
  for (int l = 0; l < K; ++l) {
    x[l] = a[(long long)i * K + l];
    y[l] = b[(long long)i * K + l];
    z[l] = 0.0;
  }
  if (op < 10) {
    switch (op) {
      case 0: md_add(x, y, z); break;
      case 1: md_sub(x, y, z); break;
      case 2: md_mul(x, y, z); break;
      case 3: md_fma(x, x, y, z); break;
      case 4: md_div(x, y, z); break;
      case 5: md_recip(x, z); break;
      case 6: md_sqrt(x, z); break;
      case 7: md_rsqrt(x, z); break;
      default: break;
    }
#pragma unroll
    for (int l = 0; l < K; ++l) r[(long long)i * K + l] = z[l];
    return;
  }
  constexpr int W = xfn::xf_words_t<K>::value;
  xfn::xf<W> u, v, w;
  xfn::xf_from_md<K, W>(x, u);
  xfn::xf_from_md<K, W>(y, v);
  switch (op) {
    case 10: xfn::xf_add(u, v, w); break;
    case 11: xfn::xf_sub(u, v, w); break;
    case 12: xfn::xf_mul(u, v, w); break;
    case 13: xfn::xf_recip(u, w); break;
    case 14: xfn::xf_rsqrt(u, w); break;
    default: w = u; break;
  }
  double o[2 * K];
  xfn::xf_to_md<2 * K, W>(w, o);
#pragma unroll
  for (int l = 0; l < 2 * K; ++l) r[(long long)i * 2 * K + l] = o[l];
}

// complex md product of pairs (a, b) -> r, each value 2K doubles (re, im)
template <int K>
__global__ void probe_cmul_kernel(int N, const double* a, const double* b, double* r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  cmd<K, 2> x, y, z;
#pragma unroll
  for (int l = 0; l < K; ++l) {
    x.re[l] = a[(long long)i * 2 * K + l];
    x.im[l] = a[(long long)i * 2 * K + K + l];
    y.re[l] = b[(long long)i * 2 * K + l];
    y.im[l] = b[(long long)i * 2 * K + K + l];
  }
  cmd_mul(x, y, z);
#pragma unroll
  for (int l = 0; l < K; ++l) {
    r[(long long)i * 2 * K + l] = z.re[l];
    r[(long long)i * 2 * K + K + l] = z.im[l];
  }
}

template <int K>
static cudaError_t run(int op, int N, const double* a, const double* b, double* r) {
  if (op == 8) probe_cmul_kernel<K><<<(N + 127) / 128, 128>>>(N, a, b, r);
  else probe_kernel<K><<<(N + 127) / 128, 128>>>(op, N, a, b, r);
  return cudaGetLastError();
}

// Host entry (test infrastructure, so it may allocate): copies the host
// arrays in, runs op on N values of K limbs and copies out `out_doubles`
// doubles.  Returns 0, or the CUDA error code.
extern "C" int md_probe(int K, int op, int N, int in_doubles, int out_doubles, const double* a, const double* b,
                        double* r) {
  // the kernels read N values of K limbs (2K for complex pairs) and write K
  // limbs (2K for xf results and complex pairs) per value
  const long long need_in = (long long)N * K * (op == 8 ? 2 : 1);
  const long long need_out = (long long)N * K * ((op == 8 || op >= 10) ? 2 : 1);
  if (N < 1 || in_doubles < need_in || out_doubles < need_out) return (int)cudaErrorInvalidValue;
  double *da = nullptr, *db = nullptr, *dr = nullptr;
  cudaError_t e = cudaMalloc(&da, sizeof(double) * in_doubles);
  if (e == cudaSuccess) e = cudaMalloc(&db, sizeof(double) * in_doubles);
  if (e == cudaSuccess) e = cudaMalloc(&dr, sizeof(double) * out_doubles);
  if (e == cudaSuccess) e = cudaMemcpy(da, a, sizeof(double) * in_doubles, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(db, b, sizeof(double) * in_doubles, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(dr, 0, sizeof(double) * out_doubles);
  if (e == cudaSuccess) {
    switch (K) {
      case 1: e = run<1>(op, N, da, db, dr); break;
      case 2: e = run<2>(op, N, da, db, dr); break;
      case 4: e = run<4>(op, N, da, db, dr); break;
      case 8: e = run<8>(op, N, da, db, dr); break;
      default: e = cudaErrorInvalidValue; break;
    }
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(r, dr, sizeof(double) * out_doubles, cudaMemcpyDeviceToHost);
  cudaFree(da);
  cudaFree(db);
  cudaFree(dr);
  return (int)e;
}
