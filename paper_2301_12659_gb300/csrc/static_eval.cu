// static_eval.cu -- f(x(t)) without a workspace: the entry point
// mdn_evaluate_static() for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc or any allocating
// routine: plug-ins inside a host application whose own pool reserves the
// device memory up front (a cudaMalloc of theirs would fail or fragment that
// pool), or real-time loops that must not allocate after start-up (cudaMalloc
// can block on the device).  For them this file
// keeps the scratch of the evaluation (the running forward products of each
// monomial, two series per equation) in one file-scope device array,
// g_scratch, of MDN_STATIC_SCRATCH_BYTES.  Every GPU that loads the library
// holds that array until the process exits.
//
// The host cannot use the symbol g_scratch as a device address (in host code
// it names a host-side stand-in), so the first call on each device looks the
// address up with cudaGetSymbolAddress, with that device current, and passes
// the pointer to the kernel.  That first call should come before any stream
// capture.  All calls share the array and it keeps the last call's contents:
// two calls whose kernels overlap on the GPU race.  The status word at the
// start of the array is cleared at every call.
#include <mutex>

#include "../../include/mdnewton.h"
#include "kernels.cuh"

namespace mdn {

constexpr size_t STATIC_DOUBLES = MDN_STATIC_SCRATCH_BYTES / sizeof(double);  // 2 MiB
// [0]: status word (as an int in the first double); the rest: per equation two
// series of [K][C][d+1] doubles.
static __device__ __align__(256) double g_scratch[STATIC_DOUBLES];

struct StaticParams {
  int n, D, M, nnz;
  const int* eq;
  const int* vptr;
  const int* vidx;
  const double* coeff;
  const double* cst;
  const double* x;
  double* f;
  double* scratch;  // device address of g_scratch
};

// One warp per equation i: the value c_m(t) prod x_v(t) of each monomial of
// equation i by forward products (ping-pong between two scratch series),
// accumulated into f_i in registers (lane t holds coefficients t and D-1-t).
template <int K, int C>
__global__ void static_eval_kernel(StaticParams p) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= p.n) return;
  const int D = p.D, P = (D + 1) / 2;
  const long long Nx = (long long)p.n * D, Nc = (long long)p.M * D;
  int* status = reinterpret_cast<int*>(p.scratch);
  double* buf = p.scratch + 32 + (size_t)i * 2 * K * C * D;  // two series, N = D each
  const int t = lane < P ? lane : 0;
  const int k1 = t, k2 = D - 1 - t;
  CAcc<K, C> acc1, acc2;
  {
    cmd<K, C> v;
    ld(p.cst, Nx, (long long)i * D + k1, v);
    cacc_set(acc1, v);
    ld(p.cst, Nx, (long long)i * D + k2, v);
    cacc_set(acc2, v);
  }
  // warp 0 checks every equation index (a monomial of no equation 0..n-1
  // would otherwise be skipped silently)
  if (i == 0) {
    for (int m = lane; m < p.M; m += 32)
      if (p.eq[m] < 0 || p.eq[m] >= p.n) atomicOr(status, 1);
  }
  for (int m = 0; m < p.M; ++m) {
    if (p.eq[m] != i) continue;
    const int vp = p.vptr[m], k = p.vptr[m + 1] - vp;
    if (vp < 0 || k < 1 || vp + k > p.nnz) {
      if (lane == 0) atomicOr(status, 1);
      continue;
    }
    SP a{const_cast<double*>(p.coeff), Nc, (long long)m * D};
    int cur = 0;
    for (int q = 0; q < k; ++q) {
      const int v = p.vidx[vp + q];
      if (v < 0 || v >= p.n) {
        if (lane == 0) atomicOr(status, 1);
        break;
      }
      SP b{const_cast<double*>(p.x), Nx, (long long)v * D};
      SP o{buf + (size_t)cur * K * C * D, D, 0};
      if (lane < P) series_product<K, C>(a, b, o, t, D);
      __syncwarp();
      a = o;
      cur ^= 1;
    }
    cmd<K, C> val;
    if (lane < P) {
      ld(a.p, a.N, a.off + k1, val);
      cacc_add(acc1, val);
      ld(a.p, a.N, a.off + k2, val);
      cacc_add(acc2, val);
    }
    __syncwarp();
  }
  cmd<K, C> r1, r2;
  cacc_get(acc1, r1);
  cacc_get(acc2, r2);
  if (lane < P) {
    st(p.f, Nx, (long long)i * D + k1, r1);
    if (k2 != k1) st(p.f, Nx, (long long)i * D + k2, r2);
  }
}

template <int K, int C>
static cudaError_t launch_static(const StaticParams& p, cudaStream_t s) {
  const int warps_per_block = 4;
  static_eval_kernel<K, C><<<(p.n + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(p);
  return cudaGetLastError();
}

// Device address of g_scratch, looked up once per device.
static std::mutex g_mutex;
static double* g_addr[128];

static cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(ptr);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace mdn

using namespace mdn;

extern "C" mdn_status mdn_evaluate_static(int limbs, int is_complex, int n, int degree, int n_monomials,
                                          int n_var_refs, const int32_t* eq_of_monomial, const int32_t* var_ptr,
                                          const int32_t* var_idx, const double* coeff, const double* const_term,
                                          const double* x, double* f_out, void* cuda_stream) {
  const int C = is_complex ? 2 : 1;
  if (!(limbs == 1 || limbs == 2 || limbs == 4 || limbs == 8) || n < 1 || n > MDN_MAX_N || degree < 0 ||
      degree > MDN_MAX_DEGREE || n_monomials < 1 || n_var_refs < 1)
    return MDN_EINVAL;
  if (!eq_of_monomial || !var_ptr || !var_idx || !coeff || !const_term || !x || !f_out) return MDN_EINVAL;
  const size_t need = sizeof(double) * (32 + (size_t)n * 2 * limbs * C * (degree + 1));
  if (need > MDN_STATIC_SCRATCH_BYTES) return MDN_ETOOLARGE;
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return MDN_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  StaticParams p{n, degree + 1, n_monomials, n_var_refs, eq_of_monomial, var_ptr, var_idx, coeff,
                 const_term, x, f_out, scratch};
  if (cudaMemsetAsync(scratch, 0, sizeof(int), st) != cudaSuccess) return MDN_ECUDA;
  cudaError_t e;
  switch (limbs * 10 + C) {
    case 11: e = launch_static<1, 1>(p, st); break;
    case 21: e = launch_static<2, 1>(p, st); break;
    case 22: e = launch_static<2, 2>(p, st); break;
    case 41: e = launch_static<4, 1>(p, st); break;
    case 42: e = launch_static<4, 2>(p, st); break;
    case 81: e = launch_static<8, 1>(p, st); break;
    case 82: e = launch_static<8, 2>(p, st); break;
    default: return MDN_EINVAL;
  }
  if (e != cudaSuccess) return MDN_ECUDA;
  int status = 0;
  if (cudaMemcpyAsync(&status, scratch, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MDN_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MDN_ECUDA;
  return status ? MDN_EINVAL : MDN_OK;
}
