// kernels.cuh -- CUDA kernels of one Newton step on truncated power series in
// multiple double arithmetic (Verschelde, arXiv 2301.12659), templated on the
// number of limbs K and on C = 1 (real) / 2 (complex).
//
// Layout (Section 1.2: one array per limb): an array of N md values is
// stored [K][C][N]; element (l, c, i) at p[(l*C + c)*N + i].  Series of
// length D = d+1 are contiguous in the last index.
//
// Kernels (the paper's Table 3 kernel types in brackets):
//   ed_kernel      evaluation and differentiation of all monomials by
//                  forward, backward and cross products [convolutions];
//   assemble_*     f(x(t)) and the Jacobian series A_j [convolutions];
//   qr_kernel      Householder QR of A0, Q^H I and back substitution, giving
//                  W = A0^{-1} [qr, qhb, bs];
//   fs_kernel      r_k = b_k - sum_{j>=1} A_j dx_{k-j} and the residual
//                  r_{k-1} - A0 dx_{k-1} [updates, residuals];
//   fx_kernel      dx_k = W r_k [bs];
//   update kernels x += dx and the norms of the step.
#pragma once
#include <cstdint>
#include "md.cuh"
#include "params.h"

namespace mdn {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// SoA access
// ---------------------------------------------------------------------------
template <int K, int C>
__device__ __forceinline__ void ld(const double* p, long long N, long long i, cmd<K, C>& v) {
#pragma unroll
  for (int l = 0; l < K; ++l) {
    v.re[l] = p[(long long)(l * C) * N + i];
    if constexpr (C == 2) v.im[l] = p[(long long)(l * C + 1) * N + i];
    else v.im[l] = 0.0;
  }
}
template <int K, int C>
__device__ __forceinline__ void st(double* p, long long N, long long i, const cmd<K, C>& v) {
#pragma unroll
  for (int l = 0; l < K; ++l) {
    p[(long long)(l * C) * N + i] = v.re[l];
    if constexpr (C == 2) p[(long long)(l * C + 1) * N + i] = v.im[l];
  }
}
template <int K>
__device__ __forceinline__ void ld_real(const double* p, long long N, long long i, double (&v)[K]) {
#pragma unroll
  for (int l = 0; l < K; ++l) v[l] = p[(long long)l * N + i];
}
template <int K>
__device__ __forceinline__ void st_real(double* p, long long N, long long i, const double (&v)[K]) {
#pragma unroll
  for (int l = 0; l < K; ++l) p[(long long)l * N + i] = v[l];
}

template <int K, int C>
__device__ __forceinline__ void cmd_shfl_xor(const cmd<K, C>& v, cmd<K, C>& o, int off) {
#pragma unroll
  for (int l = 0; l < K; ++l) {
    o.re[l] = __shfl_xor_sync(FULL, v.re[l], off);
    if constexpr (C == 2) o.im[l] = __shfl_xor_sync(FULL, v.im[l], off);
    else o.im[l] = 0.0;
  }
}
template <int K, int C>
__device__ __forceinline__ void cmd_bcast(cmd<K, C>& v, int src) {
#pragma unroll
  for (int l = 0; l < K; ++l) {
    v.re[l] = __shfl_sync(FULL, v.re[l], src);
    if constexpr (C == 2) v.im[l] = __shfl_sync(FULL, v.im[l], src);
  }
}
// Sum over the warp; every lane gets lane 0's total (a single rounding order).
template <int K, int C>
__device__ __forceinline__ void warp_sum(cmd<K, C>& v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    cmd<K, C> o;
    cmd_shfl_xor(v, o, off);
    cmd_add(v, o, v);
  }
  cmd_bcast(v, 0);
}

template <int K, int C>
__device__ __forceinline__ void cacc_select(bool c, const CAcc<K, C>& x, const CAcc<K, C>& y, CAcc<K, C>& r) {
#pragma unroll
  for (int l = 0; l < K; ++l) {
    r.re.l[l] = c ? x.re.l[l] : y.re.l[l];
    if constexpr (C == 2) r.im.l[l] = c ? x.im.l[l] : y.im.l[l];
  }
}

// ---------------------------------------------------------------------------
// memory-model helpers for the dataflow kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Warp-wide bounded wait until *flag == ep: gives up after limit_ns
// nanoseconds of wall time, records MDN_DEV_TIMEOUT in *status and returns
// false, so the kernel always terminates.
__device__ __forceinline__ bool warp_wait(const unsigned* flag, unsigned ep, long long limit_ns, int* status) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) {
    if (ld_acquire(flag) != ep) {
      const unsigned long long t0 = global_ns();
      while (ld_acquire(flag) != ep) {
        if ((long long)(global_ns() - t0) > limit_ns) {
          ok = 0;
          atomicOr(status, MDN_DEV_TIMEOUT);
          break;
        }
        __nanosleep(100);
      }
    }
  }
  ok = __shfl_sync(FULL, ok, 0);
  __syncwarp();
  return ok != 0;
}
__device__ __forceinline__ void warp_publish(unsigned* flag, unsigned ep) {
  __threadfence();
  __syncwarp();
  if ((threadIdx.x & 31) == 0) st_release(flag, ep);
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Evaluation and differentiation (Section 5.1)
// ---------------------------------------------------------------------------
struct SP {
  double* p;
  long long N;
  long long off;
};

__device__ __forceinline__ SP resolve(const EdParams& p, int code, int m, int wg) {
  const int kind = code >> 16, idx = code & 0xffff;
  SP s;
  switch (kind) {
    case SLOT_C:
      s.p = const_cast<double*>(p.coeff); s.N = p.Nc; s.off = (long long)m * p.D; break;
    case SLOT_X:
      s.p = const_cast<double*>(p.x); s.N = p.Nx;
      s.off = (long long)p.vidx[p.mono_vp[m] + idx] * p.D; break;
    case SLOT_F:
      s.p = p.scratch; s.N = p.Ns; s.off = ((long long)wg * p.Smax + (idx - 1)) * p.D; break;
    case SLOT_B:
      s.p = p.scratch; s.N = p.Ns; s.off = ((long long)wg * p.Smax + (p.kmax - 2) + (idx - 2)) * p.D; break;
    case SLOT_V:
      s.p = p.out; s.N = p.No; s.off = (long long)p.mono_sbase[m] * p.D; break;
    default:  // SLOT_P
      s.p = p.out; s.N = p.No; s.off = ((long long)p.mono_sbase[m] + 1 + idx) * p.D; break;
  }
  return s;
}

// o = a * b mod t^D computed by one group of lanes; lane t forms the
// coefficients t and D-1-t (t+1 and D-t terms: D+1 multiply-adds for every
// lane), in one loop of D-1 iterations with the accumulator picked by select.
template <int K, int C>
__device__ __forceinline__ void series_product(const SP& a, const SP& b, const SP& o, int t, int D) {
  const int k1 = t, k2 = D - 1 - t;
  cmd<K, C> av, bv;
  CAcc<K, C> acc1, acc2;
  ld(a.p, a.N, a.off, av);
  ld(b.p, b.N, b.off + k1, bv);
  cacc_mul(acc1, av, bv);
  ld(b.p, b.N, b.off + k2, bv);
  cacc_mul(acc2, av, bv);
  for (int s = 1; s < D; ++s) {
    const bool first = s <= k1;
    const int i = first ? s : s - k1;
    const int j = first ? k1 - s : k2 - i;
    ld(a.p, a.N, a.off + i, av);
    ld(b.p, b.N, b.off + j, bv);
    CAcc<K, C> acc;
    cacc_select(first, acc1, acc2, acc);
    cacc_fma(acc, av, bv);
    cacc_select(first, acc, acc1, acc1);
    cacc_select(first, acc2, acc, acc2);
  }
  cmd<K, C> r1, r2;
  cacc_get(acc1, r1);
  cacc_get(acc2, r2);
  st(o.p, o.N, o.off + k1, r1);
  if (k2 != k1) st(o.p, o.N, o.off + k2, r2);
}

template <int K, int C>
__global__ void __launch_bounds__(ED_THREADS) ed_kernel(EdParams p) {
  const int lane = threadIdx.x & 31;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int g = lane / p.P, t = lane - g * p.P;
  const bool ingroup = g < p.G;
  if (wg >= p.Wtot) return;  // whole warp: the scratch holds Wtot warps
  for (;;) {
    int q = 0;
    if (lane == 0) q = atomicAdd(p.counter, 1);
    q = __shfl_sync(FULL, q, 0);
    if (q >= p.M) break;
    const int m = p.order[q];
    const int k = p.mono_k[m];
    const int4* sc = p.sched + p.sched_off[k];
    const int nw = p.sched_nw[k];
    for (int w = 0; w < nw; ++w) {
      const int4 op = ingroup ? sc[w * p.G + g] : make_int4(0, 0, 0, 0);
      if (op.x == OP_PRODUCT) {
        series_product<K, C>(resolve(p, op.z, m, wg), resolve(p, op.w, m, wg), resolve(p, op.y, m, wg), t, p.D);
      } else if (op.x == OP_COPY) {
        const SP s = resolve(p, op.z, m, wg), d = resolve(p, op.y, m, wg);
        cmd<K, C> v;
        ld(s.p, s.N, s.off + t, v);
        st(d.p, d.N, d.off + t, v);
        ld(s.p, s.N, s.off + (p.D - 1 - t), v);
        st(d.p, d.N, d.off + (p.D - 1 - t), v);
      }
      __syncwarp();
    }
  }
}

// f_i[k] = cst_i[k] + sum of the values of the monomials of equation i.
template <int K, int C>
__global__ void assemble_f_kernel(AsmParams p) {
  const long long total = (long long)p.n * p.D;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id / p.D), kk = (int)(id - (long long)i * p.D);
    cmd<K, C> v, s;
    CAcc<K, C> acc;
    ld(p.cst, p.Nf, id, v);
    cacc_set(acc, v);
    for (int q = p.eq_ptr[i]; q < p.eq_ptr[i + 1]; ++q) {
      const int m = p.eq_mon[q];
      ld(p.out, p.No, (long long)p.mono_sbase[m] * p.D + kk, s);
      cacc_add(acc, s);
    }
    cacc_get(acc, v);
    st(p.f, p.Nf, id, v);
  }
}

// A_j[i][v] = sum over the occurrences of x_v in equation i of coefficient j
// of the partial derivative (repeated variables add up); zero elsewhere.
template <int K, int C>
__global__ void assemble_A_kernel(AsmParams p) {
  const long long nn = (long long)p.n * p.n;
  const long long total = nn * p.D;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(id / nn);
    const long long pair = id - (long long)j * nn;
    cmd<K, C> v;
    cmd_zero(v);
    const int q0 = p.pair_ptr[pair], q1 = p.pair_ptr[pair + 1];
    if (q1 > q0) {
      CAcc<K, C> acc;
      ld(p.out, p.No, (long long)p.pair_slot[q0] * p.D + j, v);
      cacc_set(acc, v);
      for (int q = q0 + 1; q < q1; ++q) {
        ld(p.out, p.No, (long long)p.pair_slot[q] * p.D + j, v);
        cacc_add(acc, v);
      }
      cacc_get(acc, v);
    }
    st(p.A, p.NA, id, v);
  }
}

// ---------------------------------------------------------------------------
// Householder QR of A0 and W = A0^{-1} = R^{-1} Q^H (Section 5.3)
// ---------------------------------------------------------------------------
// Cooperative launch: CTAs [0, nA) hold one warp per column of A0, CTAs
// [nA, 2 nA) one warp per column of the identity.  The owner of column j
// publishes reflector j (v_j, tau_j = 2 / v_j^H v_j) with a release flag;
// the other columns apply H_j = I - tau_j v_j v_j^H as soon as it appears.
// v_j = x + s |x| e_1 with s = x_0 / |x_0| (+1 for x_0 = 0), so that
// H_j x = -s |x| e_1.  tau_j = 1 / (|x| (|x| + |x_0|)).

template <int K, int C>
__device__ void qr_apply(const QrParams& p, int j, double* y, long long Ny, long long col) {
  // y[:, col] -= tau_j (v_j^H y) v_j over rows j..n-1
  const int lane = threadIdx.x & 31;
  const int n = p.n;
  CAcc<K, C> acc;
  cacc_zero(acc);
  for (int i = j + lane; i < n; i += 32) {
    cmd<K, C> v, yv;
    ld(p.Vm, p.Nnn, (long long)i * n + j, v);
    ld(y, Ny, (long long)i * n + col, yv);
    cacc_fma_conj(acc, v, yv);
  }
  cmd<K, C> w, g;
  cacc_get(acc, w);
  warp_sum(w);
  double tau[K];
  ld_real(p.tau, p.n, j, tau);
  cmd_scale(w, tau, g);
  cmd<K, C> ng;
  md_neg(g.re, ng.re);
  md_neg(g.im, ng.im);
  for (int i = j + lane; i < n; i += 32) {
    cmd<K, C> v, yv;
    ld(p.Vm, p.Nnn, (long long)i * n + j, v);
    ld(y, Ny, (long long)i * n + col, yv);
    CAcc<K, C> a2;
    cacc_set(a2, yv);
    cacc_fma(a2, ng, v);
    cacc_get(a2, yv);
    st(y, Ny, (long long)i * n + col, yv);
  }
  __syncwarp();
}

template <int K, int C>
__device__ void qr_reflector(const QrParams& p, int j, unsigned ep) {
  const int lane = threadIdx.x & 31;
  const int n = p.n;
  // |x|^2 over rows j..n-1 of column j
  Acc<K> a2;
  acc_zero(a2);
  for (int i = j + lane; i < n; i += 32) {
    cmd<K, C> x;
    ld(p.Rm, p.Nnn, (long long)i * n + j, x);
    acc_fma(a2, x.re, x.re);
    if constexpr (C == 2) acc_fma(a2, x.im, x.im);
  }
  cmd<K, C> nrm;
  acc_get(a2, nrm.re);
  md_zero(nrm.im);
  warp_sum(nrm);
  double alpha[K];
  md_sqrt(nrm.re, alpha);
  cmd<K, C> x0;
  ld(p.Rm, p.Nnn, (long long)j * n + j, x0);
  double ax0[K];
  cmd<K, C> sg;
  cmd_zero(sg);
  if constexpr (C == 1) {
    const bool neg = __double_as_longlong(x0.re[0]) < 0;
    sg.re[0] = neg ? -1.0 : 1.0;
    for (int l = 0; l < K; ++l) ax0[l] = neg ? -x0.re[l] : x0.re[l];
  } else {
    double a2x[K];
    cmd_abs2(x0, a2x);
    md_sqrt(a2x, ax0);
    if (nonzero(ax0[0])) {
      md_div(x0.re, ax0, sg.re);
      md_div(x0.im, ax0, sg.im);
    } else {
      sg.re[0] = 1.0;
    }
  }
  cmd<K, C> salpha, v0;
  cmd_scale(sg, alpha, salpha);
  cmd_add(x0, salpha, v0);
  // tau = 1 / (alpha (alpha + |x0|))
  double t1[K], t2[K], tau[K], one[K];
  md_add(alpha, ax0, t1);
  md_mul(alpha, t1, t2);
  md_zero(one);
  one[0] = 1.0;
  const bool singular = !nonzero(alpha[0]);
  if (singular) {
    md_zero(tau);
    if (lane == 0) atomicOr(p.status, MDN_DEV_SINGULAR);
  } else {
    md_div(one, t2, tau);
  }
  // reflector, R_jj = -s alpha, zeros below the diagonal
  for (int i = j + lane; i < n; i += 32) {
    cmd<K, C> x;
    if (i == j) {
      st(p.Vm, p.Nnn, (long long)i * n + j, v0);
      cmd<K, C> r;
      md_neg(salpha.re, r.re);
      md_neg(salpha.im, r.im);
      st(p.Rm, p.Nnn, (long long)i * n + j, r);
    } else {
      ld(p.Rm, p.Nnn, (long long)i * n + j, x);
      st(p.Vm, p.Nnn, (long long)i * n + j, x);
      cmd_zero(x);
      st(p.Rm, p.Nnn, (long long)i * n + j, x);
    }
  }
  if (lane == 0) st_real(p.tau, p.n, j, tau);
  warp_publish(&p.flags[j], ep);
  // 1 / R_jj for the back substitution, published separately
  cmd<K, C> r, cone, rinv;
  md_neg(salpha.re, r.re);
  md_neg(salpha.im, r.im);
  cmd_zero(cone);
  cone.re[0] = 1.0;
  if (singular) cmd_zero(rinv);
  else cmd_div(cone, r, rinv);
  if (lane == 0) st(p.rinv, p.n, j, rinv);
  warp_publish(&p.flags[p.n + j], ep);
}

template <int K, int C>
__global__ void __launch_bounds__(QR_THREADS) qr_kernel(QrParams p) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = p.n;
  const unsigned ep = *p.epoch;
  const bool colwarp = blockIdx.x < p.nA;
  const int c = (colwarp ? blockIdx.x : blockIdx.x - p.nA) * (QR_THREADS / 32) + warp;
  if (c >= n) return;
  if (colwarp) {
    // my column of A0 -> Rm
    for (int i = lane; i < n; i += 32) {
      cmd<K, C> v;
      ld(p.A0, p.NA, (long long)i * n + c, v);
      st(p.Rm, p.Nnn, (long long)i * n + c, v);
    }
    __syncwarp();
    for (int j = 0; j < c; ++j) {
      if (!warp_wait(&p.flags[j], ep, p.spin_limit, p.status)) return;
      qr_apply<K, C>(p, j, p.Rm, p.Nnn, c);
    }
    qr_reflector<K, C>(p, c, ep);
  } else {
    // column c of the identity -> Q^H e_c -> R^{-1} Q^H e_c
    for (int i = lane; i < n; i += 32) {
      cmd<K, C> v;
      cmd_zero(v);
      if (i == c) v.re[0] = 1.0;
      st(p.Y, p.Nnn, (long long)i * n + c, v);
    }
    __syncwarp();
    for (int j = 0; j < n; ++j) {
      if (!warp_wait(&p.flags[j], ep, p.spin_limit, p.status)) return;
      qr_apply<K, C>(p, j, p.Y, p.Nnn, c);
    }
    // column-oriented back substitution: x_i = y_i / R_ii, y_k -= R_ki x_i
    for (int i = n - 1; i >= 0; --i) {
      if (!warp_wait(&p.flags[n + i], ep, p.spin_limit, p.status)) return;
      cmd<K, C> yi, ri, xi;
      ld(p.Y, p.Nnn, (long long)i * n + c, yi);
      ld(p.rinv, p.n, i, ri);
      cmd_mul(yi, ri, xi);
      if (lane == 0) st(p.W, p.Nnn, (long long)i * n + c, xi);
      cmd<K, C> nx;
      md_neg(xi.re, nx.re);
      md_neg(xi.im, nx.im);
      for (int k = lane; k < i; k += 32) {
        cmd<K, C> rk, yk;
        ld(p.Rm, p.Nnn, (long long)k * n + i, rk);
        ld(p.Y, p.Nnn, (long long)k * n + c, yk);
        CAcc<K, C> a;
        cacc_set(a, yk);
        cacc_fma(a, nx, rk);
        cacc_get(a, yk);
        st(p.Y, p.Nnn, (long long)k * n + c, yk);
      }
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------
// Forward substitution on the block lower triangular Toeplitz system,
// Eq. (eqToeplitz):  A_0 dx_k = b_k - sum_{j=1..k} A_j dx_{k-j}.
// ---------------------------------------------------------------------------
template <int K, int C>
__device__ __forceinline__ void block_sum(cmd<K, C>& v, cmd<K, C>* sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  warp_sum(v);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    if (lane < nw) v = sh[lane];
    else cmd_zero(v);
    warp_sum(v);
  }
  __syncthreads();
  if (threadIdx.x == 0) sh[0] = v;
  __syncthreads();
  v = sh[0];
  __syncthreads();
}

// Row i of stage k: r_k[i] = sgn * rhs_k[i] - sum_{j=1..k} (A_j dx_{k-j})[i].
// Also the residual of stage k-1: res[i][k-1] = r_{k-1}[i] - (A_0 dx_{k-1})[i].
template <int K, int C>
__global__ void __launch_bounds__(FS_THREADS) fs_kernel(FsParams p, int k) {
  __shared__ cmd<K, C> sh[FS_THREADS / 32];
  const int i = blockIdx.x, n = p.n, D = p.D;
  const long long nn = (long long)n * n;
  CAcc<K, C> acc;
  cacc_zero(acc);
  const int terms = (k < D) ? k * n : 0;
  for (int t = threadIdx.x; t < terms; t += blockDim.x) {
    const int j = 1 + t / n, l = t - (j - 1) * n;
    cmd<K, C> a, x;
    ld(p.A, p.NA, (long long)j * nn + (long long)i * n + l, a);
    ld(p.dx, p.Nx, (long long)l * D + (k - j), x);
    cacc_fma(acc, a, x);
  }
  cmd<K, C> s;
  cacc_get(acc, s);
  block_sum(s, sh);
  if (k < D && threadIdx.x == 0) {
    cmd<K, C> b, r;
    ld(p.rhs, p.Nx, (long long)i * D + k, b);
    if (p.rhs_sign < 0) {
      md_neg(b.re, b.re);
      md_neg(b.im, b.im);
    }
    cmd_sub(b, s, r);
    st(p.r, p.Nx, (long long)i * D + k, r);
  }
  if (k >= 1) {  // residual of stage k-1
    CAcc<K, C> a2;
    cacc_zero(a2);
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
      cmd<K, C> a, x;
      ld(p.A, p.NA, (long long)i * n + l, a);
      ld(p.dx, p.Nx, (long long)l * D + (k - 1), x);
      cacc_fma(a2, a, x);
    }
    cmd<K, C> s2;
    cacc_get(a2, s2);
    block_sum(s2, sh);
    if (threadIdx.x == 0) {
      cmd<K, C> r, res;
      ld(p.r, p.Nx, (long long)i * D + (k - 1), r);
      cmd_sub(r, s2, res);
      p.resabs[(long long)i * D + (k - 1)] = (C == 2) ? hypot(res.re[0], res.im[0]) : fabs(res.re[0]);
    }
  }
}

// dx_k[i] = sum_l W[i][l] r_k[l], one warp per row.
template <int K, int C>
__global__ void fx_kernel(FsParams p, int k) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31, n = p.n, D = p.D;
  if (i >= n) return;
  CAcc<K, C> acc;
  cacc_zero(acc);
  for (int l = lane; l < n; l += 32) {
    cmd<K, C> w, r;
    ld(p.W, p.Nnn, (long long)i * n + l, w);
    ld(p.r, p.Nx, (long long)l * D + k, r);
    cacc_fma(acc, w, r);
  }
  cmd<K, C> s;
  cacc_get(acc, s);
  warp_sum(s);
  if (lane == 0) st(p.dx, p.Nx, (long long)i * D + k, s);
}

// x += dx; per-entry magnitudes of f and dx for the norms of the step.
template <int K, int C>
__global__ void update_kernel(UpdParams p) {
  const long long total = (long long)p.n * p.D;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    cmd<K, C> x, dx, f;
    ld(p.dx, p.Nx, id, dx);
    ld(p.f, p.Nx, id, f);
    ld(p.x, p.Nx, id, x);
    cmd_add(x, dx, x);
    st(p.x, p.Nx, id, x);
    bool fin = true;
#pragma unroll
    for (int l = 0; l < K; ++l) fin = fin && finite_bits(x.re[l]) && finite_bits(x.im[l]);
    if (!fin) atomicOr(p.status, MDN_DEV_NONFINITE);
    p.dxabs[id] = (C == 2) ? hypot(dx.re[0], dx.im[0]) : fabs(dx.re[0]);
    p.fabs[id] = (C == 2) ? hypot(f.re[0], f.im[0]) : fabs(f.re[0]);
  }
}

// ---------------------------------------------------------------------------
// launchers of one (K, C) instantiation
// ---------------------------------------------------------------------------
template <int K, int C>
cudaError_t launch_ed(const EdParams& p, int grid, cudaStream_t s) {
  ed_kernel<K, C><<<grid, ED_THREADS, 0, s>>>(p);
  return cudaGetLastError();
}
template <int K, int C>
int ed_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ed_kernel<K, C>, ED_THREADS, 0) != cudaSuccess) return 0;
  return nb;
}
inline int grid_for(long long work, int threads) {
  long long g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 8192) g = 8192;
  return (int)g;
}
template <int K, int C>
cudaError_t launch_assemble(const AsmParams& p, bool want_A, cudaStream_t s) {
  assemble_f_kernel<K, C><<<grid_for((long long)p.n * p.D, 128), 128, 0, s>>>(p);
  if (want_A) assemble_A_kernel<K, C><<<grid_for((long long)p.n * p.n * p.D, 128), 128, 0, s>>>(p);
  return cudaGetLastError();
}
template <int K, int C>
cudaError_t launch_qr(const QrParams& p, cudaStream_t s) {
  QrParams q = p;
  void* args[] = {(void*)&q};
  return cudaLaunchCooperativeKernel((const void*)qr_kernel<K, C>, dim3(2 * p.nA), dim3(QR_THREADS), args, 0, s);
}
template <int K, int C>
cudaError_t launch_fs(const FsParams& p, int k, cudaStream_t s) {
  fs_kernel<K, C><<<p.n, FS_THREADS, 0, s>>>(p, k);
  return cudaGetLastError();
}
template <int K, int C>
cudaError_t launch_fx(const FsParams& p, int k, cudaStream_t s) {
  const int rows = FX_THREADS / 32;
  fx_kernel<K, C><<<(p.n + rows - 1) / rows, FX_THREADS, 0, s>>>(p, k);
  return cudaGetLastError();
}
template <int K, int C>
cudaError_t launch_update(const UpdParams& p, cudaStream_t s) {
  update_kernel<K, C><<<grid_for((long long)p.n * p.D, 128), 128, 0, s>>>(p);
  return cudaGetLastError();
}

template <int K, int C>
const KernelTable* make_table() {
  static const KernelTable t = {K, C, &launch_ed<K, C>, &ed_blocks_per_sm<K, C>, &launch_assemble<K, C>,
                                &launch_qr<K, C>, &launch_fs<K, C>, &launch_fx<K, C>, &launch_update<K, C>};
  return &t;
}

}  // namespace mdn
