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
//   a0_*           the leading block A_0 = J(x_0) alone, so that its QR can
//                  run beside the full evaluation;
//   fsub_kernel    forward substitution as one dataflow launch: r_k = b_k -
//                  sum_{j>=1} A_j dx_{k-j}, dx_k = W r_k and the residuals
//                  r_k - A_0 dx_k [updates, bs, residuals];
//   update kernels x += dx and the norms of the step.
#pragma once
#include <cstdint>
#include <type_traits>
#include "md.cuh"
#include "params.h"
#include "xf.cuh"

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

// Sum of level accumulators over the warp, renormalised once; every lane
// gets lane 0's total.
template <int K, int C>
__device__ __forceinline__ void warp_sum_acc(CAcc<K, C>& a, cmd<K, C>& r) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    CAcc<K, C> o;
#pragma unroll
    for (int l = 0; l < K; ++l) {
      o.re.l[l] = __shfl_xor_sync(FULL, a.re.l[l], off);
      if constexpr (C == 2) o.im.l[l] = __shfl_xor_sync(FULL, a.im.l[l], off);
    }
    cacc_add_acc(a, o);
  }
  cacc_get(a, r);
  cmd_bcast(r, 0);
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
      }
    }
  }
  ok = __shfl_sync(FULL, ok, 0);
  __syncwarp();
  return ok != 0;
}
// The warp barrier orders every lane's earlier stores before lane 0's
// release store at GPU scope (the release is cumulative over what lane 0 has
// observed), so a reader that acquires the flag sees them: one release
// instead of a full fence in every lane.
__device__ __forceinline__ void warp_publish(unsigned* flag, unsigned ep) {
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
  // operands of term s: coefficient k1 takes s = 0..k1, coefficient k2 the rest
  auto idx = [&](int s, int& i, int& j, bool& first) {
    first = s <= k1;
    i = first ? s : s - k1;
    j = first ? k1 - s : k2 - i;
  };
  cmd<K, C> av, bv;
  CAcc<K, C> acc1, acc2;
  ld(a.p, a.N, a.off, av);
  ld(b.p, b.N, b.off + k1, bv);
  cacc_mul(acc1, av, bv);
  ld(b.p, b.N, b.off + k2, bv);
  cacc_mul(acc2, av, bv);
  constexpr bool prefetch = K * C <= 8;  // registers: keep the next operands in flight
  int i, j;
  bool first;
  if constexpr (prefetch) {
    if (D > 1) {
      idx(1, i, j, first);
      ld(a.p, a.N, a.off + i, av);
      ld(b.p, b.N, b.off + j, bv);
    }
  }
  for (int s = 1; s < D; ++s) {
    cmd<K, C> ca, cb;
    if constexpr (prefetch) {
      ca = av;
      cb = bv;
      idx(s, i, j, first);
      if (s + 1 < D) {
        int i2, j2;
        bool f2;
        idx(s + 1, i2, j2, f2);
        ld(a.p, a.N, a.off + i2, av);
        ld(b.p, b.N, b.off + j2, bv);
      }
    } else {
      idx(s, i, j, first);
      ld(a.p, a.N, a.off + i, ca);
      ld(b.p, b.N, b.off + j, cb);
    }
    CAcc<K, C> acc;
    cacc_select(first, acc1, acc2, acc);
    cacc_fma(acc, ca, cb);
    cacc_select(first, acc, acc1, acc1);
    cacc_select(first, acc2, acc, acc2);
  }
  cmd<K, C> r1, r2;
  cacc_get(acc1, r1);
  cacc_get(acc2, r2);
  st(o.p, o.N, o.off + k1, r1);
  if (k2 != k1) st(o.p, o.N, o.off + k2, r2);
}

// The same product in integer-limb extended floats (xf.cuh), for K >= 2:
// the group's lanes convert the D coefficients of a and b once into the
// group's shared memory; lane t then sums the t+1 products of coefficient
// k1 = t and the D-t products of coefficient k2 = D-1-t in fixed-point
// accumulators (one per coefficient, real and imaginary part), their scale
// set beforehand from the largest exponent sum of their terms, so a term is
// an integer product, a shift and an add on the integer pipe.  Each result
// is rounded to K limbs once.
template <int K, int C>
__device__ __forceinline__ void series_product_xf(const SP& a, const SP& b, const SP& o, int t, int D,
                                                  unsigned gmask, xfn::xf<xfn::xf_words_t<K>::value>* stage) {
  using namespace xfn;
  constexpr int W = xf_words_t<K>::value;
  xf<W>* sa = stage;          // [C][D]
  xf<W>* sb = stage + C * D;  // [C][D]
  const int k1 = t, k2 = D - 1 - t;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int k = q ? k2 : k1;
    if (q == 1 && k2 == k1) break;
    cmd<K, C> v;
    ld(a.p, a.N, a.off + k, v);
    xf_from_md<K, W>(v.re, sa[k]);
    if constexpr (C == 2) xf_from_md<K, W>(v.im, sa[D + k]);
    ld(b.p, b.N, b.off + k, v);
    xf_from_md<K, W>(v.re, sb[k]);
    if constexpr (C == 2) xf_from_md<K, W>(v.im, sb[D + k]);
  }
  __syncwarp(gmask);
  // term s = 0..D: coefficient k1 for s <= k1 (i = s), then k2 (i = s-k1-1)
  int e1r = 2 * XF_ZERO_E, e2r = 2 * XF_ZERO_E, e1i = 2 * XF_ZERO_E, e2i = 2 * XF_ZERO_E;
  for (int s = 0; s <= D; ++s) {
    const bool first = s <= k1;
    const int i = first ? s : s - k1 - 1;
    const int j = (first ? k1 : k2) - i;
    int er = sa[i].e + sb[j].e, ei = er;
    if constexpr (C == 2) {
      const int ar = sa[i].e, ai = sa[D + i].e, br = sb[j].e, bi = sb[D + j].e;
      er = max(ar + br, ai + bi);
      ei = max(ar + bi, ai + br);
    }
    if (first) {
      e1r = max(e1r, er);
      e1i = max(e1i, ei);
    } else {
      e2r = max(e2r, er);
      e2i = max(e2i, ei);
    }
  }
  xfacc<W> cr, ci, dr, di;
  xfacc_init(cr, e1r);
  if constexpr (C == 2) xfacc_init(ci, e1i);
  for (int s = 0; s <= D; ++s) {
    if (s == k1 + 1) {
      dr = cr;
      xfacc_init(cr, e2r);
      if constexpr (C == 2) {
        di = ci;
        xfacc_init(ci, e2i);
      }
    }
    const bool first = s <= k1;
    const int i = first ? s : s - k1 - 1;
    const int j = (first ? k1 : k2) - i;
    const xf<W> ar = sa[i], br = sb[j];
    xfacc_fma(cr, ar, br);
    if constexpr (C == 2) {
      const xf<W> ai = sa[D + i], bi = sb[D + j];
      xfacc_fma(cr, ai, bi, true);
      xfacc_fma(ci, ar, bi);
      xfacc_fma(ci, ai, br);
    }
  }
  cmd<K, C> r;
  xf<W> x;
  xfacc_get(dr, x);
  xf_to_md<K, W>(x, r.re);
  if constexpr (C == 2) {
    xfacc_get(di, x);
    xf_to_md<K, W>(x, r.im);
  }
  st(o.p, o.N, o.off + k1, r);
  if (k2 != k1) {
    xfacc_get(cr, x);
    xf_to_md<K, W>(x, r.re);
    if constexpr (C == 2) {
      xfacc_get(ci, x);
      xf_to_md<K, W>(x, r.im);
    }
    st(o.p, o.N, o.off + k2, r);
  }
}

template <int K, int C>
__global__ void __launch_bounds__(ED_THREADS) ed_kernel(EdParams p) {
  extern __shared__ __align__(16) unsigned char ed_smem[];
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
        if constexpr (K >= 2) {
          // shared memory: per warp G groups of 2 C len xf values (G len <= 64)
          using X = xfn::xf<xfn::xf_words_t<K>::value>;
          X* stage = reinterpret_cast<X*>(ed_smem) + ((threadIdx.x >> 5) * p.G + g) * (2 * C * p.len);
          const unsigned gmask = (p.P >= 32 ? FULL : ((1u << p.P) - 1u)) << (g * p.P);
          series_product_xf<K, C>(resolve(p, op.z, m, wg), resolve(p, op.w, m, wg), resolve(p, op.y, m, wg), t,
                                  p.len, gmask, stage);
        } else {
          series_product<K, C>(resolve(p, op.z, m, wg), resolve(p, op.w, m, wg), resolve(p, op.y, m, wg), t, p.len);
        }
      } else if (op.x == OP_COPY) {
        const SP s = resolve(p, op.z, m, wg), d = resolve(p, op.y, m, wg);
        cmd<K, C> v;
        ld(s.p, s.N, s.off + t, v);
        st(d.p, d.N, d.off + t, v);
        ld(s.p, s.N, s.off + (p.len - 1 - t), v);
        st(d.p, d.N, d.off + (p.len - 1 - t), v);
      }
      __syncwarp();
    }
  }
}

// f_i[k] = cst_i[k] + sum of the values of the monomials of equation i.
template <int K, int C>
__global__ void assemble_f_kernel(AsmParams p) {
  const long long total = (long long)p.n * p.len;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q / p.len), kk = (int)(q - (long long)i * p.len);
    const long long id = (long long)i * p.D + kk;
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
  const long long total = nn * (p.len - p.j_begin);
  for (long long id0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; id0 < total;
       id0 += (long long)gridDim.x * blockDim.x) {
    const long long id = id0 + nn * p.j_begin;
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

// A_0 = J(x_0): for every occurrence p of a variable in monomial m, the
// constant coefficient of the partial derivative, c_m(0) times the product of
// the other variables at t = 0 (one thread per occurrence).
template <int K, int C>
__global__ void a0_partials_kernel(A0Params p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.nnz) return;
  const int m = p.occ_mono[t];
  const int vp = p.mono_vp[m], k = p.mono_k[m], pos = t - vp;
  cmd<K, C> g, x;
  ld(p.coeff, p.Nc, (long long)m * p.D, g);
  for (int q = 0; q < k; ++q) {
    if (q == pos) continue;
    ld(p.x, p.Nx, (long long)p.vidx[vp + q] * p.xstride, x);
    cmd<K, C> r;
    cmd_mul(g, x, r);
    g = r;
  }
  st(p.out0, p.S, (long long)p.mono_sbase[m] + 1 + pos, g);
}
// The same partials with a warp per monomial, for monomials of many
// variables (the direct form costs k-1 products per occurrence, k^2 per
// monomial): lane l takes the occurrences [l s, (l+1) s), s = ceil(k/32);
// scans over the lanes of the chunk products give the product of the chunks
// before and after its own; a forward pass stores c (before) times the
// prefix within the chunk, a backward pass multiplies in the suffix, about
// 3k products per monomial.
template <int K, int C>
__device__ __forceinline__ void cmd_shfl_up(const cmd<K, C>& v, cmd<K, C>& o, int off) {
#pragma unroll
  for (int l = 0; l < K; ++l) {
    o.re[l] = __shfl_up_sync(FULL, v.re[l], off);
    o.im[l] = C == 2 ? __shfl_up_sync(FULL, v.im[l], off) : 0.0;
  }
}
template <int K, int C>
__device__ __forceinline__ void cmd_shfl_down(const cmd<K, C>& v, cmd<K, C>& o, int off) {
#pragma unroll
  for (int l = 0; l < K; ++l) {
    o.re[l] = __shfl_down_sync(FULL, v.re[l], off);
    o.im[l] = C == 2 ? __shfl_down_sync(FULL, v.im[l], off) : 0.0;
  }
}
template <int K, int C>
__global__ void a0_partials_warp_kernel(A0Params p) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long m = w0; m < p.M; m += nw) {
    const int vp = p.mono_vp[m], k = p.mono_k[m];
    const int s = (k + 31) / 32;
    const int lo = min(k, lane * s), hi = min(k, lo + s);
    cmd<K, C> one, x, t;
    cmd_zero(one);
    one.re[0] = 1.0;
    cmd<K, C> local = one;  // product of the own chunk
    for (int q = lo; q < hi; ++q) {
      ld(p.x, p.Nx, (long long)p.vidx[vp + q] * p.xstride, x);
      cmd_mul(local, x, t);
      local = t;
    }
    // inclusive scans of the chunk products from the left and from the right
    cmd<K, C> inc_l = local, inc_r = local, o;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      cmd_shfl_up(inc_l, o, off);
      if (lane >= off) {
        cmd_mul(o, inc_l, t);
        inc_l = t;
      }
      cmd_shfl_down(inc_r, o, off);
      if (lane + off < 32) {
        cmd_mul(inc_r, o, t);
        inc_r = t;
      }
    }
    cmd<K, C> before, after;
    cmd_shfl_up(inc_l, before, 1);
    cmd_shfl_down(inc_r, after, 1);
    if (lane == 0) before = one;
    if (lane == 31) after = one;
    cmd<K, C> run, c;
    ld(p.coeff, p.Nc, m * p.D, c);
    cmd_mul(c, before, t);
    cmd_mul(t, after, run);
    const long long slot0 = (long long)p.mono_sbase[m] + 1;
    for (int q = lo; q < hi; ++q) {  // c * before * after * prefix within the chunk
      st(p.out0, p.S, slot0 + q, run);
      ld(p.x, p.Nx, (long long)p.vidx[vp + q] * p.xstride, x);
      cmd_mul(run, x, t);
      run = t;
    }
    run = one;
    for (int q = hi - 1; q >= lo; --q) {  // times the suffix within the chunk
      cmd<K, C> v;
      ld(p.out0, p.S, slot0 + q, v);
      cmd_mul(v, run, t);
      st(p.out0, p.S, slot0 + q, t);
      ld(p.x, p.Nx, (long long)p.vidx[vp + q] * p.xstride, x);
      cmd_mul(run, x, t);
      run = t;
    }
  }
}

template <int K, int C>
__global__ void a0_assemble_kernel(A0Params p) {
  const long long nn = (long long)p.n * p.n;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < nn;
       id += (long long)gridDim.x * blockDim.x) {
    cmd<K, C> v;
    cmd_zero(v);
    const int q0 = p.pair_ptr[id], q1 = p.pair_ptr[id + 1];
    if (q1 > q0) {
      CAcc<K, C> acc;
      ld(p.out0, p.S, p.pair_slot[q0], v);
      cacc_set(acc, v);
      for (int q = q0 + 1; q < q1; ++q) {
        ld(p.out0, p.S, p.pair_slot[q], v);
        cacc_add(acc, v);
      }
      cacc_get(acc, v);
    }
    st(p.A, p.NA, id, v);  // j = 0 slice
  }
}

// ---------------------------------------------------------------------------
// Householder QR of A0 and W = A0^{-1} = R^{-1} Q^H (Section 5.3)
// ---------------------------------------------------------------------------
// Cooperative launch, one block per SM, three roles of nA blocks each:
// one warp per column of A0, one warp per column of the identity (Q^H), one
// warp per row of R^{-1}.  Every warp keeps its column or row in shared
// memory, limb by limb (structure of arrays, conflict free).
//
// Reflector j is H_j = I - tau_j v_j v_j^H with v_j = x_j + s_j |x_j| e_j,
// x_j = column j (rows j..n-1) after H_0..H_{j-1}, s_j = x_jj / |x_jj| (+1 for
// x_jj = 0), tau_j = 1 / (|x_j| (|x_j| + |x_jj|)); then H_j x_j = -s_j |x_j| e_j.
// Three flags per column (values = the launch epoch):
//   col[j]  x_j is published (rows j..n-1 of Vm column j, stored column
//           after column so that a warp reads a column in whole lines);
//   ref[j]  the scalars s_j|x_j|, v_jj and tau_j are published;
//   rinv[j] 1 / R_jj is published.
// Look-ahead: the warp of column c forms x_j^H y_c as soon as col[j]
// appears, while the owner of column j is still computing its scalars; when
// ref[j] appears, applying H_j costs
//   w = x_j^H y_c + conj(s_j|x_j|) y_c[j],   y_c -= tau_j w v_j.
// The norm of the pivot column needs no reduction on the chain: the
// reflectors are unitary, so rows j+1..n-1 of y_c after H_j hold
// |a_c|^2 - sum_{i<=j} |R_ic|^2 (a_c = column c of A0), accumulated as each
// R_ic becomes final and recomputed directly if more than 8 bits cancel.

// All arithmetic of the three roles runs in integer-limb extended floats
// (xf.cuh): on this part a warp's FP64 instruction occupies its sub-partition
// for 64 cycles, so a dependent chain of md operations on one warp is bound
// by the FP64 issue rate, while the same values carried in 64-bit integer
// words (64W >= 53K + 11 bits) move on the integer pipe.  Columns and rows
// stay in shared and global memory as md values (K limbs); they are
// converted to xf where they are read and rounded back to K limbs where they
// are stored, so every stored value is an md value correct to its precision.

// complex (or real, C = 1) extended floats
template <int W, int C>
struct cxf {
  xfn::xf<W> re, im;
};

template <int K, int W, int C>
__device__ __forceinline__ void cxf_load(const double* p, long long N, long long i, cxf<W, C>& v) {
  cmd<K, C> t;
  ld(p, N, i, t);
  xfn::xf_from_md<K, W>(t.re, v.re);
  if constexpr (C == 2) xfn::xf_from_md<K, W>(t.im, v.im);
  else xfn::xf_zero(v.im);
}
template <int K, int W, int C>
__device__ __forceinline__ void cxf_store(double* p, long long N, long long i, const cxf<W, C>& v) {
  cmd<K, C> t;
  xfn::xf_to_md<K, W>(v.re, t.re);
  if constexpr (C == 2) xfn::xf_to_md<K, W>(v.im, t.im);
  else md_zero(t.im);
  st(p, N, i, t);
}
template <int W, int C>
__device__ __forceinline__ void cxf_zero(cxf<W, C>& v) {
  xfn::xf_zero(v.re);
  xfn::xf_zero(v.im);
}
template <int W, int C>
__device__ __forceinline__ void cxf_neg(cxf<W, C>& v) {
  xfn::xf_neg(v.re);
  xfn::xf_neg(v.im);
}
// O (xf.cuh): the basic operations inline (throughput code) or called out
// of line (latency-bound chains on one warp)
template <class O = xfn::xf_ops_inline, int W, int C>
__device__ __forceinline__ void cxf_add(const cxf<W, C>& a, const cxf<W, C>& b, cxf<W, C>& r) {
  O::add(a.re, b.re, r.re);
  if constexpr (C == 2) O::add(a.im, b.im, r.im);
  else xfn::xf_zero(r.im);
}
// r = a b (conj_a: conj(a) b)
template <bool conj_a, class O = xfn::xf_ops_inline, int W, int C>
__device__ __forceinline__ void cxf_mul(const cxf<W, C>& a, const cxf<W, C>& b, cxf<W, C>& r) {
  using namespace xfn;
  if constexpr (C == 1) {
    O::mul(a.re, b.re, r.re);
    xf_zero(r.im);
  } else {
    xf<W> t1, t2, t3, t4;
    O::mul(a.re, b.re, t1);
    O::mul(a.im, b.im, t2);
    O::mul(a.re, b.im, t3);
    O::mul(a.im, b.re, t4);
    if constexpr (conj_a) {
      O::add(t1, t2, r.re);
      O::sub(t3, t4, r.im);
    } else {
      O::sub(t1, t2, r.re);
      O::add(t3, t4, r.im);
    }
  }
}
template <bool conj_a, class O = xfn::xf_ops_inline, int W, int C>
__device__ __forceinline__ void cxf_fma(cxf<W, C>& acc, const cxf<W, C>& a, const cxf<W, C>& b) {
  cxf<W, C> t;
  cxf_mul<conj_a, O>(a, b, t);
  cxf_add<O>(acc, t, acc);
}
template <class O = xfn::xf_ops_inline, int W, int C>
__device__ __forceinline__ void cxf_scale(const cxf<W, C>& a, const xfn::xf<W>& s, cxf<W, C>& r) {
  O::mul(a.re, s, r.re);
  if constexpr (C == 2) O::mul(a.im, s, r.im);
  else xfn::xf_zero(r.im);
}
// extended floats as the QR stores them: [W+1][C][N] 64-bit words, the W
// mantissa words and one word holding the exponent (low half) and sign
template <int W, int C>
__device__ __forceinline__ void xld(const uint64_t* p, long long N, long long i, cxf<W, C>& v) {
#pragma unroll
  for (int w = 0; w < W; ++w) {
    v.re.m[w] = p[(long long)(w * C) * N + i];
    if constexpr (C == 2) v.im.m[w] = p[(long long)(w * C + 1) * N + i];
  }
  const uint64_t h = p[(long long)(W * C) * N + i];
  v.re.e = (int)(unsigned)h;
  v.re.s = (int)(h >> 32);
  if constexpr (C == 2) {
    const uint64_t g = p[(long long)(W * C + 1) * N + i];
    v.im.e = (int)(unsigned)g;
    v.im.s = (int)(g >> 32);
  } else {
    xfn::xf_zero(v.im);
  }
}
template <int W, int C>
__device__ __forceinline__ void xst(uint64_t* p, long long N, long long i, const cxf<W, C>& v) {
#pragma unroll
  for (int w = 0; w < W; ++w) {
    p[(long long)(w * C) * N + i] = v.re.m[w];
    if constexpr (C == 2) p[(long long)(w * C + 1) * N + i] = v.im.m[w];
  }
  p[(long long)(W * C) * N + i] = (uint64_t)(unsigned)v.re.e | ((uint64_t)(unsigned)v.re.s << 32);
  if constexpr (C == 2)
    p[(long long)(W * C + 1) * N + i] = (uint64_t)(unsigned)v.im.e | ((uint64_t)(unsigned)v.im.s << 32);
}
// the exponents alone (for the scale of a fixed-point sum)
template <int W, int C>
__device__ __forceinline__ void xld_exp(const uint64_t* p, long long N, long long i, int& er, int& ei) {
  er = (int)(unsigned)p[(long long)(W * C) * N + i];
  ei = C == 2 ? (int)(unsigned)p[(long long)(W * C + 1) * N + i] : 2 * xfn::XF_ZERO_E;
}
template <int W, int C>
__device__ __forceinline__ void xcopy(const uint64_t* src, long long Ns, long long is, uint64_t* dst, long long Nd,
                                      long long id) {
#pragma unroll
  for (int w = 0; w < (W + 1) * C; ++w) dst[(long long)w * Nd + id] = src[(long long)w * Ns + is];
}

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(FULL, v, off));
  return v;
}
// Extra headroom bits of a fixed-point sum of `terms` products beyond the
// XF_ACC_TERMS that the accumulator's own headroom covers (0 up to 512).
__device__ __forceinline__ int acc_extra_head(long long terms) {
  int h = 0;
  while (((long long)xfn::XF_ACC_TERMS << h) < terms) ++h;
  return h;
}
// sum over the warp of fixed-point accumulators of one scale
template <int W>
__device__ __forceinline__ void xfacc_warp_sum(xfn::xfacc<W>& a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    uint64_t o[W + 2];
#pragma unroll
    for (int i = 0; i < W + 2; ++i) o[i] = __shfl_xor_sync(FULL, a.w[i], off);
    xfn::add_words<W + 2>(a.w, o, 0ULL);
  }
}

// Fixed-point dot product over the warp: sum of conj(x_i) y_i (conj_x) or
// x_i y_i for the rows the lanes pass in; the scale comes from a first
// pass over the exponents (a warp maximum), so every lane accumulates at the
// same scale and the warp sum is an integer sum.
template <bool conj_x, int W, int C>
__device__ __forceinline__ void dot_exp(int xr, int xi, int yr, int yi, int& er, int& ei) {
  er = max(er, max(xr + yr, xi + yi));
  ei = max(ei, max(xr + yi, xi + yr));
}
template <bool conj_x, class O = xfn::xf_ops_inline, int W, int C>
__device__ __forceinline__ void dot_fma(xfn::xfacc<W>& ar, xfn::xfacc<W>& ai, const cxf<W, C>& x, const cxf<W, C>& y) {
  O::acc_fma(ar, x.re, y.re);
  if constexpr (C == 2) {
    // conj(x) y = (xr yr + xi yi) + i (xr yi - xi yr);  x y = (xr yr - xi yi) + i (xr yi + xi yr)
    O::acc_fma(ar, x.im, y.im, !conj_x);
    O::acc_fma(ai, x.re, y.im);
    O::acc_fma(ai, x.im, y.re, conj_x);
  }
}
template <int W, int C>
__device__ __forceinline__ void dot_finish(xfn::xfacc<W>& ar, xfn::xfacc<W>& ai, cxf<W, C>& r) {
  xfacc_warp_sum(ar);
  xfn::xfacc_get(ar, r.re);
  if constexpr (C == 2) {
    xfacc_warp_sum(ai);
    xfn::xfacc_get(ai, r.im);
  } else {
    xfn::xf_zero(r.im);
  }
}

// The dataflow QR's warps and the pivot of the large-n QR are chains of
// dependent operations on one warp, each run once per column: from 4 words
// up they call the basic operations out of line (xf.cuh), so that their code
// stays in the instruction cache; at 1 and 2 words the inlined code is small
// and the call would cost more than it saves.
template <int W>
using QOps = typename std::conditional<(W >= 4), xfn::xf_ops_call, xfn::xf_ops_inline>::type;

// dot = sum of conj(x_j[i]) y[i] over rows i = j..n-1 (x_j from Vm); the
// rows of x_j are also staged in the warp's shared buffer xs, where the
// update by reflector j reads them (row j there becomes v_jj in qr_form_w).
template <int K, int C>
__device__ __forceinline__ void qr_lookahead(const QrParams& p, int j, const uint64_t* y, uint64_t* xs,
                                             cxf<xfn::xf_words_t<K>::value, C>& dot) {
  constexpr int W = xfn::xf_words_t<K>::value;
  using QO = QOps<W>;
  const int lane = threadIdx.x & 31;
  const int n = p.n;
  int er = 2 * xfn::XF_ZERO_E, ei = er;
  // one pass over global memory: x_j into xs (its exponents on the way)
#pragma unroll 2
  for (int i = j + lane; i < n; i += 32) {
    cxf<W, C> x;
    int yr, yi;
    xld<W, C>(p.Vm, p.Nnn, (long long)j * n + i, x);
    xst<W, C>(xs, n, i, x);
    xld_exp<W, C>(y, n, i, yr, yi);
    dot_exp<true, W, C>(x.re.e, C == 2 ? x.im.e : 2 * xfn::XF_ZERO_E, yr, yi, er, ei);
  }
  __syncwarp();
  xfn::xfacc<W> ar, ai;
  const int head = acc_extra_head(C * (n - j));
  xfn::xfacc_init(ar, warp_max(er) + head);
  if constexpr (C == 2) xfn::xfacc_init(ai, warp_max(ei) + head);
  for (int i = j + lane; i < n; i += 32) {
    cxf<W, C> x, yi;
    xld<W, C>(xs, n, i, x);
    xld<W, C>(y, n, i, yi);
    dot_fma<true, QO>(ar, ai, x, yi);
  }
  dot_finish(ar, ai, dot);
}

// |y|^2 over rows i0..n-1, every lane gets it.
template <int K, int C>
__device__ __forceinline__ void qr_norm2(const uint64_t* y, int n, int i0, xfn::xf<xfn::xf_words_t<K>::value>& nrm) {
  constexpr int W = xfn::xf_words_t<K>::value;
  using QO = QOps<W>;
  const int lane = threadIdx.x & 31;
  int er = 2 * xfn::XF_ZERO_E, ei = er;
  for (int i = i0 + lane; i < n; i += 32) {
    int yr, yi;
    xld_exp<W, C>(y, n, i, yr, yi);
    dot_exp<true, W, C>(yr, yi, yr, yi, er, ei);
  }
  xfn::xfacc<W> ar, ai;
  xfn::xfacc_init(ar, warp_max(er) + acc_extra_head(C * (n - i0)));
  for (int i = i0 + lane; i < n; i += 32) {
    cxf<W, C> v;
    xld<W, C>(y, n, i, v);
    QO::acc_fma(ar, v.re, v.re);
    if constexpr (C == 2) QO::acc_fma(ar, v.im, v.im);
  }
  xfacc_warp_sum(ar);
  xfn::xfacc_get(ar, nrm);
}

// w = dot + conj(s_j|x_j|) y[j], and v_jj into row j of xs (needs the alpha
// flag of reflector j)
template <int K, int C>
__device__ __forceinline__ void qr_form_w(const QrParams& p, int j, const uint64_t* y, uint64_t* xs,
                                          const cxf<xfn::xf_words_t<K>::value, C>& dot,
                                          cxf<xfn::xf_words_t<K>::value, C>& w) {
  constexpr int W = xfn::xf_words_t<K>::value;
  using QO = QOps<W>;
  cxf<W, C> sa, yj;
  xld<W, C>(p.salpha, p.n, j, sa);
  xld<W, C>(y, p.n, j, yj);
  if ((threadIdx.x & 31) == 0) xcopy<W, C>(p.v0, p.n, j, xs, p.n, j);
  __syncwarp();
  w = dot;
  cxf_fma<true, QO>(w, sa, yj);
}

// y -= tau_j w v_j over rows j..n-1 (needs the ref flag of reflector j).
template <int K, int C>
// With pub >= 0 (the column warp's last reflector, j = pub - 1), rows
// pub..n-1 of the result, the column x_pub that its owner publishes next,
// are also stored to Vm as they are formed.
__device__ __forceinline__ void qr_update(const QrParams& p, int j, uint64_t* y, const uint64_t* xs,
                                          const cxf<xfn::xf_words_t<K>::value, C>& w, int pub = -1) {
  constexpr int W = xfn::xf_words_t<K>::value;
  using QO = QOps<W>;
  const int lane = threadIdx.x & 31;
  const int n = p.n;
  cxf<W, 1> tau;
  xld<W, 1>(p.tau, p.n, j, tau);
  cxf<W, C> ng;
  cxf_scale<QO>(w, tau.re, ng);
  cxf_neg(ng);
  __syncwarp();
  // passes of 32 rows with a trip count uniform over the warp, and the warp
  // converged before the (out-of-line) arithmetic, so that each call runs
  // once for all lanes; a lane past the last row recomputes row j unstored
  for (int i0 = j; i0 < n; i0 += 32) {
    const int i = i0 + lane;
    const bool row = i < n;
    const int r = row ? i : j;
    cxf<W, C> v, yi;
    xld<W, C>(xs, n, r, v);  // v_j: x_j below the diagonal, v_jj on it
    xld<W, C>(y, n, r, yi);
    __syncwarp();
    cxf_fma<false, QO>(yi, ng, v);
    if (row) {
      xst<W, C>(y, n, i, yi);
      if (pub >= 0 && i >= pub) xst<W, C>(p.Vm, p.Nnn, (long long)pub * n + i, yi);
    }
  }
  __syncwarp();
}

// Column warp c: its column under the reflectors 0..c-1, then reflector c.
// Reflector j is applied in three parts: the dot product x_j^H y as soon as
// x_j is out (col[j]), w = dot + conj(s_j|x_j|) y[j] as soon as s_j|x_j| and
// v_jj are out (alpha[j]), and y -= tau_j w v_j once tau_j is out (ref[j]).  The entries
// R_jc, final as the updates go, are copied out after the pivot (off the
// chain from one column's tau to the next's).
template <int K, int C>
__device__ void qr_column(const QrParams& p, int c, uint64_t* y, uint64_t* xs, unsigned ep) {
  using namespace xfn;
  constexpr int W = xf_words_t<K>::value;
  using QO = QOps<W>;
  const int lane = threadIdx.x & 31;
  const int n = p.n;
  unsigned* fcol = p.flags;
  unsigned* fref = p.flags + n;
  unsigned* frinv = p.flags + 2 * n;
  unsigned* fal = p.flags + 3 * n;
  for (int i = lane; i < n; i += 32) {
    cxf<W, C> v;
    cxf_load<K, W, C>(p.A0, p.NA, (long long)i * n + c, v);
    xst<W, C>(y, n, i, v);
  }
  __syncwarp();
  // |a_c|^2, then minus |R_jc|^2 as each R_jc is final
  xf<W> norm0, xN;
  qr_norm2<K, C>(y, n, 0, norm0);
  xN = norm0;
  for (int j = 0; j < c; ++j) {
    if (!warp_wait(&fcol[j], ep, p.spin_limit, p.status)) return;
    cxf<W, C> dot, w;
    qr_lookahead<K, C>(p, j, y, xs, dot);
    if (!warp_wait(&fal[j], ep, p.spin_limit, p.status)) return;
    qr_form_w<K, C>(p, j, y, xs, dot, w);
    if (!warp_wait(&fref[j], ep, p.spin_limit, p.status)) return;
    qr_update<K, C>(p, j, y, xs, w, j == c - 1 ? c : -1);
    cxf<W, C> xv, q;
    xld<W, C>(y, n, j, xv);
    cxf_mul<true, QO>(xv, xv, q);
    QO::sub(xN, q.re, xN);
  }
  // publish x_c (rows c..n-1; the last update stored them for c > 0)
  if (c == 0)
    for (int i = c + lane; i < n; i += 32) xcopy<W, C>(y, n, i, p.Vm, p.Nnn, (long long)c * n + i);
  warp_publish(&fcol[c], ep);
  // N = |x_c|^2 by downdating, recomputed when it is not positive or more
  // than 8 bits cancelled
  if (c > 0 && (xN.s != 0 || xf_is_zero(xN) || xN.e + 8 < norm0.e)) qr_norm2<K, C>(y, n, c, xN);
  const bool singular = xf_is_zero(xN);
  if (singular) xf_from_double(1.0, xN);  // keep the arithmetic finite; reported below
  // The pivot scalars:
  //   |x_c| = N / sqrt(N),  s = x_cc / |x_cc| (1 if x_cc = 0),
  //   v_cc = x_cc + s|x_c|,  tau = 1 / (N + |x_c| |x_cc|),
  //   R_cc = -s|x_c|,  1 / R_cc = -conj(s) / |x_c|.
  cxf<W, C> x0;
  xld<W, C>(y, n, c, x0);
  xf<W> xry, xal, xax0;
  xf<W> sgr, sgi;  // s
  bool neg = false;
  if constexpr (C == 1) {
    neg = x0.re.s != 0;
    xax0 = x0.re;
    xax0.s = 0;
  } else {
    xf<W> t1, t2, a2x, rx;
    QO::mul(x0.re, x0.re, t1);
    QO::mul(x0.im, x0.im, t2);
    QO::add(t1, t2, a2x);
    const bool z = xf_is_zero(a2x);
    if (z) xf_from_double(1.0, a2x);
    xf_rsqrt<QO>(a2x, rx);
    QO::mul(a2x, rx, xax0);
    QO::mul(x0.re, rx, sgr);
    QO::mul(x0.im, rx, sgi);
    if (z) {
      xf_zero(xax0);
      xf_from_double(1.0, sgr);
      xf_zero(sgi);
    }
  }
  xf_rsqrt<QO>(xN, xry);
  QO::mul(xN, xry, xal);
  xf<W> sre, sim;  // s|x_c|
  if constexpr (C == 1) {
    sre = xal;
    if (neg) xf_neg(sre);
    xf_zero(sim);
  } else {
    QO::mul(sgr, xal, sre);
    QO::mul(sgi, xal, sim);
  }
  {
    cxf<W, C> sa, v0;
    sa.re = sre;
    sa.im = sim;
    QO::add(x0.re, sre, v0.re);
    if constexpr (C == 2) QO::add(x0.im, sim, v0.im);
    else xf_zero(v0.im);
    if (lane == 0) {
      xst<W, C>(p.salpha, p.n, c, sa);
      xst<W, C>(p.v0, p.n, c, v0);
    }
  }
  warp_publish(&fal[c], ep);  // the later columns form their w meanwhile
  {
    cxf<W, 1> tau;
    xf_zero(tau.im);
    xf<W> t1, t2;
    QO::mul(xal, xax0, t1);
    QO::add(xN, t1, t2);
    xf_recip<QO>(t2, tau.re);
    if (singular) {
      xf_zero(tau.re);
      if (lane == 0) atomicOr(p.status, MDN_DEV_SINGULAR);
    }
    if (lane == 0) {
      xst<W, 1>(p.tau, p.n, c, tau);
      cxf<W, C> r;
      r.re = sre;
      r.im = sim;
      cxf_neg(r);
      xst<W, C>(p.Rm, p.Nnn, (long long)c * n + c, r);
    }
  }
  warp_publish(&fref[c], ep);
  // 1 / R_cc = -conj(s) / |x_c|
  cxf<W, C> rinv;
  if constexpr (C == 1) {
    rinv.re = xry;  // s = +-1
    if (!neg) xf_neg(rinv.re);
    xf_zero(rinv.im);
  } else {
    xf_mul(sgr, xry, rinv.re);
    xf_neg(rinv.re);
    xf_mul(sgi, xry, rinv.im);
  }
  if (singular) cxf_zero(rinv);
  if (lane == 0) xst<W, C>(p.rinv, p.n, c, rinv);
  for (int i = lane; i < c; i += 32) xcopy<W, C>(y, n, i, p.Rm, p.Nnn, (long long)i * n + c);  // R_ic, i < c
  warp_publish(&frinv[c], ep);
}

// Identity warp e: Q^H e_e as the reflectors appear (column e of Y = Q^H).
template <int K, int C>
__device__ void qr_identity(const QrParams& p, int e, uint64_t* y, uint64_t* xs, unsigned ep) {
  constexpr int W = xfn::xf_words_t<K>::value;
  const int lane = threadIdx.x & 31;
  const int n = p.n;
  unsigned* fref = p.flags + n;
  for (int i = lane; i < n; i += 32) {
    cxf<W, C> v;
    cxf_zero(v);
    if (i == e) xfn::xf_from_double(1.0, v.re);
    xst<W, C>(y, n, i, v);
  }
  __syncwarp();
  for (int j = 0; j < n; ++j) {
    if (!warp_wait(&fref[j], ep, p.spin_limit, p.status)) return;
    cxf<W, C> dot, w;
    qr_lookahead<K, C>(p, j, y, xs, dot);
    qr_form_w<K, C>(p, j, y, xs, dot, w);
    qr_update<K, C>(p, j, y, xs, w);
  }
  for (int i = lane; i < n; i += 32) {
    cxf<W, C> v;
    xld<W, C>(y, n, i, v);
    cxf_store<K, W, C>(p.Y, p.Nnn, (long long)i * n + e, v);
  }
}

// Rows ia and ib of Z = R^{-1} (one warp, the rows g and n-1-g so that the
// warps share the work evenly), built column by column as R grows:
//   Z[i][i] = 1/R_ii,  Z[i][c] = -(1/R_cc) sum_{k=i..c-1} Z[i][k] R[k][c]  (c > i),
// the block inverse of the leading (c+1) x (c+1) part of R.
template <int K, int C>
__device__ void qr_rinv_rows(const QrParams& p, int ia, int ib, uint64_t* za, uint64_t* zb, unsigned ep) {
  constexpr int W = xfn::xf_words_t<K>::value;
  using QO = QOps<W>;
  const int lane = threadIdx.x & 31;
  const int n = p.n;
  unsigned* frinv = p.flags + 2 * n;
  for (int c = ia; c < n; ++c) {
    if (!warp_wait(&frinv[c], ep, p.spin_limit, p.status)) return;
    cxf<W, C> rc;
    xld<W, C>(p.rinv, p.n, c, rc);
    for (int q = 0; q < 2; ++q) {
      const int i = q ? ib : ia;
      uint64_t* z = q ? zb : za;
      if (c < i || (q == 1 && ib == ia)) continue;
      cxf<W, C> zc;
      if (c == i) {
        zc = rc;
      } else {
        int er = 2 * xfn::XF_ZERO_E, ei = er;
        for (int k = i + lane; k < c; k += 32) {
          int zr, zi, rr, ri;
          xld_exp<W, C>(z, n, k, zr, zi);
          xld_exp<W, C>(p.Rm, p.Nnn, (long long)k * n + c, rr, ri);
          dot_exp<false, W, C>(zr, zi, rr, ri, er, ei);
        }
        xfn::xfacc<W> ar, ai;
        const int head = acc_extra_head(C * (c - i));
        xfn::xfacc_init(ar, warp_max(er) + head);
        if constexpr (C == 2) xfn::xfacc_init(ai, warp_max(ei) + head);
        for (int k = i + lane; k < c; k += 32) {
          cxf<W, C> zk, rk;
          xld<W, C>(z, n, k, zk);
          xld<W, C>(p.Rm, p.Nnn, (long long)k * n + c, rk);
          dot_fma<false, QO>(ar, ai, zk, rk);
        }
        cxf<W, C> sum;
        dot_finish(ar, ai, sum);
        cxf_mul<false, QO>(sum, rc, zc);
        cxf_neg(zc);
      }
      if (lane == 0) {
        xst<W, C>(z, n, c, zc);
        cxf_store<K, W, C>(p.Z, p.Nnn, (long long)i * n + c, zc);
      }
      __syncwarp();
    }
  }
}

template <int K, int C>
__global__ void __launch_bounds__(QR_THREADS, 1) qr_kernel(QrParams p) {
  extern __shared__ __align__(16) unsigned char qr_smem[];
  uint64_t* sm = reinterpret_cast<uint64_t*>(qr_smem);
  const int warp = threadIdx.x >> 5;
  const unsigned ep = *p.epoch;
  const int n = p.n;
  const size_t col = (size_t)n * 2 * qr_xf_words(K);
  const int b = blockIdx.x;
  if (b < p.nAc) {
    const int c = b * (QR_THREADS / 32) + warp;
    if (c >= n) return;
    qr_column<K, C>(p, c, sm + warp * col, sm + (QR_THREADS / 32 + warp) * col, ep);
  } else if (b < p.nAc + p.nAi) {
    const int e = (b - p.nAc) * (QR_THREADS / 32) + warp;
    if (e >= n) return;
    qr_identity<K, C>(p, e, sm + warp * col, sm + (QR_THREADS / 32 + warp) * col, ep);
  } else {
    const int g = (b - p.nAc - p.nAi) * (QR_THREADS / 32) + warp;
    if (g > (n - 1) / 2) return;
    qr_rinv_rows<K, C>(p, g, n - 1 - g, sm + 2 * warp * col, sm + (2 * warp + 1) * col, ep);
  }
}

// ---------------------------------------------------------------------------
// The same factorization for large n (beyond what the dataflow kernel keeps
// in shared memory with all its blocks resident): column by column, the
// working columns in global memory, three plain launches per reflector step
// and no flag waits.
//   qrg_init:  Aw = A0 and Yw = I as extended floats (column-major);
//   qrg_pivot(j):  one warp: the pivot scalars of reflector j from column j
//     of Aw (rows j..n-1), the quantities of the dataflow kernel: s_j|x_j|,
//     v_jj, tau_j and 1/R_jj;
//   qrg_apply(j):  a warp per column c > j of Aw and per column of Yw:
//     w = x_j^H y + conj(s_j|x_j|) y_j, then y -= tau_j w v_j (rows j..n-1),
//     which leaves R_jc in row j of column c;
//   qrg_bsub:  a warp per column e of Yw = Q^H: W e_e = R^{-1} Q^H e_e by
//     back substitution, w_i = y_i / R_ii and y_k -= R_ki w_i for k < i,
//     i = n-1..0 (the R entries above the diagonal are in Aw).
// ---------------------------------------------------------------------------
template <int K, int C>
__global__ void qrg_init_kernel(QrParams p) {
  constexpr int W = xfn::xf_words_t<K>::value;
  const int n = p.n;
  const long long nn = (long long)n * n;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nn;
       q += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(q / n), i = (int)(q - (long long)c * n);  // q = c*n + i
    cxf<W, C> v;
    cxf_load<K, W, C>(p.A0, p.NA, (long long)i * n + c, v);
    xst<W, C>(p.Aw, nn, q, v);
    cxf_zero(v);
    if (i == c) xfn::xf_from_double(1.0, v.re);
    xst<W, C>(p.Yw, nn, q, v);
  }
}

template <int K, int C>
__device__ void qrg_pivot(const QrParams& p, int j) {
  using namespace xfn;
  constexpr int W = xf_words_t<K>::value;
  using QO = QOps<W>;
  const int lane = threadIdx.x & 31;
  const int n = p.n;
  const long long nn = (long long)n * n;
  const long long col = (long long)j * n;
  // N = |x_j|^2 over rows j..n-1 (one fixed-point sum)
  int er = 2 * XF_ZERO_E, ei = er;
  for (int i = j + lane; i < n; i += 32) {
    int yr, yi;
    xld_exp<W, C>(p.Aw, nn, col + i, yr, yi);
    dot_exp<true, W, C>(yr, yi, yr, yi, er, ei);
  }
  xfacc<W> acc;
  xfacc_init(acc, warp_max(er) + acc_extra_head(C * (n - j)));
  for (int i = j + lane; i < n; i += 32) {
    cxf<W, C> v;
    xld<W, C>(p.Aw, nn, col + i, v);
    QO::acc_fma(acc, v.re, v.re);
    if constexpr (C == 2) QO::acc_fma(acc, v.im, v.im);
  }
  xfacc_warp_sum(acc);
  xf<W> xN;
  xfacc_get(acc, xN);
  const bool singular = xf_is_zero(xN);
  if (singular) xf_from_double(1.0, xN);  // keep the arithmetic finite; reported below
  // |x| = N / sqrt(N), s = x_jj / |x_jj| (1 if x_jj = 0), v_jj = x_jj + s|x|,
  // tau = 1 / (N + |x| |x_jj|), 1 / R_jj = -conj(s) / |x|
  xf<W> xry, xal, xax0;
  xf_rsqrt<QO>(xN, xry);
  QO::mul(xN, xry, xal);
  cxf<W, C> x0;
  xld<W, C>(p.Aw, nn, col + j, x0);
  xf<W> sre, sim, sgr, sgi;
  bool neg = false;
  if constexpr (C == 1) {
    neg = x0.re.s != 0;
    xax0 = x0.re;
    xax0.s = 0;
    sre = xal;
    if (neg) xf_neg(sre);
    xf_zero(sim);
  } else {
    xf<W> t1, t2, a2x, rx;
    QO::mul(x0.re, x0.re, t1);
    QO::mul(x0.im, x0.im, t2);
    QO::add(t1, t2, a2x);
    const bool z = xf_is_zero(a2x);
    if (z) xf_from_double(1.0, a2x);
    xf_rsqrt<QO>(a2x, rx);
    QO::mul(a2x, rx, xax0);
    QO::mul(x0.re, rx, sgr);
    QO::mul(x0.im, rx, sgi);
    if (z) {
      xf_zero(xax0);
      xf_from_double(1.0, sgr);
      xf_zero(sgi);
    }
    QO::mul(sgr, xal, sre);
    QO::mul(sgi, xal, sim);
  }
  cxf<W, C> sa, v0, rinv;
  sa.re = sre;
  sa.im = sim;
  QO::add(x0.re, sre, v0.re);
  if constexpr (C == 2) QO::add(x0.im, sim, v0.im);
  else xf_zero(v0.im);
  cxf<W, 1> tau;
  xf_zero(tau.im);
  {
    xf<W> t1, t2;
    QO::mul(xal, xax0, t1);
    QO::add(xN, t1, t2);
    xf_recip<QO>(t2, tau.re);
  }
  if constexpr (C == 1) {
    rinv.re = xry;
    if (!neg) xf_neg(rinv.re);
    xf_zero(rinv.im);
  } else {
    QO::mul(sgr, xry, rinv.re);
    xf_neg(rinv.re);
    QO::mul(sgi, xry, rinv.im);
  }
  if (singular) {
    xf_zero(tau.re);
    cxf_zero(rinv);
  }
  if (lane == 0) {
    if (singular) atomicOr(p.status, MDN_DEV_SINGULAR);
    xst<W, C>(p.salpha, p.n, j, sa);
    xst<W, C>(p.v0, p.n, j, v0);
    xst<W, 1>(p.tau, p.n, j, tau);
    xst<W, C>(p.rinv, p.n, j, rinv);
  }
}

template <int K, int C>
__global__ void qrg_pivot_kernel(QrParams p, int j) {
  qrg_pivot<K, C>(p, j);
}

// Reflector j applied to the later columns of Aw and to the columns of Yw.
// Look-ahead: warp 0 takes column j+1 alone and forms the pivot scalars of
// reflector j+1 right after its update, while the other warps update the
// remaining columns; the next launch (reflector j+1) then needs no pivot
// launch of its own.
template <int K, int C>
__global__ void qrg_apply_kernel(QrParams p, int j) {
  using namespace xfn;
  constexpr int W = xf_words_t<K>::value;
  const int lane = threadIdx.x & 31;
  const int n = p.n;
  const long long nn = (long long)n * n;
  const long long xcol = (long long)j * n;
  const int na = n - 1 - j;  // columns j+1..n-1 of Aw, then the n columns of Yw
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  cxf<W, 1> tau;
  xld<W, 1>(p.tau, p.n, j, tau);
  cxf<W, C> sa, v0;
  xld<W, C>(p.salpha, p.n, j, sa);
  xld<W, C>(p.v0, p.n, j, v0);
  const int head = acc_extra_head(C * (n - j));
  // warp 0: column j+1 (t = 0) then the pivot of j+1; the others: t >= 1
  const long long tfirst = (na > 0 && nw > 1) ? (w0 == 0 ? 0 : w0) : w0;
  const long long tstep = (na > 0 && nw > 1) ? (w0 == 0 ? na + n : nw - 1) : nw;
  for (long long t = tfirst; t < na + n; t += tstep) {
    uint64_t* Y = t < na ? p.Aw : p.Yw;
    const long long ycol = (t < na ? (long long)(j + 1 + t) : (long long)(t - na)) * n;
    // dot = x_j^H y over rows j..n-1
    int er = 2 * XF_ZERO_E, ei = er;
    for (int i = j + lane; i < n; i += 32) {
      int xr, xi, yr, yi;
      xld_exp<W, C>(p.Aw, nn, xcol + i, xr, xi);
      xld_exp<W, C>(Y, nn, ycol + i, yr, yi);
      dot_exp<true, W, C>(xr, xi, yr, yi, er, ei);
    }
    xfacc<W> ar, ai;
    xfacc_init(ar, warp_max(er) + head);
    if constexpr (C == 2) xfacc_init(ai, warp_max(ei) + head);
    for (int i = j + lane; i < n; i += 32) {
      cxf<W, C> x, y;
      xld<W, C>(p.Aw, nn, xcol + i, x);
      xld<W, C>(Y, nn, ycol + i, y);
      dot_fma<true>(ar, ai, x, y);
    }
    cxf<W, C> w, yj, ng;
    dot_finish(ar, ai, w);
    xld<W, C>(Y, nn, ycol + j, yj);
    cxf_fma<true>(w, sa, yj);  // w = x^H y + conj(s|x|) y_j = v^H y
    cxf_scale(w, tau.re, ng);
    cxf_neg(ng);
    __syncwarp();
    for (int i = j + lane; i < n; i += 32) {
      cxf<W, C> v, y;
      if (i == j) v = v0;
      else xld<W, C>(p.Aw, nn, xcol + i, v);
      xld<W, C>(Y, nn, ycol + i, y);
      cxf_fma<false>(y, ng, v);
      xst<W, C>(Y, nn, ycol + i, y);
    }
    __syncwarp();
  }
  if (w0 == 0 && na > 0 && nw > 1) qrg_pivot<K, C>(p, j + 1);
}

template <int K, int C>
__global__ void qrg_bsub_kernel(QrParams p) {
  using namespace xfn;
  constexpr int W = xf_words_t<K>::value;
  const int lane = threadIdx.x & 31;
  const int n = p.n;
  const long long nn = (long long)n * n;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long e = w0; e < n; e += nw) {
    const long long ycol = e * n;
    for (int i = n - 1; i >= 0; --i) {
      cxf<W, C> yi, ri, wi;
      xld<W, C>(p.Yw, nn, ycol + i, yi);
      xld<W, C>(p.rinv, p.n, i, ri);
      cxf_mul<false>(yi, ri, wi);
      if (lane == 0) cxf_store<K, W, C>(p.W, p.Nnn, (long long)i * n + e, wi);
      cxf_neg(wi);
      for (int k = lane; k < i; k += 32) {
        cxf<W, C> r, y;
        xld<W, C>(p.Aw, nn, (long long)i * n + k, r);  // R_ki: row k of column i
        xld<W, C>(p.Yw, nn, ycol + k, y);
        cxf_fma<false>(y, r, wi);
        xst<W, C>(p.Yw, nn, ycol + k, y);
      }
      __syncwarp();
    }
  }
}

template <int K, int C>
__device__ __forceinline__ void warp_rowdot(const double* Mp, long long NM, long long row_off, int ms,
                                            const double* xp, long long Nx, int n, int D, int kx, cmd<K, C>& out);

// W = Z Y = R^{-1} Q^H: one warp per entry, lanes over k >= i (Z is upper
// triangular), one fixed-point row product each, over the whole GPU.
template <int K, int C>
__global__ void w_kernel(QrParams p) {
  const int n = p.n;
  const int lane = threadIdx.x & 31;
  const long long nn = (long long)n * n;
  const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = wid; t < nn; t += nw) {
    const int i = (int)(t / n), e = (int)(t - (long long)i * n);
    cmd<K, C> w;  // sum over k >= i of Z_ik Y_ke (Z upper triangular): column e of Y from row i
    warp_rowdot<K, C>(p.Z, p.Nnn, (long long)i * n + i, 1, p.Y + (long long)i * n, p.Nnn, n - i, n, e, w);
    if (lane == 0) st(p.W, p.Nnn, t, w);
  }
}

// ---------------------------------------------------------------------------
// Persistent forward substitution: a dataflow over the d+1 stages.
// Owner warps keep the accumulator of r_k[i] = sgn b_k[i] - sum_{m<k}
// (A_{k-m} dx_m)[i] (level sums stored in place in r) and apply the
// contribution of dx_m as soon as it is published; when the last one
// (m = k-1) is in, r_k[i] is renormalised, stored and counted in rdone[k].
// Solve warps wait for all rows of r_k, form dx_k = W r_k and count the rows
// in xdone[k].  Owners also form the residual r_k - A_0 dx_k of their rows.
// Counters are zeroed before the launch; every wait is bounded.
// ---------------------------------------------------------------------------
// One count for the warp: the warp barrier orders every lane's earlier
// stores before lane 0's release add (cumulative, as in warp_publish), so a
// reader that acquires the count sees them.
__device__ __forceinline__ void warp_count(unsigned* c) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(c) : "memory");
  __syncwarp();
}
__device__ __forceinline__ bool warp_wait_count(const unsigned* c, unsigned target, long long limit_ns, int* status) {
  return warp_wait(c, target, limit_ns, status);
}

template <int K, int C>
__device__ __forceinline__ void ld_acc(const double* p, long long N, long long i, CAcc<K, C>& a) {
  cmd<K, C> v;
  ld(p, N, i, v);
  acc_set(a.re, v.re);
  if constexpr (C == 2) acc_set(a.im, v.im);
}
template <int K, int C>
__device__ __forceinline__ void st_acc(double* p, long long N, long long i, const CAcc<K, C>& a) {
  cmd<K, C> v;
#pragma unroll
  for (int l = 0; l < K; ++l) {
    v.re[l] = a.re.l[l];
    v.im[l] = (C == 2) ? a.im.l[l] : 0.0;
  }
  st(p, N, i, v);
}

// sum_l M[row_off + l*ms] x_l over the warp (a row of a row-major n-by-n
// block for ms = 1, a column for ms = n) with x_l = coefficient kx of
// variable l; all lanes get it.
// For K >= 2 the products are summed in one fixed-point accumulator per
// part (xf.cuh) at a scale set by a warp maximum of the exponent sums, taken
// from the leading limbs (an md value is below 2^(e0+1) for a leading limb
// in [2^e0, 2^(e0+1)); one more bit covers a last-limb carry), so the warp
// sum is an integer sum and the result is rounded to K limbs once.
__device__ __forceinline__ int lead_exp(double x) {
  const int E = (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff);
  return E == 0 ? 2 * xfn::XF_ZERO_E : E - 1023;
}
template <int K, int C>
__device__ __forceinline__ void warp_rowdot(const double* Mp, long long NM, long long row_off, int ms,
                                            const double* xp, long long Nx, int n, int D, int kx, cmd<K, C>& out) {
  const int lane = threadIdx.x & 31;
  if constexpr (K >= 2) {
    constexpr int W = xfn::xf_words_t<K>::value;
    int er = 4 * xfn::XF_ZERO_E, ei = er;
    for (int l = lane; l < n; l += 32) {
      const long long ia = row_off + (long long)l * ms, ix = (long long)l * D + kx;
      const int ar = lead_exp(Mp[ia]), xr = lead_exp(xp[ix]);
      const int ai = C == 2 ? lead_exp(Mp[NM + ia]) : 2 * xfn::XF_ZERO_E;
      const int xi = C == 2 ? lead_exp(xp[Nx + ix]) : 2 * xfn::XF_ZERO_E;
      dot_exp<false, W, C>(ar, ai, xr, xi, er, ei);
    }
    xfn::xfacc<W> acr, aci;
    const int head = acc_extra_head(C * n);
    xfn::xfacc_init(acr, warp_max(er) + 1 + head);
    if constexpr (C == 2) xfn::xfacc_init(aci, warp_max(ei) + 1 + head);
    for (int l = lane; l < n; l += 32) {
      cxf<W, C> a, x;
      cxf_load<K, W, C>(Mp, NM, row_off + (long long)l * ms, a);
      cxf_load<K, W, C>(xp, Nx, (long long)l * D + kx, x);
      dot_fma<false>(acr, aci, a, x);
    }
    cxf<W, C> sum;
    dot_finish(acr, aci, sum);
    xfn::xf_to_md<K, W>(sum.re, out.re);
    if constexpr (C == 2) xfn::xf_to_md<K, W>(sum.im, out.im);
    else md_zero(out.im);
  } else {
    CAcc<K, C> acc;
    cacc_zero(acc);
    for (int l = lane; l < n; l += 32) {
      cmd<K, C> a, x;
      ld(Mp, NM, row_off + (long long)l * ms, a);
      ld(xp, Nx, (long long)l * D + kx, x);
      cacc_fma(acc, a, x);
    }
    warp_sum_acc(acc, out);
  }
}

template <int K, int C>
__global__ void __launch_bounds__(FSUB_THREADS) fsub_kernel(FsubParams p) {
  const int lane = threadIdx.x & 31;
  const int n = p.n, D = p.D;
  const long long nn = (long long)n * n;
  const int wblocks = (p.nW + 3) / 4;
  // transposed blocks: row i of M^T is column i of M; reversed stages: stage
  // k works on coefficient D-1-k of the series
  const int ms = p.transpose ? n : 1;
  auto row = [&](long long base, int i) { return base + (p.transpose ? (long long)i : (long long)i * n); };
  auto co = [&](int k) { return p.reverse ? D - 1 - k : k; };
  if ((int)blockIdx.x < wblocks) {
    // ---- solve warps: dx_k = W r_k ----
    const int w = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (w >= p.nW) return;
    for (int k = p.first_stage; k < p.nst; ++k) {
      if (!warp_wait(&p.rdone[k], (unsigned)n, p.spin_limit, p.status)) return;
      for (int i = w; i < n; i += p.nW) {
        cmd<K, C> s;
        warp_rowdot<K, C>(p.W, p.Nnn, row(0, i), ms, p.r, p.Nx, n, D, co(k), s);
        if (lane == 0) st(p.dx, p.Nx, (long long)i * D + co(k), s);
        warp_count(&p.xdone[k]);
      }
    }
    return;
  }
  // ---- owner warps ----
  const int ow = (blockIdx.x - wblocks) * 4 + (threadIdx.x >> 5);
  if (ow >= p.nOwn) return;
  const long long items = (long long)p.nst * n;
  if (ow >= items) return;  // fewer stages than owner warps (staggered orders)
  // my items q = k*n + i, q = ow, ow + nOwn, ... (increasing k)
  // initialise: acc = sgn * b_k[i]; stage 0 is final at once
  for (long long q = ow; q < items; q += p.nOwn) {
    const int k = (int)(q / n), i = (int)(q - (long long)k * n);
    if (k < p.first_stage) continue;  // r_0 stored by stage0_kernel
    cmd<K, C> b;
    ld(p.rhs, p.Nx, (long long)i * D + co(k), b);
    if (p.rhs_sign < 0) {
      md_neg(b.re, b.re);
      md_neg(b.im, b.im);
    }
    if (lane == 0) st(p.r, p.Nx, (long long)i * D + co(k), b);
    if (k == 0) {
      __syncwarp();
      warp_count(&p.rdone[0]);
    }
  }
  __syncwarp();
  // my items are in increasing k: the last one has the largest
  const long long qlast = ow + ((items - 1 - ow) / p.nOwn) * p.nOwn;
  const int kmax = (int)(qlast / n);
  for (int m = 0; m <= kmax; ++m) {
    if (!warp_wait(&p.xdone[m], (unsigned)n, p.spin_limit, p.status)) return;
    // updates first (the k = m+1 rows are on the critical path), residuals after
    for (long long q = ow; q < items; q += p.nOwn) {
      const int k = (int)(q / n), i = (int)(q - (long long)k * n);
      if (k <= m) continue;
      // r_k[i] -= (A_{k-m} dx_m)[i]
      cmd<K, C> ax;
      if constexpr (K >= 2) {
        if (k >= p.late_stage) {
          // the leading K/2 doubles of A and dx are K/2-limb values (limb
          // index outermost in the layout): the same pointers and strides
          cmd<K / 2, C> h;
          warp_rowdot<K / 2, C>(p.A, p.NA, row((long long)(k - m) * nn, i), ms, p.dx, p.Nx, n, D, co(m), h);
          cmd_zero(ax);
#pragma unroll
          for (int l = 0; l < K / 2; ++l) {
            ax.re[l] = h.re[l];
            ax.im[l] = h.im[l];
          }
        } else {
          warp_rowdot<K, C>(p.A, p.NA, row((long long)(k - m) * nn, i), ms, p.dx, p.Nx, n, D, co(m), ax);
        }
      } else {
        warp_rowdot<K, C>(p.A, p.NA, row((long long)(k - m) * nn, i), ms, p.dx, p.Nx, n, D, co(m), ax);
      }
      CAcc<K, C> a;
      ld_acc(p.r, p.Nx, (long long)i * D + co(k), a);
      cacc_add(a, ax, -1.0);
      if (k == m + 1) {
        cmd<K, C> r;
        cacc_get(a, r);
        if (lane == 0) st(p.r, p.Nx, (long long)i * D + co(k), r);
        __syncwarp();
        warp_count(&p.rdone[k]);
      } else {
        if (lane == 0) st_acc(p.r, p.Nx, (long long)i * D + co(k), a);
        __syncwarp();
      }
    }
    for (long long q = ow; q < items; q += p.nOwn) {
      const int k = (int)(q / n), i = (int)(q - (long long)k * n);
      if (k != m) continue;
      if (p.resmask && !p.resmask[i]) continue;  // a row outside the sampled monitor
      // residual of stage m: r_m[i] - (A_0 dx_m)[i]
      cmd<K, C> ax, r, res;
      warp_rowdot<K, C>(p.A0, p.NA0, row(0, i), ms, p.dx, p.Nx, n, D, co(m), ax);
      ld(p.r, p.Nx, (long long)i * D + co(k), r);
      cmd_sub(r, ax, res);
      if (lane == 0) p.resabs[(long long)i * D + co(m)] = (C == 2) ? hypot(res.re[0], res.im[0]) : fabs(res.re[0]);
    }
  }
}

// Stage 0 alone, one warp per row: r_0 = sgn b_0, dx_0 = W r_0, and the
// constant coefficients of the next series, x_0 + dx_0 (the same md addition
// as the update of x), so that the next step's A_0 and its QR can start early.
template <int K, int C>
__global__ void stage0_kernel(FsubParams p) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n = p.n, D = p.D;
  if (i >= n) return;
  const int c0 = p.reverse ? D - 1 : 0;  // coefficient of stage 0
  cmd<K, C> s;
  warp_rowdot<K, C>(p.W, p.Nnn, p.transpose ? (long long)i : (long long)i * n, p.transpose ? n : 1, p.rhs, p.Nx, n, D,
                    c0, s);
  if (p.rhs_sign < 0) {
    md_neg(s.re, s.re);
    md_neg(s.im, s.im);
  }
  if (lane == 0) {
    cmd<K, C> b;
    ld(p.rhs, p.Nx, (long long)i * D + c0, b);
    if (p.rhs_sign < 0) {
      md_neg(b.re, b.re);
      md_neg(b.im, b.im);
    }
    st(p.r, p.Nx, (long long)i * D + c0, b);
    st(p.dx, p.Nx, (long long)i * D + c0, s);
    if (p.xnext0) {
      cmd<K, C> x0, xn;
      ld(p.x, p.Nx, (long long)i * D, x0);
      cmd_add(x0, s, xn);
      st(p.xnext0, n, i, xn);
    }
  }
  warp_count(&p.xdone[0]);
}

// Stage 0 from the factors, before W = Z Y exists (Newton's pipeline: the
// next step's A_0 and QR then wait for Q^H and R^{-1} only): t = Y (sgn b_0)
// one warp per row, then dx_0 = Z t, Z upper triangular.
template <int K, int C>
__global__ void stage0y_kernel(FsubParams p) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n = p.n, D = p.D;
  if (i >= n) return;
  cmd<K, C> s;  // (Y b_0)_i
  warp_rowdot<K, C>(p.Ys, p.Nnn, (long long)i * n, 1, p.rhs, p.Nx, n, D, 0, s);
  if (lane == 0) {
    cmd<K, C> b;
    ld(p.rhs, p.Nx, (long long)i * D, b);
    if (p.rhs_sign < 0) {
      md_neg(s.re, s.re);
      md_neg(s.im, s.im);
      md_neg(b.re, b.re);
      md_neg(b.im, b.im);
    }
    st(p.r, p.Nx, (long long)i * D, b);
    st(p.t0, n, i, s);
  }
}
template <int K, int C>
__global__ void stage0z_kernel(FsubParams p) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n = p.n, D = p.D;
  if (i >= n) return;
  cmd<K, C> s;  // sum over l >= i of Z_il t0_l (Z upper triangular)
  warp_rowdot<K, C>(p.Zs, p.Nnn, (long long)i * n + i, 1, p.t0 + i, n, n - i, 1, 0, s);
  if (lane == 0) {
    st(p.dx, p.Nx, (long long)i * D, s);
    if (p.xnext0) {
      cmd<K, C> x0, xn;
      ld(p.x, p.Nx, (long long)i * D, x0);
      cmd_add(x0, s, xn);
      st(p.xnext0, n, i, xn);
    }
  }
  warp_count(&p.xdone[0]);
}

// x += dx; per-entry magnitudes of f and dx for the norms of the step.
template <int K, int C>
__global__ void update_kernel(UpdParams p) {
  const long long total = (long long)p.n * p.len;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long id = (q / p.len) * p.D + (q % p.len);
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
// Adjoint of the coefficient series (real data)
// ---------------------------------------------------------------------------
// Lane group g of warp wg takes monomial m = wg*G + g (+ multiples of
// Wtot*G): p_m = prod_v x_v by forward products (ping-pong in its two scratch
// series), then the correlation with lambda of its equation; lane t forms
// coefficients j1 = t (D-t terms) and j2 = D-1-t (t+1 terms), D+1 multiply-
// adds in one loop with the accumulator picked by select.
template <int K, int C>
__global__ void adj_coeff_kernel(AdjParams p) {
  const int lane = threadIdx.x & 31;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (wg >= p.Wtot) return;
  const int D = p.D, P = p.P, G = p.G;
  const int g = lane / P, t = lane - g * P;
  const bool ingroup = g < G;
  for (int base = wg * G; base < p.M; base += p.Wtot * G) {
    const int m = base + g;
    const bool act = ingroup && m < p.M;
    const int k = act ? p.mono_k[m] : 0;
    const int vp = act ? p.mono_vp[m] : 0;
    int kw = k;
#pragma unroll
    for (int off = 16; off; off >>= 1) kw = max(kw, __shfl_xor_sync(FULL, kw, off));
    const long long s0 = ((long long)wg * G + (ingroup ? g : 0)) * 2;
    SP cur{const_cast<double*>(p.x), p.Nx, act ? (long long)p.vidx[vp] * D : 0};
    for (int q = 2; q <= kw; ++q) {
      SP o{p.scratch, p.Ns, (s0 + (q & 1)) * D};
      if (act && q <= k) {
        SP b{const_cast<double*>(p.x), p.Nx, (long long)p.vidx[vp + q - 1] * D};
        series_product<K, C>(cur, b, o, t, D);
        cur = o;
      }
      __syncwarp();
    }
    if (act) {
      const int i = p.mono_eq[m];
      const int j1 = t, j2 = D - 1 - t;
      CAcc<K, C> acc1, acc2;
      cacc_zero(acc1);
      cacc_zero(acc2);
      for (int s = 0; s <= D; ++s) {
        const bool first = s < D - t;
        const int kk = first ? j1 + s : j2 + (s - (D - t));
        const int pj = first ? s : s - (D - t);
        cmd<K, C> lv, pv;
        ld(p.lam, p.Nx, (long long)i * D + kk, lv);
        ld(cur.p, cur.N, cur.off + pj, pv);
        CAcc<K, C> acc;
        cacc_select(first, acc1, acc2, acc);
        cacc_fma(acc, lv, pv);
        cacc_select(first, acc, acc1, acc1);
        cacc_select(first, acc2, acc, acc2);
      }
      cmd<K, C> r1, r2;
      cacc_get(acc1, r1);
      cacc_get(acc2, r2);
      md_neg(r1.re, r1.re);
      md_neg(r1.im, r1.im);
      md_neg(r2.re, r2.re);
      md_neg(r2.im, r2.im);
      st(p.grad, p.Ng, (long long)m * D + j1, r1);
      if (j2 != j1) st(p.grad, p.Ng, (long long)m * D + j2, r2);
    }
    __syncwarp();
  }
}

// L = sum_i x_{i,d}^2 + x_{0,d-1} / x_{0,d} and g = dL/dx (one block; real data,
// D >= 2): 2 x_{i,d} at coefficient d, minus x_{0,d-1} / x_{0,d}^2 for
// variable 0, and 1 / x_{0,d} at its coefficient d-1.
template <int K>
__global__ void fabry_kernel(LossParams p) {
  const int n = p.n, D = p.D, d = D - 1;
  for (long long e = threadIdx.x; e < (long long)n * D; e += blockDim.x) {
    double v[K];
    ld_real(p.x, p.Nx, e, v);
    const bool last = (e % D) == d;
#pragma unroll
    for (int l = 0; l < K; ++l) v[l] = last ? 2.0 * v[l] : 0.0;
    st_real(p.g, p.Nx, e, v);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Acc<K> s;
    acc_zero(s);
    double xd[K], xm[K], ratio[K], inv[K], t[K], g0[K], one[K];
    for (int i = 0; i < n; ++i) {
      ld_real(p.x, p.Nx, (long long)i * D + d, xd);
      acc_fma(s, xd, xd);
    }
    ld_real(p.x, p.Nx, d, xd);
    ld_real(p.x, p.Nx, d - 1, xm);
    md_zero(one);
    one[0] = 1.0;
    md_div(xm, xd, ratio);
    md_recip(xd, inv);
    acc_add(s, ratio, 1.0);
    double L[K];
    acc_get(s, L);
    md_mul(ratio, inv, t);
    ld_real(p.g, p.Nx, d, g0);
    md_sub(g0, t, g0);
    st_real(p.g, p.Nx, d, g0);
    st_real(p.g, p.Nx, d - 1, inv);
#pragma unroll
    for (int l = 0; l < K; ++l) p.loss[l] = L[l];
    (void)one;
  }
}

// ---------------------------------------------------------------------------
// Residual of the block lower triangular Toeplitz system (Eq. (eqToeplitz);
// the residual kernels of Sections 5.4 and 6): entry (i, k) is
//   r_k[i] = b_k[i] - sum_{j=0..k} sum_l A_j[i][l] dx_{k-j}[l],
// one warp per entry.  For K >= 2 the (k+1) n products and b_k[i] are summed
// in one fixed-point accumulator per part at a scale from a warp maximum of
// the leading limbs' exponents (xf.cuh), with headroom for the term count,
// and rounded to K limbs once.
// ---------------------------------------------------------------------------
template <int K, int C>
__global__ void residual_kernel(ResParams p) {
  const int lane = threadIdx.x & 31;
  const int n = p.n, D = p.D;
  const long long nn = (long long)n * n;
  const long long items = (long long)n * D;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long q = w0; q < items; q += nw) {
    const int k = (int)(q / n), i = (int)(q - (long long)k * n);
    const long long terms = (long long)(k + 1) * n;
    cmd<K, C> b, res;
    ld(p.b, p.Nx, (long long)i * D + k, b);
    if constexpr (K >= 2) {
      constexpr int W = xfn::xf_words_t<K>::value;
      int er = lead_exp(b.re[0]);
      int ei = C == 2 ? lead_exp(b.im[0]) : 2 * xfn::XF_ZERO_E;
      for (long long t = lane; t < terms; t += 32) {
        const int j = (int)(t / n), l = (int)(t - (long long)j * n);
        const long long ia = (long long)j * nn + (long long)i * n + l, ix = (long long)l * D + (k - j);
        const int ar = lead_exp(p.A[ia]), xr = lead_exp(p.dx[ix]);
        const int ai = C == 2 ? lead_exp(p.A[p.NA + ia]) : 2 * xfn::XF_ZERO_E;
        const int xi = C == 2 ? lead_exp(p.dx[p.Nx + ix]) : 2 * xfn::XF_ZERO_E;
        dot_exp<false, W, C>(ar, ai, xr, xi, er, ei);
      }
      const int head = acc_extra_head(C * terms + 1);
      xfn::xfacc<W> acr, aci;
      xfn::xfacc_init(acr, warp_max(er) + 1 + head);
      if constexpr (C == 2) xfn::xfacc_init(aci, warp_max(ei) + 1 + head);
      // acc = sum A dx - b (b once, from lane 0); the residual is -acc
      if (lane == 0) {
        xfn::xf<W> one, bx;
        xfn::xf_from_double(1.0, one);
        xfn::xf_from_md<K, W>(b.re, bx);
        xfn::xfacc_fma(acr, bx, one, true);
        if constexpr (C == 2) {
          xfn::xf_from_md<K, W>(b.im, bx);
          xfn::xfacc_fma(aci, bx, one, true);
        }
      }
      for (long long t = lane; t < terms; t += 32) {
        const int j = (int)(t / n), l = (int)(t - (long long)j * n);
        cxf<W, C> a, x;
        cxf_load<K, W, C>(p.A, p.NA, (long long)j * nn + (long long)i * n + l, a);
        cxf_load<K, W, C>(p.dx, p.Nx, (long long)l * D + (k - j), x);
        dot_fma<false>(acr, aci, a, x);
      }
      cxf<W, C> sum;
      dot_finish(acr, aci, sum);
      cxf_neg(sum);
      xfn::xf_to_md<K, W>(sum.re, res.re);
      if constexpr (C == 2) xfn::xf_to_md<K, W>(sum.im, res.im);
      else md_zero(res.im);
    } else {
      CAcc<K, C> acc;
      cacc_zero(acc);
      for (long long t = lane; t < terms; t += 32) {
        const int j = (int)(t / n), l = (int)(t - (long long)j * n);
        cmd<K, C> a, x;
        ld(p.A, p.NA, (long long)j * nn + (long long)i * n + l, a);
        ld(p.dx, p.Nx, (long long)l * D + (k - j), x);
        cacc_fma(acc, a, x);
      }
      cmd<K, C> s;
      warp_sum_acc(acc, s);
      cmd_sub(b, s, res);
    }
    if (lane == 0) {
      if (p.r) st(p.r, p.Nx, (long long)i * D + k, res);
      const bool in = !p.resmask || p.resmask[i];
      p.resabs[(long long)i * D + k] = !in ? 0.0 : (C == 2) ? hypot(res.re[0], res.im[0]) : fabs(res.re[0]);
    }
  }
}

// out = s a for every entry of an md array (md multiplication, the complex
// one for C = 2); s is one md value.
template <int K, int C>
__global__ void scale_kernel(ScaleParams p) {
  cmd<K, C> s;
  ld(p.s, 1, 0, s);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < p.N;
       q += (long long)gridDim.x * blockDim.x) {
    cmd<K, C> a, r;
    ld(p.a, p.N, q, a);
    cmd_mul(s, a, r);
    st(p.out, p.N, q, r);
  }
}

// ---------------------------------------------------------------------------
// launchers of one (K, C) instantiation
// ---------------------------------------------------------------------------
inline int grid_for(long long work, int threads) {
  long long g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 8192) g = 8192;
  return (int)g;
}
template <int K, int C>
cudaError_t launch_adjoint(const AdjParams& p, cudaStream_t s) {
  const int warps = 4;
  adj_coeff_kernel<K, C><<<(p.Wtot + warps - 1) / warps, 32 * warps, 0, s>>>(p);
  return cudaGetLastError();
}
template <int K, int C>
cudaError_t launch_fabry(const LossParams& p, cudaStream_t s) {
  fabry_kernel<K><<<1, 256, 0, s>>>(p);
  return cudaGetLastError();
}
template <int K, int C>
cudaError_t launch_ed(const EdParams& p, int grid, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(ed_kernel<K, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, QR_SMEM_RESERVE);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // the shared memory reservation sets the blocks per SM: one beside the QR
  // blocks that run at the same time on the other SMs (no block shares
  // their SMs), more otherwise
  ed_kernel<K, C><<<grid, ED_THREADS, p.smem > 0 ? p.smem : QR_SMEM_RESERVE, s>>>(p);
  return cudaGetLastError();
}
template <int K, int C>
cudaError_t launch_a0(const A0Params& p, cudaStream_t s) {
  if (p.kmax > 32) a0_partials_warp_kernel<K, C><<<grid_for((long long)p.M * 32, 128), 128, 0, s>>>(p);
  else a0_partials_kernel<K, C><<<(p.nnz + 127) / 128, 128, 0, s>>>(p);
  a0_assemble_kernel<K, C><<<grid_for((long long)p.n * p.n, 128), 128, 0, s>>>(p);
  return cudaGetLastError();
}
template <int K, int C>
int ed_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ed_kernel<K, C>, ED_THREADS, 0) != cudaSuccess) return 0;
  return nb;
}
template <int K, int C>
cudaError_t launch_assemble(const AsmParams& p, bool want_A, cudaStream_t s) {
  assemble_f_kernel<K, C><<<grid_for((long long)p.n * p.len, 128), 128, 0, s>>>(p);
  if (want_A && p.len > p.j_begin)
    assemble_A_kernel<K, C><<<grid_for((long long)p.n * p.n * (p.len - p.j_begin), 128), 128, 0, s>>>(p);
  return cudaGetLastError();
}
// Every QR block reserves most of an SM's shared memory (unused) so that no
// two blocks share an SM: each column warp then has its sub-partition's FP64
// pipe to itself, which sets the length of the sequential column chain.
template <int K, int C>
cudaError_t launch_qr_large(const QrParams& p, cudaStream_t s) {
  const int n = p.n;
  qrg_init_kernel<K, C><<<grid_for((long long)n * n, 256), 256, 0, s>>>(p);
  qrg_pivot_kernel<K, C><<<1, 32, 0, s>>>(p, 0);
  for (int j = 0; j < n; ++j) {
    // a warp per column, at least two warps (the first forms the next pivot)
    const long long cols = (long long)(n - 1 - j) + n + 1;
    qrg_apply_kernel<K, C><<<grid_for(cols * 32, 128), 128, 0, s>>>(p, j);
  }
  qrg_bsub_kernel<K, C><<<(n + 3) / 4, 128, 0, s>>>(p);
  return cudaGetLastError();
}

template <int K, int C>
cudaError_t launch_qr(const QrParams& p, cudaStream_t s) {
  if (p.large) return launch_qr_large<K, C>(p, s);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(qr_kernel<K, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, QR_SMEM_MAX);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  QrParams q = p;
  void* args[] = {(void*)&q};
  // at least the reservation, so that no two QR blocks share an SM
  size_t smem = qr_smem_bytes(p.n, K);
  if (smem < (size_t)QR_SMEM_RESERVE) smem = QR_SMEM_RESERVE;
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)qr_kernel<K, C>, dim3(p.nAc + p.nAi + p.nAz),
                                              dim3(QR_THREADS), args, smem, s);
  if (e != cudaSuccess) return e;
  if (!p.skip_w) w_kernel<K, C><<<grid_for((long long)p.n * p.n * 32, 128), 128, 0, s>>>(q);
  return cudaGetLastError();
}
template <int K, int C>
cudaError_t launch_qr_w(const QrParams& p, cudaStream_t s) {
  w_kernel<K, C><<<grid_for((long long)p.n * p.n * 32, 128), 128, 0, s>>>(p);
  return cudaGetLastError();
}
template <int K, int C>
cudaError_t launch_fsub(const FsubParams& p, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(fsub_kernel<K, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, QR_SMEM_RESERVE);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  FsubParams q = p;
  void* args[] = {(void*)&q};
  const int blocks = (p.nW + 3) / 4 + (p.nOwn + 3) / 4;
  // the shared memory reservation sets the blocks per SM (one: every warp
  // alone on its sub-partition)
  return cudaLaunchCooperativeKernel((const void*)fsub_kernel<K, C>, dim3(blocks), dim3(FSUB_THREADS), args,
                                     p.smem > 0 ? p.smem : QR_SMEM_RESERVE, s);
}
template <int K, int C>
cudaError_t launch_stage0(const FsubParams& p, cudaStream_t s) {
  if (p.Zs) {
    stage0y_kernel<K, C><<<(p.n + 3) / 4, 128, 0, s>>>(p);
    stage0z_kernel<K, C><<<(p.n + 3) / 4, 128, 0, s>>>(p);
    return cudaGetLastError();
  }
  stage0_kernel<K, C><<<(p.n + 3) / 4, 128, 0, s>>>(p);
  return cudaGetLastError();
}
template <int K, int C>
cudaError_t launch_residual(const ResParams& p, cudaStream_t s) {
  residual_kernel<K, C><<<grid_for((long long)p.n * p.D * 32, 128), 128, 0, s>>>(p);
  return cudaGetLastError();
}
template <int K, int C>
cudaError_t launch_scale(const ScaleParams& p, cudaStream_t s) {
  scale_kernel<K, C><<<grid_for(p.N, 128), 128, 0, s>>>(p);
  return cudaGetLastError();
}
template <int K, int C>
cudaError_t launch_update(const UpdParams& p, cudaStream_t s) {
  update_kernel<K, C><<<grid_for((long long)p.n * p.len, 128), 128, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace mdn
