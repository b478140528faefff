// batch.cuh -- many independent systems in one persistent launch.
//
// Every block takes whole systems from a work queue (largest estimated cost
// first) and runs Newton's method on power series (Section 2) on each until
// the stop rule holds or the step cap is reached:
//   1. evaluation and differentiation by forward, backward and cross
//      products of every monomial (Section 5.1), assembled directly into
//      f(x(t)) and the Jacobian series A_j; one warp owns an equation, so its
//      row of every A_j and its f_i are written by that warp alone;
//   2. Householder QR of A_0 (Section 5.3) with one thread per column of A_0
//      and of the identity (Q^H), then W = R^{-1} Q^H by back substitution,
//      one thread per column;
//   3. forward substitution dx_k = W (-f_k - sum_{j=1..k} A_j dx_{k-j})
//      (Section 5.4), each row's sum split over threads;
//   4. x += dx and the norms of the stop rule.
// Stop rule: ||f(x)||_inf <= tol (checked before the update) or
// ||dx||_inf <= tol * max(1, ||x||_inf) (after it); norms of the leading
// doubles.  All coordination inside a block is __syncthreads(); there are no
// waits on other blocks, so every block terminates.
#pragma once
#include "kernels.cuh"

namespace mdn {

// Per-block scratch of one system (all [K][C][N] structure of arrays).
struct BWork {
  double *A, *f, *dx, *Y, *r, *tau, *sa, *v0, *rinv, *part, *scr;
  long long NA, Nf, Nnn, Nn, NT, Ns;
};

__device__ inline BWork batch_carve(double* base, int K, int C, int n, int D, int threads, int S3) {
  const int W = threads / 32, P = (D + 1) / 2, G = 32 / P;
  const long long KC = (long long)K * C;
  BWork w;
  w.NA = (long long)D * n * n;
  w.Nf = (long long)n * D;
  w.Nnn = (long long)n * n;
  w.Nn = n;
  w.NT = threads;
  w.Ns = (long long)W * G * S3 * D;
  double* q = base;
  w.A = q;    q += KC * w.NA;
  w.f = q;    q += KC * w.Nf;
  w.dx = q;   q += KC * w.Nf;
  w.Y = q;    q += KC * w.Nnn;
  w.r = q;    q += KC * n;
  w.tau = q;  q += (long long)K * n;
  w.sa = q;   q += KC * n;
  w.v0 = q;   q += KC * n;
  w.rinv = q; q += KC * n;
  w.part = q; q += KC * threads;
  w.scr = q;
  return w;
}

__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(fabs(v));
}

// ---------------------------------------------------------------------------
// 1. evaluation and differentiation, assembled into f and the A_j
// ---------------------------------------------------------------------------
// Products of a monomial with k variables v_1..v_k and coefficient c, in the
// order one lane group runs them (F_0 = c, B_1 = x_{v_k}):
//   F_q = F_{q-1} x_{v_q}            q = 1..k         (F_k is the value)
//   B_q = B_{q-1} x_{v_{k-q+1}}      q = 2..k-1
//   d_1 = c B_{k-1}                  (k >= 2)
//   d_q = F_{q-1} B_{k-q}            q = 2..k-1
// and d_k = F_{k-1} (no product): 3k-3 products for k >= 2, one for k = 1.
// Shared memory of the evaluation's products in integer limbs (K >= 2): per
// warp its G lane groups' operands, 2 C D extended floats each (G D <= 64).
template <int K, int C>
__host__ __device__ inline size_t batch_smem_bytes(int threads) {
  if (K < 2) return 0;
  return (size_t)(threads / 32) * 2 * C * 64 * sizeof(xfn::xf<xfn::xf_words_t<K>::value>);
}

template <int K, int C>
__device__ void batch_evaluate(const BatchParams& p, const BatchSys& s, const BWork& w, double* f, long long Nf,
                               bool want_A, unsigned char* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int n = s.n, D = s.D;
  const int P = (D + 1) / 2, G = 32 / P;
  const int g = lane / P, t = lane - g * P;
  const bool ingroup = g < G;
  const int km = (p.S3 + 2) / 3;  // largest k the scratch holds
  double* xb = p.x + s.series_off;
  const long long Nx = (long long)n * D;
  const double* cb = p.coeff + s.coeff_off;
  const long long Nc = (long long)s.M * D;
  const double* csb = p.cst + s.series_off;
  const long long slot0 = (long long)(warp * G + (ingroup ? g : 0)) * p.S3;
  auto slot = [&](int i) { return SP{w.scr, w.Ns, (slot0 + i) * D}; };
  for (int i = warp; i < n; i += W) {
    for (int kk = lane; kk < D; kk += 32) {
      cmd<K, C> v;
      ld(csb, Nx, (long long)i * D + kk, v);
      st(f, Nf, (long long)i * D + kk, v);
    }
    if (want_A) {
      cmd<K, C> z;
      cmd_zero(z);
      for (int e = lane; e < D * n; e += 32) {
        const int j = e / n, v = e - j * n;
        st(w.A, w.NA, ((long long)j * n + i) * n + v, z);
      }
    }
    __syncwarp();
    const int q0 = p.eq_ptr[s.eq0 + i], q1 = p.eq_ptr[s.eq0 + i + 1];
    for (int base = q0; base < q1; base += G) {
      const int q = base + g;
      const bool act = ingroup && q < q1;
      const int m = act ? p.eq_mon[q] : 0;
      const int vp = act ? p.vptr[m] : 0;
      const int k = act ? p.vptr[m + 1] - vp : 0;
      const int nprod = !act ? 0 : (k == 1 || !want_A) ? k : 3 * k - 3;
      int npmax = nprod;
#pragma unroll
      for (int off = 16; off; off >>= 1) npmax = max(npmax, __shfl_xor_sync(FULL, npmax, off));
      const SP cf{const_cast<double*>(cb), Nc, (long long)(m - s.mono0) * D};
      auto X = [&](int qv) { return SP{xb, Nx, (long long)p.vidx[vp + qv - 1] * D}; };
      auto F = [&](int qf) { return qf == 0 ? cf : slot(qf - 1); };
      auto B = [&](int qb) { return qb == 1 ? X(k) : slot(km + qb - 2); };
      auto Dp = [&](int qd) { return slot(2 * km - 2 + qd - 1); };
      for (int step = 0; step < npmax; ++step) {
        if (step < nprod) {
          SP a, b, o;
          if (step < k) {
            a = F(step);
            b = X(step + 1);
            o = F(step + 1);
          } else if (step < 2 * k - 2) {
            const int qb = step - k + 2;
            a = B(qb - 1);
            b = X(k - qb + 1);
            o = B(qb);
          } else if (step == 2 * k - 2) {
            a = cf;
            b = B(k - 1);
            o = Dp(1);
          } else {
            const int qd = step - 2 * k + 3;
            a = F(qd - 1);
            b = B(k - qd);
            o = Dp(qd);
          }
          if constexpr (K >= 2) {
            // operands converted once into shared memory, one fixed-point
            // accumulator per coefficient (the evaluation kernel's product)
            using X = xfn::xf<xfn::xf_words_t<K>::value>;
            X* stage = reinterpret_cast<X*>(smem) + (warp * G + g) * (2 * C * D);
            const unsigned gmask = (P >= 32 ? FULL : ((1u << P) - 1u)) << (g * P);
            series_product_xf<K, C>(a, b, o, t, D, gmask, stage);
          } else {
            series_product<K, C>(a, b, o, t, D);
          }
        }
        __syncwarp();
      }
      // the groups add their monomials one after the other (they may share
      // the entries of f_i and of row i of the A_j)
      for (int gg = 0; gg < G; ++gg) {
        if (act && g == gg) {
          const int k1 = t, k2 = D - 1 - t;
          const SP val = F(k);
          for (int r = 0; r < 2; ++r) {
            const int kk = r == 0 ? k1 : k2;
            if (r == 1 && k2 == k1) break;
            cmd<K, C> a, b, c;
            ld(f, Nf, (long long)i * D + kk, a);
            ld(val.p, val.N, val.off + kk, b);
            cmd_add(a, b, c);
            st(f, Nf, (long long)i * D + kk, c);
            if (want_A) {
              for (int qv = 1; qv <= k; ++qv) {
                const SP src = (qv == k) ? F(k - 1) : Dp(qv);
                const int v = p.vidx[vp + qv - 1];
                const long long e = ((long long)kk * n + i) * n + v;
                ld(w.A, w.NA, e, a);
                ld(src.p, src.N, src.off + kk, b);
                cmd_add(a, b, c);
                st(w.A, w.NA, e, c);
              }
            }
          }
        }
        __syncwarp();
      }
    }
  }
}

// ---------------------------------------------------------------------------
// 2. Householder QR of A_0 and W = R^{-1} Q^H
// ---------------------------------------------------------------------------
// Reflector j: H_j = I - tau_j v_j v_j^H with v_j = x_j + s_j |x_j| e_j
// (x_j = rows j..n-1 of column j after H_0..H_{j-1}, s_j = x_jj / |x_jj|,
// +1 for x_jj = 0), tau_j = 1 / (|x_j| (|x_j| + |x_jj|)); H_j x_j =
// -s_j |x_j| e_j.  The entries of v_j below the diagonal stay in A_0.
// Returns false (uniformly over the block) for a zero pivot.
template <int K, int C>
__device__ bool batch_qr(const BWork& w, int n, int* sflag) {
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31;
  const long long NA = w.NA;  // A_0 is slice 0 of A: entry (i, c) at i*n + c
  for (long long e = tid; e < (long long)n * n; e += T) {
    cmd<K, C> v;
    cmd_zero(v);
    if (e / n == e % n) v.re[0] = 1.0;
    st(w.Y, w.Nnn, e, v);
  }
  if (tid == 0) *sflag = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (tid < 32) {
      // |x_j|^2 over rows j..n-1
      CAcc<K, C> ca;
      cacc_zero(ca);
      for (int i = j + lane; i < n; i += 32) {
        cmd<K, C> v;
        ld(w.A, NA, (long long)i * n + j, v);
        acc_fma(ca.re, v.re, v.re);
        if constexpr (C == 2) acc_fma(ca.re, v.im, v.im);
      }
      cmd<K, C> t;
      warp_sum_acc(ca, t);
      double N[K];
      md_copy(t.re, N);
      const bool singular = !nonzero(N[0]);
      if (singular) N[0] = 1.0;
      double ry[K], alpha[K];
      md_rsqrt(N, ry);
      md_mul(N, ry, alpha);
      cmd<K, C> x0, sg, salpha, v0;
      ld(w.A, NA, (long long)j * n + j, x0);
      double ax0[K];
      cmd_zero(sg);
      if constexpr (C == 1) {
        const bool neg = __double_as_longlong(x0.re[0]) < 0;
        sg.re[0] = neg ? -1.0 : 1.0;
#pragma unroll
        for (int l = 0; l < K; ++l) {
          ax0[l] = neg ? -x0.re[l] : x0.re[l];
          salpha.re[l] = neg ? -alpha[l] : alpha[l];
        }
        md_zero(salpha.im);
      } else {
        double a2x[K], rx[K];
        cmd_abs2(x0, a2x);
        const bool z = !nonzero(a2x[0]);
        if (z) a2x[0] = 1.0;
        md_rsqrt(a2x, rx);
        md_mul(a2x, rx, ax0);
        md_mul(x0.re, rx, sg.re);
        md_mul(x0.im, rx, sg.im);
        if (z) {
          md_zero(ax0);
          cmd_zero(sg);
          sg.re[0] = 1.0;
        }
        cmd_scale(sg, alpha, salpha);
      }
      cmd_add(x0, salpha, v0);
      double t1[K], t2[K], tau[K];
      md_mul(alpha, ax0, t1);
      md_add(N, t1, t2);
      md_recip(t2, tau);
      if (singular) md_zero(tau);
      if (lane == 0) {
        st(w.sa, w.Nn, j, salpha);
        st(w.v0, w.Nn, j, v0);
        st_real(w.tau, w.Nn, j, tau);
        if (singular) *sflag = 1;
      }
    }
    __syncthreads();
    // H_j on columns j+1..n-1 of A_0 and on every column of Y
    const int na = n - j - 1;
    cmd<K, C> v0;
    ld(w.v0, w.Nn, j, v0);
    double tau[K];
    ld_real(w.tau, w.Nn, j, tau);
    for (int u = tid; u < na + n; u += T) {
      double* yb = u < na ? w.A : w.Y;
      const long long Ny = u < na ? NA : w.Nnn;
      const int c = u < na ? j + 1 + u : u - na;
      CAcc<K, C> acc;
      cmd<K, C> yj, vi, yi;
      ld(yb, Ny, (long long)j * n + c, yj);
      cacc_zero(acc);
      cacc_fma_conj(acc, v0, yj);
      for (int i = j + 1; i < n; ++i) {
        ld(w.A, NA, (long long)i * n + j, vi);
        ld(yb, Ny, (long long)i * n + c, yi);
        cacc_fma_conj(acc, vi, yi);
      }
      cmd<K, C> wv, gm, ng;
      cacc_get(acc, wv);
      cmd_scale(wv, tau, gm);
      md_neg(gm.re, ng.re);
      md_neg(gm.im, ng.im);
      {
        CAcc<K, C> b;
        cacc_set(b, yj);
        cacc_fma(b, ng, v0);
        cacc_get(b, yj);
        st(yb, Ny, (long long)j * n + c, yj);
      }
      for (int i = j + 1; i < n; ++i) {
        ld(w.A, NA, (long long)i * n + j, vi);
        ld(yb, Ny, (long long)i * n + c, yi);
        CAcc<K, C> b;
        cacc_set(b, yi);
        cacc_fma(b, ng, vi);
        cacc_get(b, yi);
        st(yb, Ny, (long long)i * n + c, yi);
      }
    }
    __syncthreads();
  }
  const bool singular = *sflag != 0;
  // 1 / R_jj = 1 / (-s_j |x_j|)
  for (int j = tid; j < n; j += T) {
    cmd<K, C> sa, r, one, q;
    ld(w.sa, w.Nn, j, sa);
    md_neg(sa.re, r.re);
    md_neg(sa.im, r.im);
    cmd_zero(one);
    one.re[0] = 1.0;
    if (singular) r = one;
    cmd_div(one, r, q);
    st(w.rinv, w.Nn, j, q);
  }
  __syncthreads();
  // W = R^{-1} Y in place, one thread per column: rows from the bottom up
  for (int c = tid; c < n; c += T) {
    for (int i = n - 1; i >= 0; --i) {
      CAcc<K, C> acc;
      cmd<K, C> y, rl, wl, ri;
      ld(w.Y, w.Nnn, (long long)i * n + c, y);
      cacc_set(acc, y);
      for (int l = i + 1; l < n; ++l) {
        ld(w.A, NA, (long long)i * n + l, rl);  // R_il, l > i
        ld(w.Y, w.Nnn, (long long)l * n + c, wl);
        md_neg(rl.re, rl.re);
        md_neg(rl.im, rl.im);
        cacc_fma(acc, rl, wl);
      }
      cacc_get(acc, y);
      ld(w.rinv, w.Nn, i, ri);
      cmd<K, C> out;
      cmd_mul(y, ri, out);
      st(w.Y, w.Nnn, (long long)i * n + c, out);
    }
  }
  __syncthreads();
  return !singular;
}

// ---------------------------------------------------------------------------
// 3. forward substitution
// ---------------------------------------------------------------------------
// One thread's share of a dot product, sum over t < count of sgn a_t x_t
// (pair(t, a, x) loads the t-th pair), in one fixed-point accumulator per
// part at the thread's own scale (a first pass over the leading limbs'
// exponents), rounded to K limbs once (xf.cuh); plain md accumulation for
// K = 1.  With extra != null, -extra is added (once) as well.
template <int K, int C, class Pair>
__device__ __forceinline__ void thread_dot(int count, int first, int step, double sgn, Pair pair,
                                           const cmd<K, C>* extra, cmd<K, C>& out) {
  if constexpr (K >= 2) {
    constexpr int W = xfn::xf_words_t<K>::value;
    int er = 4 * xfn::XF_ZERO_E, ei = er, terms = 0;
    for (int t = first; t < count; t += step) {
      cmd<K, C> a, x;
      pair(t, a, x);
      const int ar = lead_exp(a.re[0]), xr = lead_exp(x.re[0]);
      const int ai = C == 2 ? lead_exp(a.im[0]) : 2 * xfn::XF_ZERO_E;
      const int xi = C == 2 ? lead_exp(x.im[0]) : 2 * xfn::XF_ZERO_E;
      dot_exp<false, W, C>(ar, ai, xr, xi, er, ei);
      ++terms;
    }
    if (extra) {
      er = max(er, lead_exp(extra->re[0]));
      if constexpr (C == 2) ei = max(ei, lead_exp(extra->im[0]));
    }
    const int head = acc_extra_head(C * terms + 1);
    xfn::xfacc<W> acr, aci;
    xfn::xfacc_init(acr, er + 1 + head);
    if constexpr (C == 2) xfn::xfacc_init(aci, ei + 1 + head);
    for (int t = first; t < count; t += step) {
      cmd<K, C> a, x;
      pair(t, a, x);
      cxf<W, C> ax, xx;
      xfn::xf_from_md<K, W>(a.re, ax.re);
      xfn::xf_from_md<K, W>(x.re, xx.re);
      if constexpr (C == 2) {
        xfn::xf_from_md<K, W>(a.im, ax.im);
        xfn::xf_from_md<K, W>(x.im, xx.im);
      } else {
        xfn::xf_zero(ax.im);
        xfn::xf_zero(xx.im);
      }
      if (sgn < 0) cxf_neg(ax);
      dot_fma<false>(acr, aci, ax, xx);
    }
    if (extra) {
      xfn::xf<W> one, e;
      xfn::xf_from_double(1.0, one);
      xfn::xf_from_md<K, W>(extra->re, e);
      xfn::xfacc_fma(acr, e, one, true);
      if constexpr (C == 2) {
        xfn::xf_from_md<K, W>(extra->im, e);
        xfn::xfacc_fma(aci, e, one, true);
      }
    }
    xfn::xf<W> r;
    xfn::xfacc_get(acr, r);
    xfn::xf_to_md<K, W>(r, out.re);
    if constexpr (C == 2) {
      xfn::xfacc_get(aci, r);
      xfn::xf_to_md<K, W>(r, out.im);
    } else {
      md_zero(out.im);
    }
  } else {
    CAcc<K, C> acc;
    cacc_zero(acc);
    for (int t = first; t < count; t += step) {
      cmd<K, C> a, x;
      pair(t, a, x);
      if (sgn < 0) {
        md_neg(a.re, a.re);
        md_neg(a.im, a.im);
      }
      cacc_fma(acc, a, x);
    }
    if (extra) cacc_add(acc, *extra, -1.0);
    cacc_get(acc, out);
  }
}

// Thread tid < n*pp works on row i = tid / pp with share part = tid % pp of
// the terms; partial sums meet in w.part and the first thread of the row
// adds them up.
template <int K, int C>
__device__ void batch_forward(const BWork& w, int n, int D) {
  const int tid = threadIdx.x, T = blockDim.x;
  int pp = T / n;
  if (pp > 32) pp = 32;
  if (pp < 1) pp = 1;
  const int i = tid / pp, part = tid - i * pp;
  const bool rowt = i < n;
  const long long nn = (long long)n * n;
  for (int k = 0; k < D; ++k) {
    // r_k[i] = -f_k[i] - sum_{j=1..k} (A_j dx_{k-j})[i]
    if (rowt) {
      cmd<K, C> fv, v;
      if (part == 0) ld(w.f, w.Nf, (long long)i * D + k, fv);
      thread_dot<K, C>(k * n, part, pp, -1.0,
                       [&](int e, cmd<K, C>& a, cmd<K, C>& x) {
                         const int j = 1 + e / n, l = e - (j - 1) * n;
                         ld(w.A, w.NA, (long long)j * nn + (long long)i * n + l, a);
                         ld(w.dx, w.Nf, (long long)l * D + (k - j), x);
                       },
                       part == 0 ? &fv : nullptr, v);
      st(w.part, w.NT, tid, v);
    }
    __syncthreads();
    if (rowt && part == 0) {
      CAcc<K, C> acc;
      cmd<K, C> v;
      ld(w.part, w.NT, tid, v);
      cacc_set(acc, v);
      for (int q = 1; q < pp; ++q) {
        ld(w.part, w.NT, tid + q, v);
        cacc_add(acc, v);
      }
      cacc_get(acc, v);
      st(w.r, w.Nn, i, v);
    }
    __syncthreads();
    // dx_k[i] = (W r_k)[i]
    if (rowt) {
      cmd<K, C> v;
      thread_dot<K, C>(n, part, pp, 1.0,
                       [&](int l, cmd<K, C>& a, cmd<K, C>& x) {
                         ld(w.Y, w.Nnn, (long long)i * n + l, a);
                         ld(w.r, w.Nn, l, x);
                       },
                       nullptr, v);
      st(w.part, w.NT, tid, v);
    }
    __syncthreads();
    if (rowt && part == 0) {
      CAcc<K, C> acc;
      cmd<K, C> v;
      ld(w.part, w.NT, tid, v);
      cacc_set(acc, v);
      for (int q = 1; q < pp; ++q) {
        ld(w.part, w.NT, tid + q, v);
        cacc_add(acc, v);
      }
      cacc_get(acc, v);
      st(w.dx, w.Nf, (long long)i * D + k, v);
    }
    __syncthreads();
  }
}

template <int K, int C>
__global__ void batch_kernel(BatchParams p) {
  extern __shared__ __align__(16) unsigned char batch_smem[];
  __shared__ int s_sys, s_flag;
  __shared__ unsigned long long s_max[3];
  const int tid = threadIdx.x, T = blockDim.x;
  double* base = p.work + (long long)blockIdx.x * p.work_stride;
  for (;;) {
    if (tid == 0) s_sys = atomicAdd(p.queue, 1);
    __syncthreads();
    const int q = s_sys;
    __syncthreads();
    if (q >= p.count) break;
    const int si = p.order[q];
    const BatchSys s = p.sys[si];
    const BWork w = batch_carve(base, K, C, s.n, s.D, T, p.S3);
    const long long N = (long long)s.n * s.D;
    double* xb = p.x + s.series_off;
    if (p.evaluate_only) {
      batch_evaluate<K, C>(p, s, w, p.f_out + s.series_off, N, false, batch_smem);
      __syncthreads();
      if (tid == 0) {
        p.steps_out[si] = 0;
        p.flags_out[si] = 0;
      }
      continue;
    }
    int flags = 0, steps = 0;
    for (;;) {
      __syncthreads();  // every thread has read the norms of the last step
      if (tid < 3) s_max[tid] = 0ull;
      batch_evaluate<K, C>(p, s, w, w.f, N, true, batch_smem);
      __syncthreads();
      // ||f||_inf, and a non-finite check of f
      unsigned long long fm = 0;
      for (long long e = tid; e < N; e += T) {
        cmd<K, C> v;
        ld(w.f, w.Nf, e, v);
        unsigned long long b = abs_bits(v.re[0]);
        if constexpr (C == 2) b = max(b, abs_bits(v.im[0]));
        fm = max(fm, b);
      }
      atomicMax(&s_max[0], fm);
      __syncthreads();
      const double fnorm = __longlong_as_double((long long)s_max[0]);
      if (!(fnorm <= 1.79e308)) {  // NaN or infinite
        flags |= BATCH_NONFINITE;
        break;
      }
      if (fnorm <= p.tol) {
        flags |= BATCH_CONVERGED;
        break;
      }
      if (steps >= p.max_steps) break;
      if (!batch_qr<K, C>(w, s.n, &s_flag)) {
        flags |= BATCH_SINGULAR;
        break;
      }
      batch_forward<K, C>(w, s.n, s.D);
      // x += dx, ||dx||_inf and ||x||_inf
      unsigned long long dm = 0, xm = 0;
      for (long long e = tid; e < N; e += T) {
        cmd<K, C> x, dx, r;
        ld(xb, N, e, x);
        ld(w.dx, w.Nf, e, dx);
        cmd_add(x, dx, r);
        st(xb, N, e, r);
        unsigned long long b = abs_bits(dx.re[0]), c = abs_bits(r.re[0]);
        if constexpr (C == 2) {
          b = max(b, abs_bits(dx.im[0]));
          c = max(c, abs_bits(r.im[0]));
        }
        dm = max(dm, b);
        xm = max(xm, c);
      }
      atomicMax(&s_max[1], dm);
      atomicMax(&s_max[2], xm);
      __syncthreads();
      ++steps;
      const double dnorm = __longlong_as_double((long long)s_max[1]);
      const double xnorm = __longlong_as_double((long long)s_max[2]);
      if (!(dnorm <= 1.79e308) || !(xnorm <= 1.79e308)) {
        flags |= BATCH_NONFINITE;
        break;
      }
      if (dnorm <= p.tol * fmax(1.0, xnorm)) {
        flags |= BATCH_CONVERGED;
        break;
      }
      if (steps >= p.max_steps) break;
    }
    __syncthreads();
    if (tid == 0) {
      p.steps_out[si] = steps;
      p.flags_out[si] = flags;
    }
  }
}

template <int K, int C>
static cudaError_t batch_smem_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  // the kernel's static shared memory counts against the same per-block
  // limit; larger blocks do not fit (occupancy 0)
  size_t most = batch_smem_bytes<K, C>(1024);
  if (most > (size_t)QR_SMEM_MAX - 1024) most = QR_SMEM_MAX - 1024;
  const cudaError_t e = cudaFuncSetAttribute(batch_kernel<K, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
  if (e == cudaSuccess) done = true;
  return e;
}

template <int K, int C>
cudaError_t launch_batch(const BatchParams& p, int blocks, int threads, cudaStream_t s) {
  cudaError_t e = batch_smem_attr<K, C>();
  if (e != cudaSuccess) return e;
  batch_kernel<K, C><<<blocks, threads, batch_smem_bytes<K, C>(threads), s>>>(p);
  return cudaGetLastError();
}

template <int K, int C>
int batch_occupancy(int threads) {
  int nb = 0;
  if (batch_smem_attr<K, C>() != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<K, C>, threads,
                                                    batch_smem_bytes<K, C>(threads)) != cudaSuccess)
    return 0;
  return nb;
}

template <int K, int C>
const KernelTable* make_table() {
  static const KernelTable t = {K, C, &launch_ed<K, C>, &launch_a0<K, C>, &ed_blocks_per_sm<K, C>, &launch_assemble<K, C>,
                                &launch_qr<K, C>, &launch_qr_w<K, C>, &launch_fsub<K, C>, &launch_stage0<K, C>,
                                &launch_update<K, C>, &launch_adjoint<K, C>, &launch_fabry<K, C>,
                                &launch_batch<K, C>, &batch_occupancy<K, C>, &launch_residual<K, C>,
                                &launch_scale<K, C>};
  return &t;
}

}  // namespace mdn
