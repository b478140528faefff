// md.cuh -- multiple double (md) arithmetic for sm_103a.
//
// A multiple double with K limbs (K = 1 double, 2 double double, 4 quad
// double, 8 octo double) is an unevaluated sum of K nonoverlapping doubles
// (Section 1.2 of Verschelde, arXiv 2301.12659).  Functions take the limbs as
// register arrays (the "sequence of doubles" interface of Section 6.1), so the
// global layout can stay one array per limb (structure of arrays).
//
// Algorithms, from the published literature:
//  * TwoSum: FastTwoSum of Dekker (1971) after ordering the two operands by
//    magnitude; the order is decided by an integer compare of the IEEE bit
//    patterns, so a TwoSum costs 3 FP64 instructions instead of Knuth's 6;
//  * TwoProd: the FMA error-free product p = a*b, e = fma(a, b, -p);
//  * renormalisation: the two passes of Joldes, Muller, Popescu and Tucker
//    ("Arithmetic algorithms for extended precision using floating-point
//    expansions", IEEE TC 2016): VecSum from the least significant term,
//    then a top-down pass that drops zero errors (here branch free);
//  * products and sums: the partial products a_i b_j, i + j = l, belong to
//    "level" l (magnitude ~ 2^(-53 l) |ab|, the grouping of Hida, Li and
//    Bailey's quad double multiplication, 2001).  Levels 0..K-2 are formed
//    exactly (TwoProd) and summed exactly (TwoSum) with every rounding error
//    cascaded one level down; level K-1 (and the i + j = K products) is
//    summed with plain FMA/additions; one renormalisation at the end.
//
// GB300 specifics (measured on this part): an FP64 warp instruction occupies
// the SM sub-partition's FP64 pipe for 64 cycles whatever the number of
// active lanes, an FP64 compare costs more than an add, and 32-bit integer
// instructions run ~38x faster.  Hence every comparison, select and zero test
// here is done on the integer pipe, and all FP64 work is branch free so that
// a warp never issues FP64 instructions for idle lanes.
//
// Error bounds (sloppy semantics, as for the QD library's default add): for
// K limbs, |md_add(a,b) - (a+b)| <= c_K 2^(-53K) (|a| + |b|) and
// |md_mul(a,b) - ab| <= c_K 2^(-53K) |ab| with c_K a small constant (<= 2K^2);
// the reciprocal, the quotient and the square roots to c_K 2^(-53K) relative;
// checked against exact rationals on the GPU through a test-only probe
// kernel (tests/native/md_probe.cu).
#pragma once
#include <cstdint>

namespace mdn {

// ---------------------------------------------------------------------------
// integer-pipe classification
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long mag_bits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ bool nonzero(double x) { return mag_bits(x) != 0ULL; }
__device__ __forceinline__ bool finite_bits(double x) {
  return mag_bits(x) < 0x7ff0000000000000ULL;
}

// ---------------------------------------------------------------------------
// error-free transformations
// ---------------------------------------------------------------------------
// s + e = a + b exactly, s = fl(a + b); requires |a| >= |b|.
__device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e) {
  double x = __dadd_rn(a, b);
  double z = __dsub_rn(x, a);
  e = __dsub_rn(b, z);
  s = x;
}
// s + e = a + b exactly for any a, b: order by magnitude on the integer pipe.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  const bool ge = mag_bits(a) >= mag_bits(b);
  const double hi = ge ? a : b;
  const double lo = ge ? b : a;
  fast_two_sum(hi, lo, s, e);
}
// p + e = a * b exactly (no underflow), p = fl(a * b).
__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
  double x = __dmul_rn(a, b);
  e = __fma_rn(a, b, -x);
  p = x;
}

// ---------------------------------------------------------------------------
// renormalisation of M overlapping terms (roughly decreasing) into K limbs
// ---------------------------------------------------------------------------
template <int M, int K>
__device__ __forceinline__ void renorm(double (&t)[M], double (&r)[K]) {
  double s = t[M - 1];
#pragma unroll
  for (int i = M - 2; i >= 0; --i) two_sum(t[i], s, s, t[i + 1]);
#pragma unroll
  for (int j = 0; j < K; ++j) r[j] = 0.0;
  double carry = s;
  int pos = 0;
#pragma unroll
  for (int i = 1; i < M; ++i) {
    double hi, lo;
    two_sum(carry, t[i], hi, lo);
    const bool emit = nonzero(lo);
#pragma unroll
    for (int j = 0; j < K; ++j) r[j] = (emit && pos == j) ? hi : r[j];
    carry = emit ? lo : hi;
    pos += emit ? 1 : 0;
  }
#pragma unroll
  for (int j = 0; j < K; ++j) r[j] = (pos == j) ? carry : r[j];
}

// ---------------------------------------------------------------------------
// level accumulator: K level sums whose exact total is the running value up
// to the plain additions of level K-1.
// ---------------------------------------------------------------------------
template <int K>
struct Acc {
  double l[K];
};

// Add term t that belongs to level L: exact TwoSum on levels L..K-2, each
// rounding error passed one level down; plain add on level K-1.
template <int K, int L>
__device__ __forceinline__ void cascade(Acc<K>& a, double t) {
#pragma unroll
  for (int m = L; m < K - 1; ++m) two_sum(a.l[m], t, a.l[m], t);
  a.l[K - 1] = __dadd_rn(a.l[K - 1], t);
}

template <int K>
__device__ __forceinline__ void acc_set(Acc<K>& a, const double (&x)[K]) {
#pragma unroll
  for (int i = 0; i < K; ++i) a.l[i] = x[i];
}
template <int K>
__device__ __forceinline__ void acc_zero(Acc<K>& a) {
#pragma unroll
  for (int i = 0; i < K; ++i) a.l[i] = 0.0;
}

namespace detail {
// Helpers with compile-time level indices (recursion instead of loops so the
// level of every term is a constant).
template <int K, int L>
struct AddLimbs {
  __device__ __forceinline__ static void run(Acc<K>& a, const double (&x)[K], double sgn) {
    if constexpr (L < K) {
      cascade<K, (L < K - 1 ? L : K - 1)>(a, sgn * x[L]);
      AddLimbs<K, L + 1>::run(a, x, sgn);
    }
  }
};

// Product terms of a*b of level L (i + j = L), added to the accumulator.
// For L <= K-2: exact TwoProd, hi at level L, lo at level L+1.
// For L == K-1 and L == K: plain FMA into level K-1.
template <int K, int L, int I>
struct ProdLevel {
  __device__ __forceinline__ static void run(Acc<K>& a, const double (&x)[K], const double (&y)[K]) {
    if constexpr (I <= L) {
      constexpr int J = L - I;
      if constexpr (I < K && J < K) {
        if constexpr (L <= K - 2) {
          double p, e;
          two_prod(x[I], y[J], p, e);
          cascade<K, L>(a, p);
          cascade<K, L + 1>(a, e);
        } else {
          a.l[K - 1] = __fma_rn(x[I], y[J], a.l[K - 1]);
        }
      }
      ProdLevel<K, L, I + 1>::run(a, x, y);
    }
  }
};
template <int K, int L>
struct ProdAll {
  __device__ __forceinline__ static void run(Acc<K>& a, const double (&x)[K], const double (&y)[K]) {
    if constexpr (L <= K) {
      ProdLevel<K, L, 0>::run(a, x, y);
      ProdAll<K, L + 1>::run(a, x, y);
    }
  }
};

// Initialise the accumulator with the product a*b: the (0, l) products seed
// the levels, everything else is cascaded.
template <int K, int L>
struct SeedLevels {
  __device__ __forceinline__ static void run(Acc<K>& a, double (&lo)[K], const double (&x)[K],
                                             const double (&y)[K]) {
    if constexpr (L < K - 1) {
      two_prod(x[0], y[L], a.l[L], lo[L]);
      SeedLevels<K, L + 1>::run(a, lo, x, y);
    } else if constexpr (L == K - 1) {
      a.l[K - 1] = __dmul_rn(x[0], y[K - 1]);
    }
  }
};
template <int K, int L, int I>
struct RestLevel {  // products (I, L-I) with I >= 1
  __device__ __forceinline__ static void run(Acc<K>& a, const double (&x)[K], const double (&y)[K]) {
    if constexpr (I <= L) {
      constexpr int J = L - I;
      if constexpr (I < K && J < K) {
        if constexpr (L <= K - 2) {
          double p, e;
          two_prod(x[I], y[J], p, e);
          cascade<K, L>(a, p);
          cascade<K, L + 1>(a, e);
        } else {
          a.l[K - 1] = __fma_rn(x[I], y[J], a.l[K - 1]);
        }
      }
      RestLevel<K, L, I + 1>::run(a, x, y);
    }
  }
};
template <int K, int L>
struct RestAll {
  __device__ __forceinline__ static void run(Acc<K>& a, const double (&lo)[K], const double (&x)[K],
                                             const double (&y)[K]) {
    if constexpr (L <= K) {
      if constexpr (L >= 1 && L - 1 <= K - 2) cascade<K, (L < K - 1 ? L : K - 1)>(a, lo[L - 1]);
      RestLevel<K, L, 1>::run(a, x, y);
      RestAll<K, L + 1>::run(a, lo, x, y);
    }
  }
};
}  // namespace detail

// a.l += sgn * x  (x an md number, limb i at level i)
template <int K>
__device__ __forceinline__ void acc_add(Acc<K>& a, const double (&x)[K], double sgn = 1.0) {
  detail::AddLimbs<K, 0>::run(a, x, sgn);
}
// a.l += b.l (two accumulators: every level of b enters at its level)
template <int K>
__device__ __forceinline__ void acc_add_acc(Acc<K>& a, const Acc<K>& b) {
  detail::AddLimbs<K, 0>::run(a, b.l, 1.0);
}
// a.l += x * y
template <int K>
__device__ __forceinline__ void acc_fma(Acc<K>& a, const double (&x)[K], const double (&y)[K]) {
  if constexpr (K == 1) {
    a.l[0] = __fma_rn(x[0], y[0], a.l[0]);
  } else {
    detail::ProdAll<K, 0>::run(a, x, y);
  }
}
// a.l = x * y (level sums, not renormalised)
template <int K>
__device__ __forceinline__ void acc_mul(Acc<K>& a, const double (&x)[K], const double (&y)[K]) {
  if constexpr (K == 1) {
    a.l[0] = __dmul_rn(x[0], y[0]);
  } else {
    double lo[K];
    detail::SeedLevels<K, 0>::run(a, lo, x, y);
    detail::RestAll<K, 0>::run(a, lo, x, y);
  }
}
// r = renormalised value of the accumulator
template <int K>
__device__ __forceinline__ void acc_get(Acc<K>& a, double (&r)[K]) {
  double t[K];
#pragma unroll
  for (int i = 0; i < K; ++i) t[i] = a.l[i];
  renorm<K, K>(t, r);
}

// ---------------------------------------------------------------------------
// md operations
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void md_zero(double (&r)[K]) {
#pragma unroll
  for (int i = 0; i < K; ++i) r[i] = 0.0;
}
template <int K>
__device__ __forceinline__ void md_copy(const double (&a)[K], double (&r)[K]) {
#pragma unroll
  for (int i = 0; i < K; ++i) r[i] = a[i];
}
template <int K>
__device__ __forceinline__ void md_neg(const double (&a)[K], double (&r)[K]) {
#pragma unroll
  for (int i = 0; i < K; ++i) r[i] = -a[i];
}
template <int K>
__device__ __forceinline__ void md_add(const double (&a)[K], const double (&b)[K], double (&r)[K]) {
  Acc<K> s;
  acc_set(s, a);
  acc_add(s, b, 1.0);
  acc_get(s, r);
}
template <int K>
__device__ __forceinline__ void md_sub(const double (&a)[K], const double (&b)[K], double (&r)[K]) {
  Acc<K> s;
  acc_set(s, a);
  acc_add(s, b, -1.0);
  acc_get(s, r);
}
template <int K>
__device__ __forceinline__ void md_mul(const double (&a)[K], const double (&b)[K], double (&r)[K]) {
  Acc<K> s;
  acc_mul(s, a, b);
  acc_get(s, r);
}
// r = c + a*b
template <int K>
__device__ __forceinline__ void md_fma(const double (&c)[K], const double (&a)[K], const double (&b)[K],
                                       double (&r)[K]) {
  Acc<K> s;
  acc_set(s, c);
  acc_fma(s, a, b);
  acc_get(s, r);
}
// r = a * d for a double d
template <int K>
__device__ __forceinline__ void md_mul_d(const double (&a)[K], double d, double (&r)[K]) {
  double b[K];
  md_zero(b);
  b[0] = d;
  md_mul(a, b, r);
}

// Term t of level L (a runtime value that is constant after unrolling).
template <int K>
__device__ __forceinline__ void cascade_at(Acc<K>& a, int L, double t) {
#pragma unroll
  for (int m = 0; m < K - 1; ++m)
    if (m >= L) two_sum(a.l[m], t, a.l[m], t);
  a.l[K - 1] = __dadd_rn(a.l[K - 1], t);
}

// r = x * y for y with KB <= K limbs (the partial products x_i y_j, j < KB,
// in the same level scheme as md_mul).
template <int K, int KB>
__device__ __forceinline__ void md_mul_part(const double (&x)[K], const double (&y)[KB], double (&r)[K]) {
  if constexpr (KB == K) {
    md_mul(x, y, r);
  } else {
    Acc<K> a;
    double lo[K];
#pragma unroll
    for (int L = 0; L < K; ++L) {  // seeds: x_L y_0 at level L
      if (L <= K - 2) two_prod(x[L], y[0], a.l[L], lo[L]);
      else a.l[K - 1] = __dmul_rn(x[K - 1], y[0]);
    }
#pragma unroll
    for (int L = 0; L <= K - 2; ++L) cascade_at(a, L + 1, lo[L]);
#pragma unroll
    for (int j = 1; j < KB; ++j)
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int L = i + j;
        if (L > K) continue;
        if (L <= K - 2) {
          double p, e;
          two_prod(x[i], y[j], p, e);
          cascade_at(a, L, p);
          cascade_at(a, L + 1, e);
        } else {
          a.l[K - 1] = __fma_rn(x[i], y[j], a.l[K - 1]);
        }
      }
    acc_get(a, r);
  }
}

// y = 1 / b: the reciprocal at K/2 limbs, then one Newton correction
// y = y_h + y_h (1 - b y_h) whose residual is formed at K limbs and whose
// product is formed at K/2 limbs (the residual is ~2^(-53 K/2)), after
// Karp and Markstein ("High-precision division and square root", ACM TOMS
// 1997).  Seed: the correctly rounded double reciprocal.
template <int K>
__device__ __forceinline__ void md_recip(const double (&b)[K], double (&y)[K]) {
  if constexpr (K == 1) {
    y[0] = __drcp_rn(b[0]);
  } else {
    constexpr int H = K / 2;
    double bh[H], yh[H];
#pragma unroll
    for (int l = 0; l < H; ++l) bh[l] = b[l];
    md_recip<H>(bh, yh);
    double p[K], one[K], e[K];
    md_mul_part<K, H>(b, yh, p);
    md_zero(one);
    one[0] = 1.0;
    md_sub(one, p, e);
    double eh[H], corr[H];
#pragma unroll
    for (int l = 0; l < H; ++l) eh[l] = e[l];
    md_mul<H>(yh, eh, corr);
    double t[K];
#pragma unroll
    for (int l = 0; l < H; ++l) {
      t[l] = yh[l];
      t[H + l] = corr[l];
    }
    renorm<K, K>(t, y);
  }
}
// r = a / b = a * (1/b)
template <int K>
__device__ __forceinline__ void md_div(const double (&a)[K], const double (&b)[K], double (&r)[K]) {
  double y[K];
  md_recip(b, y);
  md_mul(a, y, r);
}

// One Newton correction y += y (1 - a y^2) / 2 with every product at K limbs.
template <int K>
__device__ __forceinline__ void md_rsqrt_refine(const double (&a)[K], double (&y)[K]) {
  double q[K], p[K], one[K], e[K], c[K];
  md_mul(a, y, q);
  md_mul(q, y, p);
  md_zero(one);
  one[0] = 1.0;
  md_sub(one, p, e);
#pragma unroll
  for (int l = 0; l < K; ++l) e[l] *= 0.5;  // exact
  md_mul(y, e, c);
  md_add(y, c, y);
}

// y = 1 / sqrt(a), a > 0: the same scheme with y = y_h + y_h (1 - a y_h^2) / 2.
// The seed 1/sqrt in double carries two roundings, and each level squares the
// error of the level below (times 3/2), so the half-width value gets one more
// correction at its own width before the step to K limbs (K >= 4): without
// it the octo double result would keep only about 406 of its 424 bits.
template <int K>
__device__ __forceinline__ void md_rsqrt(const double (&a)[K], double (&y)[K]) {
  if constexpr (K == 1) {
    y[0] = __drcp_rn(__dsqrt_rn(a[0]));
  } else {
    constexpr int H = K / 2;
    double ah[H], yh[H];
#pragma unroll
    for (int l = 0; l < H; ++l) ah[l] = a[l];
    md_rsqrt<H>(ah, yh);
    if constexpr (H >= 2) md_rsqrt_refine<H>(ah, yh);
    double q[K], p[K], one[K], e[K];
    md_mul_part<K, H>(a, yh, q);
    md_mul_part<K, H>(q, yh, p);
    md_zero(one);
    one[0] = 1.0;
    md_sub(one, p, e);
    double eh[H], corr[H];
#pragma unroll
    for (int l = 0; l < H; ++l) eh[l] = 0.5 * e[l];  // exact
    md_mul<H>(yh, eh, corr);
    double t[K];
#pragma unroll
    for (int l = 0; l < H; ++l) {
      t[l] = yh[l];
      t[H + l] = corr[l];
    }
    renorm<K, K>(t, y);
  }
}
// r = sqrt(a) = a / sqrt(a) for a > 0, r = 0 for a = 0
template <int K>
__device__ __forceinline__ void md_sqrt(const double (&a)[K], double (&r)[K]) {
  const bool z = !nonzero(a[0]);
  double aa[K], y[K];
#pragma unroll
  for (int l = 0; l < K; ++l) aa[l] = z ? (l == 0 ? 1.0 : 0.0) : a[l];
  md_rsqrt(aa, y);
  md_mul(aa, y, r);
#pragma unroll
  for (int l = 0; l < K; ++l) r[l] = z ? 0.0 : r[l];
}

// ---------------------------------------------------------------------------
// complex md (C = 2) and real md (C = 1) through one interface
// ---------------------------------------------------------------------------
template <int K, int C>
struct cmd {
  double re[K];
  double im[K];
};

template <int K, int C>
struct CAcc {
  Acc<K> re, im;
};

template <int K, int C>
__device__ __forceinline__ void cmd_zero(cmd<K, C>& r) {
  md_zero(r.re);
  md_zero(r.im);
}

template <int K, int C>
__device__ __forceinline__ void cacc_zero(CAcc<K, C>& a) {
  acc_zero(a.re);
  if constexpr (C == 2) acc_zero(a.im);
}
template <int K, int C>
__device__ __forceinline__ void cacc_set(CAcc<K, C>& a, const cmd<K, C>& x) {
  acc_set(a.re, x.re);
  if constexpr (C == 2) acc_set(a.im, x.im);
}
template <int K, int C>
__device__ __forceinline__ void cacc_add_acc(CAcc<K, C>& a, const CAcc<K, C>& b) {
  acc_add_acc(a.re, b.re);
  if constexpr (C == 2) acc_add_acc(a.im, b.im);
}
template <int K, int C>
__device__ __forceinline__ void cacc_add(CAcc<K, C>& a, const cmd<K, C>& x, double sgn = 1.0) {
  acc_add(a.re, x.re, sgn);
  if constexpr (C == 2) acc_add(a.im, x.im, sgn);
}
// a += x * y (4M complex product: R*R - I*I, R*I + I*R)
template <int K, int C>
__device__ __forceinline__ void cacc_fma(CAcc<K, C>& a, const cmd<K, C>& x, const cmd<K, C>& y) {
  acc_fma(a.re, x.re, y.re);
  if constexpr (C == 2) {
    double nim[K];
    md_neg(x.im, nim);
    acc_fma(a.re, nim, y.im);
    acc_fma(a.im, x.re, y.im);
    acc_fma(a.im, x.im, y.re);
  }
}
// a += conj(x) * y
template <int K, int C>
__device__ __forceinline__ void cacc_fma_conj(CAcc<K, C>& a, const cmd<K, C>& x, const cmd<K, C>& y) {
  acc_fma(a.re, x.re, y.re);
  if constexpr (C == 2) {
    double nim[K];
    md_neg(x.im, nim);
    acc_fma(a.re, x.im, y.im);
    acc_fma(a.im, x.re, y.im);
    acc_fma(a.im, nim, y.re);
  }
}
// a = x * y
template <int K, int C>
__device__ __forceinline__ void cacc_mul(CAcc<K, C>& a, const cmd<K, C>& x, const cmd<K, C>& y) {
  acc_mul(a.re, x.re, y.re);
  if constexpr (C == 2) {
    double nim[K];
    md_neg(x.im, nim);
    acc_fma(a.re, nim, y.im);
    acc_mul(a.im, x.re, y.im);
    acc_fma(a.im, x.im, y.re);
  }
}
template <int K, int C>
__device__ __forceinline__ void cacc_get(CAcc<K, C>& a, cmd<K, C>& r) {
  acc_get(a.re, r.re);
  if constexpr (C == 2) acc_get(a.im, r.im); else md_zero(r.im);
}

template <int K, int C>
__device__ __forceinline__ void cmd_add(const cmd<K, C>& a, const cmd<K, C>& b, cmd<K, C>& r) {
  md_add(a.re, b.re, r.re);
  if constexpr (C == 2) md_add(a.im, b.im, r.im);
}
template <int K, int C>
__device__ __forceinline__ void cmd_sub(const cmd<K, C>& a, const cmd<K, C>& b, cmd<K, C>& r) {
  md_sub(a.re, b.re, r.re);
  if constexpr (C == 2) md_sub(a.im, b.im, r.im);
}
template <int K, int C>
__device__ __forceinline__ void cmd_mul(const cmd<K, C>& a, const cmd<K, C>& b, cmd<K, C>& r) {
  CAcc<K, C> s;
  cacc_mul(s, a, b);
  cacc_get(s, r);
}
// r = a * s for a real md s
template <int K, int C>
__device__ __forceinline__ void cmd_scale(const cmd<K, C>& a, const double (&s)[K], cmd<K, C>& r) {
  md_mul(a.re, s, r.re);
  if constexpr (C == 2) md_mul(a.im, s, r.im); else md_zero(r.im);
}
// |a|^2 as a real md
template <int K, int C>
__device__ __forceinline__ void cmd_abs2(const cmd<K, C>& a, double (&r)[K]) {
  Acc<K> s;
  acc_mul(s, a.re, a.re);
  if constexpr (C == 2) acc_fma(s, a.im, a.im);
  acc_get(s, r);
}
// r = a / b (complex: a conj(b) / |b|^2)
template <int K, int C>
__device__ __forceinline__ void cmd_div(const cmd<K, C>& a, const cmd<K, C>& b, cmd<K, C>& r) {
  if constexpr (C == 1) {
    md_div(a.re, b.re, r.re);
    md_zero(r.im);
  } else {
    double den[K];
    cmd_abs2(b, den);
    CAcc<K, C> s;
    cacc_zero(s);
    cacc_fma_conj(s, b, a);  // conj(b) * a
    cmd<K, C> num;
    cacc_get(s, num);
    md_div(num.re, den, r.re);
    md_div(num.im, den, r.im);
  }
}

}  // namespace mdn
