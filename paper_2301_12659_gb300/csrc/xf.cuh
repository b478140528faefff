// xf.cuh -- extended floats with 64-bit integer limbs, for the scalar chains
// of the multiple double (md) kernels.
//
// On this part an FP64 warp instruction costs 64 cycles in its SM
// sub-partition while a 32-bit integer multiply-add runs 38x faster (the
// measured rates behind md.cuh).  A dependent chain of md operations on one
// warp (the pivot scalars of a Householder reflector: a reciprocal square
// root, a reciprocal, a few products) therefore waits on the FP64 pipe for
// microseconds per operation.  An xf carries the same value with W 64-bit
// words of mantissa and integer exponent and sign, and runs its arithmetic on
// the integer pipe:
//
//   value = (-1)^s * (M / 2^(64W-1)) * 2^e,   M = m[W-1]..m[0], top bit set
//
// (zero: M = 0, e = XF_ZERO_E, s = 0).  W is chosen so that 64W exceeds the
// 53K bits of a K-limb md value by at least 11 bits (xf_words_t<K>), so a
// conversion md -> xf is exact unless gaps between the limbs make them span
// more than 64W bits (then bits below 2^(1-64W) relative are dropped), and
// every xf operation rounds (truncates) far below the md precision:
//   * add/sub: operands aligned with one guard word, so a difference with
//     cancellation is exact; error < 2^(2-64W) relative to the result;
//   * mul: the columns of the 2W-word product below word W-2 are dropped;
//     error < 2^(3-64W) relative;
//   * reciprocal and reciprocal square root: Newton's iterations for 1/a
//     and 1/sqrt(a) (y += y(1 - ay), y += y(1 - ay^2)/2), started from the
//     double precision reciprocal / reciprocal square root of the leading
//     53 bits, each step at the narrowest width that holds the bits it
//     makes correct: both to a few bits short of 64W, at least 53K + 8
//     correct bits;
//   * xf -> md: K times, the leading 53 bits rounded to nearest give a limb
//     and the exact remainder goes on, so the limbs are nonoverlapping with
//     |limb_{l+1}| <= ulp(limb_l)/2.
// Values must stay within the normal double range (no subnormal limbs;
// a limb below 2^-1022 is flushed to zero).  The functions are __host__
// __device__ so that the host build tests them against exact rationals.
#pragma once
#include <cstdint>
#if !defined(__CUDA_ARCH__)
#include <cmath>
#include <cstring>
#endif

#if defined(__CUDACC__)
#define XF_FN __host__ __device__ __forceinline__
#else
#define XF_FN inline
#endif

namespace xfn {

constexpr int XF_ZERO_E = -(1 << 28);

// 64-bit mantissa words of the xf that carries a K-limb md value
XF_FN constexpr int xf_words_of(int K) { return K == 1 ? 1 : K == 2 ? 2 : K == 4 ? 4 : 7; }
template <int K>
struct xf_words_t {
  static constexpr int value = xf_words_of(K);
};

template <int W>
struct xf {
  uint64_t m[W];  // m[W-1] most significant
  int e;
  int s;
};

// ---------------------------------------------------------------------------
// portable word operations
// ---------------------------------------------------------------------------
XF_FN uint64_t umulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}
XF_FN int clz64(uint64_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return __builtin_clzll(x);
#endif
}
XF_FN uint64_t dbits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}
XF_FN double bitsd(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}
XF_FN double drecip(double x) {
#if defined(__CUDA_ARCH__)
  return __drcp_rn(x);
#else
  return 1.0 / x;
#endif
}
XF_FN double drsqrt(double x) {
#if defined(__CUDA_ARCH__)
  return rsqrt(x);
#else
  return 1.0 / std::sqrt(x);
#endif
}
// (hi:lo) >> b for 0 <= b < 64
XF_FN uint64_t fshr(uint64_t lo, uint64_t hi, int b) {
  return b == 0 ? lo : ((lo >> b) | (hi << (64 - b)));
}
// (hi:lo) << b, the high word, for 0 <= b < 64
XF_FN uint64_t fshl(uint64_t lo, uint64_t hi, int b) {
  return b == 0 ? hi : ((hi << b) | (lo >> (64 - b)));
}

// Carry chains.  On the device they are single inline-PTX blocks of add.cc /
// addc.cc, so the carry travels in the condition code from word to word
// (one add per word) instead of being rebuilt from unsigned compares; the
// condition code lives only inside each block.  The first add of a block,
// cin + (2^64 - 1), sets the carry flag to cin (0 or 1); the last one reads
// the carry out of the top word.
#if defined(__CUDACC__)
template <int N>
struct addc_ptx;
template <>
struct addc_ptx<2> {
  static __device__ __forceinline__ uint64_t run(uint64_t (&a)[2], const uint64_t (&b)[2], uint64_t cin) {
    uint64_t cout;
    asm("{\n\t"
        ".reg .u64 t;\n\t"
        "add.cc.u64 t, %5, 0xffffffffffffffff;\n\t"
        "addc.cc.u64 %0, %0, %3;\n\t"
        "addc.cc.u64 %1, %1, %4;\n\t"
        "addc.u64 %2, 0, 0;\n\t"
        "}"
        : "+l"(a[0]), "+l"(a[1]), "=l"(cout)
        : "l"(b[0]), "l"(b[1]), "l"(cin));
    return cout;
  }
};
template <>
struct addc_ptx<3> {
  static __device__ __forceinline__ uint64_t run(uint64_t (&a)[3], const uint64_t (&b)[3], uint64_t cin) {
    uint64_t cout;
    asm("{\n\t"
        ".reg .u64 t;\n\t"
        "add.cc.u64 t, %7, 0xffffffffffffffff;\n\t"
        "addc.cc.u64 %0, %0, %4;\n\t"
        "addc.cc.u64 %1, %1, %5;\n\t"
        "addc.cc.u64 %2, %2, %6;\n\t"
        "addc.u64 %3, 0, 0;\n\t"
        "}"
        : "+l"(a[0]), "+l"(a[1]), "+l"(a[2]), "=l"(cout)
        : "l"(b[0]), "l"(b[1]), "l"(b[2]), "l"(cin));
    return cout;
  }
};
template <>
struct addc_ptx<4> {
  static __device__ __forceinline__ uint64_t run(uint64_t (&a)[4], const uint64_t (&b)[4], uint64_t cin) {
    uint64_t cout;
    asm("{\n\t"
        ".reg .u64 t;\n\t"
        "add.cc.u64 t, %9, 0xffffffffffffffff;\n\t"
        "addc.cc.u64 %0, %0, %5;\n\t"
        "addc.cc.u64 %1, %1, %6;\n\t"
        "addc.cc.u64 %2, %2, %7;\n\t"
        "addc.cc.u64 %3, %3, %8;\n\t"
        "addc.u64 %4, 0, 0;\n\t"
        "}"
        : "+l"(a[0]), "+l"(a[1]), "+l"(a[2]), "+l"(a[3]), "=l"(cout)
        : "l"(b[0]), "l"(b[1]), "l"(b[2]), "l"(b[3]), "l"(cin));
    return cout;
  }
};
template <>
struct addc_ptx<5> {
  static __device__ __forceinline__ uint64_t run(uint64_t (&a)[5], const uint64_t (&b)[5], uint64_t cin) {
    uint64_t cout;
    asm("{\n\t"
        ".reg .u64 t;\n\t"
        "add.cc.u64 t, %11, 0xffffffffffffffff;\n\t"
        "addc.cc.u64 %0, %0, %6;\n\t"
        "addc.cc.u64 %1, %1, %7;\n\t"
        "addc.cc.u64 %2, %2, %8;\n\t"
        "addc.cc.u64 %3, %3, %9;\n\t"
        "addc.cc.u64 %4, %4, %10;\n\t"
        "addc.u64 %5, 0, 0;\n\t"
        "}"
        : "+l"(a[0]), "+l"(a[1]), "+l"(a[2]), "+l"(a[3]), "+l"(a[4]), "=l"(cout)
        : "l"(b[0]), "l"(b[1]), "l"(b[2]), "l"(b[3]), "l"(b[4]), "l"(cin));
    return cout;
  }
};
template <>
struct addc_ptx<6> {
  static __device__ __forceinline__ uint64_t run(uint64_t (&a)[6], const uint64_t (&b)[6], uint64_t cin) {
    uint64_t cout;
    asm("{\n\t"
        ".reg .u64 t;\n\t"
        "add.cc.u64 t, %13, 0xffffffffffffffff;\n\t"
        "addc.cc.u64 %0, %0, %7;\n\t"
        "addc.cc.u64 %1, %1, %8;\n\t"
        "addc.cc.u64 %2, %2, %9;\n\t"
        "addc.cc.u64 %3, %3, %10;\n\t"
        "addc.cc.u64 %4, %4, %11;\n\t"
        "addc.cc.u64 %5, %5, %12;\n\t"
        "addc.u64 %6, 0, 0;\n\t"
        "}"
        : "+l"(a[0]), "+l"(a[1]), "+l"(a[2]), "+l"(a[3]), "+l"(a[4]), "+l"(a[5]), "=l"(cout)
        : "l"(b[0]), "l"(b[1]), "l"(b[2]), "l"(b[3]), "l"(b[4]), "l"(b[5]), "l"(cin));
    return cout;
  }
};
template <>
struct addc_ptx<7> {
  static __device__ __forceinline__ uint64_t run(uint64_t (&a)[7], const uint64_t (&b)[7], uint64_t cin) {
    uint64_t cout;
    asm("{\n\t"
        ".reg .u64 t;\n\t"
        "add.cc.u64 t, %15, 0xffffffffffffffff;\n\t"
        "addc.cc.u64 %0, %0, %8;\n\t"
        "addc.cc.u64 %1, %1, %9;\n\t"
        "addc.cc.u64 %2, %2, %10;\n\t"
        "addc.cc.u64 %3, %3, %11;\n\t"
        "addc.cc.u64 %4, %4, %12;\n\t"
        "addc.cc.u64 %5, %5, %13;\n\t"
        "addc.cc.u64 %6, %6, %14;\n\t"
        "addc.u64 %7, 0, 0;\n\t"
        "}"
        : "+l"(a[0]), "+l"(a[1]), "+l"(a[2]), "+l"(a[3]), "+l"(a[4]), "+l"(a[5]), "+l"(a[6]), "=l"(cout)
        : "l"(b[0]), "l"(b[1]), "l"(b[2]), "l"(b[3]), "l"(b[4]), "l"(b[5]), "l"(b[6]), "l"(cin));
    return cout;
  }
};
template <>
struct addc_ptx<8> {
  static __device__ __forceinline__ uint64_t run(uint64_t (&a)[8], const uint64_t (&b)[8], uint64_t cin) {
    uint64_t cout;
    asm("{\n\t"
        ".reg .u64 t;\n\t"
        "add.cc.u64 t, %17, 0xffffffffffffffff;\n\t"
        "addc.cc.u64 %0, %0, %9;\n\t"
        "addc.cc.u64 %1, %1, %10;\n\t"
        "addc.cc.u64 %2, %2, %11;\n\t"
        "addc.cc.u64 %3, %3, %12;\n\t"
        "addc.cc.u64 %4, %4, %13;\n\t"
        "addc.cc.u64 %5, %5, %14;\n\t"
        "addc.cc.u64 %6, %6, %15;\n\t"
        "addc.cc.u64 %7, %7, %16;\n\t"
        "addc.u64 %8, 0, 0;\n\t"
        "}"
        : "+l"(a[0]), "+l"(a[1]), "+l"(a[2]), "+l"(a[3]), "+l"(a[4]), "+l"(a[5]), "+l"(a[6]), "+l"(a[7]), "=l"(cout)
        : "l"(b[0]), "l"(b[1]), "l"(b[2]), "l"(b[3]), "l"(b[4]), "l"(b[5]), "l"(b[6]), "l"(b[7]), "l"(cin));
    return cout;
  }
};
template <>
struct addc_ptx<9> {
  static __device__ __forceinline__ uint64_t run(uint64_t (&a)[9], const uint64_t (&b)[9], uint64_t cin) {
    uint64_t cout;
    asm("{\n\t"
        ".reg .u64 t;\n\t"
        "add.cc.u64 t, %19, 0xffffffffffffffff;\n\t"
        "addc.cc.u64 %0, %0, %10;\n\t"
        "addc.cc.u64 %1, %1, %11;\n\t"
        "addc.cc.u64 %2, %2, %12;\n\t"
        "addc.cc.u64 %3, %3, %13;\n\t"
        "addc.cc.u64 %4, %4, %14;\n\t"
        "addc.cc.u64 %5, %5, %15;\n\t"
        "addc.cc.u64 %6, %6, %16;\n\t"
        "addc.cc.u64 %7, %7, %17;\n\t"
        "addc.cc.u64 %8, %8, %18;\n\t"
        "addc.u64 %9, 0, 0;\n\t"
        "}"
        : "+l"(a[0]), "+l"(a[1]), "+l"(a[2]), "+l"(a[3]), "+l"(a[4]), "+l"(a[5]), "+l"(a[6]), "+l"(a[7]), "+l"(a[8]), "=l"(cout)
        : "l"(b[0]), "l"(b[1]), "l"(b[2]), "l"(b[3]), "l"(b[4]), "l"(b[5]), "l"(b[6]), "l"(b[7]), "l"(b[8]), "l"(cin));
    return cout;
  }
};

#endif

// a = a + b + cin (mod 2^(64N)), cin in {0, 1}; returns the carry out
template <int N>
XF_FN uint64_t add_words(uint64_t (&a)[N], const uint64_t (&b)[N], uint64_t cin) {
#if defined(__CUDA_ARCH__)
  if constexpr (N >= 2 && N <= 9) return addc_ptx<N>::run(a, b, cin);
#endif
  uint64_t c = cin;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const uint64_t u = a[i] + b[i];
    const uint64_t c1 = u < b[i];
    const uint64_t v = u + c;
    c = c1 | (v < u);
    a[i] = v;
  }
  return c;
}

// (c:s) += v: a word added into a sum s whose carries are counted in c
XF_FN void add_count(uint64_t& s, uint64_t& c, uint64_t v) {
#if defined(__CUDA_ARCH__)
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(s), "+l"(c) : "l"(v));
#else
  s += v;
  c += s < v;
#endif
}

// ---------------------------------------------------------------------------
// mantissa shifts and normalisation
// ---------------------------------------------------------------------------
// r[0..W] = the W-word a shifted right by s >= 0 bits into W+1 words, r[0]
// receiving the first word of bits shifted out (a guard word).
template <int W>
XF_FN void shr_guard(const uint64_t (&a)[W], int s, uint64_t (&r)[W + 1]) {
  uint64_t t[W + 1];
  t[0] = 0;
#pragma unroll
  for (int i = 0; i < W; ++i) t[i + 1] = a[i];
  const int q = s >> 6;
  const int b = s & 63;
#pragma unroll
  for (int st = 1; st <= W; st <<= 1) {
    const bool on = (q & st) != 0;
#pragma unroll
    for (int i = 0; i <= W; ++i) t[i] = on ? (i + st <= W ? t[i + st] : 0ULL) : t[i];
  }
  const bool gone = q > W;
#pragma unroll
  for (int i = 0; i <= W; ++i) {
    const uint64_t v = fshr(t[i], i + 1 <= W ? t[i + 1] : 0ULL, b);
    r[i] = gone ? 0ULL : v;
  }
}

// leading zero bits of the N-word a (64N if zero)
template <int N>
XF_FN int lzcount(const uint64_t (&a)[N]) {
  int lz = 64 * N;
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (a[i] != 0ULL) lz = 64 * (N - 1 - i) + clz64(a[i]);
  return lz;
}

// a <<= s for 0 <= s < 64N (in place)
template <int N>
XF_FN void shl_inplace(uint64_t (&a)[N], int s) {
  const int q = s >> 6;
  const int b = s & 63;
#pragma unroll
  for (int st = 1; st < N; st <<= 1) {
    const bool on = (q & st) != 0;
#pragma unroll
    for (int i = N - 1; i >= 0; --i) a[i] = on ? (i - st >= 0 ? a[i - st] : 0ULL) : a[i];
  }
#pragma unroll
  for (int i = N - 1; i >= 0; --i) a[i] = fshl(i > 0 ? a[i - 1] : 0ULL, a[i], b);
}

template <int W>
XF_FN void xf_zero(xf<W>& r) {
#pragma unroll
  for (int i = 0; i < W; ++i) r.m[i] = 0ULL;
  r.e = XF_ZERO_E;
  r.s = 0;
}
template <int W>
XF_FN bool xf_is_zero(const xf<W>& a) {
  return a.m[W - 1] == 0ULL;
}
template <int W>
XF_FN void xf_neg(xf<W>& a) {
  a.s = xf_is_zero(a) ? 0 : a.s ^ 1;
}

// The W+1-word g, worth G / 2^(64W+63) * 2^e with G = sum g[i] 2^(64i),
// normalised into r (truncated to W words), or zero.
template <int W>
XF_FN void xf_pack(uint64_t (&g)[W + 1], int e, int s, xf<W>& r) {
  const int lz = lzcount<W + 1>(g);
  const bool z = lz >= 64 * (W + 1);
  shl_inplace<W + 1>(g, z ? 0 : lz);
#pragma unroll
  for (int i = 0; i < W; ++i) r.m[i] = z ? 0ULL : g[i + 1];
  r.e = z ? XF_ZERO_E : e - lz;
  r.s = z ? 0 : s;
}

// xf_pack for a g whose leading bit is bit 63 or 62 of its top word (the
// product of two mantissas in [1, 2), or a sum without cancellation): a
// one-bit normalisation instead of the general count and shift.
template <int W>
XF_FN void xf_pack_near(const uint64_t (&g)[W + 1], int e, int s, xf<W>& r) {
  const bool top = (g[W] >> 63) != 0ULL;
#pragma unroll
  for (int i = 0; i < W; ++i) r.m[i] = top ? g[i + 1] : ((g[i + 1] << 1) | (g[i] >> 63));
  r.e = top ? e : e - 1;
  r.s = s;
}

// Whether every lane of the warp (on the host: this value) can take the
// one-bit normalisation: the leading bit of g sits in bit 63 or 62 of its
// top word.  On the device the decision is warp-uniform, so a warp whose
// lanes disagree takes the general path together.
template <int W>
XF_FN bool pack_near_ok(const uint64_t (&g)[W + 1]) {
  const bool near = (g[W] >> 62) != 0ULL;
#if defined(__CUDA_ARCH__)
  return __all_sync(__activemask(), near);
#else
  return near;
#endif
}

// ---------------------------------------------------------------------------
// arithmetic
// ---------------------------------------------------------------------------
// |a| < |b|
template <int W>
XF_FN bool mag_less(const xf<W>& a, const xf<W>& b) {
  bool lt = false, decided = false;
  if (a.e != b.e) {
    lt = a.e < b.e;
    decided = true;
  }
#pragma unroll
  for (int i = W - 1; i >= 0; --i) {
    if (!decided && a.m[i] != b.m[i]) {
      lt = a.m[i] < b.m[i];
      decided = true;
    }
  }
  return lt;
}

template <int W>
XF_FN void xf_add(const xf<W>& a, const xf<W>& b, xf<W>& r) {
  const bool sw = mag_less(a, b);
  const xf<W>& x = sw ? b : a;  // larger magnitude
  const xf<W>& y = sw ? a : b;
  const int d = x.e - y.e;  // >= 0 (zero has the least exponent)
  uint64_t ys[W + 1];
  shr_guard<W>(y.m, d, ys);
  uint64_t g[W + 2];
  if (x.s == y.s) {
    uint64_t t[W], u[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
      t[i] = x.m[i];
      u[i] = ys[i + 1];
    }
    g[0] = ys[0];
    g[W + 1] = add_words<W>(t, u, 0ULL);
#pragma unroll
    for (int i = 0; i < W; ++i) g[i + 1] = t[i];
  } else {
    // (x.m with a zero guard word) - ys = (x.m : 0) + ~ys + 1; no borrow
    // since |x| >= |y|
    uint64_t t[W + 1], u[W + 1];
    t[0] = 0ULL;
#pragma unroll
    for (int i = 0; i < W; ++i) t[i + 1] = x.m[i];
#pragma unroll
    for (int i = 0; i <= W; ++i) u[i] = ~ys[i];
    add_words<W + 1>(t, u, 1ULL);
#pragma unroll
    for (int i = 0; i <= W; ++i) g[i] = t[i];
    g[W + 1] = 0ULL;
  }
  // g (W+2 words) has its leading bit at 64(W+1) or below; the value is
  // g / 2^(64W+63) * 2^(x.e) with the top bit of word W+1 worth 2^(x.e+1)
  uint64_t h[W + 1];
  const bool carry = g[W + 1] != 0ULL;
#pragma unroll
  for (int i = 0; i <= W; ++i) h[i] = carry ? fshr(g[i], g[i + 1], 1) : g[i];
  // a sum of like signs, and a difference that cancels at most one bit, has
  // its leading bit in bit 63 or 62 of h[W]
  if (pack_near_ok<W>(h)) xf_pack_near<W>(h, x.e + (carry ? 1 : 0), x.s, r);
  else xf_pack<W>(h, x.e + (carry ? 1 : 0), x.s, r);
}

template <int W>
XF_FN void xf_sub(const xf<W>& a, const xf<W>& b, xf<W>& r) {
  xf<W> nb = b;
  xf_neg(nb);
  xf_add(a, nb, r);
}

// The top W+1 words of the product of the mantissas of a and b, worth
// H / 2^(64W+63) * 2^(a.e + b.e + 1): the columns W-2 .. 2W-1 of the
// 2W-word product (column k weighs 2^(64k)); the products landing below
// column W-2 are dropped.
template <int W>
XF_FN void xf_mul_core(const xf<W>& a, const xf<W>& b, uint64_t (&h)[W + 1]) {
  uint64_t carry = 0;
#pragma unroll
  for (int k = W - 2; k <= 2 * W - 1; ++k) {
    uint64_t s = carry, c = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const int j = k - i;
      if (j >= 0 && j < W) add_count(s, c, a.m[i] * b.m[j]);
      const int jh = k - 1 - i;
      if (jh >= 0 && jh < W && k - 1 >= W - 2) add_count(s, c, umulhi(a.m[i], b.m[jh]));
    }
    if (k >= W - 1) h[k - (W - 1)] = s;
    carry = c;
  }
}

template <int W>
XF_FN void xf_mul(const xf<W>& a, const xf<W>& b, xf<W>& r) {
  // the product of two mantissas in [1, 2) is in [1, 4): its leading bit is
  // bit 63 or 62 of the top word
  uint64_t h[W + 1];
  xf_mul_core(a, b, h);
  const bool z = xf_is_zero(a) || xf_is_zero(b);
  if (z) {
    xf_zero(r);
    return;
  }
  xf_pack_near<W>(h, a.e + b.e + 1, a.s ^ b.s, r);
}

// r = a >> s for s >= 0 (N words, truncated; s >= 64N gives zero)
template <int N>
XF_FN void shr_words(const uint64_t (&a)[N], int s, uint64_t (&r)[N]) {
  const int q = s >> 6;
  const int b = s & 63;
#pragma unroll
  for (int i = 0; i < N; ++i) r[i] = a[i];
#pragma unroll
  for (int st = 1; st < N; st <<= 1) {
    const bool on = (q & st) != 0;
#pragma unroll
    for (int i = 0; i < N; ++i) r[i] = on ? (i + st < N ? r[i + st] : 0ULL) : r[i];
  }
  const bool gone = q >= N;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const uint64_t v = fshr(r[i], i + 1 < N ? r[i + 1] : 0ULL, b);
    r[i] = gone ? 0ULL : v;
  }
}

// ---------------------------------------------------------------------------
// fixed-point accumulation of products (dot products, convolutions)
// ---------------------------------------------------------------------------
// A sum of fewer than XF_ACC_TERMS products a_i b_i in a two's complement
// integer T of W+2 words, worth T / 2^(64W+63) * 2^E.  E is fixed before the
// first product from the largest exponent sum e_max = max(a_i.e + b_i.e):
// E = e_max + 1 + XF_ACC_HEAD, so every product (< 2^(e_max+2)) enters
// below 2^(64W+64-XF_ACC_HEAD) with a right shift of at least XF_ACC_HEAD
// bits, and the magnitude of the sum stays below 2^(64W+64) (W+1 words).
// The sum is exact but for the bits shifted out below the W+1 words, so its
// error is below (terms) 2^(XF_ACC_HEAD+1-64(W+1)) times the largest term:
// the accuracy of an md dot product (error relative to the sum of
// magnitudes), with 64 - XF_ACC_HEAD bits to spare.
constexpr int XF_ACC_HEAD = 9;
constexpr int XF_ACC_TERMS = 1 << XF_ACC_HEAD;

template <int W>
struct xfacc {
  uint64_t w[W + 2];
  int E;
};

template <int W>
XF_FN void xfacc_init(xfacc<W>& a, int e_max) {
#pragma unroll
  for (int i = 0; i < W + 2; ++i) a.w[i] = 0ULL;
  a.E = e_max + 1 + XF_ACC_HEAD;
}

// the exponent sum that xfacc_init wants for the product x y (very negative
// when either is zero)
template <int W>
XF_FN int xf_prod_exp(const xf<W>& x, const xf<W>& y) {
  return x.e + y.e;
}

// a += x y (neg: a -= x y)
template <int W>
XF_FN void xfacc_fma(xfacc<W>& a, const xf<W>& x, const xf<W>& y, bool neg = false) {
  uint64_t h[W + 1], r[W + 1];
  xf_mul_core(x, y, h);
  const bool z = xf_is_zero(x) || xf_is_zero(y);
  const int d = a.E - (x.e + y.e + 1);
  shr_words<W + 1>(h, z ? 64 * (W + 1) : d, r);
  const uint64_t mask = ((x.s ^ y.s) != 0) != neg ? ~0ULL : 0ULL;
  // a.w += (r, sign-extended to W+2 words, negated in two's complement
  // when mask is set)
  uint64_t yv[W + 2];
#pragma unroll
  for (int i = 0; i <= W; ++i) yv[i] = r[i] ^ mask;
  yv[W + 1] = mask;
  add_words<W + 2>(a.w, yv, mask & 1ULL);
}

// ---------------------------------------------------------------------------
// inline or out-of-line calls of the basic operations
// ---------------------------------------------------------------------------
// Every inlined operation is a new copy of its code (a few hundred
// instructions at W = 4).  Code that one warp runs once per value, such as
// the pivot scalars of a Householder reflector, is then bound by
// instruction fetch: its copies are not in the instruction cache the next
// time they run.  Called out of line, one copy per width serves every call
// site and stays cached.  Arguments and results go by value, in registers.
// xf_ops_inline suits throughput code (independent operations interleave);
// xf_ops_call suits latency-bound chains on one warp.
#if defined(__CUDACC__)
template <int W>
__device__ __noinline__ xf<W> xf_mul_ol(const xf<W> a, const xf<W> b) {
  xf<W> r;
  xf_mul(a, b, r);
  return r;
}
template <int W>
__device__ __noinline__ xf<W> xf_add_ol(const xf<W> a, const xf<W> b) {
  xf<W> r;
  xf_add(a, b, r);
  return r;
}
template <int W>
__device__ __noinline__ xf<W> xf_sub_ol(const xf<W> a, const xf<W> b) {
  xf<W> r;
  xf_sub(a, b, r);
  return r;
}
template <int W>
__device__ __noinline__ xfacc<W> xfacc_fma_ol(xfacc<W> acc, const xf<W> x, const xf<W> y, const bool neg) {
  xfacc_fma(acc, x, y, neg);
  return acc;
}
#endif

struct xf_ops_inline {
  static constexpr bool call = false;
  template <int W>
  static XF_FN void mul(const xf<W>& a, const xf<W>& b, xf<W>& r) { xf_mul(a, b, r); }
  template <int W>
  static XF_FN void add(const xf<W>& a, const xf<W>& b, xf<W>& r) { xf_add(a, b, r); }
  template <int W>
  static XF_FN void sub(const xf<W>& a, const xf<W>& b, xf<W>& r) { xf_sub(a, b, r); }
  template <int W>
  static XF_FN void acc_fma(xfacc<W>& acc, const xf<W>& x, const xf<W>& y, bool neg = false) {
    xfacc_fma(acc, x, y, neg);
  }
};

struct xf_ops_call {
  static constexpr bool call = true;
#if defined(__CUDA_ARCH__)
  template <int W>
  static __device__ __forceinline__ void mul(const xf<W>& a, const xf<W>& b, xf<W>& r) { r = xf_mul_ol<W>(a, b); }
  template <int W>
  static __device__ __forceinline__ void add(const xf<W>& a, const xf<W>& b, xf<W>& r) { r = xf_add_ol<W>(a, b); }
  template <int W>
  static __device__ __forceinline__ void sub(const xf<W>& a, const xf<W>& b, xf<W>& r) { r = xf_sub_ol<W>(a, b); }
  template <int W>
  static __device__ __forceinline__ void acc_fma(xfacc<W>& acc, const xf<W>& x, const xf<W>& y, bool neg = false) {
    acc = xfacc_fma_ol<W>(acc, x, y, neg);
  }
#else
  template <int W>
  static XF_FN void mul(const xf<W>& a, const xf<W>& b, xf<W>& r) { xf_mul(a, b, r); }
  template <int W>
  static XF_FN void add(const xf<W>& a, const xf<W>& b, xf<W>& r) { xf_add(a, b, r); }
  template <int W>
  static XF_FN void sub(const xf<W>& a, const xf<W>& b, xf<W>& r) { xf_sub(a, b, r); }
  template <int W>
  static XF_FN void acc_fma(xfacc<W>& acc, const xf<W>& x, const xf<W>& y, bool neg = false) {
    xfacc_fma(acc, x, y, neg);
  }
#endif
};

template <int W>
XF_FN void xfacc_get(const xfacc<W>& a, xf<W>& r) {
  const bool neg = (a.w[W + 1] >> 63) != 0ULL;
  uint64_t g[W + 1];
  uint64_t c = neg ? 1ULL : 0ULL;
  const uint64_t mask = neg ? ~0ULL : 0ULL;
#pragma unroll
  for (int i = 0; i <= W; ++i) {
    const uint64_t v = (a.w[i] ^ mask) + c;
    c = (c != 0ULL && v == 0ULL) ? 1ULL : 0ULL;
    g[i] = v;
  }
  xf_pack<W>(g, a.E, neg ? 1 : 0, r);
}

template <int W>
XF_FN void xf_mul_pow2(xf<W>& a, int k) {
  a.e = xf_is_zero(a) ? XF_ZERO_E : a.e + k;
}

// ---------------------------------------------------------------------------
// conversions
// ---------------------------------------------------------------------------
template <int W>
XF_FN void xf_from_double(double x, xf<W>& r) {
  const uint64_t b = dbits(x);
  const int E = (int)((b >> 52) & 0x7ff);
  const bool z = E == 0;  // zero (subnormals are flushed)
#pragma unroll
  for (int i = 0; i < W - 1; ++i) r.m[i] = 0ULL;
  r.m[W - 1] = z ? 0ULL : (((b & 0xfffffffffffffULL) | 0x10000000000000ULL) << 11);
  r.e = z ? XF_ZERO_E : E - 1023;
  r.s = z ? 0 : (int)(b >> 63);
}

// md -> xf: limb 0 fixes the sign and exponent; each lower limb is added
// (same sign) or subtracted (opposite sign) at its offset below limb 0 in
// a fixed-point number of W+2 words (a guard word below the mantissa and a
// carry word above), which stays positive because limb 0 dominates the sum
// of the others; one normalisation at the end.
template <int K, int W>
XF_FN void xf_from_md(const double (&a)[K], xf<W>& r) {
  const uint64_t b0 = dbits(a[0]);
  const int E0 = (int)((b0 >> 52) & 0x7ff);
  if (E0 == 0) {
    xf_zero(r);
    return;
  }
  uint64_t g[W + 2];
#pragma unroll
  for (int i = 0; i < W; ++i) g[i] = 0ULL;
  g[W] = ((b0 & 0xfffffffffffffULL) | 0x10000000000000ULL) << 11;
  g[W + 1] = 0ULL;
  const uint64_t s0 = b0 >> 63;
#pragma unroll
  for (int l = 1; l < K; ++l) {
    const uint64_t bl = dbits(a[l]);
    const int El = (int)((bl >> 52) & 0x7ff);
    uint64_t top[W];
#pragma unroll
    for (int i = 0; i < W - 1; ++i) top[i] = 0ULL;
    top[W - 1] = El == 0 ? 0ULL : (((bl & 0xfffffffffffffULL) | 0x10000000000000ULL) << 11);
    uint64_t ys[W + 1];
    shr_guard<W>(top, E0 - El, ys);
    const uint64_t mask = ((bl >> 63) ^ s0) ? ~0ULL : 0ULL;
    uint64_t yv[W + 2];
#pragma unroll
    for (int i = 0; i <= W; ++i) yv[i] = ys[i] ^ mask;
    yv[W + 1] = mask;
    add_words<W + 2>(g, yv, mask & 1ULL);
  }
  uint64_t h[W + 1];
  const bool carry = g[W + 1] != 0ULL;
#pragma unroll
  for (int i = 0; i <= W; ++i) h[i] = carry ? fshr(g[i], g[i + 1], 1) : g[i];
  xf_pack<W>(h, E0 - 1023 + (carry ? 1 : 0), (int)s0, r);
}

// the leading limb: the 53 leading bits rounded to nearest, as a double, and
// the exact remainder a - limb.
template <int W>
XF_FN double xf_take_limb(xf<W>& a) {
  if (xf_is_zero(a)) return 0.0;
  const uint64_t top = a.m[W - 1];
  const uint64_t up = (top >> 10) & 1ULL;
  uint64_t mant = (top >> 11) + up;
  int e = a.e;
  const bool ovf = mant == (1ULL << 53);
  mant = ovf ? (1ULL << 52) : mant;
  e += ovf ? 1 : 0;
  const bool flush = e < -1022;
  const double limb = flush ? 0.0
                            : bitsd(((uint64_t)a.s << 63) | ((uint64_t)(e + 1023) << 52) |
                                    (mant & 0xfffffffffffffULL));
  if (flush) {
    xf_zero(a);
    return 0.0;
  }
  // remainder: the bits below the 53 leading ones, minus 2^(64W-53) if
  // rounded up (then of the opposite sign)
  uint64_t g[W + 1];
  g[0] = 0ULL;
#pragma unroll
  for (int i = 0; i < W; ++i) g[i + 1] = a.m[i];
  g[W] &= (1ULL << 11) - 1ULL;
  if (up) {
    uint64_t c = 1;
#pragma unroll
    for (int i = 0; i <= W; ++i) {
      const uint64_t v = ~g[i] + c;
      c = (c != 0ULL && v == 0ULL) ? 1ULL : 0ULL;
      g[i] = v;
    }
    g[W] &= (1ULL << 11) - 1ULL;
  }
  xf_pack<W>(g, a.e, up ? a.s ^ 1 : a.s, a);
  return limb;
}

template <int K, int W>
XF_FN void xf_to_md(const xf<W>& a, double (&r)[K]) {
  xf<W> t = a;
#pragma unroll
  for (int l = 0; l < K; ++l) r[l] = xf_take_limb(t);
}

// the double nearest to the leading 53 bits of a mantissa in [1, 2)
template <int W>
XF_FN double xf_mant_double(const xf<W>& a) {
  const uint64_t top = a.m[W - 1];
  return bitsd((1023ULL << 52) | ((top >> 11) & 0xfffffffffffffULL));
}

// ---------------------------------------------------------------------------
// reciprocal and reciprocal square root: Newton's iteration in fixed point
// ---------------------------------------------------------------------------
// Columns LO .. NA+NB-1 of the product of the NA-word a and the NB-word b
// (column k weighs 2^(64k)) into out[0 .. NA+NB-1-LO].  Below column LO only
// the products of column LO-1 enter (their high halves, and the carry of
// their low halves), so out[0] may fall short of the exact column by fewer
// than NA + NB units.
template <int NA, int NB, int LO>
XF_FN void mul_top(const uint64_t (&a)[NA], const uint64_t (&b)[NB], uint64_t (&out)[NA + NB - LO]) {
  uint64_t carry = 0;
#pragma unroll
  for (int k = LO - 1; k <= NA + NB - 1; ++k) {
    uint64_t s = carry, c = 0;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const int j = k - i;
      if (j >= 0 && j < NB) add_count(s, c, a[i] * b[j]);
      const int jh = k - 1 - i;
      if (k > LO - 1 && jh >= 0 && jh < NB) add_count(s, c, umulhi(a[i], b[jh]));
    }
    if (k >= LO) out[k - LO] = s;
    carry = c;
  }
}

// Y += sgn C over N words, sgn = -1 when neg (two's complement, no
// branch).  A sum that reaches 2^(64N) (y = 1 - ulp, the leading words of m
// exactly 1, so that the iteration heads for 1 itself) stays at 2^(64N) - 1.
template <int N>
XF_FN void add_signed(uint64_t (&Y)[N], const uint64_t (&C)[N], bool neg) {
  const uint64_t mask = neg ? ~0ULL : 0ULL;
  uint64_t t[N];
#pragma unroll
  for (int i = 0; i < N; ++i) t[i] = C[i] ^ mask;
  const uint64_t cy = add_words<N>(Y, t, mask & 1ULL);
  const uint64_t sat = (!neg && cy != 0ULL) ? ~0ULL : 0ULL;
#pragma unroll
  for (int i = 0; i < N; ++i) Y[i] |= sat;
}

// D = 2^(64V+63+sh) - P over V+1 words (two's complement), then |D| in
// place; returns whether D < 0.  sh = 0 or -1.
template <int V>
XF_FN bool newton_residual(const uint64_t (&P)[V + 1], int sh, uint64_t (&D)[V + 1]) {
  uint64_t one[V + 1];
#pragma unroll
  for (int i = 0; i <= V; ++i) {
    D[i] = ~P[i];
    one[i] = 0ULL;
  }
  one[V] = sh == 0 ? (1ULL << 63) : (1ULL << 62);
  add_words<V + 1>(D, one, 1ULL);  // 2^(...) + ~P + 1 = 2^(...) - P
  const bool neg = (D[V] >> 63) != 0ULL;
  const uint64_t mask = neg ? ~0ULL : 0ULL;
  uint64_t z[V + 1];
#pragma unroll
  for (int i = 0; i <= V; ++i) {
    D[i] ^= mask;
    z[i] = 0ULL;
  }
  add_words<V + 1>(D, z, mask & 1ULL);
  return neg;
}

// One Newton step for y = 1/m at width V:  m = A / 2^(64V-1) in [1, 2) (A:
// the leading V words of the mantissa), y = Y / 2^(64V) in (1/2, 1);
//   D = 1 - m y (a signed fixed-point number, small),  y += y D.
// With k correct bits in y, |D| < 2^(1-k) and the step leaves about 2k
// (up to the 64V of the width): the products are formed to the words
// that the result keeps.
template <int V>
XF_FN void recip_fx_step(const uint64_t (&A)[V], uint64_t (&Y)[V]) {
  uint64_t P[V + 1], D[V + 1], U[V + 1], C[V];
  mul_top<V, V, V - 1>(A, Y, P);  // m y = P / 2^(64V+63)
  const bool neg = newton_residual<V>(P, 0, D);
  mul_top<V, V + 1, V>(Y, D, U);  // y |D| = (U / 2^63) / 2^(64V)
#pragma unroll
  for (int i = 0; i < V; ++i) C[i] = (U[i] >> 63) | (U[i + 1] << 1);
  add_signed<V>(Y, C, neg);
}

// One Newton step for y = 1/sqrt(m) at width V:  m = A / 2^(64V-1-odd) in
// [1, 4), y = Y / 2^(64V) in (1/2, 1];  D = 1 - m y^2,  y += y D / 2.
template <int V>
XF_FN void rsqrt_fx_step(const uint64_t (&A)[V], bool odd, uint64_t (&Y)[V]) {
  uint64_t Q[V], P[V + 1], D[V + 1], U[V + 1], C[V];
  mul_top<V, V, V>(Y, Y, Q);  // y^2 = Q / 2^(64V)
  mul_top<V, V, V - 1>(A, Q, P);  // m y^2 = P / 2^(64V+63-odd)
  const bool neg = newton_residual<V>(P, odd ? -1 : 0, D);
  mul_top<V, V + 1, V>(Y, D, U);
  // y D / 2 = U / 2^(64V+64-odd) (as Y's fixed point)
#pragma unroll
  for (int i = 0; i < V; ++i) C[i] = odd ? ((U[i] >> 63) | (U[i + 1] << 1)) : U[i + 1];
  add_signed<V>(Y, C, neg);
}

// The leading V words of the W-word mantissa, and Y from width V to V2.
template <int V, int W>
XF_FN void lead_words(const uint64_t (&m)[W], uint64_t (&A)[V]) {
#pragma unroll
  for (int i = 0; i < V; ++i) A[i] = m[W - V + i];
}
template <int V2, int V>
XF_FN void widen(const uint64_t (&Y)[V], uint64_t (&Y2)[V2]) {
#pragma unroll
  for (int i = 0; i < V2; ++i) Y2[i] = i < V2 - V ? 0ULL : Y[i - (V2 - V)];
}

// the step at width V on the iterate Yp of width VP < V
template <bool RSQRT, int V, int W, int VP>
XF_FN void fx_step_at(const uint64_t (&m)[W], bool odd, const uint64_t (&Yp)[VP], uint64_t (&Y)[V]) {
  uint64_t A[V];
  widen<V>(Yp, Y);
  lead_words<V>(m, A);
  if constexpr (RSQRT) rsqrt_fx_step<V>(A, odd, Y);
  else recip_fx_step<V>(A, Y);
}

// The steps at widths 1, 2, 4, ... up to W from a double seed y0 in (0, 1):
// the seed has about 52 correct bits and each step doubles them, up to the
// width it runs at (62, 122, 242, 440 bits after the steps at 1, 2, 4, 7
// words; each step's truncations cost a few bits below its width), at least
// 53K + 8 bits for the K = 1, 2, 4, 8 limbs that W = 1, 2, 4, 7 serve.  The
// reciprocal square root's step leaves 3/2 of the squared error, so at
// W = 4 it takes a step at 3 words before the last (122 -> 186 -> 256).
template <bool RSQRT, int W>
XF_FN void newton_fx(const uint64_t (&m)[W], bool odd, double y0, uint64_t (&Y)[W]) {
  uint64_t Y1[1], A1[1];
  Y1[0] = (uint64_t)(y0 * 18446744073709551616.0);  // y0 2^64 < 2^64, exact
  lead_words<1>(m, A1);
  if constexpr (RSQRT) rsqrt_fx_step<1>(A1, odd, Y1);
  else recip_fx_step<1>(A1, Y1);
  if constexpr (W == 1) {
    Y[0] = Y1[0];
    return;
  } else {
    uint64_t Y2[2];
    fx_step_at<RSQRT, 2>(m, odd, Y1, Y2);
    if constexpr (W == 2) {
      Y[0] = Y2[0];
      Y[1] = Y2[1];
    } else if constexpr (W == 4 && RSQRT) {
      uint64_t Y3[3];
      fx_step_at<RSQRT, 3>(m, odd, Y2, Y3);
      fx_step_at<RSQRT, 4>(m, odd, Y3, Y);
    } else if constexpr (W == 4) {
      fx_step_at<RSQRT, 4>(m, odd, Y2, Y);
    } else {
      uint64_t Y4[4];
      fx_step_at<RSQRT, 4>(m, odd, Y2, Y4);
      fx_step_at<RSQRT, W>(m, odd, Y4, Y);
    }
  }
}

// Y / 2^(64W) (y in (1/2, 1), or a few units below 1/2) as an xf value of
// exponent e - 1: normalised by one bit where the top bit is clear.
template <int W>
XF_FN void fx_to_xf(const uint64_t (&Y)[W], int e, int s, xf<W>& r) {
  const bool top = (Y[W - 1] >> 63) != 0ULL;
#pragma unroll
  for (int i = 0; i < W; ++i) r.m[i] = top ? Y[i] : ((Y[i] << 1) | (i > 0 ? Y[i - 1] >> 63 : 0ULL));
  r.e = top ? e - 1 : e - 2;
  r.s = s;
}

// whether the mantissa is exactly 2^(64W-1) (the value a power of two)
template <int W>
XF_FN bool mant_is_pow2(const xf<W>& a) {
  bool p = a.m[W - 1] == (1ULL << 63);
#pragma unroll
  for (int i = 0; i < W - 1; ++i) p = p && a.m[i] == 0ULL;
  return p;
}

// r = 1 / a, a nonzero:  1/a = (1/m) 2^(-e) for a = m 2^e, m in [1, 2).
template <int W>
XF_FN void xf_recip_fx(const xf<W>& a, xf<W>& r) {
  if (mant_is_pow2(a)) {  // 1/m = 1 exactly
    xf_from_double(1.0, r);
    r.e = -a.e;
    r.s = a.s;
    return;
  }
  double y0 = drecip(xf_mant_double(a));  // in (1/2, 1]; below 1 since m > 1
  y0 = y0 < 1.0 ? y0 : 1.0 - 0x1p-53;
  uint64_t Y[W];
  newton_fx<false>(a.m, false, y0, Y);
  fx_to_xf(Y, -a.e, a.s, r);
}

// r = 1 / sqrt(a), a > 0:  a = m' 2^e' with e' even and m' = m or 2m in
// [1, 4), 1/sqrt(a) = (1/sqrt(m')) 2^(-e'/2).
template <int W>
XF_FN void xf_rsqrt_fx(const xf<W>& a, xf<W>& r) {
  const bool odd = (a.e & 1) != 0;
  const int eh = (odd ? a.e - 1 : a.e) / 2;
  if (!odd && mant_is_pow2(a)) {  // m' = 1
    xf_from_double(1.0, r);
    r.e = -eh;
    return;
  }
  const double md = xf_mant_double(a);
  double y0 = drsqrt(odd ? 2.0 * md : md);
  y0 = y0 < 1.0 ? y0 : 1.0 - 0x1p-53;
  uint64_t Y[W];
  newton_fx<true>(a.m, odd, y0, Y);
  fx_to_xf(Y, -eh, 0, r);
}

#if defined(__CUDACC__)
template <int W>
__device__ __noinline__ xf<W> xf_recip_ol(const xf<W> a) {
  xf<W> r;
  xf_recip_fx(a, r);
  return r;
}
template <int W>
__device__ __noinline__ xf<W> xf_rsqrt_ol(const xf<W> a) {
  xf<W> r;
  xf_rsqrt_fx(a, r);
  return r;
}
#endif

// r = 1 / a, a nonzero, and r = 1 / sqrt(a), a > 0 (O: inline, or one
// out-of-line call on the device)
template <class O = xf_ops_inline, int W>
XF_FN void xf_recip(const xf<W>& a, xf<W>& r) {
#if defined(__CUDA_ARCH__)
  if constexpr (O::call) {
    r = xf_recip_ol<W>(a);
    return;
  }
#endif
  xf_recip_fx(a, r);
}
template <class O = xf_ops_inline, int W>
XF_FN void xf_rsqrt(const xf<W>& a, xf<W>& r) {
#if defined(__CUDA_ARCH__)
  if constexpr (O::call) {
    r = xf_rsqrt_ol<W>(a);
    return;
  }
#endif
  xf_rsqrt_fx(a, r);
}

}  // namespace xfn
