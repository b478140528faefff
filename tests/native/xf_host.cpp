// Host build of the integer-limb extended floats (xf.cuh) for the CPU tests:
// md inputs are converted to xf, one operation runs, and the result comes
// back as an md value of KO limbs (KO = K + 1 shows the xf result itself,
// below the md precision).
#include "../../paper_2301_12659_gb300/csrc/xf.cuh"

using namespace xfn;

template <int K, int W, int KO>
static void run(int op, const double* a, const double* b, double* out) {
  double la[K], lb[K], r[KO];
  for (int l = 0; l < K; ++l) {
    la[l] = a[l];
    lb[l] = b[l];
  }
  xf<W> x, y, z;
  xf_from_md<K, W>(la, x);
  xf_from_md<K, W>(lb, y);
  switch (op) {
    case 0: z = x; break;
    case 1: xf_add(x, y, z); break;
    case 2: xf_sub(x, y, z); break;
    case 3: xf_mul(x, y, z); break;
    case 4: xf_recip(x, z); break;
    case 5: xf_rsqrt(x, z); break;
    default: xf_zero(z);
  }
  xf_to_md<KO, W>(z, r);
  for (int l = 0; l < KO; ++l) out[l] = r[l];
}

// op: 0 round trip, 1 add, 2 sub, 3 mul, 4 reciprocal, 5 rsqrt.
// extra = 0: K output limbs; extra = 1: K + 1 output limbs.
extern "C" int xf_host_op(int K, int extra, int op, const double* a, const double* b, double* out) {
  if (extra) {
    switch (K) {
      case 1: run<1, 1, 2>(op, a, b, out); return 0;
      case 2: run<2, 2, 3>(op, a, b, out); return 0;
      case 4: run<4, 4, 5>(op, a, b, out); return 0;
      case 8: run<8, 7, 9>(op, a, b, out); return 0;
    }
  } else {
    switch (K) {
      case 1: run<1, 1, 1>(op, a, b, out); return 0;
      case 2: run<2, 2, 2>(op, a, b, out); return 0;
      case 4: run<4, 4, 4>(op, a, b, out); return 0;
      case 8: run<8, 7, 8>(op, a, b, out); return 0;
    }
  }
  return 1;
}

// c = a * b mod t^D for md series a, b ([D][K] limbs each) with one
// fixed-point accumulator per coefficient; c as [D][KO] limbs.
template <int K, int W, int KO>
static void conv(int D, const double* a, const double* b, double* out) {
  xf<W> xa[64], xb[64];
  for (int i = 0; i < D; ++i) {
    double la[K], lb[K];
    for (int l = 0; l < K; ++l) {
      la[l] = a[i * K + l];
      lb[l] = b[i * K + l];
    }
    xf_from_md<K, W>(la, xa[i]);
    xf_from_md<K, W>(lb, xb[i]);
  }
  for (int k = 0; k < D; ++k) {
    int e = XF_ZERO_E * 2;
    for (int i = 0; i <= k; ++i) {
      const int ei = xf_prod_exp(xa[i], xb[k - i]);
      e = ei > e ? ei : e;
    }
    xfacc<W> acc;
    xfacc_init(acc, e);
    for (int i = 0; i <= k; ++i) xfacc_fma(acc, xa[i], xb[k - i], (i & 1) != 0 && k == D - 1);
    xf<W> r;
    xfacc_get(acc, r);
    double o[KO];
    xf_to_md<KO, W>(r, o);
    for (int l = 0; l < KO; ++l) out[k * KO + l] = o[l];
  }
}

// The last coefficient alternates the signs of its terms (exercises the
// subtracting path of the accumulator).
extern "C" int xf_host_conv(int K, int D, const double* a, const double* b, double* out) {
  if (D < 1 || D > 64) return 1;
  switch (K) {
    case 1: conv<1, 1, 2>(D, a, b, out); return 0;
    case 2: conv<2, 2, 3>(D, a, b, out); return 0;
    case 4: conv<4, 4, 5>(D, a, b, out); return 0;
    case 8: conv<8, 7, 9>(D, a, b, out); return 0;
  }
  return 1;
}

// a + b + cin over N 64-bit words (a, b, out: N words, least significant
// first); returns the carry out, or -1 for an unsupported N.
template <int N>
static int addw(const uint64_t* a, const uint64_t* b, uint64_t cin, uint64_t* out) {
  uint64_t x[N], y[N];
  for (int i = 0; i < N; ++i) {
    x[i] = a[i];
    y[i] = b[i];
  }
  const uint64_t c = add_words<N>(x, y, cin);
  for (int i = 0; i < N; ++i) out[i] = x[i];
  return (int)c;
}

extern "C" int xf_host_add_words(int N, const uint64_t* a, const uint64_t* b, uint64_t cin, uint64_t* out) {
  switch (N) {
    case 1: return addw<1>(a, b, cin, out);
    case 2: return addw<2>(a, b, cin, out);
    case 3: return addw<3>(a, b, cin, out);
    case 4: return addw<4>(a, b, cin, out);
    case 5: return addw<5>(a, b, cin, out);
    case 6: return addw<6>(a, b, cin, out);
    case 7: return addw<7>(a, b, cin, out);
    case 8: return addw<8>(a, b, cin, out);
    case 9: return addw<9>(a, b, cin, out);
  }
  return -1;
}

// (c:s) += v for each v of vals[count]; returns s, c in out[0], out[1].
extern "C" void xf_host_add_count(int count, const uint64_t* vals, uint64_t s0, uint64_t c0, uint64_t* out) {
  uint64_t s = s0, c = c0;
  for (int i = 0; i < count; ++i) add_count(s, c, vals[i]);
  out[0] = s;
  out[1] = c;
}

// Columns LO .. NA+NB-1 of the product of two word arrays (mul_top); out
// receives NA+NB-LO words.  Returns 1 for a shape not instantiated here.
template <int NA, int NB, int LO>
static void mtop(const uint64_t* a, const uint64_t* b, uint64_t* out) {
  uint64_t x[NA], y[NB], r[NA + NB - LO];
  for (int i = 0; i < NA; ++i) x[i] = a[i];
  for (int i = 0; i < NB; ++i) y[i] = b[i];
  mul_top<NA, NB, LO>(x, y, r);
  for (int i = 0; i < NA + NB - LO; ++i) out[i] = r[i];
}

extern "C" int xf_host_mul_top(int NA, int NB, int LO, const uint64_t* a, const uint64_t* b, uint64_t* out) {
  const int key = NA * 100 + NB * 10 + LO;
  switch (key) {
    case 110: mtop<1, 1, 0>(a, b, out); return 0;
    case 121: mtop<1, 2, 1>(a, b, out); return 0;
    case 221: mtop<2, 2, 1>(a, b, out); return 0;
    case 222: mtop<2, 2, 2>(a, b, out); return 0;
    case 232: mtop<2, 3, 2>(a, b, out); return 0;
    case 332: mtop<3, 3, 2>(a, b, out); return 0;
    case 333: mtop<3, 3, 3>(a, b, out); return 0;
    case 343: mtop<3, 4, 3>(a, b, out); return 0;
    case 443: mtop<4, 4, 3>(a, b, out); return 0;
    case 444: mtop<4, 4, 4>(a, b, out); return 0;
    case 454: mtop<4, 5, 4>(a, b, out); return 0;
    case 776: mtop<7, 7, 6>(a, b, out); return 0;
    case 777: mtop<7, 7, 7>(a, b, out); return 0;
    case 787: mtop<7, 8, 7>(a, b, out); return 0;
  }
  return 1;
}
