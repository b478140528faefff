/*
 * mdoracle.c -- CPU oracle for Newton's method on truncated power series in
 * multiple double arithmetic (arXiv 2301.12659).  TEST INFRASTRUCTURE ONLY:
 * the tests, the smoke check and the CPU-baseline leg of bench.py load it; the
 * product path never does.  It shares no code with the CUDA library.
 *
 * Design: every multiple double (md) result is the exact value of its defining
 * expression rounded once to K limbs.  Exactness comes from Shewchuk's
 * expansion arithmetic (J. R. Shewchuk, "Adaptive precision floating-point
 * arithmetic and fast robust geometric predicates", 1997): a growing,
 * nonoverlapping expansion to which doubles are added with Knuth's TwoSum, and
 * products enter as Dekker's exact TwoProduct (T. J. Dekker, "A floating-point
 * technique for extending the available precision", 1971; Veltkamp splitting,
 * no FMA, so the oracle does not depend on the fused multiply-add the GPU
 * uses).  Rounding to K limbs peels off the leading double of the exact value
 * K times.  Division is long division with an exact remainder and the square
 * root is Newton's iteration with an exact residual.  The whole file must be
 * compiled with -ffp-contract=off so no a*b+c is fused.
 *
 * The method steps follow the paper:
 *   Section 5.1     truncated series products (c_k = sum a_i b_{k-i}) and the
 *                   evaluation and differentiation of monomials; the oracle
 *                   multiplies the factors of every partial derivative
 *                   directly, without the forward/backward/cross reuse;
 *   Section 2       Eq. (eqToeplitz), the block lower triangular Toeplitz
 *                   system, solved by forward substitution, and the Newton
 *                   pseudo code;
 *   Section 5.3     Householder QR of A0, Q^H b and back substitution;
 *   Sections 5.4, 6 residuals ||b - A dx||_1 in md.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "mdoracle.h"

#define KMAX 8
/* A nonoverlapping expansion has components on disjoint bit ranges of the
 * double exponent range (2098 bit positions), so it never has more parts. */
#define ACC_CAP 2112

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ESINGULAR = 2, ORC_ENONFINITE = 3, ORC_ECAP = 4 };

/* ------------------------------------------------------------------------- */
/* Error-free transformations                                                 */
/* ------------------------------------------------------------------------- */

/* Knuth's TwoSum: s = fl(a+b) and s + e = a + b exactly. */
static void two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *e = (a - av) + (b - bv);
    *s = x;
}

/* Veltkamp's splitting: a = hi + lo with hi, lo of at most 26 bits. */
static void split(double a, double *hi, double *lo) {
    double c = 134217729.0 * a; /* 2^27 + 1 */
    double h = c - (c - a);
    *hi = h;
    *lo = a - h;
}

/* Dekker's TwoProduct: p = fl(a*b) and p + e = a*b exactly. */
static void two_prod(double a, double b, double *p, double *e) {
    double x = a * b, ah, al, bh, bl;
    split(a, &ah, &al);
    split(b, &bh, &bl);
    double err1 = x - ah * bh;
    double err2 = err1 - al * bh;
    double err3 = err2 - ah * bl;
    *e = al * bl - err3;
    *p = x;
}

/* ------------------------------------------------------------------------- */
/* Exact accumulator: a Shewchuk expansion, components in increasing magnitude */
/* ------------------------------------------------------------------------- */

typedef struct {
    int len;
    int bad; /* 1: a non-finite input was added; 2: capacity exceeded */
    double c[ACC_CAP];
} acc_t;

static void acc_init(acc_t *a) { a->len = 0; a->bad = 0; }

/* Shewchuk's GROW-EXPANSION with zero elimination, in place. */
static void acc_add(acc_t *a, double b) {
    if (b == 0.0) return;
    if (!isfinite(b)) { a->bad |= 1; return; }
    double q = b;
    int h = 0;
    for (int i = 0; i < a->len; ++i) {
        double s, e;
        two_sum(q, a->c[i], &s, &e);
        if (e != 0.0) a->c[h++] = e;
        q = s;
    }
    if (q != 0.0) {
        if (h < ACC_CAP) a->c[h++] = q;
        else a->bad |= 2;
    }
    a->len = h;
}

/* A double close to the value of the expansion (sum from the smallest part). */
static double acc_estimate(const acc_t *a) {
    double v = 0.0;
    for (int i = 0; i < a->len; ++i) v += a->c[i];
    return v;
}

static void acc_add_md(acc_t *a, const double *x, int K, double sgn) {
    for (int l = 0; l < K; ++l) acc_add(a, sgn * x[l]);
}

/* a += sgn * x * y, every limb product x_i*y_j entered exactly. */
static void acc_add_prod(acc_t *a, const double *x, const double *y, int K, double sgn) {
    for (int i = 0; i < K; ++i) {
        if (x[i] == 0.0) continue;
        for (int j = 0; j < K; ++j) {
            if (y[j] == 0.0) continue;
            double p, e;
            two_prod(x[i], sgn * y[j], &p, &e);
            if (!isfinite(p)) { a->bad |= 1; continue; }
            acc_add(a, p);
            acc_add(a, e);
        }
    }
}

/* Round the exact value to K limbs: peel off the leading double K times.
 * Each limb is within a few ulps of the remaining exact value, so the limbs
 * are nonoverlapping and the dropped remainder is below ~2 ulp of the last. */
static acc_t *acc_scratch(void);
static void acc_round(const acc_t *a, int K, double *out) {
    for (int l = 0; l < KMAX; ++l) out[l] = 0.0;
    if (a->bad) {
        for (int l = 0; l < K; ++l) out[l] = NAN;
        return;
    }
    acc_t *t = acc_scratch();
    t->len = a->len;
    t->bad = 0;
    memcpy(t->c, a->c, sizeof(double) * (size_t)a->len);
    for (int l = 0; l < K; ++l) {
        double v = acc_estimate(t);
        out[l] = v;
        if (v == 0.0) break;
        acc_add(t, -v);
    }
}

/* One scratch expansion per thread for acc_round (keeps stacks small). */
static acc_t *acc_scratch(void) {
    static _Thread_local acc_t *buf = NULL;
    if (!buf) buf = (acc_t *)malloc(sizeof(acc_t));
    return buf;
}

/* ------------------------------------------------------------------------- */
/* md scalars (real and complex)                                              */
/* ------------------------------------------------------------------------- */

typedef struct {
    double re[KMAX];
    double im[KMAX];
} mdc;

typedef struct {
    acc_t re, im;
} cacc_t;

static void mdc_zero(mdc *x) { memset(x, 0, sizeof(mdc)); }
static int mdc_finite(const mdc *x, int K) {
    for (int l = 0; l < K; ++l)
        if (!isfinite(x->re[l]) || !isfinite(x->im[l])) return 0;
    return 1;
}

static void cacc_init(cacc_t *a) { acc_init(&a->re); acc_init(&a->im); }
static void cacc_add(cacc_t *a, const mdc *x, int K, int C, double sgn) {
    acc_add_md(&a->re, x->re, K, sgn);
    if (C == 2) acc_add_md(&a->im, x->im, K, sgn);
}
/* a += sgn * x * y (complex product written out: 4 real products). */
static void cacc_add_prod(cacc_t *a, const mdc *x, const mdc *y, int K, int C, double sgn) {
    acc_add_prod(&a->re, x->re, y->re, K, sgn);
    if (C == 2) {
        acc_add_prod(&a->re, x->im, y->im, K, -sgn);
        acc_add_prod(&a->im, x->re, y->im, K, sgn);
        acc_add_prod(&a->im, x->im, y->re, K, sgn);
    }
}
/* a += sgn * conj(x) * y. */
static void cacc_add_conjprod(cacc_t *a, const mdc *x, const mdc *y, int K, int C, double sgn) {
    acc_add_prod(&a->re, x->re, y->re, K, sgn);
    if (C == 2) {
        acc_add_prod(&a->re, x->im, y->im, K, sgn);
        acc_add_prod(&a->im, x->re, y->im, K, sgn);
        acc_add_prod(&a->im, x->im, y->re, K, -sgn);
    }
}
static void cacc_round(const cacc_t *a, int K, int C, mdc *out) {
    mdc_zero(out);
    acc_round(&a->re, K, out->re);
    if (C == 2) acc_round(&a->im, K, out->im);
}

/* Long division: quotient digits q_s = fl(r / b_0) with the remainder
 * r = a - (q_0 + ... + q_s) b kept exact, K+2 digits, rounded once. */
static int md_div_real(const double *a, const double *b, int K, double *q) {
    for (int l = 0; l < KMAX; ++l) q[l] = 0.0;
    if (b[0] == 0.0) {
        q[0] = NAN;
        return ORC_ESINGULAR;
    }
    acc_t *r = (acc_t *)malloc(sizeof(acc_t));
    acc_t *qs = (acc_t *)malloc(sizeof(acc_t));
    acc_init(r);
    acc_init(qs);
    acc_add_md(r, a, K, 1.0);
    for (int s = 0; s < K + 2; ++s) {
        double rv = acc_estimate(r);
        if (rv == 0.0) break;
        double qd = rv / b[0];
        acc_add(qs, qd);
        for (int j = 0; j < K; ++j) {
            if (b[j] == 0.0) continue;
            double p, e;
            two_prod(qd, b[j], &p, &e);
            acc_add(r, -p);
            acc_add(r, -e);
        }
    }
    if (r->bad) qs->bad |= r->bad;
    acc_round(qs, K, q);
    int bad = qs->bad;
    free(r);
    free(qs);
    return bad ? ORC_ENONFINITE : ORC_OK;
}

/* Square root by Newton's iteration x <- x + (a - x^2)/(2x), the residual
 * a - x^2 formed exactly; quadratic convergence from the double sqrt(a_0). */
static int md_sqrt_real(const double *a, int K, double *r) {
    for (int l = 0; l < KMAX; ++l) r[l] = 0.0;
    if (a[0] == 0.0) return ORC_OK;
    if (!(a[0] > 0.0) || !isfinite(a[0])) {
        r[0] = NAN;
        return ORC_ENONFINITE;
    }
    double x[KMAX] = {0};
    x[0] = sqrt(a[0]);
    int iters = 2;
    while ((1 << (iters - 1)) < K) ++iters; /* 53 * 2^(iters-1) > 53 K bits, plus one */
    acc_t *t = (acc_t *)malloc(sizeof(acc_t));
    int rc = ORC_OK;
    for (int it = 0; it < iters; ++it) {
        double res[KMAX], twox[KMAX], dlt[KMAX];
        acc_init(t);
        acc_add_md(t, a, K, 1.0);
        acc_add_prod(t, x, x, K, -1.0);
        acc_round(t, K, res);
        for (int l = 0; l < KMAX; ++l) twox[l] = 2.0 * x[l];
        rc |= md_div_real(res, twox, K, dlt);
        acc_init(t);
        acc_add_md(t, x, K, 1.0);
        acc_add_md(t, dlt, K, 1.0);
        acc_round(t, K, x);
    }
    free(t);
    memcpy(r, x, sizeof(x));
    return rc;
}

/* q = a / b for complex md: a * conj(b) / |b|^2 (each part rounded once
 * before the real divisions). */
static int mdc_div(const mdc *a, const mdc *b, int K, int C, mdc *q) {
    mdc_zero(q);
    if (C == 1) return md_div_real(a->re, b->re, K, q->re);
    cacc_t *num = (cacc_t *)malloc(sizeof(cacc_t));
    acc_t *den = (acc_t *)malloc(sizeof(acc_t));
    cacc_init(num);
    acc_init(den);
    acc_add_prod(&num->re, a->re, b->re, K, 1.0);
    acc_add_prod(&num->re, a->im, b->im, K, 1.0);
    acc_add_prod(&num->im, a->im, b->re, K, 1.0);
    acc_add_prod(&num->im, a->re, b->im, K, -1.0);
    acc_add_prod(den, b->re, b->re, K, 1.0);
    acc_add_prod(den, b->im, b->im, K, 1.0);
    double nre[KMAX], nim[KMAX], dd[KMAX];
    acc_round(&num->re, K, nre);
    acc_round(&num->im, K, nim);
    acc_round(den, K, dd);
    free(num);
    free(den);
    int rc = md_div_real(nre, dd, K, q->re);
    rc |= md_div_real(nim, dd, K, q->im);
    return rc;
}

/* |x| for complex md, sqrt(re^2 + im^2). */
static int mdc_abs(const mdc *x, int K, int C, double *out) {
    acc_t *s = (acc_t *)malloc(sizeof(acc_t));
    acc_init(s);
    acc_add_prod(s, x->re, x->re, K, 1.0);
    if (C == 2) acc_add_prod(s, x->im, x->im, K, 1.0);
    double s2[KMAX];
    acc_round(s, K, s2);
    free(s);
    return md_sqrt_real(s2, K, out);
}

/* ------------------------------------------------------------------------- */
/* Layout conversion: product SoA [K][C][N] <-> oracle arrays of mdc          */
/* ------------------------------------------------------------------------- */

static void soa_to_mdc(const double *src, int K, int C, long N, mdc *dst) {
    for (long i = 0; i < N; ++i) {
        mdc_zero(&dst[i]);
        for (int l = 0; l < K; ++l) {
            dst[i].re[l] = src[((long)l * C + 0) * N + i];
            if (C == 2) dst[i].im[l] = src[((long)l * C + 1) * N + i];
        }
    }
}

static void mdc_to_soa(const mdc *src, int K, int C, long N, double *dst) {
    for (long i = 0; i < N; ++i)
        for (int l = 0; l < K; ++l) {
            dst[((long)l * C + 0) * N + i] = src[i].re[l];
            if (C == 2) dst[((long)l * C + 1) * N + i] = src[i].im[l];
        }
}

/* ------------------------------------------------------------------------- */
/* Truncated power series                                                     */
/* ------------------------------------------------------------------------- */

/* c = a * b mod t^(d+1); c may alias a or b. */
static void series_mul(const mdc *a, const mdc *b, mdc *c, int d, int K, int C) {
    mdc *tmp = (mdc *)malloc(sizeof(mdc) * (size_t)(d + 1));
    cacc_t *acc = (cacc_t *)malloc(sizeof(cacc_t));
    for (int k = 0; k <= d; ++k) {
        cacc_init(acc);
        for (int i = 0; i <= k; ++i) cacc_add_prod(acc, &a[i], &b[k - i], K, C, 1.0);
        cacc_round(acc, K, C, &tmp[k]);
    }
    memcpy(c, tmp, sizeof(mdc) * (size_t)(d + 1));
    free(acc);
    free(tmp);
}

/* ------------------------------------------------------------------------- */
/* Evaluation and differentiation of the system                               */
/* ------------------------------------------------------------------------- */

typedef struct {
    int K, C, n, d, M;
    const int32_t *eq, *vptr, *vidx;
    const mdc *coeff; /* [M][d+1] */
    const mdc *cst;   /* [n][d+1] or NULL */
} sys_t;

static int check_structure(int n, int d, int M, const int32_t *eq, const int32_t *vptr,
                           const int32_t *vidx) {
    if (n < 1 || d < 0 || M < 0 || !eq || !vptr || (M > 0 && !vidx)) return ORC_EINVAL;
    if (vptr[0] != 0) return ORC_EINVAL;
    for (int m = 0; m < M; ++m) {
        if (eq[m] < 0 || eq[m] >= n) return ORC_EINVAL;
        if (vptr[m + 1] <= vptr[m]) return ORC_EINVAL;
        for (int p = vptr[m]; p < vptr[m + 1]; ++p)
            if (vidx[p] < 0 || vidx[p] >= n) return ORC_EINVAL;
    }
    return ORC_OK;
}

/* f_i = sum of monomial values + cst_i; A_j[i][v] = sum over the occurrences
 * of x_v of the coefficient j of the product of the other factors. */
static int evaluate(const sys_t *S, const mdc *X, mdc *F, mdc *A) {
    const int n = S->n, d = S->d, K = S->K, C = S->C, M = S->M, D = d + 1;
    int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
    int *list = (int *)malloc(sizeof(int) * (size_t)(M > 0 ? M : 1));
    for (int m = 0; m < M; ++m) cnt[S->eq[m] + 1]++;
    for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    {
        int *fill = (int *)calloc((size_t)n, sizeof(int));
        for (int m = 0; m < M; ++m) list[cnt[S->eq[m]] + fill[S->eq[m]]++] = m;
        free(fill);
    }
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int i = 0; i < n; ++i) {
        int nm = cnt[i + 1] - cnt[i];
        int slots = 0;
        for (int q = 0; q < nm; ++q) {
            int m = list[cnt[i] + q];
            slots += S->vptr[m + 1] - S->vptr[m];
        }
        mdc *val = (mdc *)malloc(sizeof(mdc) * (size_t)(nm > 0 ? nm : 1) * D);
        mdc *par = (mdc *)malloc(sizeof(mdc) * (size_t)(slots > 0 ? slots : 1) * D);
        int *slot_var = (int *)malloc(sizeof(int) * (size_t)(slots > 0 ? slots : 1));
        cacc_t *acc = (cacc_t *)malloc(sizeof(cacc_t));
        int s = 0;
        for (int q = 0; q < nm; ++q) {
            int m = list[cnt[i] + q];
            int p0 = S->vptr[m], k = S->vptr[m + 1] - p0;
            mdc *v = &val[(size_t)q * D];
            memcpy(v, &S->coeff[(size_t)m * D], sizeof(mdc) * D);
            for (int p = 0; p < k; ++p) series_mul(v, &X[(size_t)S->vidx[p0 + p] * D], v, d, K, C);
            for (int jj = 0; A && jj < k; ++jj, ++s) {
                mdc *g = &par[(size_t)s * D];
                slot_var[s] = S->vidx[p0 + jj];
                memcpy(g, &S->coeff[(size_t)m * D], sizeof(mdc) * D);
                for (int p = 0; p < k; ++p)
                    if (p != jj) series_mul(g, &X[(size_t)S->vidx[p0 + p] * D], g, d, K, C);
            }
        }
        for (int kk = 0; kk < D; ++kk) {
            cacc_init(acc);
            if (S->cst) cacc_add(acc, &S->cst[(size_t)i * D + kk], K, C, 1.0);
            for (int q = 0; q < nm; ++q) cacc_add(acc, &val[(size_t)q * D + kk], K, C, 1.0);
            cacc_round(acc, K, C, &F[(size_t)i * D + kk]);
            if (!mdc_finite(&F[(size_t)i * D + kk], K)) err |= 1;
        }
        if (A) {
            for (int vv = 0; vv < n; ++vv)
                for (int j = 0; j < D; ++j) {
                    mdc *out = &A[((size_t)j * n + i) * n + vv];
                    cacc_init(acc);
                    for (int t = 0; t < slots; ++t)
                        if (slot_var[t] == vv) cacc_add(acc, &par[(size_t)t * D + j], K, C, 1.0);
                    cacc_round(acc, K, C, out);
                    if (!mdc_finite(out, K)) err |= 1;
                }
        }
        free(acc);
        free(slot_var);
        free(par);
        free(val);
    }
    free(list);
    free(cnt);
    return err ? ORC_ENONFINITE : ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Householder QR of A0, Q^H b, back substitution                             */
/* ------------------------------------------------------------------------- */

typedef struct {
    int n, K, C;
    mdc *R;   /* n*n row-major, upper triangular */
    mdc *V;   /* n*n row-major: reflector j in rows j..n-1 of column j */
    mdc *tau; /* n: 2 / (v^H v), real (in .re) */
} qr_t;

static void qr_free(qr_t *Q) {
    free(Q->R);
    free(Q->V);
    free(Q->tau);
}

/* H_j = I - tau_j v_j v_j^H with v_j = x + s |x| e_1, s = x_0/|x_0| (s = +1 when
 * x_0 = 0, the sign of x_0 for real data), so that H_j x = -s |x| e_1. */
static int qr_factor(const mdc *A0, int n, int K, int C, qr_t *Q) {
    Q->n = n;
    Q->K = K;
    Q->C = C;
    Q->R = (mdc *)calloc((size_t)n * n, sizeof(mdc));
    Q->V = (mdc *)calloc((size_t)n * n, sizeof(mdc));
    Q->tau = (mdc *)calloc((size_t)n, sizeof(mdc));
    mdc *W = (mdc *)malloc(sizeof(mdc) * (size_t)n * n);
    memcpy(W, A0, sizeof(mdc) * (size_t)n * n);
    int rc = ORC_OK;
    acc_t *s = (acc_t *)malloc(sizeof(acc_t));
    for (int j = 0; j < n && rc == ORC_OK; ++j) {
        double nrm2[KMAX], alpha[KMAX];
        acc_init(s);
        for (int i = j; i < n; ++i) {
            acc_add_prod(s, W[(size_t)i * n + j].re, W[(size_t)i * n + j].re, K, 1.0);
            if (C == 2) acc_add_prod(s, W[(size_t)i * n + j].im, W[(size_t)i * n + j].im, K, 1.0);
        }
        acc_round(s, K, nrm2);
        if (!isfinite(nrm2[0])) { rc = ORC_ENONFINITE; break; }
        if (nrm2[0] == 0.0) { rc = ORC_ESINGULAR; break; }
        rc |= md_sqrt_real(nrm2, K, alpha);
        mdc x0 = W[(size_t)j * n + j], sg, salpha;
        mdc_zero(&sg);
        if (C == 1) {
            sg.re[0] = (x0.re[0] < 0.0) ? -1.0 : 1.0;
        } else {
            double ax[KMAX];
            rc |= mdc_abs(&x0, K, C, ax);
            if (ax[0] == 0.0) {
                sg.re[0] = 1.0;
            } else {
                rc |= md_div_real(x0.re, ax, K, sg.re);
                rc |= md_div_real(x0.im, ax, K, sg.im);
            }
        }
        { /* salpha = s * alpha */
            cacc_t *t = (cacc_t *)malloc(sizeof(cacc_t));
            mdc al;
            mdc_zero(&al);
            memcpy(al.re, alpha, sizeof(alpha));
            cacc_init(t);
            cacc_add_prod(t, &sg, &al, K, C, 1.0);
            cacc_round(t, K, C, &salpha);
            /* v_j = x + s alpha e_1 */
            for (int i = j + 1; i < n; ++i) Q->V[(size_t)i * n + j] = W[(size_t)i * n + j];
            cacc_init(t);
            cacc_add(t, &x0, K, C, 1.0);
            cacc_add(t, &salpha, K, C, 1.0);
            cacc_round(t, K, C, &Q->V[(size_t)j * n + j]);
            free(t);
        }
        { /* tau_j = 2 / (v^H v) */
            double vn2[KMAX], two[KMAX] = {2.0};
            acc_init(s);
            for (int i = j; i < n; ++i) {
                acc_add_prod(s, Q->V[(size_t)i * n + j].re, Q->V[(size_t)i * n + j].re, K, 1.0);
                if (C == 2) acc_add_prod(s, Q->V[(size_t)i * n + j].im, Q->V[(size_t)i * n + j].im, K, 1.0);
            }
            acc_round(s, K, vn2);
            mdc_zero(&Q->tau[j]);
            rc |= md_div_real(two, vn2, K, Q->tau[j].re);
        }
        /* W[j:, c] -= tau (v^H W[j:, c]) v for the columns right of j */
#pragma omp parallel for schedule(dynamic, 1)
        for (int c = j + 1; c < n; ++c) {
            cacc_t *t = (cacc_t *)malloc(sizeof(cacc_t));
            mdc w, g;
            cacc_init(t);
            for (int i = j; i < n; ++i) cacc_add_conjprod(t, &Q->V[(size_t)i * n + j], &W[(size_t)i * n + c], K, C, 1.0);
            cacc_round(t, K, C, &w);
            cacc_init(t);
            cacc_add_prod(t, &Q->tau[j], &w, K, C, 1.0);
            cacc_round(t, K, C, &g);
            for (int i = j; i < n; ++i) {
                cacc_init(t);
                cacc_add(t, &W[(size_t)i * n + c], K, C, 1.0);
                cacc_add_prod(t, &g, &Q->V[(size_t)i * n + j], K, C, -1.0);
                cacc_round(t, K, C, &W[(size_t)i * n + c]);
            }
            free(t);
        }
        /* column j becomes -s alpha e_1 */
        for (int l = 0; l < KMAX; ++l) {
            W[(size_t)j * n + j].re[l] = -salpha.re[l];
            W[(size_t)j * n + j].im[l] = -salpha.im[l];
        }
        for (int i = j + 1; i < n; ++i) mdc_zero(&W[(size_t)i * n + j]);
    }
    free(s);
    for (int i = 0; i < n; ++i)
        for (int c = i; c < n; ++c) Q->R[(size_t)i * n + c] = W[(size_t)i * n + c];
    free(W);
    return rc;
}

/* y := H_j y for one reflector. */
static void qr_reflect(const qr_t *Q, int j, mdc *y) {
    const int n = Q->n, K = Q->K, C = Q->C;
    cacc_t *t = (cacc_t *)malloc(sizeof(cacc_t));
    mdc w, g;
    cacc_init(t);
    for (int i = j; i < n; ++i) cacc_add_conjprod(t, &Q->V[(size_t)i * n + j], &y[i], K, C, 1.0);
    cacc_round(t, K, C, &w);
    cacc_init(t);
    cacc_add_prod(t, &Q->tau[j], &w, K, C, 1.0);
    cacc_round(t, K, C, &g);
    for (int i = j; i < n; ++i) {
        cacc_init(t);
        cacc_add(t, &y[i], K, C, 1.0);
        cacc_add_prod(t, &g, &Q->V[(size_t)i * n + j], K, C, -1.0);
        cacc_round(t, K, C, &y[i]);
    }
    free(t);
}

/* y := Q^H y = H_{n-1} ... H_0 y. */
static void qr_apply_qh(const qr_t *Q, mdc *y) {
    for (int j = 0; j < Q->n; ++j) qr_reflect(Q, j, y);
}

/* Solve R x = y by back substitution. */
static int back_sub(const qr_t *Q, const mdc *y, mdc *x) {
    const int n = Q->n, K = Q->K, C = Q->C;
    cacc_t *t = (cacc_t *)malloc(sizeof(cacc_t));
    int rc = ORC_OK;
    for (int i = n - 1; i >= 0; --i) {
        mdc num;
        cacc_init(t);
        cacc_add(t, &y[i], K, C, 1.0);
        for (int c = i + 1; c < n; ++c) cacc_add_prod(t, &Q->R[(size_t)i * n + c], &x[c], K, C, -1.0);
        cacc_round(t, K, C, &num);
        rc |= mdc_div(&num, &Q->R[(size_t)i * n + i], K, C, &x[i]);
    }
    free(t);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Block lower triangular Toeplitz solve, Eq. (eqToeplitz)                    */
/* ------------------------------------------------------------------------- */

/* x rounded to L <= K limbs. */
static void mdc_round_to(const mdc *x, int K, int C, int L, mdc *out) {
    cacc_t *t = (cacc_t *)malloc(sizeof(cacc_t));
    cacc_init(t);
    cacc_add(t, x, K, C, 1.0);
    cacc_round(t, L, C, out);
    free(t);
}

/* A [(d+1)][n][n], B and DX [n][d+1]: sum_{j<=k} A_j DX_{k-j} = B_k. */
/* Forward substitution of Section 5.4.  Stages k >= late_stage (the
 * stated-accuracy variant) form their update sum_{j>=1} A_j dx_{k-j} in
 * late_K limbs: every operand rounded to late_K limbs, the sum rounded to
 * late_K limbs, then subtracted from b_k in K limbs.  late_stage > d: the
 * plain method. */
static int block_stages(int K, int C, int n, int d, const mdc *A, const mdc *B, mdc *DX, int late_stage,
                        int late_K, const qr_t *QQ);
static int block_solve(int K, int C, int n, int d, const mdc *A, const mdc *B, mdc *DX, int late_stage,
                       int late_K) {
    qr_t Q;
    int rc = qr_factor(A, n, K, C, &Q);
    if (rc == ORC_OK) rc = block_stages(K, C, n, d, A, B, DX, late_stage, late_K, &Q);
    qr_free(&Q);
    return rc;
}

/* The d+1 stages with a given factorization of A_0. */
static int block_stages(int K, int C, int n, int d, const mdc *A, const mdc *B, mdc *DX, int late_stage,
                        int late_K, const qr_t *QQ) {
    const int D = d + 1;
    const qr_t Q = *QQ;
    int rc = ORC_OK;
    mdc *r = (mdc *)malloc(sizeof(mdc) * (size_t)n);
    mdc *xk = (mdc *)malloc(sizeof(mdc) * (size_t)n);
    for (int k = 0; k < D; ++k) {
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) {
            cacc_t *t = (cacc_t *)malloc(sizeof(cacc_t));
            cacc_init(t);
            cacc_add(t, &B[(size_t)i * D + k], K, C, 1.0);
            if (k >= late_stage && late_K < K) {
                cacc_t *u = (cacc_t *)malloc(sizeof(cacc_t));
                cacc_init(u);
                for (int j = 1; j <= k; ++j)
                    for (int l = 0; l < n; ++l) {
                        mdc a, x;
                        mdc_round_to(&A[((size_t)j * n + i) * n + l], K, C, late_K, &a);
                        mdc_round_to(&DX[(size_t)l * D + (k - j)], K, C, late_K, &x);
                        cacc_add_prod(u, &a, &x, late_K, C, 1.0);
                    }
                mdc upd;
                cacc_round(u, late_K, C, &upd);
                cacc_add(t, &upd, late_K, C, -1.0);
                free(u);
            } else {
                for (int j = 1; j <= k; ++j)
                    for (int l = 0; l < n; ++l)
                        cacc_add_prod(t, &A[((size_t)j * n + i) * n + l], &DX[(size_t)l * D + (k - j)], K, C,
                                      -1.0);
            }
            cacc_round(t, K, C, &r[i]);
            free(t);
        }
        qr_apply_qh(&Q, r);
        rc |= back_sub(&Q, r, xk);
        for (int i = 0; i < n; ++i) DX[(size_t)i * D + k] = xk[i];
    }
    free(xk);
    free(r);
    return rc;
}

static double norm1(const mdc *v, long N, int C) {
    double s = 0.0;
    for (long i = 0; i < N; ++i) s += (C == 2) ? hypot(v[i].re[0], v[i].im[0]) : fabs(v[i].re[0]);
    return s;
}

/* ||B - T DX||_1 with T the block Toeplitz matrix, every entry in md:
   entry (i, k) of the residual is b_k[i] - sum_{j=0..k} (A_j dx_{k-j})[i]
   (Eq. (eqToeplitz)), its exact value rounded once.  R (may be NULL) receives
   the md residual series.  With rows != NULL only the `count` rows listed
   enter the norm, scaled by n / count (the sampled monitor of Section 5.4).
   The entries' magnitudes are summed in row-major order after the parallel
   loop, so the reported norm does not depend on the thread count. */
static double toeplitz_residual_rows(int K, int C, int n, int d, const mdc *A, const mdc *B, const mdc *DX,
                                     mdc *R, const int32_t *rows, int count) {
    const int D = d + 1;
    double *mag = (double *)calloc((size_t)n * D, sizeof(double));
    char *in = (char *)calloc((size_t)n, 1);
    if (rows) {
        for (int q = 0; q < count; ++q) in[rows[q]] = 1;
    } else {
        memset(in, 1, (size_t)n);
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        if (!in[i] && !R) continue;
        cacc_t *t = (cacc_t *)malloc(sizeof(cacc_t));
        for (int k = 0; k < D; ++k) {
            mdc r;
            cacc_init(t);
            cacc_add(t, &B[(size_t)i * D + k], K, C, 1.0);
            for (int j = 0; j <= k; ++j)
                for (int l = 0; l < n; ++l)
                    cacc_add_prod(t, &A[((size_t)j * n + i) * n + l], &DX[(size_t)l * D + (k - j)], K, C, -1.0);
            cacc_round(t, K, C, &r);
            if (R) R[(size_t)i * D + k] = r;
            if (in[i]) mag[(size_t)i * D + k] = norm1(&r, 1, C);
        }
        free(t);
    }
    double total = 0.0;
    for (long e = 0; e < (long)n * D; ++e) total += mag[e];
    free(mag);
    free(in);
    return rows ? total * ((double)n / count) : total;
}

static double toeplitz_residual(int K, int C, int n, int d, const mdc *A, const mdc *B, const mdc *DX) {
    return toeplitz_residual_rows(K, C, n, d, A, B, DX, NULL, NULL, 0);
}

/* ------------------------------------------------------------------------- */
/* Exported entry points                                                      */
/* ------------------------------------------------------------------------- */

void orc_set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int check_kc(int K, int C) { return (K >= 1 && K <= KMAX && (C == 1 || C == 2)) ? ORC_OK : ORC_EINVAL; }

int orc_md_binary(int op, int K, int C, int N, const double *a, const double *b, double *r) {
    if (check_kc(K, C) || N < 0 || op < 0 || op > 3) return ORC_EINVAL;
    mdc *x = (mdc *)malloc(sizeof(mdc) * (size_t)(N > 0 ? N : 1));
    mdc *y = (mdc *)malloc(sizeof(mdc) * (size_t)(N > 0 ? N : 1));
    mdc *z = (mdc *)malloc(sizeof(mdc) * (size_t)(N > 0 ? N : 1));
    soa_to_mdc(a, K, C, N, x);
    soa_to_mdc(b, K, C, N, y);
    int rc = ORC_OK;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : rc)
    for (int i = 0; i < N; ++i) {
        if (op == 3) {
            rc |= mdc_div(&x[i], &y[i], K, C, &z[i]);
        } else {
            cacc_t *t = (cacc_t *)malloc(sizeof(cacc_t));
            cacc_init(t);
            if (op == 2) {
                cacc_add_prod(t, &x[i], &y[i], K, C, 1.0);
            } else {
                cacc_add(t, &x[i], K, C, 1.0);
                cacc_add(t, &y[i], K, C, op == 1 ? -1.0 : 1.0);
            }
            cacc_round(t, K, C, &z[i]);
            free(t);
        }
    }
    mdc_to_soa(z, K, C, N, r);
    free(x);
    free(y);
    free(z);
    return rc;
}

int orc_md_sqrt(int K, int N, const double *a, double *r) {
    if (check_kc(K, 1) || N < 0) return ORC_EINVAL;
    int rc = ORC_OK;
    for (int i = 0; i < N; ++i) {
        double x[KMAX] = {0}, y[KMAX];
        for (int l = 0; l < K; ++l) x[l] = a[(long)l * N + i];
        rc |= md_sqrt_real(x, K, y);
        for (int l = 0; l < K; ++l) r[(long)l * N + i] = y[l];
    }
    return rc;
}

int orc_series_mul(int K, int C, int d, const double *a, const double *b, double *c) {
    if (check_kc(K, C) || d < 0) return ORC_EINVAL;
    const long D = d + 1;
    mdc *x = (mdc *)malloc(sizeof(mdc) * D), *y = (mdc *)malloc(sizeof(mdc) * D);
    soa_to_mdc(a, K, C, D, x);
    soa_to_mdc(b, K, C, D, y);
    series_mul(x, y, x, d, K, C);
    mdc_to_soa(x, K, C, D, c);
    free(x);
    free(y);
    return ORC_OK;
}

int orc_evaluate(int K, int C, int n, int d, int M, const int32_t *eq, const int32_t *vptr,
                 const int32_t *vidx, const double *coeff, const double *cst, const double *x,
                 double *f, double *A) {
    if (check_kc(K, C) || check_structure(n, d, M, eq, vptr, vidx)) return ORC_EINVAL;
    const long D = d + 1;
    mdc *CF = (mdc *)malloc(sizeof(mdc) * (size_t)(M > 0 ? M : 1) * D);
    mdc *CS = cst ? (mdc *)malloc(sizeof(mdc) * (size_t)n * D) : NULL;
    mdc *X = (mdc *)malloc(sizeof(mdc) * (size_t)n * D);
    mdc *F = (mdc *)malloc(sizeof(mdc) * (size_t)n * D);
    mdc *AA = A ? (mdc *)malloc(sizeof(mdc) * (size_t)D * n * n) : NULL;
    soa_to_mdc(coeff, K, C, (long)M * D, CF);
    if (cst) soa_to_mdc(cst, K, C, (long)n * D, CS);
    soa_to_mdc(x, K, C, (long)n * D, X);
    sys_t S = {K, C, n, d, M, eq, vptr, vidx, CF, CS};
    int rc = evaluate(&S, X, F, AA);
    mdc_to_soa(F, K, C, (long)n * D, f);
    if (A) mdc_to_soa(AA, K, C, D * n * n, A);
    free(AA);
    free(F);
    free(X);
    free(CS);
    free(CF);
    return rc;
}

int orc_planted_constant(int K, int C, int n, int d, int M, const int32_t *eq,
                         const int32_t *vptr, const int32_t *vidx, const double *coeff,
                         const double *xstar, double *cst) {
    if (check_kc(K, C) || check_structure(n, d, M, eq, vptr, vidx)) return ORC_EINVAL;
    const long D = d + 1;
    mdc *CF = (mdc *)malloc(sizeof(mdc) * (size_t)(M > 0 ? M : 1) * D);
    mdc *X = (mdc *)malloc(sizeof(mdc) * (size_t)n * D);
    mdc *F = (mdc *)malloc(sizeof(mdc) * (size_t)n * D);
    soa_to_mdc(coeff, K, C, (long)M * D, CF); /* zero padded to KMAX limbs */
    soa_to_mdc(xstar, K, C, (long)n * D, X);
    sys_t S = {KMAX, C, n, d, M, eq, vptr, vidx, CF, NULL};
    int rc = evaluate(&S, X, F, NULL);
    for (long i = 0; i < (long)n * D; ++i)
        for (int l = 0; l < KMAX; ++l) {
            F[i].re[l] = -F[i].re[l];
            F[i].im[l] = -F[i].im[l];
        }
    mdc_to_soa(F, K, C, (long)n * D, cst); /* leading K limbs of the octo double */
    free(F);
    free(X);
    free(CF);
    return rc;
}

int orc_qr(int K, int C, int n, const double *A0, double *Qout, double *Rout) {
    if (check_kc(K, C) || n < 1) return ORC_EINVAL;
    const long N = (long)n * n;
    mdc *A = (mdc *)malloc(sizeof(mdc) * N);
    soa_to_mdc(A0, K, C, N, A);
    qr_t Q;
    int rc = qr_factor(A, n, K, C, &Q);
    if (rc == ORC_OK) {
        /* column c of Q is H_0 H_1 ... H_{n-1} e_c */
        mdc *Qm = (mdc *)calloc((size_t)N, sizeof(mdc));
        mdc *y = (mdc *)malloc(sizeof(mdc) * (size_t)n);
        for (int c = 0; c < n; ++c) {
            for (int i = 0; i < n; ++i) mdc_zero(&y[i]);
            y[c].re[0] = 1.0;
            for (int j = n - 1; j >= 0; --j) qr_reflect(&Q, j, y);
            for (int i = 0; i < n; ++i) Qm[(size_t)i * n + c] = y[i];
        }
        mdc_to_soa(Qm, K, C, N, Qout);
        mdc_to_soa(Q.R, K, C, N, Rout);
        free(y);
        free(Qm);
    }
    qr_free(&Q);
    free(A);
    return rc;
}

int orc_solve(int K, int C, int n, int d, const double *A, const double *b, double *dx) {
    return orc_solve_late(K, C, n, d, A, b, d + 1, K, dx);
}

int orc_solve_late(int K, int C, int n, int d, const double *A, const double *b, int late_stage, int late_K,
                   double *dx) {
    if (check_kc(K, C) || n < 1 || d < 0 || late_K < 1 || late_K > K) return ORC_EINVAL;
    const long D = d + 1;
    mdc *AA = (mdc *)malloc(sizeof(mdc) * (size_t)D * n * n);
    mdc *B = (mdc *)malloc(sizeof(mdc) * (size_t)n * D);
    mdc *X = (mdc *)calloc((size_t)n * D, sizeof(mdc));
    soa_to_mdc(A, K, C, D * n * n, AA);
    soa_to_mdc(b, K, C, (long)n * D, B);
    int rc = block_solve(K, C, n, d, AA, B, X, late_stage, late_K);
    mdc_to_soa(X, K, C, (long)n * D, dx);
    free(X);
    free(B);
    free(AA);
    return rc;
}

int orc_toeplitz_residual(int K, int C, int n, int d, const double *A, const double *b, const double *dx,
                          const int32_t *rows, int count, double *r, double *norm) {
    if (check_kc(K, C) || n < 1 || d < 0 || !norm) return ORC_EINVAL;
    if (rows) {
        if (count < 1 || count > n) return ORC_EINVAL;
        for (int q = 0; q < count; ++q)
            if (rows[q] < 0 || rows[q] >= n) return ORC_EINVAL;
    }
    const long D = d + 1;
    mdc *AA = (mdc *)malloc(sizeof(mdc) * (size_t)D * n * n);
    mdc *B = (mdc *)malloc(sizeof(mdc) * (size_t)n * D);
    mdc *X = (mdc *)malloc(sizeof(mdc) * (size_t)n * D);
    mdc *R = r ? (mdc *)malloc(sizeof(mdc) * (size_t)n * D) : NULL;
    soa_to_mdc(A, K, C, D * n * n, AA);
    soa_to_mdc(b, K, C, (long)n * D, B);
    soa_to_mdc(dx, K, C, (long)n * D, X);
    *norm = toeplitz_residual_rows(K, C, n, d, AA, B, X, R, rows, count);
    if (R) {
        mdc_to_soa(R, K, C, (long)n * D, r);
        free(R);
    }
    free(X);
    free(B);
    free(AA);
    return ORC_OK;
}

int orc_newton(int K, int C, int n, int d, int M, const int32_t *eq, const int32_t *vptr,
               const int32_t *vidx, const double *coeff, const double *cst, const double *x0,
               int steps, double *x_out, double *hist) {
    return orc_newton_late(K, C, n, d, M, eq, vptr, vidx, coeff, cst, x0, steps, d + 1, K, x_out, hist);
}

int orc_newton_late(int K, int C, int n, int d, int M, const int32_t *eq, const int32_t *vptr,
                    const int32_t *vidx, const double *coeff, const double *cst, const double *x0,
                    int steps, int late_stage, int late_K, double *x_out, double *hist) {
    if (check_kc(K, C) || check_structure(n, d, M, eq, vptr, vidx) || steps < 0 || late_K < 1 || late_K > K)
        return ORC_EINVAL;
    const long D = d + 1, N = (long)n * D;
    mdc *CF = (mdc *)malloc(sizeof(mdc) * (size_t)(M > 0 ? M : 1) * D);
    mdc *CS = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *X = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *F = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *B = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *DX = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *AA = (mdc *)malloc(sizeof(mdc) * (size_t)D * n * n);
    soa_to_mdc(coeff, K, C, (long)M * D, CF);
    soa_to_mdc(cst, K, C, N, CS);
    soa_to_mdc(x0, K, C, N, X);
    sys_t S = {K, C, n, d, M, eq, vptr, vidx, CF, CS};
    int rc = ORC_OK;
    for (int s = 0; s < steps && rc == ORC_OK; ++s) {
        rc = evaluate(&S, X, F, AA);
        if (rc != ORC_OK) break;
        hist[3 * s + 0] = norm1(F, N, C);
        for (long i = 0; i < N; ++i)
            for (int l = 0; l < KMAX; ++l) {
                B[i].re[l] = -F[i].re[l];
                B[i].im[l] = -F[i].im[l];
            }
        for (long i = 0; i < N; ++i) mdc_zero(&DX[i]);
        rc = block_solve(K, C, n, d, AA, B, DX, late_stage, late_K);
        if (rc != ORC_OK) break;
        hist[3 * s + 1] = toeplitz_residual(K, C, n, d, AA, B, DX);
        cacc_t *t = (cacc_t *)malloc(sizeof(cacc_t));
        for (long i = 0; i < N; ++i) {
            cacc_init(t);
            cacc_add(t, &X[i], K, C, 1.0);
            cacc_add(t, &DX[i], K, C, 1.0);
            cacc_round(t, K, C, &X[i]);
        }
        free(t);
        hist[3 * s + 2] = norm1(DX, N, C);
    }
    mdc_to_soa(X, K, C, N, x_out);
    free(AA);
    free(DX);
    free(B);
    free(F);
    free(X);
    free(CS);
    free(CF);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of the converged series (real systems)                             */
/* ------------------------------------------------------------------------- */

/* Fabry-ratio loss (the ratio theorem of Section 1.3: c_d / c_{d+1} of a
 * series tends to its nearest singularity):
 *   L = sum_i x_{i,d}^2 + x_{0,d-1} / x_{0,d},
 * and g = dL/dx: 2 x_{i,d} at coefficient d of every variable, plus
 * -x_{0,d-1} / x_{0,d}^2 there for variable 0 and 1 / x_{0,d} at its
 * coefficient d-1; zero elsewhere.  Real data, d >= 1. */
int orc_fabry_loss(int K, int n, int d, const double *x, double *loss, double *g) {
    if (check_kc(K, 1) || n < 1 || d < 1) return ORC_EINVAL;
    const long D = d + 1, N = (long)n * D;
    mdc *X = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *G = (mdc *)calloc((size_t)N, sizeof(mdc));
    soa_to_mdc(x, K, 1, N, X);
    int rc = ORC_OK;
    acc_t *s = (acc_t *)malloc(sizeof(acc_t));
    acc_init(s);
    for (int i = 0; i < n; ++i) {
        const mdc *xd = &X[(size_t)i * D + d];
        acc_add_prod(s, xd->re, xd->re, K, 1.0);
        for (int l = 0; l < K; ++l) G[(size_t)i * D + d].re[l] = 2.0 * xd->re[l];
    }
    double ratio[KMAX] = {0}, inv[KMAX] = {0}, one[KMAX] = {1.0}, t[KMAX] = {0};
    rc |= md_div_real(X[d - 1].re, X[d].re, K, ratio);
    rc |= md_div_real(one, X[d].re, K, inv);
    acc_add_md(s, ratio, K, 1.0);
    double L[KMAX];
    acc_round(s, K, L);
    memcpy(G[d - 1].re, inv, sizeof(double) * K);
    /* -ratio / x_{0,d} added to 2 x_{0,d} */
    rc |= md_div_real(ratio, X[d].re, K, t);
    acc_init(s);
    acc_add_md(s, G[d].re, K, 1.0);
    acc_add_md(s, t, K, -1.0);
    acc_round(s, K, G[d].re);
    for (int l = 0; l < K; ++l) loss[l] = L[l];
    mdc_to_soa(G, K, 1, N, g);
    free(s);
    free(G);
    free(X);
    return rc;
}

/* Gradient of a loss of the converged series with respect to every
 * coefficient series of the system.  At the solution f(x(c), c) = 0, so
 * dL/dc = -lambda^T df/dc with J^T lambda = g, J the block lower triangular
 * Toeplitz Jacobian of Eq. (eqToeplitz) (blocks A_0 .. A_d).  J^T is block
 * upper triangular:
 *   lambda_k = A_0^{-T} (g_k - sum_{j=1..d-k} A_j^T lambda_{k+j}),  k = d..0,
 * with A_0^{-T} = Q R^{-T} from the Householder QR of A_0 (Section 5.3).
 * Coefficient j of c_m enters f_{eq(m),k} through [t^{k-j}] p_m, p_m the
 * product of the monomial's variables, so
 *   grad c_{m,j} = -sum_{k=j..d} lambda_{eq(m),k} p_m[k-j]   (a correlation).
 * x and g [K][1][n][d+1], grad [K][1][M][d+1]; real data. */
int orc_adjoint(int K, int C, int n, int d, int M, const int32_t *eq, const int32_t *vptr,
                const int32_t *vidx, const double *coeff, const double *x, const double *g, double *grad) {
    if (check_kc(K, C) || C != 1 || check_structure(n, d, M, eq, vptr, vidx)) return ORC_EINVAL;
    const long D = d + 1, N = (long)n * D;
    mdc *CF = (mdc *)malloc(sizeof(mdc) * (size_t)(M > 0 ? M : 1) * D);
    mdc *X = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *G = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *F = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *AA = (mdc *)malloc(sizeof(mdc) * (size_t)D * n * n);
    mdc *LAM = (mdc *)calloc((size_t)N, sizeof(mdc));
    mdc *GR = (mdc *)calloc((size_t)(M > 0 ? M : 1) * D, sizeof(mdc));
    soa_to_mdc(coeff, K, C, (long)M * D, CF);
    soa_to_mdc(x, K, C, N, X);
    soa_to_mdc(g, K, C, N, G);
    sys_t S = {K, C, n, d, M, eq, vptr, vidx, CF, NULL};
    int rc = evaluate(&S, X, F, AA);
    qr_t Q;
    memset(&Q, 0, sizeof Q);
    if (rc == ORC_OK) rc = qr_factor(AA, n, K, C, &Q);
    if (rc == ORC_OK) {
        mdc *r = (mdc *)malloc(sizeof(mdc) * (size_t)n);
        mdc *y = (mdc *)malloc(sizeof(mdc) * (size_t)n);
        cacc_t *t = (cacc_t *)malloc(sizeof(cacc_t));
        for (int k = d; k >= 0 && rc == ORC_OK; --k) {
            for (int i = 0; i < n; ++i) {
                cacc_init(t);
                cacc_add(t, &G[(size_t)i * D + k], K, C, 1.0);
                for (int j = 1; j <= d - k; ++j)
                    for (int l = 0; l < n; ++l)
                        cacc_add_prod(t, &AA[((size_t)j * n + l) * n + i], &LAM[(size_t)l * D + k + j], K, C, -1.0);
                cacc_round(t, K, C, &r[i]);
            }
            /* R^T y = r: forward substitution */
            for (int i = 0; i < n; ++i) {
                mdc num;
                cacc_init(t);
                cacc_add(t, &r[i], K, C, 1.0);
                for (int l = 0; l < i; ++l) cacc_add_prod(t, &Q.R[(size_t)l * n + i], &y[l], K, C, -1.0);
                cacc_round(t, K, C, &num);
                rc |= mdc_div(&num, &Q.R[(size_t)i * n + i], K, C, &y[i]);
            }
            /* lambda_k = Q y = H_0 H_1 ... H_{n-1} y (real reflectors are symmetric) */
            for (int j = n - 1; j >= 0; --j) qr_reflect(&Q, j, y);
            for (int i = 0; i < n; ++i) LAM[(size_t)i * D + k] = y[i];
        }
        free(t);
        free(y);
        free(r);
    }
    if (rc == ORC_OK) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int m = 0; m < M; ++m) {
            const int i = eq[m];
            mdc *p = (mdc *)calloc((size_t)D, sizeof(mdc));
            p[0].re[0] = 1.0;
            for (int q = vptr[m]; q < vptr[m + 1]; ++q) series_mul(p, &X[(size_t)vidx[q] * D], p, d, K, C);
            cacc_t *t = (cacc_t *)malloc(sizeof(cacc_t));
            for (int j = 0; j < D; ++j) {
                cacc_init(t);
                for (int k = j; k < D; ++k) cacc_add_prod(t, &LAM[(size_t)i * D + k], &p[k - j], K, C, -1.0);
                cacc_round(t, K, C, &GR[(size_t)m * D + j]);
            }
            free(t);
            free(p);
        }
        mdc_to_soa(GR, K, C, (long)M * D, grad);
    }
    qr_free(&Q);
    free(GR);
    free(LAM);
    free(AA);
    free(F);
    free(G);
    free(X);
    free(CF);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Staggered orders with the QR of A_0 once (Sections 4 and 5.3)              */
/* ------------------------------------------------------------------------- */

/* Number of coefficients of step s: 1 for s < first_steps (Newton on x_0
 * alone until it is accurate), then L := min(D, L + 1 + L/2) per step (the
 * growth of Section 4, optimistic about quadratic convergence). */
static int stagger_order(int s, int first_steps, int D) {
    if (s < first_steps) return 1;
    int L = 1;
    for (int t = first_steps; t <= s; ++t) {
        L = L + 1 + L / 2;
        if (L >= D) return D;
    }
    return L;
}

/* Newton's method with staggered orders: step s works on the coefficients
 * 0..L_s-1 only (the truncated system is the system mod t^{L_s}: f, A_j and
 * the update of those coefficients depend on no higher one).  Steps
 * s < first_steps factor A_0 at their own x_0; later steps reuse the last of
 * those factorizations (the QR once, valid when x_0 is accurate to about half
 * the working precision).  hist [steps][3] as in orc_newton over the active
 * coefficients; orders [steps] receives L_s. */
int orc_newton_staggered(int K, int C, int n, int d, int M, const int32_t *eq, const int32_t *vptr,
                         const int32_t *vidx, const double *coeff, const double *cst, const double *x0,
                         int steps, int first_steps, double *x_out, double *hist, int32_t *orders) {
    if (check_kc(K, C) || check_structure(n, d, M, eq, vptr, vidx) || steps < 0 || first_steps < 1)
        return ORC_EINVAL;
    const int D = d + 1;
    const long N = (long)n * D;
    mdc *CF = (mdc *)malloc(sizeof(mdc) * (size_t)(M > 0 ? M : 1) * D);
    mdc *CS = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *X = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    soa_to_mdc(coeff, K, C, (long)M * D, CF);
    soa_to_mdc(cst, K, C, N, CS);
    soa_to_mdc(x0, K, C, N, X);
    /* truncated copies, [.][L] */
    mdc *CFL = (mdc *)malloc(sizeof(mdc) * (size_t)(M > 0 ? M : 1) * D);
    mdc *CSL = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *XL = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *F = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *B = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *DX = (mdc *)malloc(sizeof(mdc) * (size_t)N);
    mdc *AA = (mdc *)malloc(sizeof(mdc) * (size_t)D * n * n);
    qr_t Q;
    memset(&Q, 0, sizeof Q);
    int have_q = 0, rc = ORC_OK;
    for (int s = 0; s < steps && rc == ORC_OK; ++s) {
        const int L = stagger_order(s, first_steps, D);
        orders[s] = L;
        for (int m = 0; m < M; ++m)
            for (int k = 0; k < L; ++k) CFL[(size_t)m * L + k] = CF[(size_t)m * D + k];
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < L; ++k) {
                CSL[(size_t)i * L + k] = CS[(size_t)i * D + k];
                XL[(size_t)i * L + k] = X[(size_t)i * D + k];
            }
        sys_t S = {K, C, n, L - 1, M, eq, vptr, vidx, CFL, CSL};
        rc = evaluate(&S, XL, F, AA);
        if (rc != ORC_OK) break;
        const long NL = (long)n * L;
        hist[3 * s + 0] = norm1(F, NL, C);
        for (long i = 0; i < NL; ++i)
            for (int l = 0; l < KMAX; ++l) {
                B[i].re[l] = -F[i].re[l];
                B[i].im[l] = -F[i].im[l];
            }
        for (long i = 0; i < NL; ++i) mdc_zero(&DX[i]);
        if (s < first_steps) {
            if (have_q) qr_free(&Q);
            rc = qr_factor(AA, n, K, C, &Q);
            have_q = 1;
            if (rc != ORC_OK) break;
        }
        rc = block_stages(K, C, n, L - 1, AA, B, DX, L, K, &Q);
        if (rc != ORC_OK) break;
        hist[3 * s + 1] = toeplitz_residual(K, C, n, L - 1, AA, B, DX);
        cacc_t *t = (cacc_t *)malloc(sizeof(cacc_t));
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < L; ++k) {
                mdc *xv = &X[(size_t)i * D + k];
                cacc_init(t);
                cacc_add(t, xv, K, C, 1.0);
                cacc_add(t, &DX[(size_t)i * L + k], K, C, 1.0);
                cacc_round(t, K, C, xv);
            }
        free(t);
        hist[3 * s + 2] = norm1(DX, NL, C);
    }
    if (have_q) qr_free(&Q);
    mdc_to_soa(X, K, C, N, x_out);
    free(AA);
    free(DX);
    free(B);
    free(F);
    free(XL);
    free(CSL);
    free(CFL);
    free(X);
    free(CS);
    free(CF);
    return rc;
}
