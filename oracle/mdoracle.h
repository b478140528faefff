/*
 * mdoracle.h -- C interface of the CPU oracle (test infrastructure only).
 *
 * The oracle is a plain, slow, obviously-correct CPU implementation of Newton's
 * method on truncated power series in multiple double arithmetic (Verschelde,
 * "GPU Accelerated Newton for Taylor Series Solutions of Polynomial Homotopies
 * in Multiple Double Precision", arXiv 2301.12659).  Only the tests, the smoke
 * check and the CPU-baseline leg of bench.py may load it; the product library
 * (include/mdnewton.h) shares no code with it and never links it.
 *
 * Every array argument is a host pointer in the same structure-of-arrays
 * layout the product uses (Section 1.2: one array per limb), limb-major:
 *   series   x[K][C][n][d+1]      coefficient k of variable v at ((l*C+c)*n+v)*(d+1)+k
 *   coeffs   c[K][C][M][d+1]
 *   matrices A[K][C][d+1][n][n]  entry (j,i,v) at (((l*C+c)*(d+1)+j)*n+i)*n+v
 * with K limbs (2 double double, 4 quad double, 8 octo double), C = 1 (real)
 * or 2 (complex; c = 0 real part, c = 1 imaginary part), n variables and
 * equations, truncation degree d (d+1 coefficients), M monomials.
 *
 * Return codes: 0 ok, 1 invalid argument, 2 zero pivot in the QR of A0,
 * 3 non-finite value, 4 expansion capacity exceeded (cannot happen for finite
 * doubles; kept as a guard).
 */
#ifndef MDORACLE_H
#define MDORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

void orc_set_threads(int nthreads);
int orc_get_threads(void);

/* Elementwise md arithmetic on N values stored [K][C][N] (pins and tests).
 * op: 0 add, 1 sub, 2 mul, 3 div.  Complex (C = 2) supported for all four. */
int orc_md_binary(int op, int K, int C, int N, const double *a, const double *b, double *r);
/* Square root of N real md values [K][N] (a >= 0). */
int orc_md_sqrt(int K, int N, const double *a, double *r);

/* Truncated series product c = a*b mod t^(d+1) for one series pair [K][C][d+1]
 * (Section 5.1: c_k = sum_{i=0..k} a_i b_{k-i}). */
int orc_series_mul(int K, int C, int d, const double *a, const double *b, double *c);

/* Evaluation and differentiation (Section 5.1) of the system
 *   f_i(x(t)) = sum_{m : eq[m] = i} coeff_m(t) * prod_{p} x_{vidx[p]}(t) + cst_i(t)
 * at x(t): f[K][C][n][d+1], and when A != NULL the Jacobian series
 * A[K][C][d+1][n][n], A_j[i][v] = [t^j] d f_i / d x_v.  Monomial m uses
 * variables vidx[vptr[m] .. vptr[m+1]-1]; a repeated variable is a power. */
int orc_evaluate(int K, int C, int n, int d, int M, const int32_t *eq, const int32_t *vptr,
                 const int32_t *vidx, const double *coeff, const double *cst, const double *x,
                 double *f, double *A);

/* Constant term that plants x*(t) as a solution: cst = -(f(x*) with cst = 0),
 * evaluated in octo double from the K-limb inputs and rounded to K limbs. */
int orc_planted_constant(int K, int C, int n, int d, int M, const int32_t *eq,
                         const int32_t *vptr, const int32_t *vidx, const double *coeff,
                         const double *xstar, double *cst);

/* Householder QR of one n-by-n md matrix A0 [K][C][n][n] (Section 5.3).
 * Outputs the explicit unitary Q [K][C][n][n] and upper triangular R. */
int orc_qr(int K, int C, int n, const double *A0, double *Q, double *R);

/* Solve the block lower triangular Toeplitz system of Eq. (eqToeplitz),
 *   sum_{j=0..k} A_j dx_{k-j} = b_k   (k = 0..d),
 * by Householder QR of A0 and forward substitution.  A [K][C][d+1][n][n],
 * b and dx [K][C][n][d+1]. */
int orc_solve(int K, int C, int n, int d, const double *A, const double *b, double *dx);
/* The same with the stated-accuracy variant of the updates: stages
 * k >= late_stage form sum_{j>=1} A_j dx_{k-j} in late_K limbs (operands and
 * sum rounded to late_K limbs), everything else in K limbs. */
int orc_solve_late(int K, int C, int n, int d, const double *A, const double *b, int late_stage, int late_K,
                   double *dx);

/* Residual of the block lower triangular Toeplitz system of Eq. (eqToeplitz)
 * (the residuals of Sections 5.4 and 6): r_k = b_k - sum_{j=0..k} A_j dx_{k-j},
 * each entry its exact value rounded once to K limbs, into r [K][C][n][d+1]
 * (may be NULL), and *norm = its 1-norm of leading doubles (|re| or hypot).
 * With rows != NULL only the `count` distinct rows listed enter the norm,
 * scaled by n / count (the sampled monitor of Section 5.4). */
int orc_toeplitz_residual(int K, int C, int n, int d, const double *A, const double *b, const double *dx,
                          const int32_t *rows, int count, double *r, double *norm);

/* Newton's method on power series (Section 2 pseudo code): `steps` iterations
 * from x0, no early exit.  x_out [K][C][n][d+1]; hist [steps][3] holds per
 * step ||f(x)||_1 before the update, the monitor ||b - A dx||_1 and ||dx||_1
 * (each the 1-norm of the leading doubles of the md entries). */
int orc_newton(int K, int C, int n, int d, int M, const int32_t *eq, const int32_t *vptr,
               const int32_t *vidx, const double *coeff, const double *cst, const double *x0,
               int steps, double *x_out, double *hist);
/* Newton with the late-update variant of orc_solve_late in every step. */
int orc_newton_late(int K, int C, int n, int d, int M, const int32_t *eq, const int32_t *vptr,
                    const int32_t *vidx, const double *coeff, const double *cst, const double *x0,
                    int steps, int late_stage, int late_K, double *x_out, double *hist);

/* Newton with staggered orders and the QR once (Sections 4 and 5.3): step s
 * works on the first L_s coefficients, L_s = 1 for s < first_steps and then
 * L := min(d+1, L + 1 + L/2) per step; steps s < first_steps factor A_0, later
 * steps reuse the last factorization.  orders [steps] receives L_s. */
int orc_newton_staggered(int K, int C, int n, int d, int M, const int32_t *eq, const int32_t *vptr,
                         const int32_t *vidx, const double *coeff, const double *cst, const double *x0,
                         int steps, int first_steps, double *x_out, double *hist, int32_t *orders);

/* Fabry-ratio loss L = sum_i x_{i,d}^2 + x_{0,d-1} / x_{0,d} of a real series
 * x [K][1][n][d+1] (d >= 1): loss [K] and g = dL/dx [K][1][n][d+1]. */
int orc_fabry_loss(int K, int n, int d, const double *x, double *loss, double *g);

/* Adjoint: gradient [K][1][M][d+1] of a loss with dL/dx = g with respect to
 * the coefficient series of a real system, at a converged series x:
 * lambda = J^{-T} g by the transposed block triangular solve with
 * A_0^{-T} = Q R^{-T}, then grad c_{m,j} = -sum_{k>=j} lambda_{eq(m),k}
 * [t^{k-j}] prod_{v in m} x_v. */
int orc_adjoint(int K, int C, int n, int d, int M, const int32_t *eq, const int32_t *vptr,
                const int32_t *vidx, const double *coeff, const double *x, const double *g, double *grad);

#ifdef __cplusplus
}
#endif
#endif
