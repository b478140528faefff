// params.h -- kernel parameter blocks shared by the host runtime and the
// CUDA kernels of libmdnewton.  Arrays of md values use the [K][C][N] layout;
// the N of each array is stored beside its pointer.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "xf.cuh"

namespace mdn {

constexpr int ED_THREADS = 128;  // 4 warps: one per SM sub-partition
constexpr int QR_THREADS = 128;  // 4 warps: one per SM sub-partition
constexpr int QR_SMEM_RESERVE = 116 * 1024;  // any two reserving blocks exceed an SM's shared memory
constexpr int QR_SMEM_MAX = 227 * 1024;      // dynamic shared memory a block may use
constexpr int FSUB_THREADS = 128;  // 4 warps per block, one block per SM
constexpr int FSUB_WBLOCKS = 16;   // blocks of solve warps

// device status bits (OR-ed by kernels, mapped to mdn_status by the host)
constexpr int MDN_DEV_SINGULAR = 1;
constexpr int MDN_DEV_NONFINITE = 2;
constexpr int MDN_DEV_TIMEOUT = 4;

// slot kinds of the evaluation/differentiation schedule: code = kind<<16 | index
enum SlotKind { SLOT_NONE = 0, SLOT_C = 1, SLOT_X = 2, SLOT_F = 3, SLOT_B = 4, SLOT_V = 5, SLOT_P = 6 };
enum OpKind { OP_NONE = 0, OP_PRODUCT = 1, OP_COPY = 2 };

struct EdParams {
  int n, D, M, P, G, kmax, Smax, Wtot;
  int len;  // coefficients computed (<= D, the stride); P and G are those of len
  int smem;  // shared memory each block reserves (sets the blocks per SM)
  const double* x;
  long long Nx;  // n*D
  const double* coeff;
  long long Nc;  // M*D
  double* out;
  long long No;  // S*D (value and partials of every monomial)
  double* scratch;
  long long Ns;  // Wtot*Smax*D (forward/backward products, per warp)
  const int* order;
  const int* mono_k;
  const int* mono_vp;
  const int* mono_sbase;
  const int* vidx;
  const int4* sched;
  const int* sched_off;
  const int* sched_nw;
  int* counter;
};

// Leading Jacobian block A_0 = J(x_0) from the constant coefficients only.
struct A0Params {
  int n, D, M;
  const double* x;
  long long Nx;
  int xstride;  // distance between the constant coefficients of two variables in x
  const double* coeff;
  long long Nc;
  const int* mono_k;
  const int* mono_vp;
  const int* mono_sbase;
  const int* vidx;
  int nnz;
  const int* occ_mono;  // [nnz] monomial of each occurrence
  double* out0;         // [K][C][S] partial at t^0 of every slot
  long long S;
  const int* pair_ptr;
  const int* pair_slot;
  double* A;            // A_0 written into the j = 0 slice of [K][C][D][n][n]
  long long NA;
  int kmax;             // largest monomial: beyond 32 variables a warp per monomial
};

struct AsmParams {
  int n, D, j_begin;
  int len;  // coefficients assembled (<= D)
  const double* out;
  long long No;
  const double* cst;
  double* f;
  long long Nf;  // n*D
  double* A;
  long long NA;  // D*n*n
  const int* eq_ptr;
  const int* eq_mon;
  const int* mono_sbase;
  const int* pair_ptr;
  const int* pair_slot;
};

struct QrParams {
  int n;
  int nAc, nAi, nAz;  // blocks: columns of A0 (4 each), identity columns (4), rows of R^{-1} (8)
  const double* A0;
  long long NA;   // stride of the A array the A0 slice lives in
  long long Nnn;  // n*n
  uint64_t* Rm;  // R and the reflectors x_j, as extended floats [W+1][C][n][n]
  uint64_t* Vm;  // (W mantissa words and a word of exponent and sign); Vm column-major
  double* Y;  // Q^H (identity columns under all reflectors)
  double* Z;  // R^{-1}
  double* W;
  // scalars of reflector j, as extended floats ([W+1][n] or [W+1][C][n])
  uint64_t* tau;
  uint64_t* rinv;    // 1 / R_jj
  uint64_t* salpha;  // s_j |x_j| (R_jj = -salpha_j)
  uint64_t* v0;      // leading entry of reflector j
  unsigned* flags;  // [4n]: column, reflector (tau), 1/R_jj, and s_j|x_j| with v_jj published
  const unsigned* epoch;
  int* status;
  long long spin_limit;  // nanoseconds a flag wait may last
  int skip_w;  // 1: the launcher leaves W = Z Y to the w launcher (Newton's pipeline)
  // column-by-column variant for large n (no waits): the columns of A0 and
  // of the identity under the reflectors, as extended floats, column-major
  // ([W+1][C][n columns][n rows], element (i, c) at c*n + i)
  int large;
  uint64_t* Aw;
  uint64_t* Yw;
};

// Persistent forward substitution (one cooperative launch per solve).
struct FsubParams {
  int n, D, rhs_sign;
  int first_stage;  // 1 when stage 0 (dx_0 = W r_0) was done by stage0_kernel
  int nW;       // solve warps (dx_k = W r_k), on the first nW/4 blocks
  int nOwn;     // owner warps of the r_k[i] accumulators
  int late_stage;  // stages k >= late_stage form their updates in K/2 limbs (D: never)
  int nst;         // stages solved (<= D; staggered orders)
  int smem;        // shared memory each block reserves (sets the blocks per SM)
  const int* resmask;  // rows whose residual the monitor forms (null: all)
  int transpose;   // 1: use A_j^T and W^T (the adjoint's solve with J^T)
  int reverse;     // 1: stage k works on coefficient D-1-k (J^T is block upper triangular)
  const double* A;
  long long NA;  // D*n*n (slices j >= 1 are read)
  const double* A0;
  long long NA0;  // stride of the array holding A_0
  const double* W;
  long long Nnn;
  const double* rhs;
  double* r;     // accumulators, then r_k[i]   [K][C][n][D]
  const double* Zs;  // stage 0 from the factors: dx_0 = Z (Y r_0) when not null
  const double* Ys;  //   (Z = R^{-1}, Y = Q^H, before W = Z Y is formed)
  double* t0;        //   Y r_0 [K][C][n]
  const double* x;   // stage0_kernel: current series, x_0 + dx_0 goes to xnext0
  double* xnext0;    // [K][C][n]
  double* dx;
  long long Nx;  // n*D
  double* resabs;
  unsigned* rdone;  // [D] rows of r_k finished
  unsigned* xdone;  // [D] rows of dx_k finished
  int* status;
  long long spin_limit;
};

struct UpdParams {
  int n, D;
  int len;  // coefficients updated (<= D)
  double* x;
  const double* dx;
  const double* f;
  long long Nx;
  double* dxabs;
  double* fabs;
  int* status;
};

struct NormParams {
  long long count;
  const double* fabs;
  const double* resabs;
  const double* dxabs;
  double res_scale;  // n / sampled rows of the residual monitor
  double* hist;  // 3 values
};

// Launchers of one (K, C) instantiation.
// Adjoint of the coefficient series: grad[m][j] = -sum_{k>=j} lam_{eq(m),k} [t^{k-j}] prod x_v.
struct AdjParams {
  int n, D, M, P, G, Wtot;
  const int* mono_eq;
  const int* mono_vp;
  const int* mono_k;
  const int* vidx;
  const double* x;
  long long Nx;      // n*D
  const double* lam;
  double* grad;      // [K][C][M][D]
  long long Ng;      // M*D
  double* scratch;   // per warp 2*G series of D
  long long Ns;
};
// Fabry-ratio loss of a real series and its gradient.
struct LossParams {
  int n, D;
  const double* x;
  long long Nx;
  double* loss;  // [K]
  double* g;     // [K][1][n][D]
};

// Residual of the block Toeplitz system (mdn_residual): one warp per entry.
struct ResParams {
  int n, D;
  const double* A;
  long long NA;  // D*n*n
  const double* b;
  const double* dx;
  long long Nx;  // n*D
  double* r;         // md residual series [K][C][n][D] (may be null)
  double* resabs;    // |leading double| per entry, zero outside the row sample
  const int* resmask;  // rows in the sampled norm (null: all)
};

// out = s * a for one md scalar s and an md array a (mdn_md_scale).
struct ScaleParams {
  const double* s;  // [K][C] (N = 1)
  const double* a;
  double* out;
  long long N;
};

// ---- batched systems (one persistent launch) ----
struct BatchSys {
  int n, D, M, mono0;      // monomials mono0 .. mono0+M-1 (global numbering)
  int eq0;                 // eq_ptr[eq0 .. eq0+n] delimit the monomials of each equation
  int pad;
  long long coeff_off;     // doubles: start of this system's [K][C][M][D] coefficients
  long long series_off;    // doubles: start of its [K][C][n][D] series (x, constant term, f)
};

enum : int { BATCH_CONVERGED = 1, BATCH_SINGULAR = 2, BATCH_NONFINITE = 4 };

struct BatchParams {
  int count, max_steps, evaluate_only, S3;  // S3: scratch series per lane group
  double tol;
  const BatchSys* sys;
  const int* order;    // systems in decreasing estimated cost
  const int* eq_ptr;   // per system n+1 offsets into eq_mon
  const int* eq_mon;   // monomials grouped by equation, larger ones first
  const int* vptr;     // [Mtot+1] CSR offsets (global)
  const int* vidx;     // variable of each occurrence (local to its system)
  const double* coeff;
  const double* cst;
  double* x;           // packed series, updated in place
  double* f_out;       // evaluate_only: packed f(x)
  double* work;        // per-block scratch
  long long work_stride;  // doubles per block
  int* queue;
  int* steps_out;
  int* flags_out;
};

__host__ __device__ inline long long batch_work_doubles(int K, int C, int n, int D, int threads, int S3) {
  const int W = threads / 32, P = (D + 1) / 2, G = 32 / P;
  const long long KC = (long long)K * C;
  const long long nn = (long long)n * n;
  long long s = 0;
  s += KC * D * nn;                      // A
  s += 2 * KC * n * D;                   // f, dx
  s += KC * nn;                          // Y, then W
  s += KC * n;                           // r
  s += (long long)K * n;                 // tau
  s += 3 * KC * n;                       // s|x|, v0, 1/R_jj
  s += KC * threads;                     // partial sums
  s += KC * (long long)W * G * S3 * D;   // products of the evaluation
  return s + 64;
}


// 64-bit words of one real extended float as the QR stores it: the
// mantissa words and one word of exponent and sign.
__host__ __device__ inline int qr_xf_words(int K) { return xfn::xf_words_of(K) + 1; }
// Shared memory of a QR block: four columns of A0 or of the identity, or
// eight rows of R^{-1} (n complex extended floats each).
__host__ __device__ inline size_t qr_smem_bytes(int n, int K) {
  return 8 * (size_t)n * 2 * qr_xf_words(K) * sizeof(uint64_t);
}
// Blocks of the QR launch: columns of A0 (4 per block), columns of the
// identity (4 per block), pairs of rows of R^{-1} (4 pairs per block).
__host__ __device__ inline int qr_blocks_for(int n) { return (n + 3) / 4 + (n + 3) / 4 + ((n + 1) / 2 + 3) / 4; }

struct KernelTable {
  int K, C;
  cudaError_t (*ed)(const EdParams&, int grid, cudaStream_t);
  cudaError_t (*a0)(const A0Params&, cudaStream_t);
  int (*ed_blocks_per_sm)();
  cudaError_t (*assemble)(const AsmParams&, bool want_A, cudaStream_t);
  cudaError_t (*qr)(const QrParams&, cudaStream_t);  // QR, Q^H, R^{-1}, then W = R^{-1} Q^H
  cudaError_t (*qr_w)(const QrParams&, cudaStream_t);  // W = Z Y alone
  cudaError_t (*fsub)(const FsubParams&, cudaStream_t);
  cudaError_t (*stage0)(const FsubParams&, cudaStream_t);
  cudaError_t (*update)(const UpdParams&, cudaStream_t);
  cudaError_t (*adjoint)(const AdjParams&, cudaStream_t);
  cudaError_t (*fabry)(const LossParams&, cudaStream_t);
  cudaError_t (*batch)(const BatchParams&, int blocks, int threads, cudaStream_t);
  int (*batch_occupancy)(int threads);  // resident blocks per SM
  cudaError_t (*residual)(const ResParams&, cudaStream_t);
  cudaError_t (*scale)(const ScaleParams&, cudaStream_t);
};

const KernelTable* kernels_for(int K, int C);

}  // namespace mdn
