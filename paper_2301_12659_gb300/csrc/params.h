// params.h -- kernel parameter blocks shared by the host runtime and the
// CUDA kernels of libmdnewton.  Arrays of md values use the [K][C][N] layout;
// the N of each array is stored beside its pointer.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mdn {

constexpr int ED_THREADS = 256;
constexpr int QR_THREADS = 128;  // 4 warps: one per SM sub-partition
constexpr int FS_THREADS = 256;
constexpr int FX_THREADS = 128;

// device status bits (OR-ed by kernels, mapped to mdn_status by the host)
constexpr int MDN_DEV_SINGULAR = 1;
constexpr int MDN_DEV_NONFINITE = 2;
constexpr int MDN_DEV_TIMEOUT = 4;

// slot kinds of the evaluation/differentiation schedule: code = kind<<16 | index
enum SlotKind { SLOT_NONE = 0, SLOT_C = 1, SLOT_X = 2, SLOT_F = 3, SLOT_B = 4, SLOT_V = 5, SLOT_P = 6 };
enum OpKind { OP_NONE = 0, OP_PRODUCT = 1, OP_COPY = 2 };

struct EdParams {
  int n, D, M, P, G, kmax, Smax, Wtot;
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

struct AsmParams {
  int n, D;
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
  int n, nA;
  const double* A0;
  long long NA;   // stride of the A array the A0 slice lives in
  long long Nnn;  // n*n
  double* Rm;
  double* Vm;
  double* Y;
  double* W;
  double* tau;   // [K][n]
  double* rinv;  // [K][C][n]
  unsigned* flags;  // [2n]
  const unsigned* epoch;
  int* status;
  long long spin_limit;  // nanoseconds a flag wait may last
};

struct FsParams {
  int n, D, rhs_sign;
  const double* A;
  long long NA;
  const double* W;
  long long Nnn;
  const double* rhs;
  double* r;
  double* dx;
  long long Nx;
  double* resabs;
};

struct UpdParams {
  int n, D;
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
  double* hist;  // 3 values
};

// Launchers of one (K, C) instantiation.
struct KernelTable {
  int K, C;
  cudaError_t (*ed)(const EdParams&, int grid, cudaStream_t);
  int (*ed_blocks_per_sm)();
  cudaError_t (*assemble)(const AsmParams&, bool want_A, cudaStream_t);
  cudaError_t (*qr)(const QrParams&, cudaStream_t);
  cudaError_t (*fs)(const FsParams&, int k, cudaStream_t);
  cudaError_t (*fx)(const FsParams&, int k, cudaStream_t);
  cudaError_t (*update)(const UpdParams&, cudaStream_t);
};

const KernelTable* kernels_for(int K, int C);

}  // namespace mdn
