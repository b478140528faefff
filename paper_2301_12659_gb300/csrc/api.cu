// api.cu -- host runtime of libmdnewton: the C-ABI of include/mdnewton.h.
//
// The runtime owns no device memory.  mdn_load_system() lays out the
// caller's workspace, builds on the host the tables the kernels read
// (monomial order for the dynamic work queue, the product schedule of every
// monomial size, the gather lists of f and A) and copies them in.  A Newton
// step (Section 2) is then a fixed sequence of launches on the caller's
// stream: evaluation and differentiation, assembly, QR of A0 and its
// inverse, d+1 forward substitution stages, update and norms.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mdnewton.h"
#include "params.h"

namespace mdn {
const KernelTable* kernels_k1_c1();
const KernelTable* kernels_k2_c1();
const KernelTable* kernels_k2_c2();
const KernelTable* kernels_k4_c1();
const KernelTable* kernels_k4_c2();
const KernelTable* kernels_k8_c1();
const KernelTable* kernels_k8_c2();

const KernelTable* kernels_for(int K, int C) {
  if (K == 1 && C == 1) return kernels_k1_c1();
  if (K == 2 && C == 1) return kernels_k2_c1();
  if (K == 2 && C == 2) return kernels_k2_c2();
  if (K == 4 && C == 1) return kernels_k4_c1();
  if (K == 4 && C == 2) return kernels_k4_c2();
  if (K == 8 && C == 1) return kernels_k8_c1();
  if (K == 8 && C == 2) return kernels_k8_c2();
  return nullptr;
}

// Largest monomial for which the schedules of every product length are built.
constexpr int STAGGER_KMAX = 64;

// Bounded waits of the dataflow kernels: two seconds of wall time at most by
// default (mdn_set_wait_limit_ns changes it per context).
constexpr long long SPIN_LIMIT = 2000000000LL;

__global__ void bump_kernel(unsigned* epoch) { *epoch += 1u; }

// Deterministic sums of three magnitude arrays into hist[0..2] (one block,
// fixed order: strided partial sums, then a tree).
__global__ void norms_kernel(NormParams p) {
  __shared__ double sh[3][1024];
  const int t = threadIdx.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (long long i = t; i < p.count; i += blockDim.x) {
    s0 += p.fabs[i];
    s1 += p.resabs[i];
    s2 += p.dxabs[i];
  }
  sh[0][t] = s0;
  sh[1][t] = s1;
  sh[2][t] = s2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (t < w) {
      sh[0][t] += sh[0][t + w];
      sh[1][t] += sh[1][t + w];
      sh[2][t] += sh[2][t + w];
    }
    __syncthreads();
  }
  if (t == 0) {
    p.hist[0] = sh[0][0];
    p.hist[1] = sh[1][0] * p.res_scale;
    p.hist[2] = sh[2][0];
  }
}

// ---------------------------------------------------------------------------
// Product schedule of one monomial with k variables (Section 5.1): forward
// products F_j = F_{j-1} x_j (F_0 = c, F_k = value), backward products
// B_j = B_{j-1} x_{k-j+1} (B_1 = x_k) and cross products d_j = F_{j-1} B_{k-j}
// (d_1 = c B_{k-1}, d_k = F_{k-1}): 3k-3 truncated products for k >= 2.
// Tasks are list-scheduled in waves of at most G products that run at once
// in one warp (G groups of lanes), longest remaining chain first.
// ---------------------------------------------------------------------------
static int code(int kind, int idx) { return (kind << 16) | idx; }

static void build_schedule(int k, int G, std::vector<int4>& waves_out, int& nwaves) {
  struct Task {
    int type, dst, a, b;
    std::vector<int> deps;
    int prio;
  };
  std::vector<Task> T;
  auto fcode = [&](int j) {
    if (j == 0) return code(SLOT_C, 0);
    if (j == k) return code(SLOT_V, 0);
    if (j == k - 1) return code(SLOT_P, k - 1);
    return code(SLOT_F, j);
  };
  auto bcode = [&](int j) { return j == 1 ? code(SLOT_X, k - 1) : code(SLOT_B, j); };
  if (k == 1) {
    T.push_back({OP_PRODUCT, code(SLOT_V, 0), code(SLOT_C, 0), code(SLOT_X, 0), {}, 0});
    T.push_back({OP_COPY, code(SLOT_P, 0), code(SLOT_C, 0), 0, {}, 0});
  } else {
    std::vector<int> fidx(k + 1, -1), bidx(k + 1, -1);
    for (int j = 1; j <= k; ++j) {
      Task t{OP_PRODUCT, fcode(j), fcode(j - 1), code(SLOT_X, j - 1), {}, 0};
      if (j >= 2) t.deps.push_back(fidx[j - 1]);
      fidx[j] = (int)T.size();
      T.push_back(t);
    }
    for (int j = 2; j <= k - 1; ++j) {
      Task t{OP_PRODUCT, bcode(j), bcode(j - 1), code(SLOT_X, k - j), {}, 0};
      if (j >= 3) t.deps.push_back(bidx[j - 1]);
      bidx[j] = (int)T.size();
      T.push_back(t);
    }
    for (int p = 0; p <= k - 2; ++p) {
      const int bj = k - 1 - p;
      Task t{OP_PRODUCT, code(SLOT_P, p), fcode(p), bcode(bj), {}, 0};
      if (p >= 1) t.deps.push_back(fidx[p]);
      if (bj >= 2) t.deps.push_back(bidx[bj]);
      T.push_back(t);
    }
  }
  // priority: length of the longest chain of dependents (tasks only depend on
  // earlier tasks, so a reverse sweep suffices)
  const int nt = (int)T.size();
  std::vector<int> longest(nt, 1);
  for (int i = nt - 1; i >= 0; --i)
    for (int d : T[i].deps) longest[d] = std::max(longest[d], longest[i] + 1);
  // list scheduling: each wave takes the G ready tasks of longest chain (ties
  // by index); tasks that become ready join the next wave
  std::vector<std::vector<int>> dependents(nt);
  std::vector<int> indeg(nt, 0);
  for (int i = 0; i < nt; ++i) {
    indeg[i] = (int)T[i].deps.size();
    for (int d : T[i].deps) dependents[d].push_back(i);
  }
  auto later = [&](int a, int b) { return longest[a] != longest[b] ? longest[a] < longest[b] : a > b; };
  std::vector<int> heap;  // max-heap under `later`
  for (int i = 0; i < nt; ++i)
    if (indeg[i] == 0) heap.push_back(i);
  std::make_heap(heap.begin(), heap.end(), later);
  nwaves = 0;
  std::vector<int> wave;
  while (!heap.empty()) {
    wave.clear();
    while ((int)wave.size() < G && !heap.empty()) {
      std::pop_heap(heap.begin(), heap.end(), later);
      wave.push_back(heap.back());
      heap.pop_back();
    }
    for (int g = 0; g < G; ++g) {
      if (g < (int)wave.size()) {
        const Task& t = T[wave[g]];
        waves_out.push_back(make_int4(t.type, t.dst, t.a, t.b));
      } else {
        waves_out.push_back(make_int4(OP_NONE, 0, 0, 0));
      }
    }
    for (int i : wave)  // finished at the end of this wave
      for (int d : dependents[i])
        if (--indeg[d] == 0) {
          heap.push_back(d);
          std::push_heap(heap.begin(), heap.end(), later);
        }
    ++nwaves;
  }
}

}  // namespace mdn

using namespace mdn;

struct Layout {
  size_t total = 0;
  size_t o_order, o_mono_k, o_mono_vp, o_mono_sbase, o_vidx, o_sched, o_sched_off, o_sched_nw, o_eq_ptr,
      o_eq_mon, o_pair_ptr, o_pair_slot, o_occ, o_counter, o_status, o_flags, o_epoch, o_done;
  size_t o_mono_eq, o_adj, o_resmask;
  size_t o_x, o_f, o_dx, o_r, o_out, o_out0, o_scratch, o_A, o_A0b, o_Rm, o_Vm, o_Y, o_Z, o_W, o_xn0, o_tau, o_rinv, o_salpha, o_v0, o_fabs, o_dxabs,
      o_resabs, o_hist, o_rnorm, o_t0;
};

struct mdn_ctx {
  int K, C, n, d, D;
  const KernelTable* kt = nullptr;
  int num_sms = 0, ed_grid = 0, Wtot = 0;
  int P = 1, G = 1;
  // system (host tables)
  int M = 0, nnz = 0, S = 0, kmax = 1, Smax = 1;
  std::vector<int> order, mono_k, mono_vp, mono_sbase, mono_eq, vidx, sched_off, sched_nw, eq_ptr, eq_mon, pair_ptr,
      pair_slot, occ;
  std::vector<int4> sched;
  bool loaded = false, has_series = false;
  bool solves = true;  // n small enough for the QR of A0 (else evaluation only)
  bool large_qr = false;  // the QR runs column by column in global memory
  int late_stage = 1 << 30;  // stages from here form their updates in K/2 limbs
  int res_rows = 0;          // rows of the sampled residual monitor (0: all)
  int stagger_first = 0;     // staggered orders: order-1 steps with a QR each (0: off)
  long long wait_limit_ns = SPIN_LIMIT;  // bound of every device wait
  int fsub_per_sm = 2;             // owner blocks per SM of the forward substitution
  int ed_per_sm = 1;               // evaluation blocks per SM
  bool qr_running_beside = false;  // a QR of A0 runs on the side stream meanwhile
  std::vector<int> gvals, gidx_of_len;  // lane-group counts of the product lengths 1..D
  const double* coeff = nullptr;
  const double* cst = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;  // the QR of A0 overlaps the evaluation on this stream
  cudaStream_t side2 = nullptr;  // W = Z Y of the pipelined QR, off its critical loop
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_w = nullptr;
  char* ws = nullptr;
  Layout L;
  std::string err;
  // phase timers (mdn_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_rec;
  cudaEvent_t open_ev_of[MDN_NUM_PHASES] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  long long launches[MDN_NUM_PHASES] = {0, 0, 0, 0, 0};
  template <class T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(ws + off);
  }
};

static mdn_status fail(const mdn_ctx* c, mdn_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    const_cast<mdn_ctx*>(c)->err = buf;
  }
  return s;
}

#define CU(call)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return fail(ctx, MDN_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static cudaEvent_t prof_event(mdn_ctx* ctx) {
  if (ctx->ev_used == ctx->ev_pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    ctx->ev_pool.push_back(e);
  }
  return ctx->ev_pool[ctx->ev_used++];
}
// Open a phase: record its start event when the timers run.
static void ph_begin(mdn_ctx* ctx, int phase, cudaStream_t st = nullptr) {
  if (!ctx->prof) return;
  cudaEvent_t e = prof_event(ctx);
  if (!e) return;
  cudaEventRecord(e, st ? st : ctx->stream);
  ctx->open_ev_of[phase] = e;
}
static void ph_end(mdn_ctx* ctx, int phase, int launches, cudaStream_t st = nullptr) {
  ctx->launches[phase] += launches;
  if (!ctx->prof || !ctx->open_ev_of[phase]) return;
  cudaEvent_t e = prof_event(ctx);
  if (!e) return;
  cudaEventRecord(e, st ? st : ctx->stream);
  ctx->prof_rec.push_back({phase, {ctx->open_ev_of[phase], e}});
  ctx->open_ev_of[phase] = nullptr;
}

// Tables that depend only on the structure of the system.
static mdn_status build_tables(mdn_ctx* ctx, int M, const int32_t* eq, const int32_t* vptr, const int32_t* vidx) {
  const int n = ctx->n;
  if (M < 1 || !vptr) return fail(ctx, MDN_EINVAL, "need at least one monomial and var_ptr");
  if (vptr[0] != 0) return fail(ctx, MDN_EINVAL, "var_ptr[0] must be 0");
  int kmax = 1;
  for (int m = 0; m < M; ++m) {
    const int k = vptr[m + 1] - vptr[m];
    if (k < 1) return fail(ctx, MDN_EINVAL, "monomial %d has no variable", m);
    if (k > 4096) return fail(ctx, MDN_EINVAL, "monomial %d has %d variables (max 4096)", m, k);
    kmax = std::max(kmax, k);
  }
  ctx->M = M;
  ctx->nnz = vptr[M];
  ctx->kmax = kmax;
  ctx->Smax = std::max(1, 2 * kmax - 4);
  ctx->mono_k.assign(M, 0);
  ctx->mono_vp.assign(M, 0);
  ctx->mono_sbase.assign(M, 0);
  int S = 0;
  for (int m = 0; m < M; ++m) {
    ctx->mono_k[m] = vptr[m + 1] - vptr[m];
    ctx->mono_vp[m] = vptr[m];
    ctx->mono_sbase[m] = S;
    S += ctx->mono_k[m] + 1;
  }
  ctx->S = S;
  // Evaluation blocks per SM: two (more warps per sub-partition hide the
  // latency of the integer-limb products) when the products spread over the
  // warps of one block per SM come to well over the longest single chain
  // (the 3k-3 products of the largest monomial, which the warps sharing its
  // sub-partition would slow down); one otherwise.
  {
    long long total = 0, longest = 1;
    for (int m = 0; m < M; ++m) {
      const long long pr = ctx->mono_k[m] == 1 ? 1 : 3LL * ctx->mono_k[m] - 3;
      total += pr;
      longest = std::max(longest, pr);
    }
    const long long warps1 = 4LL * std::max(1, ctx->num_sms);
    ctx->ed_per_sm = (2 * total > 3 * longest * warps1) ? 2 : 1;
    ctx->ed_grid = std::max(1, ctx->num_sms) * ctx->ed_per_sm;
  }
  // work queue order: most expensive monomials first (longest processing time)
  ctx->order.resize(M);
  for (int m = 0; m < M; ++m) ctx->order[m] = m;
  std::stable_sort(ctx->order.begin(), ctx->order.end(),
                   [&](int a, int b) { return ctx->mono_k[a] > ctx->mono_k[b]; });
  // schedules for every size 1..kmax and every lane-group count G that a
  // product length 1..D uses (G(len) = 32 / ceil(len/2); shorter lengths run
  // with staggered orders); with monomials of more than STAGGER_KMAX
  // variables only the full length (the tables grow with G * kmax^2)
  ctx->gvals.clear();
  ctx->gidx_of_len.assign(ctx->D + 1, -1);
  for (int len = 1; len <= ctx->D; ++len) {
    if (kmax > STAGGER_KMAX && len != ctx->D) continue;
    const int g = 32 / ((len + 1) / 2);
    int gi = (int)(std::find(ctx->gvals.begin(), ctx->gvals.end(), g) - ctx->gvals.begin());
    if (gi == (int)ctx->gvals.size()) ctx->gvals.push_back(g);
    ctx->gidx_of_len[len] = gi;
  }
  const int ng = (int)ctx->gvals.size();
  ctx->sched.clear();
  ctx->sched_off.assign((size_t)ng * (kmax + 1), 0);
  ctx->sched_nw.assign((size_t)ng * (kmax + 1), 0);
  for (int gi = 0; gi < ng; ++gi)
    for (int k = 1; k <= kmax; ++k) {
      ctx->sched_off[(size_t)gi * (kmax + 1) + k] = (int)ctx->sched.size();
      int nw = 0;
      build_schedule(k, ctx->gvals[gi], ctx->sched, nw);
      ctx->sched_nw[(size_t)gi * (kmax + 1) + k] = nw;
    }
  if (eq && vidx) {
    for (int m = 0; m < M; ++m)
      if (eq[m] < 0 || eq[m] >= n) return fail(ctx, MDN_EINVAL, "eq_of_monomial[%d] = %d out of range", m, eq[m]);
    for (int q = 0; q < ctx->nnz; ++q)
      if (vidx[q] < 0 || vidx[q] >= n) return fail(ctx, MDN_EINVAL, "var_idx[%d] = %d out of range", q, vidx[q]);
    ctx->vidx.assign(vidx, vidx + ctx->nnz);
    ctx->mono_eq.assign(eq, eq + M);
    ctx->occ.assign(ctx->nnz, 0);
    for (int m = 0; m < M; ++m)
      for (int q = vptr[m]; q < vptr[m + 1]; ++q) ctx->occ[q] = m;
    // equation lists (monomials in index order)
    ctx->eq_ptr.assign(n + 1, 0);
    for (int m = 0; m < M; ++m) ctx->eq_ptr[eq[m] + 1]++;
    for (int i = 0; i < n; ++i) ctx->eq_ptr[i + 1] += ctx->eq_ptr[i];
    ctx->eq_mon.assign(M, 0);
    {
      std::vector<int> fill(ctx->eq_ptr.begin(), ctx->eq_ptr.end() - 1);
      for (int m = 0; m < M; ++m) ctx->eq_mon[fill[eq[m]]++] = m;
    }
    // (row, variable) gather lists of the Jacobian: slot of every occurrence
    const long long nn = (long long)n * n;
    ctx->pair_ptr.assign(nn + 1, 0);
    for (int m = 0; m < M; ++m)
      for (int q = vptr[m]; q < vptr[m + 1]; ++q) ctx->pair_ptr[(long long)eq[m] * n + vidx[q] + 1]++;
    for (long long t = 0; t < nn; ++t) ctx->pair_ptr[t + 1] += ctx->pair_ptr[t];
    ctx->pair_slot.assign(ctx->nnz, 0);
    {
      std::vector<int> fill(ctx->pair_ptr.begin(), ctx->pair_ptr.end() - 1);
      for (int i = 0; i < n; ++i)
        for (int e = ctx->eq_ptr[i]; e < ctx->eq_ptr[i + 1]; ++e) {
          const int m = ctx->eq_mon[e];
          for (int q = vptr[m]; q < vptr[m + 1]; ++q)
            ctx->pair_slot[fill[(long long)i * n + vidx[q]]++] = ctx->mono_sbase[m] + 1 + (q - vptr[m]);
        }
    }
  }
  return MDN_OK;
}

static void compute_layout(mdn_ctx* ctx) {
  Layout& L = ctx->L;
  const size_t KC = (size_t)ctx->K * ctx->C;
  const size_t n = ctx->n, D = ctx->D, M = ctx->M;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + std::max<size_t>(bytes, 8));
    return at;
  };
  L.o_order = take(4 * M);
  L.o_mono_k = take(4 * M);
  L.o_mono_vp = take(4 * M);
  L.o_mono_sbase = take(4 * M);
  L.o_mono_eq = take(4 * M);
  L.o_vidx = take(4 * (size_t)ctx->nnz);
  L.o_sched = take(sizeof(int4) * ctx->sched.size());
  L.o_sched_off = take(4 * ctx->sched_off.size());
  L.o_sched_nw = take(4 * ctx->sched_nw.size());
  L.o_eq_ptr = take(4 * (n + 1));
  L.o_eq_mon = take(4 * M);
  L.o_pair_ptr = take(4 * (n * n + 1));
  L.o_pair_slot = take(4 * (size_t)ctx->nnz);
  L.o_occ = take(4 * (size_t)ctx->nnz);
  L.o_counter = take(4);
  L.o_status = take(4);
  L.o_flags = take(4 * 4 * n);
  L.o_epoch = take(4);
  L.o_done = take(4 * 2 * D);
  const size_t ser = 8 * KC * n * D;
  L.o_x = take(ser);
  L.o_f = take(ser);
  L.o_dx = take(ser);
  L.o_r = take(ser);
  L.o_out = take(8 * KC * (size_t)ctx->S * D);
  L.o_out0 = take(8 * KC * (size_t)ctx->S);
  L.o_scratch = take(8 * KC * (size_t)ctx->Wtot * ctx->Smax * D);
  L.o_adj = take(8 * KC * (size_t)ctx->Wtot * 2 * ctx->G * D);  // products of the adjoint
  L.o_A = take(8 * KC * D * n * n);
  L.o_A0b = take(8 * KC * n * n * 2);  // A_0 of this step and of the next (pipelined QR)
  L.o_Rm = take(8 * (size_t)qr_xf_words(ctx->K) * ctx->C * n * n);  // extended floats
  L.o_Vm = take(8 * (size_t)qr_xf_words(ctx->K) * ctx->C * n * n);
  L.o_Y = take(8 * KC * n * n * 2);  // Q^H and R^{-1} of this step and of the next
  L.o_Z = take(8 * KC * n * n * 2);
  L.o_t0 = take(8 * KC * n);
  L.o_W = take(8 * KC * n * n * 2);    // A_0^{-1} of this step and of the next
  L.o_xn0 = take(8 * KC * n);          // constant coefficients of the next series
  L.o_tau = take(8 * (size_t)qr_xf_words(ctx->K) * n);  // extended floats
  L.o_rinv = take(8 * (size_t)qr_xf_words(ctx->K) * ctx->C * n);
  L.o_salpha = take(8 * (size_t)qr_xf_words(ctx->K) * ctx->C * n);
  L.o_v0 = take(8 * (size_t)qr_xf_words(ctx->K) * ctx->C * n);
  L.o_fabs = take(8 * n * D);
  L.o_dxabs = take(8 * n * D);
  L.o_resabs = take(8 * n * D);
  L.o_resmask = take(4 * n);
  L.o_hist = take(8 * 3 * MDN_MAX_STEPS);
  L.o_rnorm = take(8 * 3);
  L.total = o;
}

extern "C" {

mdn_status mdn_create(mdn_ctx** out, int limbs, int is_complex, int n, int degree) {
  if (!out) return MDN_EINVAL;
  *out = nullptr;
  const int C = is_complex ? 2 : 1;
  const KernelTable* kt = kernels_for(limbs, C);
  if (!kt || n < 1 || n > MDN_MAX_N_EVAL || degree < 0 || degree > MDN_MAX_DEGREE) return MDN_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MDN_ECUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MDN_ECUDA;
  // the dataflow QR keeps its columns and rows in shared memory with all its
  // blocks resident, one per SM; larger systems (up to MDN_MAX_N) take the
  // column-by-column QR in global memory; beyond that a context only
  // evaluates
  const bool small_qr = n <= MDN_MAX_N_DATAFLOW && qr_smem_bytes(n, limbs) <= (size_t)QR_SMEM_MAX &&
                        qr_blocks_for(n) <= sms;
  const bool solves = n <= MDN_MAX_N;
  mdn_ctx* ctx = new (std::nothrow) mdn_ctx();
  if (!ctx) return MDN_EINVAL;
  ctx->K = limbs;
  ctx->C = C;
  ctx->n = n;
  ctx->d = degree;
  ctx->D = degree + 1;
  ctx->kt = kt;
  ctx->num_sms = sms;
  ctx->solves = solves;
  ctx->large_qr = !small_qr;
  ctx->P = (ctx->D + 1) / 2;  // lanes per product: coefficient pairs (k, D-1-k)
  ctx->G = 32 / ctx->P;       // products in flight per warp
  // one evaluation warp per SM sub-partition: four warps already fill an SM's
  // FP64 pipes, and fewer warps than monomials let the largest-first work
  // queue balance the load
  ctx->ed_grid = sms * ctx->ed_per_sm;
  if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->side2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_w, cudaEventDisableTiming) != cudaSuccess) {
    delete ctx;
    return MDN_ECUDA;
  }
  *out = ctx;
  return MDN_OK;
}

size_t mdn_workspace_bytes(const mdn_ctx* cctx, int n_monomials, const int32_t* var_ptr) {
  if (!cctx || !var_ptr || n_monomials < 1) return 0;
  mdn_ctx tmp = *cctx;
  tmp.err.clear();
  if (build_tables(&tmp, n_monomials, nullptr, var_ptr, nullptr) != MDN_OK) return 0;
  tmp.nnz = var_ptr[n_monomials];
  tmp.Wtot = std::min(tmp.ed_grid * (ED_THREADS / 32), n_monomials);
  compute_layout(&tmp);
  return tmp.L.total;
}

mdn_status mdn_load_system(mdn_ctx* ctx, int M, const int32_t* eq, const int32_t* vptr, const int32_t* vidx,
                           const double* coeff, const double* cst, void* workspace, size_t ws_bytes,
                           void* cuda_stream) {
  if (!ctx) return MDN_EINVAL;
  ctx->loaded = false;
  ctx->has_series = false;
  if (!eq || !vptr || !vidx || !coeff || !cst || !workspace)
    return fail(ctx, MDN_EINVAL, "null pointer argument");
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return fail(ctx, MDN_EINVAL, "workspace not 256-byte aligned");
  mdn_status s = build_tables(ctx, M, eq, vptr, vidx);
  if (s != MDN_OK) return s;
  // more warps than monomials would only idle
  ctx->Wtot = std::min(ctx->ed_grid * (ED_THREADS / 32), M);
  compute_layout(ctx);
  if (ws_bytes < ctx->L.total)
    return fail(ctx, MDN_EWORKSPACE, "workspace has %zu bytes, needs %zu", ws_bytes, ctx->L.total);
  ctx->ws = static_cast<char*>(workspace);
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->coeff = coeff;
  ctx->cst = cst;
  const Layout& L = ctx->L;
  cudaStream_t st = ctx->stream;
  auto put = [&](size_t off, const void* src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(ctx->ws + off, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
  };
  CU(put(L.o_order, ctx->order.data(), 4 * ctx->order.size()));
  CU(put(L.o_mono_k, ctx->mono_k.data(), 4 * ctx->mono_k.size()));
  CU(put(L.o_mono_vp, ctx->mono_vp.data(), 4 * ctx->mono_vp.size()));
  CU(put(L.o_mono_sbase, ctx->mono_sbase.data(), 4 * ctx->mono_sbase.size()));
  CU(put(L.o_mono_eq, ctx->mono_eq.data(), 4 * ctx->mono_eq.size()));
  CU(put(L.o_vidx, ctx->vidx.data(), 4 * ctx->vidx.size()));
  CU(put(L.o_sched, ctx->sched.data(), sizeof(int4) * ctx->sched.size()));
  CU(put(L.o_sched_off, ctx->sched_off.data(), 4 * ctx->sched_off.size()));
  CU(put(L.o_sched_nw, ctx->sched_nw.data(), 4 * ctx->sched_nw.size()));
  CU(put(L.o_eq_ptr, ctx->eq_ptr.data(), 4 * ctx->eq_ptr.size()));
  CU(put(L.o_eq_mon, ctx->eq_mon.data(), 4 * ctx->eq_mon.size()));
  CU(put(L.o_pair_ptr, ctx->pair_ptr.data(), 4 * ctx->pair_ptr.size()));
  CU(put(L.o_pair_slot, ctx->pair_slot.data(), 4 * ctx->pair_slot.size()));
  CU(put(L.o_occ, ctx->occ.data(), 4 * ctx->occ.size()));
  CU(cudaMemsetAsync(ctx->ws + L.o_counter, 0, 4, st));
  CU(cudaMemsetAsync(ctx->ws + L.o_status, 0, 4, st));
  CU(cudaMemsetAsync(ctx->ws + L.o_flags, 0, 4 * 4 * (size_t)ctx->n, st));
  CU(cudaMemsetAsync(ctx->ws + L.o_epoch, 0, 4, st));
  CU(cudaMemsetAsync(ctx->ws + L.o_dx, 0, 8 * (size_t)ctx->K * ctx->C * ctx->n * ctx->D, st));
  CU(cudaStreamSynchronize(st));  // host tables may be reused after return
  ctx->res_rows = 0;
  ctx->loaded = true;
  ctx->err.clear();
  return MDN_OK;
}

mdn_status mdn_set_series(mdn_ctx* ctx, const double* x) {
  if (!ctx) return MDN_EINVAL;
  if (!ctx->loaded) return fail(ctx, MDN_ESTATE, "no system loaded");
  if (!x) return fail(ctx, MDN_EINVAL, "null series");
  CU(cudaMemcpyAsync(ctx->at<double>(ctx->L.o_x), x, 8 * (size_t)ctx->K * ctx->C * ctx->n * ctx->D,
                     cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->has_series = true;
  return MDN_OK;
}

mdn_status mdn_get_series(const mdn_ctx* cctx, double* x_out) {
  mdn_ctx* ctx = const_cast<mdn_ctx*>(cctx);
  if (!ctx) return MDN_EINVAL;
  if (!ctx->has_series) return fail(ctx, MDN_ESTATE, "no series set");
  if (!x_out) return fail(ctx, MDN_EINVAL, "null output");
  CU(cudaMemcpyAsync(x_out, ctx->at<double>(ctx->L.o_x), 8 * (size_t)ctx->K * ctx->C * ctx->n * ctx->D,
                     cudaMemcpyDeviceToDevice, ctx->stream));
  return MDN_OK;
}

// ---- launch sequences -------------------------------------------------------

// A_0 = J(x_0) into the j = 0 slice of A (constant coefficients only).
// x: constant coefficients every xstride doubles in limb arrays of Nx doubles;
// A_0 is written with limb stride NA (n*n for a separate matrix, D*n*n for
// the j = 0 slice of a Jacobian series).
static mdn_status run_a0(mdn_ctx* ctx, const double* x, long long Nx, int xstride, double* A, long long NA,
                         cudaStream_t st) {
  const Layout& L = ctx->L;
  const long long D = ctx->D;
  A0Params a{};
  a.n = ctx->n;
  a.D = ctx->D;
  a.M = ctx->M;
  a.x = x;
  a.Nx = Nx;
  a.xstride = xstride;
  a.coeff = ctx->coeff;
  a.Nc = (long long)ctx->M * D;
  a.mono_k = ctx->at<int>(L.o_mono_k);
  a.mono_vp = ctx->at<int>(L.o_mono_vp);
  a.mono_sbase = ctx->at<int>(L.o_mono_sbase);
  a.vidx = ctx->at<int>(L.o_vidx);
  a.nnz = ctx->nnz;
  a.occ_mono = ctx->at<int>(L.o_occ);
  a.out0 = ctx->at<double>(L.o_out0);
  a.S = ctx->S;
  a.pair_ptr = ctx->at<int>(L.o_pair_ptr);
  a.pair_slot = ctx->at<int>(L.o_pair_slot);
  a.A = A;
  a.NA = NA;
  a.kmax = ctx->kmax;
  CU(ctx->kt->a0(a, st));
  return MDN_OK;
}

// Evaluation and differentiation of all monomials, then f and the Jacobian
// slices j >= 1 (slice 0 comes from run_a0) on `blocks` SMs.
// Evaluation of the first `len` coefficients (all by default; fewer with
// staggered orders: the truncated products of the first len coefficients
// need no higher one).
static mdn_status run_evaluate(mdn_ctx* ctx, const double* x, double* f, double* A, int blocks, int len = 0) {
  const Layout& L = ctx->L;
  const long long D = ctx->D, n = ctx->n;
  if (len <= 0 || len > ctx->D) len = ctx->D;
  int gi = ctx->gidx_of_len[len];
  int G = 32 / ((len + 1) / 2);
  if (gi < 0) {
    // monomials too large for a schedule per product length: the schedule of
    // the full length, whose fewer groups per warp leave lanes idle at this
    // length (G (len+1)/2 <= 32 still holds)
    gi = ctx->gidx_of_len[ctx->D];
    if (gi < 0) return fail(ctx, MDN_EINVAL, "no product schedule for %d coefficients", len);
    G = ctx->gvals[gi];
  }
  EdParams e{};
  e.n = ctx->n;
  e.D = ctx->D;
  e.len = len;
  e.M = ctx->M;
  e.P = (len + 1) / 2;
  e.G = G;
  e.kmax = ctx->kmax;
  e.Smax = ctx->Smax;
  const int per_sm = (ctx->qr_running_beside || ctx->ed_per_sm < 1) ? 1 : ctx->ed_per_sm;
  e.smem = per_sm == 1 ? QR_SMEM_RESERVE : per_sm == 2 ? 100 * 1024 : 70 * 1024;
  e.Wtot = std::min(blocks * per_sm * (ED_THREADS / 32), ctx->Wtot);
  e.x = x;
  e.Nx = n * D;
  e.coeff = ctx->coeff;
  e.Nc = (long long)ctx->M * D;
  e.out = ctx->at<double>(L.o_out);
  e.No = (long long)ctx->S * D;
  e.scratch = ctx->at<double>(L.o_scratch);
  e.Ns = (long long)ctx->Wtot * ctx->Smax * D;
  e.order = ctx->at<int>(L.o_order);
  e.mono_k = ctx->at<int>(L.o_mono_k);
  e.mono_vp = ctx->at<int>(L.o_mono_vp);
  e.mono_sbase = ctx->at<int>(L.o_mono_sbase);
  e.vidx = ctx->at<int>(L.o_vidx);
  e.sched = ctx->at<int4>(L.o_sched);
  e.sched_off = ctx->at<int>(L.o_sched_off) + (size_t)gi * (ctx->kmax + 1);
  e.sched_nw = ctx->at<int>(L.o_sched_nw) + (size_t)gi * (ctx->kmax + 1);
  e.counter = ctx->at<int>(L.o_counter);
  ph_begin(ctx, MDN_PHASE_EVALUATE);
  CU(cudaMemsetAsync(e.counter, 0, 4, ctx->stream));
  const int grid = (e.Wtot + (ED_THREADS / 32) - 1) / (ED_THREADS / 32);
  CU(ctx->kt->ed(e, grid, ctx->stream));
  ph_end(ctx, MDN_PHASE_EVALUATE, 1);
  AsmParams a{};
  a.n = ctx->n;
  a.D = ctx->D;
  a.len = len;
  a.j_begin = 1;
  a.out = e.out;
  a.No = e.No;
  a.cst = ctx->cst;
  a.f = f;
  a.Nf = n * D;
  a.A = A;
  a.NA = D * n * n;
  a.eq_ptr = ctx->at<int>(L.o_eq_ptr);
  a.eq_mon = ctx->at<int>(L.o_eq_mon);
  a.mono_sbase = e.mono_sbase;
  a.pair_ptr = ctx->at<int>(L.o_pair_ptr);
  a.pair_slot = ctx->at<int>(L.o_pair_slot);
  ph_begin(ctx, MDN_PHASE_ASSEMBLE);
  CU(ctx->kt->assemble(a, A != nullptr, ctx->stream));
  ph_end(ctx, MDN_PHASE_ASSEMBLE, (A != nullptr && len > 1) ? 2 : 1);
  return MDN_OK;
}

// Parameters of the QR of A0 into the Y/Z buffer pair `buf` with W out.
static QrParams qr_params(mdn_ctx* ctx, const double* A0, long long NA0, double* W, int buf) {
  const Layout& L = ctx->L;
  const long long n = ctx->n, KC = (long long)ctx->K * ctx->C;
  QrParams q{};
  q.n = ctx->n;
  q.nAc = (ctx->n + 3) / 4;
  q.nAi = (ctx->n + 3) / 4;
  q.nAz = ((ctx->n + 1) / 2 + 3) / 4;
  q.A0 = A0;
  q.NA = NA0;
  q.Nnn = n * n;
  q.Rm = ctx->at<uint64_t>(L.o_Rm);
  q.Vm = ctx->at<uint64_t>(L.o_Vm);
  q.Y = ctx->at<double>(L.o_Y) + buf * KC * n * n;
  q.Z = ctx->at<double>(L.o_Z) + buf * KC * n * n;
  q.W = W;
  q.tau = ctx->at<uint64_t>(L.o_tau);
  q.rinv = ctx->at<uint64_t>(L.o_rinv);
  q.salpha = ctx->at<uint64_t>(L.o_salpha);
  q.v0 = ctx->at<uint64_t>(L.o_v0);
  q.flags = ctx->at<unsigned>(L.o_flags);
  q.epoch = ctx->at<unsigned>(L.o_epoch);
  q.status = ctx->at<int>(L.o_status);
  q.spin_limit = ctx->wait_limit_ns;
  q.large = ctx->large_qr ? 1 : 0;
  q.Aw = q.Rm;  // the large variant's working columns take the place of R and the reflectors
  q.Yw = q.Vm;
  return q;
}

// Householder QR of A0 (the j = 0 slice of A) and, unless skip_w, W = A0^{-1}
// on stream st.  With skip_w the factors Z = R^{-1} and Y = Q^H are left in
// buffer `buf` and run_qr_w forms W from them.
static mdn_status run_qr(mdn_ctx* ctx, const double* A0, long long NA0, double* W, cudaStream_t st, int buf = 0,
                         bool skip_w = false) {
  bump_kernel<<<1, 1, 0, st>>>(ctx->at<unsigned>(ctx->L.o_epoch));
  CU(cudaGetLastError());
  QrParams q = qr_params(ctx, A0, NA0, W, buf);
  q.skip_w = skip_w ? 1 : 0;
  CU(ctx->kt->qr(q, st));
  return MDN_OK;
}
static mdn_status run_qr_w(mdn_ctx* ctx, double* W, int buf, cudaStream_t st) {
  QrParams q = qr_params(ctx, nullptr, 0, W, buf);
  CU(ctx->kt->qr_w(q, st));
  return MDN_OK;
}

// SMs the QR occupies: the dataflow kernel's blocks, or all of them for the
// column-by-column variant (which then does not overlap the evaluation)
static int qr_blocks(const mdn_ctx* ctx) { return ctx->large_qr ? ctx->num_sms : qr_blocks_for(ctx->n); }
// Kernel launches of A_0 and its QR: two for A_0, the epoch bump, then the
// dataflow kernel and W, or the column-by-column sequence (initialisation,
// the first pivot, an update launch per column that also forms the next
// pivot, the back substitution).
static int qr_launches(const mdn_ctx* ctx) { return 3 + (ctx->large_qr ? ctx->n + 3 : 2); }

// Forward substitution for dx with right hand side sgn * rhs: stage 0 alone
// (dx_0 = W r_0, and x_0 + dx_0 into the xnext0 buffer when x is given), the
// event e0 recorded after it when not null, then the remaining stages on
// `blocks` SMs.
// With factors >= 0, stage 0 is formed from Z = R^{-1} and Y = Q^H of that
// buffer (dx_0 = Z (Y r_0)) and the later stages wait for the event w_ready
// (W formed on another stream) before they start.
static mdn_status run_forward(mdn_ctx* ctx, const double* A, const double* A0, long long NA0, const double* W,
                              const double* rhs, int sgn, double* dx, const double* x, cudaEvent_t e0, int blocks,
                              bool transposed = false, int nst = 0, int factors = -1, cudaEvent_t w_ready = nullptr) {
  const Layout& L = ctx->L;
  const long long D = ctx->D, n = ctx->n;
  ph_begin(ctx, MDN_PHASE_FORWARD);
  FsubParams u{};
  u.n = ctx->n;
  u.D = ctx->D;
  u.rhs_sign = sgn;
  u.first_stage = 1;
  u.nW = std::min(ctx->n, 4 * FSUB_WBLOCKS);
  const int wb = (u.nW + 3) / 4;
  const int nst_eff = (nst > 0 && nst <= ctx->D) ? nst : ctx->D;
  // owner blocks per SM: one beside a concurrent QR (whose chain wants its
  // SMs alone); otherwise ctx->fsub_per_sm, so that more warps share each
  // sub-partition and hide the latency of the integer-limb row products
  const int per_sm = (ctx->qr_running_beside || ctx->fsub_per_sm < 1) ? 1 : ctx->fsub_per_sm;
  u.smem = per_sm == 1 ? QR_SMEM_RESERVE : per_sm == 2 ? 100 * 1024 : 70 * 1024;
  u.nOwn = (int)std::min<long long>(4LL * per_sm * std::max(1, blocks - wb), (long long)ctx->n * nst_eff);
  u.late_stage = transposed ? ctx->D : std::min(ctx->late_stage, ctx->D);
  u.transpose = transposed ? 1 : 0;
  u.reverse = transposed ? 1 : 0;
  u.nst = nst_eff;
  u.A = A;
  u.NA = D * n * n;
  u.A0 = A0;
  u.NA0 = NA0;
  u.W = W;
  u.Nnn = n * n;
  u.rhs = rhs;
  u.r = ctx->at<double>(L.o_r);
  u.dx = dx;
  u.Nx = n * D;
  u.x = x;
  u.xnext0 = x ? ctx->at<double>(L.o_xn0) : nullptr;
  u.resabs = ctx->at<double>(L.o_resabs);
  u.resmask = ctx->res_rows ? ctx->at<int>(L.o_resmask) : nullptr;
  u.rdone = ctx->at<unsigned>(L.o_done);
  u.xdone = u.rdone + ctx->D;
  u.status = ctx->at<int>(L.o_status);
  u.spin_limit = ctx->wait_limit_ns;
  if (factors >= 0) {
    const long long off = (long long)factors * ctx->K * ctx->C * n * n;
    u.Zs = ctx->at<double>(L.o_Z) + off;
    u.Ys = ctx->at<double>(L.o_Y) + off;
    u.t0 = ctx->at<double>(L.o_t0);
  }
  CU(cudaMemsetAsync(u.rdone, 0, 4 * 2 * (size_t)ctx->D, ctx->stream));
  CU(ctx->kt->stage0(u, ctx->stream));
  if (e0) CU(cudaEventRecord(e0, ctx->stream));
  if (w_ready) CU(cudaStreamWaitEvent(ctx->stream, w_ready, 0));
  // stages 1..nst-1 and the residuals of all stages (with one stage, the
  // residual of stage 0 alone)
  CU(ctx->kt->fsub(u, ctx->stream));
  ph_end(ctx, MDN_PHASE_FORWARD, factors >= 0 ? 3 : 2);
  return MDN_OK;
}

// Newton steps with the QR of A_0 pipelined across steps.  Step s needs
// W_s = (A_0 at x^(s))^{-1}; x^(s) has the constant coefficients
// x_0^(s-1) + dx_0^(s-1), known right after stage 0 of step s-1.  So the A_0
// and QR of step s run on the side stream (on a third of the SMs) beside the
// later stages of step s-1, its update and the evaluation of step s (on the
// other SMs).  A_0 and W alternate between two buffers by step parity.
// Staggered orders (Section 4): coefficients worked on by step s; the first
// stagger_first steps work on x_0 alone, then L := min(D, L + 1 + L/2).
static int stagger_len(const mdn_ctx* ctx, int s) {
  const int f = ctx->stagger_first;
  if (f <= 0) return ctx->D;
  if (s < f) return 1;
  int L = 1;
  for (int t = f; t <= s; ++t) {
    L = L + 1 + L / 2;
    if (L >= ctx->D) return ctx->D;
  }
  return L;
}
// Whether step s forms its own QR of A_0 (with staggered orders only the
// order-1 steps do; later steps reuse the last one: the QR once of
// Section 5.3, valid once x_0 is accurate to about half the precision).
static bool qr_at(const mdn_ctx* ctx, int s) { return ctx->stagger_first <= 0 || s < ctx->stagger_first; }

static mdn_status run_steps(mdn_ctx* ctx, int steps, double tol, int* done_out, bool* converged) {
  const Layout& L = ctx->L;
  const long long D = ctx->D, n = ctx->n, nn = n * n, KC = (long long)ctx->K * ctx->C;
  double* x = ctx->at<double>(L.o_x);
  double* f = ctx->at<double>(L.o_f);
  double* dx = ctx->at<double>(L.o_dx);
  double* A = ctx->at<double>(L.o_A);
  double* hist = ctx->at<double>(L.o_hist);
  double* A0b[2] = {ctx->at<double>(L.o_A0b), ctx->at<double>(L.o_A0b) + KC * nn};
  double* Wb[2] = {ctx->at<double>(L.o_W), ctx->at<double>(L.o_W) + KC * nn};
  const int qb = qr_blocks(ctx);
  const bool overlap = ctx->side && qb <= (ctx->num_sms * 3) / 8;
  const int rest = overlap ? ctx->num_sms - qb : ctx->num_sms;
  // W = Z Y on a third stream: the next step's stage 0 takes dx_0 from the
  // factors, so the loop of QRs (stage 0 -> A_0 -> QR -> stage 0) does not
  // wait for W; only the later stages of the forward substitution do
  const bool split_w = overlap && !ctx->large_qr && ctx->side2;
  mdn_status r;
  *converged = false;
  auto launch_w = [&](int buf) -> mdn_status {
    CU(cudaStreamWaitEvent(ctx->side2, ctx->ev_join, 0));
    ph_begin(ctx, MDN_PHASE_QR, ctx->side2);
    mdn_status rr = run_qr_w(ctx, Wb[buf], buf, ctx->side2);
    if (rr != MDN_OK) return rr;
    ph_end(ctx, MDN_PHASE_QR, 1, ctx->side2);
    CU(cudaEventRecord(ctx->ev_w, ctx->side2));
    return MDN_OK;
  };
  // A_0 and QR of the first step
  if (overlap) {
    CU(cudaEventRecord(ctx->ev_fork, ctx->stream));
    CU(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  }
  cudaStream_t qs = overlap ? ctx->side : ctx->stream;
  ph_begin(ctx, MDN_PHASE_QR, qs);
  if ((r = run_a0(ctx, x, n * D, ctx->D, A0b[0], nn, qs)) != MDN_OK) return r;
  if ((r = run_qr(ctx, A0b[0], nn, Wb[0], qs, 0, split_w)) != MDN_OK) return r;
  ph_end(ctx, MDN_PHASE_QR, qr_launches(ctx) - (split_w ? 1 : 0), qs);
  if (overlap) CU(cudaEventRecord(ctx->ev_join, ctx->side));
  if (split_w && (r = launch_w(0)) != MDN_OK) return r;
  if (ctx->stagger_first > 0) {
    // inactive coefficients contribute nothing to the norms of the step
    CU(cudaMemsetAsync(ctx->at<double>(L.o_fabs), 0, 8 * (size_t)n * D, ctx->stream));
    CU(cudaMemsetAsync(ctx->at<double>(L.o_dxabs), 0, 8 * (size_t)n * D, ctx->stream));
    CU(cudaMemsetAsync(ctx->at<double>(L.o_resabs), 0, 8 * (size_t)n * D, ctx->stream));
  }
  for (int s = 0; s < steps; ++s) {
    const int b = qr_at(ctx, s) ? (s & 1) : ((ctx->stagger_first - 1) & 1);
    const int len = stagger_len(ctx, s);
    ctx->qr_running_beside = overlap;
    r = run_evaluate(ctx, x, f, A, rest, len);
    ctx->qr_running_beside = false;
    if (r != MDN_OK) return r;
    if (overlap) CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
    const bool next = s + 1 < steps && qr_at(ctx, s + 1);
    // with no QR to run beside it the forward substitution takes every SM
    ctx->qr_running_beside = overlap && next;
    r = run_forward(ctx, A, A0b[b], nn, Wb[b], f, -1, dx, x, (overlap && next) ? ctx->ev_fork : nullptr,
                    (overlap && next) ? rest : ctx->num_sms, false, len, split_w ? b : -1,
                    split_w ? ctx->ev_w : nullptr);
    ctx->qr_running_beside = false;
    if (r != MDN_OK) return r;
    if (next) {
      // A_0 and QR of step s+1 from x_0 + dx_0
      if (overlap) CU(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
      ph_begin(ctx, MDN_PHASE_QR, qs);
      if ((r = run_a0(ctx, ctx->at<double>(L.o_xn0), n, 1, A0b[b ^ 1], nn, qs)) != MDN_OK) return r;
      if ((r = run_qr(ctx, A0b[b ^ 1], nn, Wb[b ^ 1], qs, b ^ 1, split_w)) != MDN_OK) return r;
      ph_end(ctx, MDN_PHASE_QR, qr_launches(ctx) - (split_w ? 1 : 0), qs);
      if (overlap) CU(cudaEventRecord(ctx->ev_join, ctx->side));
      if (split_w && (r = launch_w(b ^ 1)) != MDN_OK) return r;
    }
    UpdParams u{};
    u.n = ctx->n;
    u.D = ctx->D;
    u.len = len;
    u.x = x;
    u.dx = dx;
    u.f = f;
    u.Nx = n * D;
    u.dxabs = ctx->at<double>(L.o_dxabs);
    u.fabs = ctx->at<double>(L.o_fabs);
    u.status = ctx->at<int>(L.o_status);
    ph_begin(ctx, MDN_PHASE_UPDATE);
    CU(ctx->kt->update(u, ctx->stream));
    NormParams np{};
    np.count = n * D;
    np.fabs = u.fabs;
    np.resabs = ctx->at<double>(L.o_resabs);
    np.res_scale = ctx->res_rows ? (double)ctx->n / ctx->res_rows : 1.0;
    np.dxabs = u.dxabs;
    np.hist = hist + 3 * s;
    norms_kernel<<<1, 1024, 0, ctx->stream>>>(np);
    CU(cudaGetLastError());
    ph_end(ctx, MDN_PHASE_UPDATE, 2);
    *done_out = s + 1;
    if (tol > 0.0) {
      double h[3];
      CU(cudaMemcpyAsync(h, hist + 3 * s, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
      CU(cudaStreamSynchronize(ctx->stream));
      if (h[2] <= tol && len == ctx->D) {
        *converged = true;
        break;
      }
    }
  }
  // the QR of a step that is not run must be finished before returning
  if (overlap) CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
  if (split_w) CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_w, 0));
  return MDN_OK;
}

static mdn_status read_status(mdn_ctx* ctx) {
  int st = 0;
  CU(cudaMemcpyAsync(&st, ctx->at<int>(ctx->L.o_status), 4, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (st & MDN_DEV_TIMEOUT) return fail(ctx, MDN_ETIMEOUT, "a bounded device wait timed out");
  // a non-finite value makes the pivots of the QR meaningless too: it is
  // the cause to report when both are set
  if (st & MDN_DEV_NONFINITE) return fail(ctx, MDN_ENONFINITE, "non-finite value in the series");
  if (st & MDN_DEV_SINGULAR) return fail(ctx, MDN_ESINGULAR, "zero pivot in the Householder QR of A0");
  return MDN_OK;
}

mdn_status mdn_newton(mdn_ctx* ctx, int max_steps, double tol, int* steps_done, double* res_hist) {
  if (!ctx) return MDN_EINVAL;
  if (steps_done) *steps_done = 0;
  if (!ctx->loaded) return fail(ctx, MDN_ESTATE, "no system loaded");
  if (!ctx->has_series) return fail(ctx, MDN_ESTATE, "no series set");
  if (max_steps < 1 || max_steps > MDN_MAX_STEPS) return fail(ctx, MDN_EINVAL, "max_steps out of range");
  if (!ctx->solves) return fail(ctx, MDN_EINVAL, "n = %d > MDN_MAX_N: this context only evaluates", ctx->n);
  const Layout& L = ctx->L;
  double* hist = ctx->at<double>(L.o_hist);
  CU(cudaMemsetAsync(ctx->at<int>(L.o_status), 0, 4, ctx->stream));
  int done = 0;
  bool converged = false;
  mdn_status r = run_steps(ctx, max_steps, tol, &done, &converged);
  if (r != MDN_OK) return r;
  if (res_hist) CU(cudaMemcpyAsync(res_hist, hist, sizeof(double) * 3 * done, cudaMemcpyDeviceToHost, ctx->stream));
  mdn_status st = read_status(ctx);
  if (steps_done) *steps_done = done;
  if (st != MDN_OK) return st;
  if (tol > 0.0 && !converged) return fail(ctx, MDN_ENOTCONVERGED, "||dx||_1 above tol after %d steps", done);
  return MDN_OK;
}

mdn_status mdn_get_residual(mdn_ctx* ctx, double* f_out) {
  if (!ctx) return MDN_EINVAL;
  if (!ctx->loaded || !ctx->has_series) return fail(ctx, MDN_ESTATE, "no system or series");
  if (!f_out) return fail(ctx, MDN_EINVAL, "null output");
  return run_evaluate(ctx, ctx->at<double>(ctx->L.o_x), f_out, nullptr, ctx->num_sms);
}

mdn_status mdn_evaluate(mdn_ctx* ctx, const double* x, double* f_out, double* A_out) {
  if (!ctx) return MDN_EINVAL;
  if (!ctx->loaded) return fail(ctx, MDN_ESTATE, "no system loaded");
  if (!x || !f_out) return fail(ctx, MDN_EINVAL, "null pointer argument");
  mdn_status r;
  if (A_out && (r = run_a0(ctx, x, (long long)ctx->n * ctx->D, ctx->D, A_out,
                           (long long)ctx->D * ctx->n * ctx->n, ctx->stream)) != MDN_OK)
    return r;
  return run_evaluate(ctx, x, f_out, A_out, ctx->num_sms);
}

mdn_status mdn_solve(mdn_ctx* ctx, const double* A, const double* b, double* dx) {
  if (!ctx) return MDN_EINVAL;
  if (!ctx->loaded) return fail(ctx, MDN_ESTATE, "no system loaded");
  if (!A || !b || !dx) return fail(ctx, MDN_EINVAL, "null pointer argument");
  if (!ctx->solves) return fail(ctx, MDN_EINVAL, "n = %d > MDN_MAX_N: this context only evaluates", ctx->n);
  CU(cudaMemsetAsync(ctx->at<int>(ctx->L.o_status), 0, 4, ctx->stream));
  const long long DNN = (long long)ctx->D * ctx->n * ctx->n;
  double* W = ctx->at<double>(ctx->L.o_W);
  ph_begin(ctx, MDN_PHASE_QR);
  mdn_status r = run_qr(ctx, A, DNN, W, ctx->stream);
  if (r != MDN_OK) return r;
  ph_end(ctx, MDN_PHASE_QR, qr_launches(ctx) - 2);
  if ((r = run_forward(ctx, A, A, DNN, W, b, +1, dx, nullptr, nullptr, ctx->num_sms)) != MDN_OK) return r;
  return read_status(ctx);
}

mdn_status mdn_fabry_loss(mdn_ctx* ctx, const double* x, double* loss_out, double* g_out) {
  if (!ctx) return MDN_EINVAL;
  if (!ctx->loaded) return fail(ctx, MDN_ESTATE, "no system loaded");
  if (!x || !loss_out || !g_out) return fail(ctx, MDN_EINVAL, "null pointer argument");
  if (ctx->C != 1 || ctx->D < 2) return fail(ctx, MDN_EINVAL, "the loss needs real data and degree >= 1");
  LossParams lp{};
  lp.n = ctx->n;
  lp.D = ctx->D;
  lp.x = x;
  lp.Nx = (long long)ctx->n * ctx->D;
  lp.loss = loss_out;
  lp.g = g_out;
  CU(ctx->kt->fabry(lp, ctx->stream));
  return MDN_OK;
}

// dL/dc = -lambda^T df/dc with J^T lambda = g (J the block lower triangular
// Jacobian of Eq. (eqToeplitz) at x): A(t) and A_0^{-1} at x, the solve with
// J^T as the forward substitution with transposed blocks in reversed stage
// order (A_0^{-T} = W^T), then the correlations of the coefficient adjoints.
mdn_status mdn_adjoint(mdn_ctx* ctx, const double* x, const double* g, double* grad_out) {
  if (!ctx) return MDN_EINVAL;
  if (!ctx->loaded) return fail(ctx, MDN_ESTATE, "no system loaded");
  if (!x || !g || !grad_out) return fail(ctx, MDN_EINVAL, "null pointer argument");
  if (ctx->C != 1) return fail(ctx, MDN_EINVAL, "the adjoint is defined for real data");
  if (!ctx->solves) return fail(ctx, MDN_EINVAL, "n = %d > MDN_MAX_N: this context only evaluates", ctx->n);
  const Layout& L = ctx->L;
  const long long n = ctx->n, D = ctx->D, DNN = D * n * n;
  CU(cudaMemsetAsync(ctx->at<int>(L.o_status), 0, 4, ctx->stream));
  double* A = ctx->at<double>(L.o_A);
  double* f = ctx->at<double>(L.o_f);
  double* W = ctx->at<double>(L.o_W);
  double* lam = ctx->at<double>(L.o_dx);
  mdn_status r;
  // A_0 and its QR on the side stream beside the evaluation of A(t)
  const int qb = qr_blocks(ctx);
  const bool overlap = ctx->side && qb <= (ctx->num_sms * 3) / 8;
  cudaStream_t qs = overlap ? ctx->side : ctx->stream;
  double* A0 = ctx->at<double>(L.o_A0b);
  if (overlap) {
    CU(cudaEventRecord(ctx->ev_fork, ctx->stream));
    CU(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  }
  ph_begin(ctx, MDN_PHASE_QR, qs);
  if ((r = run_a0(ctx, x, n * D, ctx->D, A0, n * n, qs)) != MDN_OK) return r;
  if ((r = run_qr(ctx, A0, n * n, W, qs)) != MDN_OK) return r;
  ph_end(ctx, MDN_PHASE_QR, qr_launches(ctx), qs);
  if (overlap) CU(cudaEventRecord(ctx->ev_join, ctx->side));
  // A_1..A_d (the solve with J^T reads A_0 from the QR's copy)
  ctx->qr_running_beside = overlap;
  r = run_evaluate(ctx, x, f, A, overlap ? ctx->num_sms - qb : ctx->num_sms);
  ctx->qr_running_beside = false;
  if (r != MDN_OK) return r;
  if (overlap) CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
  if ((r = run_forward(ctx, A, A0, n * n, W, g, +1, lam, nullptr, nullptr, ctx->num_sms, true)) != MDN_OK) return r;
  AdjParams a{};
  a.n = ctx->n;
  a.D = ctx->D;
  a.M = ctx->M;
  a.P = ctx->P;
  a.G = ctx->G;
  a.Wtot = ctx->Wtot;
  a.mono_eq = ctx->at<int>(L.o_mono_eq);
  a.mono_vp = ctx->at<int>(L.o_mono_vp);
  a.mono_k = ctx->at<int>(L.o_mono_k);
  a.vidx = ctx->at<int>(L.o_vidx);
  a.x = x;
  a.Nx = n * D;
  a.lam = lam;
  a.grad = grad_out;
  a.Ng = (long long)ctx->M * D;
  a.scratch = ctx->at<double>(L.o_adj);
  a.Ns = (long long)ctx->Wtot * 2 * ctx->G * D;
  ph_begin(ctx, MDN_PHASE_EVALUATE);
  CU(ctx->kt->adjoint(a, ctx->stream));
  ph_end(ctx, MDN_PHASE_EVALUATE, 1);
  return read_status(ctx);
}

mdn_status mdn_residual(mdn_ctx* ctx, const double* A, const double* b, const double* dx, double* r_out,
                        double* norm_out) {
  if (!ctx) return MDN_EINVAL;
  if (!ctx->loaded) return fail(ctx, MDN_ESTATE, "no system loaded");
  if (!A || !b || !dx) return fail(ctx, MDN_EINVAL, "null pointer argument");
  const Layout& L = ctx->L;
  const long long n = ctx->n, D = ctx->D;
  ResParams rp{};
  rp.n = ctx->n;
  rp.D = ctx->D;
  rp.A = A;
  rp.NA = D * n * n;
  rp.b = b;
  rp.dx = dx;
  rp.Nx = n * D;
  rp.r = r_out;
  rp.resabs = ctx->at<double>(L.o_resabs);
  rp.resmask = ctx->res_rows ? ctx->at<int>(L.o_resmask) : nullptr;
  CU(ctx->kt->residual(rp, ctx->stream));
  NormParams np{};
  np.count = n * D;
  np.fabs = rp.resabs;
  np.resabs = rp.resabs;
  np.dxabs = rp.resabs;
  np.res_scale = ctx->res_rows ? (double)ctx->n / ctx->res_rows : 1.0;
  np.hist = ctx->at<double>(L.o_rnorm);
  norms_kernel<<<1, 1024, 0, ctx->stream>>>(np);
  CU(cudaGetLastError());
  double h[3];
  CU(cudaMemcpyAsync(h, np.hist, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (norm_out) *norm_out = h[1];
  return MDN_OK;
}

mdn_status mdn_md_scale(mdn_ctx* ctx, const double* s, const double* a, int64_t count, double* out) {
  if (!ctx) return MDN_EINVAL;
  if (!ctx->loaded) return fail(ctx, MDN_ESTATE, "no system loaded");
  if (!s || !a || !out || count < 0) return fail(ctx, MDN_EINVAL, "bad argument");
  if (count == 0) return MDN_OK;
  ScaleParams sp{};
  sp.s = s;
  sp.a = a;
  sp.out = out;
  sp.N = count;
  CU(ctx->kt->scale(sp, ctx->stream));
  return MDN_OK;
}

mdn_status mdn_set_wait_limit_ns(mdn_ctx* ctx, int64_t limit_ns) {
  if (!ctx) return MDN_EINVAL;
  if (limit_ns < 1) return fail(ctx, MDN_EINVAL, "the wait limit must be positive");
  ctx->wait_limit_ns = limit_ns;
  return MDN_OK;
}

mdn_status mdn_set_residual_rows(mdn_ctx* ctx, const int32_t* rows, int count) {
  if (!ctx) return MDN_EINVAL;
  if (!ctx->loaded) return fail(ctx, MDN_ESTATE, "no system loaded");
  if (count < 0 || count > ctx->n || (count > 0 && !rows)) return fail(ctx, MDN_EINVAL, "bad row count");
  std::vector<int> mask(ctx->n, count ? 0 : 1);
  for (int q = 0; q < count; ++q) {
    if (rows[q] < 0 || rows[q] >= ctx->n) return fail(ctx, MDN_EINVAL, "row %d out of range", rows[q]);
    if (mask[rows[q]]) return fail(ctx, MDN_EINVAL, "row %d listed twice", rows[q]);
    mask[rows[q]] = 1;
  }
  const Layout& L = ctx->L;
  CU(cudaMemcpyAsync(ctx->at<int>(L.o_resmask), mask.data(), 4 * (size_t)ctx->n, cudaMemcpyHostToDevice,
                     ctx->stream));
  // rows outside the sample contribute zero to the monitor
  CU(cudaMemsetAsync(ctx->at<double>(L.o_resabs), 0, 8 * (size_t)ctx->n * ctx->D, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  ctx->res_rows = (count == ctx->n) ? 0 : count;
  return MDN_OK;
}

mdn_status mdn_set_stagger(mdn_ctx* ctx, int first_steps) {
  if (!ctx) return MDN_EINVAL;
  if (first_steps < 0 || first_steps > MDN_MAX_STEPS) return fail(ctx, MDN_EINVAL, "first_steps out of range");
  ctx->stagger_first = first_steps;
  return MDN_OK;
}

mdn_status mdn_set_late_updates(mdn_ctx* ctx, int first_stage, int limbs) {
  if (!ctx) return MDN_EINVAL;
  if (first_stage < 1) return fail(ctx, MDN_EINVAL, "first_stage must be >= 1");
  if (limbs == ctx->K) {
    ctx->late_stage = 1 << 30;
    return MDN_OK;
  }
  if (ctx->K < 2 || limbs != ctx->K / 2) return fail(ctx, MDN_EINVAL, "limbs must be K or K/2");
  ctx->late_stage = first_stage;
  return MDN_OK;
}

mdn_status mdn_status_word(mdn_ctx* ctx) {
  if (!ctx) return MDN_EINVAL;
  if (!ctx->loaded) return fail(ctx, MDN_ESTATE, "no system loaded");
  return read_status(ctx);
}

mdn_status mdn_profile(mdn_ctx* ctx, int enable, double* ms_out, int64_t* launches_out) {
  if (!ctx) return MDN_EINVAL;
  if (enable) {
    ctx->prof = true;
    ctx->prof_rec.clear();
    ctx->ev_used = 0;
    for (int i = 0; i < MDN_NUM_PHASES; ++i) ctx->open_ev_of[i] = nullptr;
    for (int i = 0; i < MDN_NUM_PHASES; ++i) ctx->launches[i] = 0;
    return MDN_OK;
  }
  ctx->prof = false;
  double ms[MDN_NUM_PHASES] = {0, 0, 0, 0, 0};
  if (!ctx->prof_rec.empty()) {
    CU(cudaEventSynchronize(ctx->prof_rec.back().second.second));
    for (auto& r : ctx->prof_rec) {
      float t = 0.f;
      CU(cudaEventElapsedTime(&t, r.second.first, r.second.second));
      ms[r.first] += t;
    }
  }
  for (int i = 0; i < MDN_NUM_PHASES; ++i) {
    if (ms_out) ms_out[i] = ms[i];
    if (launches_out) launches_out[i] = ctx->launches[i];
  }
  ctx->prof_rec.clear();
  ctx->ev_used = 0;
  return MDN_OK;
}

const char* mdn_last_error(const mdn_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

mdn_status mdn_ed_schedule(int k, int groups, int32_t* ops, int capacity, int* n_waves) {
  if (k < 1 || k > 4096 || groups < 1 || groups > 32 || !n_waves || capacity < 0) return MDN_EINVAL;
  std::vector<int4> w;
  int nw = 0;
  build_schedule(k, groups, w, nw);
  *n_waves = nw;
  if (!ops) return MDN_OK;
  if ((size_t)capacity < w.size()) return MDN_EINVAL;
  for (size_t i = 0; i < w.size(); ++i) {
    ops[4 * i] = w[i].x;
    ops[4 * i + 1] = w[i].y;
    ops[4 * i + 2] = w[i].z;
    ops[4 * i + 3] = w[i].w;
  }
  return MDN_OK;
}

void mdn_destroy(mdn_ctx* ctx) {
  if (!ctx) return;
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->ev_w) cudaEventDestroy(ctx->ev_w);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->side2) cudaStreamDestroy(ctx->side2);
  delete ctx;
}

}  // extern "C"
