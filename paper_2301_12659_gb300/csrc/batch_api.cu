// batch_api.cu -- host runtime of the batched systems (mdn_batch_* of
// include/mdnewton.h): validation, the tables of the persistent kernel
// (monomials grouped by equation, largest first; systems in decreasing
// estimated cost for the work queue), the per-block scratch, and the CUDA
// graph that replays the solve launch.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/mdnewton.h"
#include "params.h"

namespace mdn {
const KernelTable* kernels_for(int K, int C);
}
using namespace mdn;

namespace {
constexpr int BATCH_MAX_N = 128;
constexpr int BATCH_MAX_K = 16;
size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
}  // namespace

struct mdn_batch {
  int K = 0, C = 0, count = 0;
  const KernelTable* kt = nullptr;
  int threads = 256, blocks_per_sm = 1, num_sms = 0;
  std::vector<int> n, D, M;
  std::vector<long long> mono0, coeff_off, series_off;
  long long Mtot = 0, nnz = 0, series_total = 0;
  int kmax = 1, S3 = 1;
  long long work_stride = 0;
  // host tables (kept alive for the asynchronous copies)
  std::vector<BatchSys> h_sys;
  std::vector<int> h_order, h_eq_ptr, h_eq_mon, h_vptr, h_vidx;
  size_t o_sys = 0, o_order = 0, o_eq_ptr = 0, o_eq_mon = 0, o_vptr = 0, o_vidx = 0, o_queue = 0, o_steps = 0,
         o_flags = 0, o_work = 0, total = 0;
  char* ws = nullptr;
  const double* coeff = nullptr;
  const double* cst = nullptr;
  cudaStream_t stream = nullptr;   // the caller's
  cudaStream_t gstream = nullptr;  // graph launches (capturable)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool loaded = false;
  // the captured solve and what it was captured for
  cudaGraphExec_t gexec = nullptr;
  const double* g_x0 = nullptr;
  double* g_x = nullptr;
  int g_steps = -1;
  double g_tol = -1.0;
  std::string err;
  template <class T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(ws + off);
  }
};

static mdn_status bfail(const mdn_batch* b, mdn_status s, const char* fmt, ...) {
  if (b) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    const_cast<mdn_batch*>(b)->err = buf;
  }
  return s;
}

#define BCU(call)                                                                                \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return bfail(b, MDN_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static int kmax_of(const mdn_batch* b, const int32_t* vptr) {
  int km = 1;
  for (long long m = 0; m < b->Mtot; ++m) km = std::max(km, vptr[m + 1] - vptr[m]);
  return km;
}

static void layout(mdn_batch* b) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t r = o;
    o = al256(o + bytes);
    return r;
  };
  long long eqp = 0;
  for (int s = 0; s < b->count; ++s) eqp += b->n[s] + 1;
  b->o_sys = take(sizeof(BatchSys) * b->count);
  b->o_order = take(sizeof(int) * b->count);
  b->o_eq_ptr = take(sizeof(int) * eqp);
  b->o_eq_mon = take(sizeof(int) * b->Mtot);
  b->o_vptr = take(sizeof(int) * (b->Mtot + 1));
  b->o_vidx = take(sizeof(int) * std::max<long long>(1, b->nnz));
  b->o_queue = take(sizeof(int) * 4);
  b->o_steps = take(sizeof(int) * b->count);
  b->o_flags = take(sizeof(int) * b->count);
  long long stride = 0;
  for (int s = 0; s < b->count; ++s)
    stride = std::max(stride, batch_work_doubles(b->K, b->C, b->n[s], b->D[s], b->threads, b->S3));
  b->work_stride = (stride + 31) / 32 * 32;
  b->o_work = take(sizeof(double) * (size_t)b->work_stride * b->blocks_per_sm * b->num_sms);
  b->total = o;
}

extern "C" {

mdn_status mdn_batch_create(mdn_batch** out, int limbs, int is_complex, int count, const int32_t* n,
                            const int32_t* degree, const int32_t* n_monomials, int threads_per_block,
                            int blocks_per_sm) {
  if (!out) return MDN_EINVAL;
  *out = nullptr;
  const int C = is_complex ? 2 : 1;
  const KernelTable* kt = kernels_for(limbs, C);
  if (!kt || count < 1 || !n || !degree || !n_monomials) return MDN_EINVAL;
  int nmax = 1;
  for (int s = 0; s < count; ++s) {
    if (n[s] < 1 || n[s] > BATCH_MAX_N || degree[s] < 0 || degree[s] > MDN_MAX_DEGREE || n_monomials[s] < 1)
      return MDN_EINVAL;
    nmax = std::max(nmax, (int)n[s]);
  }
  const int threads = threads_per_block ? threads_per_block : std::max(256, (nmax + 31) / 32 * 32);
  if (threads % 32 || threads < 128 || threads > 1024 || threads < nmax) return MDN_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MDN_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MDN_ECUDA;
  const int occ = kt->batch_occupancy(threads);
  if (occ < 1) return MDN_EINVAL;
  const int bps = blocks_per_sm ? blocks_per_sm : occ;
  if (bps < 1 || bps > occ) return MDN_EINVAL;
  mdn_batch* b = new (std::nothrow) mdn_batch();
  if (!b) return MDN_EINVAL;
  b->K = limbs;
  b->C = C;
  b->count = count;
  b->kt = kt;
  b->threads = threads;
  b->blocks_per_sm = bps;
  b->num_sms = sms;
  b->n.assign(n, n + count);
  b->M.assign(n_monomials, n_monomials + count);
  b->D.resize(count);
  b->mono0.resize(count);
  b->coeff_off.resize(count);
  b->series_off.resize(count);
  long long m0 = 0, co = 0, so = 0;
  const long long KC = (long long)limbs * C;
  for (int s = 0; s < count; ++s) {
    b->D[s] = degree[s] + 1;
    b->mono0[s] = m0;
    b->coeff_off[s] = co;
    b->series_off[s] = so;
    m0 += b->M[s];
    co += KC * b->M[s] * b->D[s];
    so += KC * (long long)b->n[s] * b->D[s];
  }
  b->Mtot = m0;
  b->series_total = so;
  if (cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    mdn_batch_destroy(b);
    return MDN_ECUDA;
  }
  *out = b;
  return MDN_OK;
}

size_t mdn_batch_workspace_bytes(const mdn_batch* cb, const int32_t* var_ptr) {
  if (!cb || !var_ptr || var_ptr[0] != 0) return 0;
  mdn_batch* b = const_cast<mdn_batch*>(cb);
  for (long long m = 0; m < b->Mtot; ++m)
    if (var_ptr[m + 1] - var_ptr[m] < 1 || var_ptr[m + 1] - var_ptr[m] > BATCH_MAX_K) return 0;
  b->nnz = var_ptr[b->Mtot];
  b->kmax = kmax_of(b, var_ptr);
  b->S3 = 3 * b->kmax - 2;
  layout(b);
  return b->total;
}

mdn_status mdn_batch_load(mdn_batch* b, const int32_t* eq, const int32_t* vptr, const int32_t* vidx,
                          const double* coeff, const double* cst, void* workspace, size_t ws_bytes,
                          void* cuda_stream) {
  if (!b) return MDN_EINVAL;
  b->loaded = false;
  if (!eq || !vptr || !vidx || !coeff || !cst || !workspace) return bfail(b, MDN_EINVAL, "null argument");
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return bfail(b, MDN_EINVAL, "workspace not 256-byte aligned");
  const size_t need = mdn_batch_workspace_bytes(b, vptr);
  if (!need) return bfail(b, MDN_EINVAL, "bad var_ptr (monomials of 1..16 variables)");
  if (ws_bytes < need) return bfail(b, MDN_EWORKSPACE, "workspace %zu < %zu bytes", ws_bytes, need);
  // structure checks and the tables
  b->h_sys.resize(b->count);
  b->h_eq_ptr.clear();
  b->h_eq_mon.clear();
  b->h_eq_mon.reserve(b->Mtot);
  std::vector<double> cost(b->count);
  for (int s = 0; s < b->count; ++s) {
    const int n = b->n[s], D = b->D[s];
    const long long m0 = b->mono0[s], m1 = m0 + b->M[s];
    std::vector<std::vector<int>> byeq(n);
    double c = 0.0;
    for (long long m = m0; m < m1; ++m) {
      if (eq[m] < 0 || eq[m] >= n) return bfail(b, MDN_EINVAL, "system %d: equation index out of range", s);
      for (int q = vptr[m]; q < vptr[m + 1]; ++q)
        if (vidx[q] < 0 || vidx[q] >= n) return bfail(b, MDN_EINVAL, "system %d: variable index out of range", s);
      byeq[eq[m]].push_back((int)m);
      const int k = vptr[m + 1] - vptr[m];
      c += (k == 1 ? 1.0 : 3.0 * k - 3.0) * D * (D + 1) / 2.0;
    }
    c += (double)n * n * D * (D + 1) / 2.0 + 2.0 * n * n * n;  // updates, QR and W
    cost[s] = c;
    BatchSys& y = b->h_sys[s];
    y.n = n;
    y.D = D;
    y.M = b->M[s];
    y.mono0 = (int)m0;
    y.eq0 = (int)b->h_eq_ptr.size();
    y.pad = 0;
    y.coeff_off = b->coeff_off[s];
    y.series_off = b->series_off[s];
    for (int i = 0; i < n; ++i) {
      b->h_eq_ptr.push_back((int)b->h_eq_mon.size());
      std::stable_sort(byeq[i].begin(), byeq[i].end(),
                       [&](int a, int c2) { return vptr[a + 1] - vptr[a] > vptr[c2 + 1] - vptr[c2]; });
      b->h_eq_mon.insert(b->h_eq_mon.end(), byeq[i].begin(), byeq[i].end());
    }
    b->h_eq_ptr.push_back((int)b->h_eq_mon.size());
  }
  b->h_order.resize(b->count);
  std::iota(b->h_order.begin(), b->h_order.end(), 0);
  std::stable_sort(b->h_order.begin(), b->h_order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  b->h_vptr.assign(vptr, vptr + b->Mtot + 1);
  b->h_vidx.assign(vidx, vidx + std::max<long long>(1, b->nnz));
  if (b->nnz == 0) b->h_vidx[0] = 0;
  b->ws = static_cast<char*>(workspace);
  b->coeff = coeff;
  b->cst = cst;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaStream_t st = b->stream;
  BCU(cudaMemcpyAsync(b->at<BatchSys>(b->o_sys), b->h_sys.data(), sizeof(BatchSys) * b->count,
                      cudaMemcpyHostToDevice, st));
  BCU(cudaMemcpyAsync(b->at<int>(b->o_order), b->h_order.data(), sizeof(int) * b->count, cudaMemcpyHostToDevice, st));
  BCU(cudaMemcpyAsync(b->at<int>(b->o_eq_ptr), b->h_eq_ptr.data(), sizeof(int) * b->h_eq_ptr.size(),
                      cudaMemcpyHostToDevice, st));
  BCU(cudaMemcpyAsync(b->at<int>(b->o_eq_mon), b->h_eq_mon.data(), sizeof(int) * b->h_eq_mon.size(),
                      cudaMemcpyHostToDevice, st));
  BCU(cudaMemcpyAsync(b->at<int>(b->o_vptr), b->h_vptr.data(), sizeof(int) * b->h_vptr.size(),
                      cudaMemcpyHostToDevice, st));
  BCU(cudaMemcpyAsync(b->at<int>(b->o_vidx), b->h_vidx.data(), sizeof(int) * b->h_vidx.size(),
                      cudaMemcpyHostToDevice, st));
  BCU(cudaStreamSynchronize(st));
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  b->loaded = true;
  return MDN_OK;
}

static BatchParams params_of(const mdn_batch* b, double* x, double* f_out, int max_steps, double tol, int eval) {
  BatchParams p{};
  p.count = b->count;
  p.max_steps = max_steps;
  p.evaluate_only = eval;
  p.S3 = b->S3;
  p.tol = tol;
  p.sys = b->at<BatchSys>(b->o_sys);
  p.order = b->at<int>(b->o_order);
  p.eq_ptr = b->at<int>(b->o_eq_ptr);
  p.eq_mon = b->at<int>(b->o_eq_mon);
  p.vptr = b->at<int>(b->o_vptr);
  p.vidx = b->at<int>(b->o_vidx);
  p.coeff = b->coeff;
  p.cst = b->cst;
  p.x = x;
  p.f_out = f_out;
  p.work = b->at<double>(b->o_work);
  p.work_stride = b->work_stride;
  p.queue = b->at<int>(b->o_queue);
  p.steps_out = b->at<int>(b->o_steps);
  p.flags_out = b->at<int>(b->o_flags);
  return p;
}

mdn_status mdn_batch_evaluate(mdn_batch* b, const double* x, double* f_out) {
  if (!b) return MDN_EINVAL;
  if (!b->loaded) return bfail(b, MDN_ESTATE, "no systems loaded");
  if (!x || !f_out) return bfail(b, MDN_EINVAL, "null argument");
  const BatchParams p = params_of(b, const_cast<double*>(x), f_out, 0, 0.0, 1);
  BCU(cudaMemsetAsync(p.queue, 0, sizeof(int), b->stream));
  BCU(b->kt->batch(p, b->blocks_per_sm * b->num_sms, b->threads, b->stream));
  BCU(cudaStreamSynchronize(b->stream));
  return MDN_OK;
}

mdn_status mdn_batch_solve(mdn_batch* b, const double* x0, double* x, int max_steps, double tol, int32_t* steps_out,
                           int32_t* flags_out) {
  if (!b) return MDN_EINVAL;
  if (!b->loaded) return bfail(b, MDN_ESTATE, "no systems loaded");
  if (!x0 || !x) return bfail(b, MDN_EINVAL, "null argument");
  if (max_steps < 0 || max_steps > MDN_MAX_STEPS || !(tol >= 0.0)) return bfail(b, MDN_EINVAL, "max_steps or tol");
  if (!b->gexec || b->g_x0 != x0 || b->g_x != x || b->g_steps != max_steps || b->g_tol != tol) {
    if (b->gexec) {
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
    const BatchParams p = params_of(b, x, nullptr, max_steps, tol, 0);
    cudaGraph_t graph = nullptr;
    BCU(cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    if (x != x0)
      e = cudaMemcpyAsync(x, x0, sizeof(double) * (size_t)b->series_total, cudaMemcpyDeviceToDevice, b->gstream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.queue, 0, sizeof(int), b->gstream);
    if (e == cudaSuccess) e = b->kt->batch(p, b->blocks_per_sm * b->num_sms, b->threads, b->gstream);
    const cudaError_t e2 = cudaStreamEndCapture(b->gstream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return bfail(b, MDN_ECUDA, "capturing the solve: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(b, MDN_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    b->g_x0 = x0;
    b->g_x = x;
    b->g_steps = max_steps;
    b->g_tol = tol;
  }
  // the caller's stream orders the graph launch before and after
  BCU(cudaEventRecord(b->ev_in, b->stream));
  BCU(cudaStreamWaitEvent(b->gstream, b->ev_in, 0));
  BCU(cudaGraphLaunch(b->gexec, b->gstream));
  BCU(cudaEventRecord(b->ev_out, b->gstream));
  BCU(cudaStreamWaitEvent(b->stream, b->ev_out, 0));
  if (steps_out)
    BCU(cudaMemcpyAsync(steps_out, b->at<int>(b->o_steps), sizeof(int) * b->count, cudaMemcpyDeviceToHost,
                        b->stream));
  if (flags_out)
    BCU(cudaMemcpyAsync(flags_out, b->at<int>(b->o_flags), sizeof(int) * b->count, cudaMemcpyDeviceToHost,
                        b->stream));
  BCU(cudaStreamSynchronize(b->stream));
  return MDN_OK;
}

mdn_status mdn_batch_tiles(const mdn_batch* b, int* threads_per_block, int* blocks_per_sm) {
  if (!b) return MDN_EINVAL;
  if (threads_per_block) *threads_per_block = b->threads;
  if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
  return MDN_OK;
}

const char* mdn_batch_last_error(const mdn_batch* b) { return b ? b->err.c_str() : "null batch"; }

void mdn_batch_destroy(mdn_batch* b) {
  if (!b) return;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->gstream) cudaStreamDestroy(b->gstream);
  delete b;
}

}  // extern "C"
