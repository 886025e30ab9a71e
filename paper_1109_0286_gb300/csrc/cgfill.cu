// C-ABI implementation: plans, device memory, and the PCG control flow of the
// constrained-realization fill-in (Bucher & Louis, Sects. 2.1-2.4).
//
// Every numerical step runs in the pass kernels (cg_kernels.cuh); this file
// validates inputs, builds the tables, owns the buffers and sequences the
// passes on the plan's stream.  The CG loop runs in chunks of iterations
// replayed from a captured CUDA graph; each kernel of a converged instance
// returns at once, so the host only polls the per-instance `done` flags
// between chunks.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cgfill.h"
#include "cg_launch.h"
#include "cg_types.h"

using namespace cgf;

namespace {

thread_local std::string g_last_error;

fill_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return FILL_ECUDA;
}

#define CK(expr)                                          \
  do {                                                    \
    cudaError_t e_ = (expr);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr);   \
  } while (0)

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// W_kLmax^m = exp(-2 pi i m / kLmax) from quadrant-reduced angles.
void twiddles_host(std::vector<double>& tw) {
  const int N = kLmax, Q = N / 4;
  tw.resize(2 * size_t(N));
  for (int m = 0; m < N; ++m) {
    const int q = m / Q, r = m % Q;
    const double th = 2.0 * M_PI * double(r) / double(N);
    const double c0 = std::cos(th), s0 = std::sin(th);
    double c, s;
    switch (q) {
      case 0: c = c0; s = s0; break;
      case 1: c = -s0; s = c0; break;
      case 2: c = -c0; s = -s0; break;
      default: c = s0; s = -c0; break;
    }
    tw[2 * m] = c;
    tw[2 * m + 1] = -s;
  }
}

template <typename T>
struct Precision {
  // device buffers (instance-major slabs of batch * npix)
  T* r = nullptr; T* p = nullptr; T* q = nullptr; T* z = nullptr;
  T* u = nullptr; T* y = nullptr; T* b = nullptr; T* spec = nullptr;
  T* t_inv = nullptr; T* t_sqrt = nullptr; T* tw = nullptr;
  CgState* st = nullptr;        // device, batch
  CgState* hst = nullptr;       // pinned mirror
  double* partial = nullptr;
  double* hist = nullptr;
  InstDesc<T>* desc = nullptr;  // device, batch
  InstDesc<T>* hdesc = nullptr; // pinned
  int rows = 0, ffts = 0;
  bool used = false;
  cudaGraphExec_t iter_graph = nullptr;
  int iter_graph_chunk = 0;
  long long iter_graph_kernels = 0;
};

}  // namespace

struct fill_plan {
  int ny = 0, nx = 0, log_l = 0, log_n = 0, batch = 1;
  long long npix = 0, nmasked = 0;
  fill_opts o{};
  cudaStream_t s = nullptr;      // caller's stream
  cudaStream_t cap = nullptr;    // plan-owned stream for graph capture
  uint32_t* obs = nullptr;
  long long launches = 0;        // kernels issued by the current call
  Precision<float> f;
  Precision<double> g;
  std::vector<void*> dev;
  std::vector<void*> host;
  ~fill_plan() {
    if (f.iter_graph) cudaGraphExecDestroy(f.iter_graph);
    if (g.iter_graph) cudaGraphExecDestroy(g.iter_graph);
    for (void* p : dev) cudaFree(p);
    for (void* p : host) cudaFreeHost(p);
    if (cap) cudaStreamDestroy(cap);
  }
  template <typename X>
  cudaError_t dalloc(X** p, size_t count) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, count * sizeof(X) + 256);
    if (e == cudaSuccess) {
      dev.push_back(v);
      *p = reinterpret_cast<X*>(v);
    }
    return e;
  }
  template <typename X>
  cudaError_t halloc(X** p, size_t count) {
    void* v = nullptr;
    cudaError_t e = cudaMallocHost(&v, count * sizeof(X) + 64);
    if (e == cudaSuccess) {
      host.push_back(v);
      *p = reinterpret_cast<X*>(v);
    }
    return e;
  }
};

namespace {

// ----------------------------------------------------------------- schedules
template <typename T>
int default_rows(int log_l, int ny) {
  const int TT = (1 << log_l) / 16;
  int rows = std::max(16, 256 / TT);
  rows = std::min(rows, Launch<T>::max_threads() / TT);
  while (rows > 1 && Launch<T>::row_smem(log_l, rows) > 210 * 1024) rows /= 2;
  return std::min(rows, ny);
}

template <typename T>
int default_ffts(int log_n, int nkx) {
  const int TT = (1 << log_n) / 16;
  int f = std::max(1, 256 / TT);
  f = std::min(f, std::max(1, Launch<T>::max_threads() / TT));
  while (f > 1 && Launch<T>::col_smem(log_n, f) > 100 * 1024) f /= 2;
  return std::min(f, nkx);
}

// ----------------------------------------------------------------- small kernels
__global__ void k_state_init(CgState* st, int n, double tol2, int max_iter, double* hist,
                             int hist_cap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  CgState s{};
  s.tol2 = tol2;
  s.max_iter = max_iter;
  s.first = 1;
  s.hist_cap = hist_cap;
  s.hist = hist ? hist + size_t(i) * hist_cap : nullptr;
  st[i] = s;
}

// Prepares the FP32 inner solve of a refinement step: accumulate the finished
// solve's iteration count, skip converged instances, and set the inner
// tolerance to what the outer target still needs (floored by inner_tol).
__global__ void k_inner_reset(CgState* st32, CgState* st64, int n, double tol, double floor_tol,
                              int max_iter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  CgState& a = st32[i];
  CgState& g = st64[i];
  g.total_iter += a.iter;
  a.iter = 0;
  a.status = 0;
  a.first = 1;
  a.ticket = 0;
  a.alpha = a.beta = 0.0;
  a.max_iter = max_iter;
  if (g.done) {
    a.done = 1;
    return;
  }
  double need = (g.rr > 0.0 && g.bb > 0.0) ? 0.5 * tol * sqrt(g.bb / g.rr) : 1.0;
  need = fmin(fmax(need, floor_tol), 0.5);
  a.tol2 = need * need;
  a.done = 0;
}

__global__ void k_inner_collect(CgState* st32, CgState* st64, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  st64[i].total_iter += st32[i].iter;
  st32[i].iter = 0;
}

// ----------------------------------------------------------------- pass helpers
template <typename T>
Precision<T>& prec(fill_plan* p);
template <>
Precision<float>& prec<float>(fill_plan* p) { return p->f; }
template <>
Precision<double>& prec<double>(fill_plan* p) { return p->g; }

template <typename T>
cudaError_t row(fill_plan* p, cudaStream_t s, int op, int sop, bool in_spec, bool out_spec,
                bool check_done, int ninst = -1) {
  Precision<T>& P = prec<T>(p);
  ++p->launches;
  RowArgs a{p->ny, p->nx, P.rows, op, sop, check_done ? 1 : 0};
  return Launch<T>::row(p->log_l, in_spec, out_spec, P.desc, ninst < 0 ? p->batch : ninst, a,
                        P.tw, s);
}

template <typename T>
cudaError_t col(fill_plan* p, cudaStream_t s, int table, bool check_done, int ninst = -1) {
  Precision<T>& P = prec<T>(p);
  ++p->launches;
  ColArgs a{p->ny, p->nx / 2 + 1, P.ffts, table, check_done ? 1 : 0};
  return Launch<T>::col(p->log_n, P.desc, ninst < 0 ? p->batch : ninst, a, P.tw, s);
}

template <typename T>
cudaError_t vec(fill_plan* p, cudaStream_t s, int op, int sop, bool check_done) {
  Precision<T>& P = prec<T>(p);
  ++p->launches;
  VecArgs a{p->npix, op, sop, check_done ? 1 : 0};
  long long pairs = p->npix / 2;
  int nblk = (int)std::min<long long>((pairs + 255) / 256, 1024);
  return Launch<T>::vec(P.desc, p->batch, a, nblk, s);
}

#define CE(expr)                              \
  do {                                        \
    cudaError_t e_ = (expr);                  \
    if (e_ != cudaSuccess) return e_;         \
  } while (0)

// Unconstrained draw and right-hand side (Sects. 2.3, 2.1):
//   y = F^-1 sqrt(P) F xi;  b = -P_x F^-1 (1/P) F [(d - y) on U].
template <typename T>
cudaError_t draw_and_rhs(fill_plan* p, cudaStream_t s, bool plain_cg) {
  CE(row<T>(p, s, OP_XI, SC_NONE, false, true, false));
  CE(col<T>(p, s, 1, false));
  CE(row<T>(p, s, OP_Y_W, SC_NONE, true, true, false));
  CE(col<T>(p, s, 0, false));
  return row<T>(p, s, OP_B, plain_cg ? SC_BB_RHO : SC_BB, true, false, false);
}

// First preconditioned residual z0 = S S r0 and rho0 = r0^T z0.
template <typename T>
cudaError_t pcg_start(fill_plan* p, cudaStream_t s, int load_sop) {
  if (!p->o.precond) {
    if (load_sop == SC_NONE) return cudaSuccess;
    // plain CG inner solve: rho = bb = ||r||^2, beta = 0
    return row<T>(p, s, OP_LOAD_R, SC_BB_RHO, false, true, true);
  }
  CE(row<T>(p, s, OP_LOAD_R, load_sop, false, true, true));
  CE(col<T>(p, s, 1, true));
  CE(row<T>(p, s, OP_MASK, SC_NONE, true, true, true));
  CE(col<T>(p, s, 1, true));
  return row<T>(p, s, OP_Z, SC_BETA, true, false, true);
}

// One CG iteration (Sect. 2.4).  Preconditioned form with B = S S:
//   p = z + beta p; q = A p; alpha = rho / p^T q; u += alpha p; r -= alpha q;
//   z = S S r; beta = r^T z / rho.
template <typename T>
cudaError_t pcg_iter(fill_plan* p, cudaStream_t s) {
  if (p->o.precond) {
    CE(row<T>(p, s, OP_P_UPD_Z, SC_NONE, false, true, true));
    CE(col<T>(p, s, 0, true));
    CE(row<T>(p, s, OP_Q, SC_ALPHA, true, false, true));
    CE(row<T>(p, s, OP_R_UPD, SC_RCHECK, false, true, true));
    CE(col<T>(p, s, 1, true));
    CE(row<T>(p, s, OP_MASK, SC_NONE, true, true, true));
    CE(col<T>(p, s, 1, true));
    return row<T>(p, s, OP_Z, SC_BETA, true, false, true);
  }
  CE(row<T>(p, s, OP_P_UPD_R, SC_NONE, false, true, true));
  CE(col<T>(p, s, 0, true));
  CE(row<T>(p, s, OP_Q, SC_ALPHA, true, false, true));
  return vec<T>(p, s, VOP_UPDATE, SC_RCHECK_BETA, true);
}

template <typename T>
fill_status build_iter_graph(fill_plan* p, int chunk) {
  Precision<T>& P = prec<T>(p);
  if (P.iter_graph && P.iter_graph_chunk == chunk) return FILL_OK;
  if (P.iter_graph) {
    cudaGraphExecDestroy(P.iter_graph);
    P.iter_graph = nullptr;
  }
  cudaGraph_t graph = nullptr;
  const long long before = p->launches;
  CK(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < chunk && e == cudaSuccess; ++c) e = pcg_iter<T>(p, p->cap);
  cudaError_t e2 = cudaStreamEndCapture(p->cap, &graph);
  P.iter_graph_kernels = p->launches - before;
  p->launches = before;
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(e, "capture pcg_iter");
  }
  CK(e2);
  e = cudaGraphInstantiate(&P.iter_graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  P.iter_graph_chunk = chunk;
  return FILL_OK;
}

// Runs CG iterations until every instance's state is done.
template <typename T>
fill_status run_pcg(fill_plan* p) {
  Precision<T>& P = prec<T>(p);
  const int chunk = 8;
  fill_status fs = build_iter_graph<T>(p, chunk);
  if (fs != FILL_OK) return fs;
  const int limit = p->o.max_iter / chunk + 2;
  for (int c = 0; c <= limit; ++c) {
    CK(cudaMemcpyAsync(P.hst, P.st, sizeof(CgState) * p->batch, cudaMemcpyDeviceToHost, p->s));
    CK(cudaStreamSynchronize(p->s));
    bool all = true;
    for (int i = 0; i < p->batch; ++i) all = all && P.hst[i].done;
    if (all) return FILL_OK;
    CK(cudaGraphLaunch(P.iter_graph, p->s));
    p->launches += P.iter_graph_kernels;
  }
  return FILL_OK;
}

template <typename T>
void fill_desc(fill_plan* p, const void* d, long long d_stride, const uint64_t* seeds, void* out) {
  Precision<T>& P = prec<T>(p);
  for (int i = 0; i < p->batch; ++i) {
    InstDesc<T>& D = P.hdesc[i];
    const size_t off = size_t(i) * p->npix;
    D.d = d ? reinterpret_cast<const T*>(d) + size_t(d_stride) * i : nullptr;
    D.out = out ? reinterpret_cast<T*>(out) + off : nullptr;
    D.seed = seeds ? (unsigned long long)seeds[i] : 0ull;
  }
}

template <typename T>
cudaError_t upload_desc(fill_plan* p) {
  Precision<T>& P = prec<T>(p);
  return cudaMemcpyAsync(P.desc, P.hdesc, sizeof(InstDesc<T>) * p->batch, cudaMemcpyHostToDevice,
                         p->s);
}

template <typename T>
fill_status setup_precision(fill_plan* p, const std::vector<double>& tinv,
                            const std::vector<double>& tsqrt, const std::vector<double>& tw) {
  Precision<T>& P = prec<T>(p);
  P.used = true;
  const size_t B = p->batch, n = p->npix;
  const size_t nspec = 2 * size_t(p->nx / 2 + 1) * p->ny;
  T** vecs[] = {&P.r, &P.p, &P.q, &P.z, &P.u, &P.y, &P.b};
  for (T** v : vecs)
    if (p->dalloc(v, B * n) != cudaSuccess) return FILL_ENOMEM;
  if (p->dalloc(&P.spec, B * nspec) != cudaSuccess) return FILL_ENOMEM;
  const size_t ntab = size_t(p->nx / 2 + 1) * p->ny;
  if (p->dalloc(&P.t_inv, ntab) != cudaSuccess || p->dalloc(&P.t_sqrt, ntab) != cudaSuccess ||
      p->dalloc(&P.tw, 2 * size_t(kLmax)) != cudaSuccess)
    return FILL_ENOMEM;
  if (p->dalloc(&P.st, B) != cudaSuccess || p->halloc(&P.hst, B) != cudaSuccess ||
      p->dalloc(&P.partial, B * kMaxPartials) != cudaSuccess ||
      p->dalloc(&P.desc, B) != cudaSuccess || p->halloc(&P.hdesc, B) != cudaSuccess)
    return FILL_ENOMEM;
  const int hc = std::max(p->o.history_cap, 1);
  if (p->dalloc(&P.hist, B * hc) != cudaSuccess) return FILL_ENOMEM;
  std::vector<T> a(ntab), b2(ntab), w(2 * size_t(kLmax));
  for (size_t i = 0; i < ntab; ++i) {
    a[i] = (T)tinv[i];
    b2[i] = (T)tsqrt[i];
  }
  for (size_t i = 0; i < w.size(); ++i) w[i] = (T)tw[i];
  CK(cudaMemcpy(P.t_inv, a.data(), ntab * sizeof(T), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(P.t_sqrt, b2.data(), ntab * sizeof(T), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(P.tw, w.data(), w.size() * sizeof(T), cudaMemcpyHostToDevice));
  CK(cudaMemset(P.u, 0, B * n * sizeof(T)));
  CK(cudaMemset(P.p, 0, B * n * sizeof(T)));
  P.rows = p->o.rows_per_cta > 0 ? std::min(p->o.rows_per_cta, p->ny) : default_rows<T>(p->log_l, p->ny);
  P.ffts = p->o.ffts_per_cta > 0 ? p->o.ffts_per_cta : default_ffts<T>(p->log_n, p->nx / 2 + 1);
  const int TT = (1 << p->log_l) / 16;
  if (P.rows * TT > Launch<T>::max_threads() || p->ny % P.rows != 0 ||
      p->ny / P.rows > kMaxPartials || Launch<T>::row_smem(p->log_l, P.rows) > 227 * 1024 ||
      P.ffts * ((1 << p->log_n) / 16) > Launch<T>::max_threads() ||
      Launch<T>::col_smem(p->log_n, P.ffts) > 227 * 1024)
    return FILL_EINVAL;
  CK(Launch<T>::prepare());
  for (size_t i = 0; i < B; ++i) {
    InstDesc<T> D{};
    D.obs = p->obs;
    D.t_inv = P.t_inv;
    D.t_sqrt = P.t_sqrt;
    D.spec = P.spec + i * nspec;
    D.r = P.r + i * n;
    D.p = P.p + i * n;
    D.q = P.q + i * n;
    D.z = P.z + i * n;
    D.u = P.u + i * n;
    D.y = P.y + i * n;
    D.b = P.b + i * n;
    D.st = P.st + i;
    D.partial = P.partial + i * kMaxPartials;
    P.hdesc[i] = D;
  }
  return FILL_OK;
}

template <typename T>
cudaError_t init_states(fill_plan* p, double tol) {
  Precision<T>& P = prec<T>(p);
  const int hc = std::max(p->o.history_cap, 1);
  ++p->launches;
  k_state_init<<<(p->batch + 127) / 128, 128, 0, p->s>>>(P.st, p->batch, tol * tol,
                                                        p->o.max_iter, P.hist, hc);
  return cudaGetLastError();
}

void collect_stats(fill_plan* p, fill_stats* stats, double ms, fill_status* worst) {
  const bool mixed = p->o.mode == FILL_MODE_MIXED;
  for (int i = 0; i < p->batch; ++i) {
    fill_stats st{};
    if (mixed) {
      const CgState& a = p->f.hst[i];
      const CgState& g = p->g.hst[i];
      st.iters = g.total_iter;
      st.refine_steps = g.refine;
      const bool conv = g.rr <= g.tol2 * g.bb;
      st.status = g.status ? g.status : (conv ? FILL_OK : FILL_ENOTCONV);
      st.rel_resid = a.bb > 0 ? std::sqrt(a.rr / a.bb) : 0.0;
      st.true_rel_resid = g.bb > 0 ? std::sqrt(g.rr / g.bb) : 0.0;
    } else {
      const CgState& a = p->o.mode == FILL_MODE_FP32 ? p->f.hst[i] : p->g.hst[i];
      st.iters = a.iter;
      st.status = a.status;
      st.rel_resid = a.bb > 0 ? std::sqrt(a.rr / a.bb) : 0.0;
      st.true_rel_resid = -1.0;
    }
    st.ms = ms;
    st.launches = (int)p->launches;
    if (st.status > *worst) *worst = (fill_status)st.status;
    if (stats) stats[i] = st;
  }
}

}  // namespace

// =================================================================== C ABI
extern "C" {

void fill_opts_default(fill_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->mode = FILL_MODE_MIXED;
  o->precond = 1;
  o->batch = 1;
  o->max_iter = 10000;
  o->max_refine = 10;
  o->inner_tol = 1e-6;
  o->history_cap = 0;
}

fill_status fill_init(fill_plan** out, int ny, int nx, const double* P_half,
                      const uint8_t* observed, const fill_opts* opts, void* stream) {
  if (!out || !P_half || !observed) return FILL_EINVAL;
  *out = nullptr;
  if (!pow2(nx) || !pow2(ny) || nx < 32 || nx > 8192 || ny < 16 || ny > 8192) return FILL_EINVAL;
  fill_opts o;
  if (opts)
    o = *opts;
  else
    fill_opts_default(&o);
  if (o.mode < 0 || o.mode > 2 || o.batch < 1 || o.batch > 65535 || o.max_iter < 1 ||
      o.max_refine < 1 || !(o.inner_tol > 0.0) || o.history_cap < 0 || o.rows_per_cta < 0 ||
      o.ffts_per_cta < 0)
    return FILL_EINVAL;
  const int nkx = nx / 2 + 1;
  // P: finite, positive, real-symmetric on the self-conjugate columns.
  for (long long i = 0; i < (long long)ny * nkx; ++i)
    if (!(std::isfinite(P_half[i]) && P_half[i] > 0.0)) return FILL_EINVAL;
  for (int col : {0, nx / 2})
    for (int my = 0; my < ny; ++my) {
      const double a = P_half[(size_t)my * nkx + col], b = P_half[(size_t)((ny - my) % ny) * nkx + col];
      if (std::fabs(a - b) > 1e-12 * std::fabs(a)) return FILL_EINVAL;
    }
  const long long npix = (long long)ny * nx;
  long long nmasked = 0;
  std::vector<uint32_t> bits((npix + 31) / 32, 0u);
  for (long long i = 0; i < npix; ++i) {
    if (observed[i] > 1) return FILL_EINVAL;
    if (observed[i])
      bits[i >> 5] |= 1u << (i & 31);
    else
      ++nmasked;
  }
  fill_plan* p = new (std::nothrow) fill_plan();
  if (!p) return FILL_ENOMEM;
  p->ny = ny;
  p->nx = nx;
  p->log_l = ilog2(nx / 2);
  p->log_n = ilog2(ny);
  p->batch = o.batch;
  p->npix = npix;
  p->nmasked = nmasked;
  p->o = o;
  p->s = reinterpret_cast<cudaStream_t>(stream);
  fill_status fs = FILL_OK;
  auto fail = [&](fill_status st) {
    delete p;
    return st;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamCreate"));
  if (p->dalloc(&p->obs, bits.size()) != cudaSuccess) return fail(FILL_ENOMEM);
  e = cudaMemcpy(p->obs, bits.data(), bits.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_fail(e, "upload mask"));
  // Tables [kx][ky] with the inverse DFT's 1/n folded in.
  std::vector<double> tinv((size_t)nkx * ny), tsqrt((size_t)nkx * ny), tw;
  for (int ky = 0; ky < ny; ++ky)
    for (int kx = 0; kx < nkx; ++kx) {
      const double P = P_half[(size_t)ky * nkx + kx];
      tinv[(size_t)kx * ny + ky] = 1.0 / (P * double(npix));
      tsqrt[(size_t)kx * ny + ky] = std::sqrt(P) / double(npix);
    }
  twiddles_host(tw);
  if (o.mode == FILL_MODE_FP32 || o.mode == FILL_MODE_MIXED) {
    fs = setup_precision<float>(p, tinv, tsqrt, tw);
    if (fs != FILL_OK) return fail(fs);
  }
  if (o.mode == FILL_MODE_FP64 || o.mode == FILL_MODE_MIXED) {
    fs = setup_precision<double>(p, tinv, tsqrt, tw);
    if (fs != FILL_OK) return fail(fs);
  }
  if (o.mode == FILL_MODE_MIXED) {
    for (int i = 0; i < p->batch; ++i) {
      p->g.hdesc[i].dlt = p->f.hdesc[i].u;
      p->g.hdesc[i].r32 = p->f.hdesc[i].r;
    }
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(cuda_fail(e, "fill_init"));
  *out = p;
  return FILL_OK;
}

fill_status fill_realize(fill_plan* p, const void* d, long long d_stride, const uint64_t* seeds,
                         double tol, void* out, fill_stats* stats) {
  if (!p || !d || !seeds || !out || !(tol >= 0.0) || d_stride < 0) return FILL_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  const int B = p->batch;
  p->launches = 0;
  const size_t n = p->npix;
  fill_status worst = FILL_OK;
  if (p->nmasked == 0) {  // nothing to fill: out = d
    const size_t esz = p->o.mode == FILL_MODE_FP32 ? sizeof(float) : sizeof(double);
    for (int i = 0; i < B; ++i)
      CK(cudaMemcpyAsync((char*)out + i * n * esz, (const char*)d + size_t(d_stride) * i * esz,
                         n * esz, cudaMemcpyDeviceToDevice, p->s));
    CK(cudaStreamSynchronize(p->s));
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (stats)
      for (int i = 0; i < B; ++i) stats[i] = fill_stats{0, 0, FILL_OK, 0, 0.0, 0.0, ms};
    return FILL_OK;
  }
  fill_status fs;
  if (p->o.mode == FILL_MODE_FP32 || p->o.mode == FILL_MODE_FP64) {
    const bool f32 = p->o.mode == FILL_MODE_FP32;
    if (f32) {
      fill_desc<float>(p, d, d_stride, seeds, out);
      CK(upload_desc<float>(p));
      CK(init_states<float>(p, tol));
      CK(cudaMemsetAsync(p->f.u, 0, B * n * sizeof(float), p->s));
      CK(cudaMemsetAsync(p->f.p, 0, B * n * sizeof(float), p->s));
      CK(draw_and_rhs<float>(p, p->s, !p->o.precond));
      CK(pcg_start<float>(p, p->s, SC_NONE));
      fs = run_pcg<float>(p);
      if (fs != FILL_OK) return fs;
      CK(vec<float>(p, p->s, VOP_ASSEMBLE, SC_NONE, false));
      CK(cudaMemcpyAsync(p->f.hst, p->f.st, sizeof(CgState) * B, cudaMemcpyDeviceToHost, p->s));
    } else {
      fill_desc<double>(p, d, d_stride, seeds, out);
      CK(upload_desc<double>(p));
      CK(init_states<double>(p, tol));
      CK(cudaMemsetAsync(p->g.u, 0, B * n * sizeof(double), p->s));
      CK(cudaMemsetAsync(p->g.p, 0, B * n * sizeof(double), p->s));
      CK(draw_and_rhs<double>(p, p->s, !p->o.precond));
      CK(pcg_start<double>(p, p->s, SC_NONE));
      fs = run_pcg<double>(p);
      if (fs != FILL_OK) return fs;
      CK(vec<double>(p, p->s, VOP_ASSEMBLE, SC_NONE, false));
      CK(cudaMemcpyAsync(p->g.hst, p->g.st, sizeof(CgState) * B, cudaMemcpyDeviceToHost, p->s));
    }
  } else {
    // Mixed: FP64 draw / RHS / residual, FP32 inner PCG, FP64 refinement.
    fill_desc<double>(p, d, d_stride, seeds, out);
    fill_desc<float>(p, nullptr, 0, seeds, nullptr);
    CK(upload_desc<double>(p));
    CK(upload_desc<float>(p));
    CK(init_states<double>(p, tol));
    CK(init_states<float>(p, p->o.inner_tol));
    CK(cudaMemsetAsync(p->g.u, 0, B * n * sizeof(double), p->s));
    CK(draw_and_rhs<double>(p, p->s, false));
    const int nb = (B + 127) / 128;
    for (int outer = 0; outer < p->o.max_refine; ++outer) {
      ++p->launches;
      k_inner_reset<<<nb, 128, 0, p->s>>>(p->f.st, p->g.st, B, tol, p->o.inner_tol, p->o.max_iter);
      CK(cudaGetLastError());
      CK(cudaMemsetAsync(p->f.u, 0, B * n * sizeof(float), p->s));
      CK(cudaMemsetAsync(p->f.p, 0, B * n * sizeof(float), p->s));
      CK(pcg_start<float>(p, p->s, SC_BB));
      fs = run_pcg<float>(p);
      if (fs != FILL_OK) return fs;
      // u += delta (FP64), r = b - A u (FP64 true residual), r32 = (float) r
      CK(row<double>(p, p->s, OP_U64_UPD, SC_NONE, false, true, true));
      CK(col<double>(p, p->s, 0, true));
      CK(row<double>(p, p->s, OP_RES, SC_RES, true, false, true));
      CK(cudaMemcpyAsync(p->g.hst, p->g.st, sizeof(CgState) * B, cudaMemcpyDeviceToHost, p->s));
      CK(cudaStreamSynchronize(p->s));
      bool all = true;
      for (int i = 0; i < B; ++i) all = all && p->g.hst[i].done;
      if (all) break;
    }
    ++p->launches;
    k_inner_collect<<<nb, 128, 0, p->s>>>(p->f.st, p->g.st, B);
    CK(cudaGetLastError());
    CK(vec<double>(p, p->s, VOP_ASSEMBLE, SC_NONE, false));
    CK(cudaMemcpyAsync(p->g.hst, p->g.st, sizeof(CgState) * B, cudaMemcpyDeviceToHost, p->s));
    CK(cudaMemcpyAsync(p->f.hst, p->f.st, sizeof(CgState) * B, cudaMemcpyDeviceToHost, p->s));
  }
  CK(cudaStreamSynchronize(p->s));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  collect_stats(p, stats, ms, &worst);
  return worst;
}

fill_status fill_draw(fill_plan* p, const uint64_t* seeds, void* out) {
  if (!p || !seeds || !out) return FILL_EINVAL;
  const size_t n = p->npix;
  if (p->o.mode == FILL_MODE_FP32) {
    fill_desc<float>(p, nullptr, 0, seeds, nullptr);
    CK(upload_desc<float>(p));
    CK(init_states<float>(p, 0.0));
    CK(row<float>(p, p->s, OP_XI, SC_NONE, false, true, false));
    CK(col<float>(p, p->s, 1, false));
    CK(row<float>(p, p->s, OP_STORE_Y, SC_NONE, true, false, false));
    CK(cudaMemcpyAsync(out, p->f.y, p->batch * n * sizeof(float), cudaMemcpyDeviceToDevice, p->s));
  } else {
    fill_desc<double>(p, nullptr, 0, seeds, nullptr);
    CK(upload_desc<double>(p));
    CK(init_states<double>(p, 0.0));
    CK(row<double>(p, p->s, OP_XI, SC_NONE, false, true, false));
    CK(col<double>(p, p->s, 1, false));
    CK(row<double>(p, p->s, OP_STORE_Y, SC_NONE, true, false, false));
    CK(cudaMemcpyAsync(out, p->g.y, p->batch * n * sizeof(double), cudaMemcpyDeviceToDevice, p->s));
  }
  CK(cudaStreamSynchronize(p->s));
  return FILL_OK;
}

}  // extern "C"

namespace {
template <typename T>
fill_status apply_t(fill_plan* p, int which, const void* in, void* out) {
  Precision<T>& P = prec<T>(p);
  const size_t n = p->npix;
  fill_desc<T>(p, nullptr, 0, nullptr, nullptr);
  CK(upload_desc<T>(p));
  CK(init_states<T>(p, 0.0));
  CK(cudaMemcpyAsync(P.r, in, n * sizeof(T), cudaMemcpyDeviceToDevice, p->s));
  const bool masked = which >= 2;
  const int table = (which == 0 || which == 2) ? 0 : 1;
  CK(row<T>(p, p->s, masked ? OP_LOAD_R_MASK : OP_LOAD_R, SC_NONE, false, true, false, 1));
  CK(col<T>(p, p->s, table, false, 1));
  CK(row<T>(p, p->s, masked ? OP_Z : OP_STORE_Y, SC_NONE, true, false, false, 1));
  CK(cudaMemcpyAsync(out, masked ? P.z : P.y, n * sizeof(T), cudaMemcpyDeviceToDevice, p->s));
  CK(cudaStreamSynchronize(p->s));
  return FILL_OK;
}
}  // namespace

extern "C" {

fill_status fill_apply(fill_plan* p, int which, const void* in, void* out) {
  if (!p || !in || !out || which < 0 || which > 3 || in == out) return FILL_EINVAL;
  return p->o.mode == FILL_MODE_FP32 ? apply_t<float>(p, which, in, out)
                                     : apply_t<double>(p, which, in, out);
}

fill_status fill_history(fill_plan* p, int inst, double* hist, int cap, int* count) {
  if (!p || !hist || inst < 0 || inst >= p->batch || cap < 0) return FILL_EINVAL;
  const int hc = std::max(p->o.history_cap, 1);
  int m = 0;
  const double* src = nullptr;
  if (p->o.mode == FILL_MODE_MIXED) {
    m = p->g.hst[inst].refine + 1;  // FP64 true residual after each refinement step
    src = p->g.hist;
  } else if (p->o.mode == FILL_MODE_FP32) {
    m = p->f.hst[inst].iter + 1;
    src = p->f.hist;
  } else {
    m = p->g.hst[inst].iter + 1;
    src = p->g.hist;
  }
  m = p->o.history_cap == 0 ? 0 : std::min(std::min(cap, hc), m);
  if (m > 0) CK(cudaMemcpy(hist, src + size_t(inst) * hc, m * sizeof(double), cudaMemcpyDeviceToHost));
  if (count) *count = m;
  return FILL_OK;
}

}  // extern "C"

namespace {
template <typename T>
fill_status time_pass_t(fill_plan* p, int pass, int reps, double* ms, double* bytes) {
  Precision<T>& P = prec<T>(p);
  if (!P.used) return FILL_EINVAL;
  fill_desc<T>(p, nullptr, 0, nullptr, nullptr);
  CK(upload_desc<T>(p));
  CK(init_states<T>(p, 0.0));
  const double n = double(p->npix), S = double(p->nx / 2 + 1) * p->ny, t = sizeof(T);
  const double SB = 2.0 * S * t;
  auto launch = [&](cudaStream_t s) -> cudaError_t {
    switch (pass) {
      case 0: return col<T>(p, s, 0, false);
      case 1: return row<T>(p, s, OP_R_UPD, SC_RCHECK, false, true, false);
      case 2: return row<T>(p, s, OP_P_UPD_Z, SC_NONE, false, true, false);
      case 3: return row<T>(p, s, OP_Q, SC_ALPHA, true, false, false);
      default: return row<T>(p, s, OP_MASK, SC_NONE, true, true, false);
    }
  };
  double b = 0.0;
  switch (pass) {
    case 0: b = 2.0 * SB + S * t; break;
    case 1: b = 6.0 * n * t + SB; break;
    case 2: b = 3.0 * n * t + SB; break;
    case 3: b = SB + 2.0 * n * t + n / 8.0; break;
    default: b = 2.0 * SB + n / 8.0; break;
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(launch(p->s));
  CK(cudaEventRecord(e0, p->s));
  for (int i = 0; i < reps; ++i) CK(launch(p->s));
  CK(cudaEventRecord(e1, p->s));
  CK(cudaEventSynchronize(e1));
  float m = 0.f;
  CK(cudaEventElapsedTime(&m, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = double(m) / reps;
  *bytes = b * p->batch;
  return FILL_OK;
}
}  // namespace

extern "C" {

fill_status fill_time_pass(fill_plan* p, int pass, int precision, int reps, double* ms,
                           double* bytes) {
  if (!p || !ms || !bytes || pass < 0 || pass > 4 || reps < 1 || precision < 0 || precision > 1)
    return FILL_EINVAL;
  return precision == 0 ? time_pass_t<float>(p, pass, reps, ms, bytes)
                        : time_pass_t<double>(p, pass, reps, ms, bytes);
}

long long fill_masked_count(const fill_plan* p) { return p ? p->nmasked : -1; }

void fill_destroy(fill_plan* p) {
  if (!p) return;
  cudaStreamSynchronize(p->s);
  delete p;
}

const char* fill_strerror(fill_status s) {
  switch (s) {
    case FILL_OK: return "ok";
    case FILL_EINVAL: return "invalid argument";
    case FILL_ENOMEM: return "out of memory";
    case FILL_ENOTCONV: return "not converged within max_iter";
    case FILL_EBREAKDOWN: return "CG breakdown (non-positive curvature or non-finite value)";
    case FILL_ETIMEOUT: return "device wait timed out";
    case FILL_ECUDA: return "CUDA error";
  }
  return "unknown status";
}

const char* fill_last_error(void) { return g_last_error.c_str(); }

int fill_version(void) { return CGFILL_VERSION; }

}  // extern "C"
