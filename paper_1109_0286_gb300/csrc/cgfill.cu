// C-ABI implementation: plans, device memory, and the PCG control flow of the
// constrained-realization fill-in (Bucher & Louis, Sects. 2.1-2.4).
//
// Every numerical step runs in the pass kernels (cg_kernels.cuh); this file
// validates inputs, builds the tables, owns the buffers and sequences the
// passes on the plan's stream.  A whole CG loop is one launch of a captured
// CUDA graph with a conditional WHILE node: kernels of converged instances
// return at once, and a one-CTA control kernel ends the loop when every
// instance is done (or after a hard iteration limit).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/cgfill.h"
#include "cg_common.cuh"
#include "cg_generic.h"
#include "cg_launch.h"
#include "cg_schedule.h"
#include "cg_types.h"

using namespace cgf;

namespace {

thread_local std::string g_last_error;

}  // namespace

void cgf_set_last_error(const char* msg) { g_last_error = msg; }

namespace {

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

// exp(-2 pi i num / den) in FP64 from an angle reduced to [0, pi/4]
// (octant symmetry), so the result carries the full accuracy of cos / sin.
void unit_root(long long num, long long den, double* re, double* im) {
  const long long m = 8 * (((num % den) + den) % den);
  const int o = (int)(m / den);                 // octant 0..7
  const double f = double(m % den) / double(den);
  const double th = (o & 1) ? (1.0 - f) * M_PI / 4.0 : f * M_PI / 4.0;
  const double c0 = std::cos(th), s0 = std::sin(th);
  double c, sn;
  switch (o) {
    case 0: c = c0; sn = s0; break;
    case 1: c = s0; sn = c0; break;
    case 2: c = -s0; sn = c0; break;
    case 3: c = -c0; sn = s0; break;
    case 4: c = -c0; sn = -s0; break;
    case 5: c = -s0; sn = -c0; break;
    case 6: c = s0; sn = -c0; break;
    default: c = c0; sn = -s0; break;
  }
  *re = c;
  *im = -sn;
}

// W_kLmax^m = exp(-2 pi i m / kLmax) from quadrant-reduced angles, followed
// by the per-stage tables of every power-of-two length (stw_* in cg_types.h).
void twiddles_host(std::vector<double>& tw) {
  const int N = kLmax, Q = N / 4;
  tw.resize(2 * size_t(kTwEntries));
  for (int l = 4; l <= 13; ++l)
    for (int st = stw_first(l); st < l / 4; ++st) {
      const int ns = stw_ns(l, st);
      const size_t base = size_t(kLmax) + stw_base(l) + stw_stage_off(l, st);
      for (int r = 1; r < 16; ++r)
        for (int jm = 0; jm < ns; ++jm) {
          const size_t e = base + size_t(r - 1) * ns + jm;
          unit_root((long long)jm * r, 16LL * ns, &tw[2 * e], &tw[2 * e + 1]);
        }
    }
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
  T* w = nullptr; T* spec2 = nullptr;              // backward buffers
  int* band = nullptr; T* coef1 = nullptr; T* coef2 = nullptr;
  double* bpart = nullptr; double* bsum = nullptr; // band partials, sums
  int nbands = 0;
  T* t_inv = nullptr; T* t_sqrt = nullptr; T* tw = nullptr;
  CgState* st = nullptr;        // device, batch
  CgState* hst = nullptr;       // pinned mirror
  double* partial = nullptr;
  double* hist = nullptr;
  double* coef = nullptr;       // CG coefficients, 2 history_cap per instance
  T* kt = nullptr;              // kernel tables of the Sect. 6.3 solver
  int nk = 0, nk_cap = 0;
  T* gwl = nullptr; T* gwx = nullptr; T* gwn = nullptr;   // mixed-radix twiddles
  InstDesc<T>* desc = nullptr;  // device, batch
  InstDesc<T>* hdesc = nullptr; // pinned
  int rows = 0, ffts = 0;
  int col_variant = 0;          // column kernel of the table passes (ColArgs::variant)
  bool used = false;
  cudaGraphExec_t iter_graph = nullptr;   // CG loop graph (conditional WHILE node)
  long long iter_graph_kernels = 0;       // kernels per loop body
  CgState** stp = nullptr;                // device: state pointer of each instance
};

}  // namespace

constexpr int kMaxLanes = 8;   // CG-loop lanes of a plan (fill_opts::lanes)

struct fill_plan {
  int ny = 0, nx = 0, log_l = 0, log_n = 0, batch = 1;
  bool gen = false;              // mixed-radix grid (cg_generic.h kernels)
  cgf::GenLen grow{}, gcol{};    // its row (nx/2) and column (ny) transforms
  long long npix = 0, nmasked = 0;
  fill_opts o{};
  cudaStream_t s = nullptr;      // caller's stream
  cudaStream_t cap = nullptr;    // plan-owned stream for graph capture
  cudaStream_t cap2 = nullptr;   // second capture stream (conditional bodies)
  int nlanes = 1;                // CG-loop lanes (fill_opts::lanes)
  cudaStream_t lane_s[kMaxLanes] = {};
  cudaEvent_t lane_join[kMaxLanes] = {};
  cudaEvent_t lane_fork = nullptr, lane_fork_cap = nullptr;
  uint2* mw = nullptr;           // mask words: observed bits, compact offset
  long long nv = 0;              // compact vector stride per instance (>= nmasked)
  std::vector<double> P_half;    // host copy of the spectrum
  double* P_dev = nullptr;       // device copy (fill_set_spectrum builds the tables from it)
  double* sig_dev = nullptr;     // device copy of the band templates' S(k) (fill_set_bands)
  std::vector<int32_t> band_idx; // band templates of fill_set_bands (host copies), so
  std::vector<double> band_sig;  // that fill_set_spectrum can rebuild the gradient weights
  int nbands = 0;
  struct fill_group* batch_group = nullptr;     // cached group of fill_realize_batch
  std::vector<unsigned long long> batch_key;    // serials of its plans, in order
  unsigned long long serial = 0;                // unique id of this plan
  long long launches = 0;        // kernels issued by the current call
  double relax_a = 0.0;          // max_k 1/P(k): white level of C^-1 (Sect. 5 relaxation)
  cudaGraphExec_t mixed_graph = nullptr;   // reliable-update mixed CG loop
  long long mixed_graph_kernels = 0;
  int* dev_err = nullptr;        // device: set by a kernel whose bounded wait gave up
  int* loop_counter = nullptr;   // device [2]: loop bodies, IF bodies of the last loop graph
  int* hloop = nullptr;          // pinned: loop counters [0..1], device error flag [2]
  long long if_kernels = 0;      // kernels inside the update IF node
  Precision<float> f;
  Precision<double> g;           // FP64 mode
  Precision<df> h;               // mixed mode's high precision (double-float)
  std::vector<void*> dev;
  std::vector<void*> host;
  ~fill_plan() {
    if (batch_group) fill_group_destroy(batch_group);
    if (mixed_graph) cudaGraphExecDestroy(mixed_graph);
    if (f.iter_graph) cudaGraphExecDestroy(f.iter_graph);
    if (g.iter_graph) cudaGraphExecDestroy(g.iter_graph);
    if (h.iter_graph) cudaGraphExecDestroy(h.iter_graph);
    for (void* p : dev) cudaFree(p);
    for (void* p : host) cudaFreeHost(p);
    if (cap) cudaStreamDestroy(cap);
    if (cap2) cudaStreamDestroy(cap2);
    for (int l = 0; l < kMaxLanes; ++l) {
      if (lane_s[l]) cudaStreamDestroy(lane_s[l]);
      if (lane_join[l]) cudaEventDestroy(lane_join[l]);
    }
    if (lane_fork) cudaEventDestroy(lane_fork);
    if (lane_fork_cap) cudaEventDestroy(lane_fork_cap);
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

// ----------------------------------------------------------------- small kernels
template <typename T>
__global__ void k_state_init(const InstDesc<T>* desc, int n, double tol2, int max_iter,
                             int hist_cap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  CgState s{};
  s.tol2 = tol2;
  s.max_iter = max_iter;
  s.first = 1;
  s.hist_cap = hist_cap;
  s.hist = desc[i].hist;
  s.coef = desc[i].coef;
  *desc[i].st = s;
}

template <typename T>
__global__ void k_gather_states(const InstDesc<T>* desc, int n, CgState* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = *desc[i].st;
}

// Prepares the FP32 inner solve of a refinement step: accumulate the finished
// solve's iteration count, skip converged instances, and set the inner
// tolerance to what the outer target still needs (floored by inner_tol).
// (States reached through the FP32 and double-float descriptors of the same
// instances, which need not be contiguous: a group's class spans plans.)
__global__ void k_inner_reset(const InstDesc<float>* lo, const InstDesc<df>* hi, int n,
                              double tol, double floor_tol, int max_iter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  CgState& a = *lo[i].st;
  CgState& g = *hi[i].st;
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

__global__ void k_inner_collect(const InstDesc<float>* lo, const InstDesc<df>* hi, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  CgState& a = *lo[i].st;
  hi[i].st->total_iter += a.iter;
  a.last_iter = a.iter;
  a.iter = 0;
}

// Spectral tables of one precision from P on the device (fill_set_spectrum):
// 1/(nP) and sqrt(P)/n in the transposed [kx][ky] layout and, with band
// templates, the band-gradient weights wt S / (2 n sqrt P) and wt S / (n P^2)
// (wt = 1 on the self-conjugate columns kx = 0, nx/2, else 2), in FP64 and
// rounded to T once -- the values the host path computes.
template <typename T>
__global__ void k_spectral_tables(const double* P, const double* sig, int ny, int nkx, int nx,
                                  T* t_inv, T* t_sqrt, T* c1, T* c2) {
  const long long total = (long long)ny * nkx;
  const double n = double(ny) * double(nx);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(t / ny), ky = (int)(t % ny);
    const long long h = (long long)ky * nkx + kx;
    const double p = P[h];
    t_inv[t] = (T)(1.0 / (p * n));
    t_sqrt[t] = (T)(sqrt(p) / n);
    if (c1) {
      const double wt = (kx == 0 || kx == nx / 2) ? 1.0 : 2.0, sg = sig[h];
      c1[t] = (T)(wt * sg / (2.0 * n * sqrt(p)));
      c2[t] = (T)(wt * sg / (n * p * p));
    }
  }
}

// ----------------------------------------------------------------- pass helpers
template <typename T>
Precision<T>& prec(fill_plan* p);
template <>
Precision<float>& prec<float>(fill_plan* p) { return p->f; }
template <>
Precision<double>& prec<double>(fill_plan* p) { return p->g; }
template <>
Precision<df>& prec<df>(fill_plan* p) { return p->h; }

// Launch context: one grid size, one descriptor array (a plan's instances or
// a size class of a group).
template <typename T>
struct Ctx {
  int ny, nx, log_l, log_n, rows, ffts, ninst, precond;
  int col_variant;
  long long npix;
  const InstDesc<T>* desc;
  const T* tw;
  long long* launches;
  int* err = nullptr;             // device error flag of bounded waits
  const GenLen* grow = nullptr;   // mixed-radix grids: transforms and twiddles
  const GenLen* gcol = nullptr;
  const T* gwl = nullptr;
  const T* gwx = nullptr;
  const T* gwn = nullptr;
};

template <typename T>
Ctx<T> ctx(fill_plan* p, int ninst = -1) {
  Precision<T>& P = prec<T>(p);
  Ctx<T> c{p->ny, p->nx, p->log_l, p->log_n, P.rows, P.ffts,
           ninst < 0 ? p->batch : ninst, p->o.precond, P.col_variant, p->npix, P.desc, P.tw,
           &p->launches, p->dev_err};
  if (p->gen) {
    c.grow = &p->grow;
    c.gcol = &p->gcol;
    c.gwl = P.gwl;
    c.gwx = P.gwx;
    c.gwn = P.gwn;
  }
  return c;
}

template <typename T>
cudaError_t row(const Ctx<T>& c, cudaStream_t s, int op, int sop, bool in_spec, bool out_spec,
                int skip, int spec_sel = 0, int param = 0) {
  ++*c.launches;
  RowArgs a{c.ny, c.nx, c.rows, ilog2(c.rows), op, sop, skip, spec_sel, param};
  if (c.grow)
    return GenLaunch<T>::row(in_spec, out_spec, c.desc, c.ninst, a, *c.grow, c.gwl, c.gwx, s);
  return Launch<T>::row(c.log_l, in_spec, out_spec, c.desc, c.ninst, a, c.tw, s);
}

template <typename T>
cudaError_t col(const Ctx<T>& c, cudaStream_t s, int table, int skip, int spec_sel = 0,
                int pre = 0) {
  ++*c.launches;
  ColArgs a{c.ny, c.nx / 2 + 1, c.ffts, table, skip, spec_sel, pre, c.err, c.col_variant};
  if (c.gcol) return GenLaunch<T>::col(c.desc, c.ninst, a, *c.gcol, c.gwn, s);
  return Launch<T>::col(c.log_n, c.desc, c.ninst, a, c.tw, s);
}

template <typename T>
cudaError_t vec(const Ctx<T>& c, cudaStream_t s, int op, int sop, int skip, double p0 = 0.0,
                double p1 = 0.0) {
  ++*c.launches;
  VecArgs a{c.npix, op, sop, skip, p0, p1, c.nx};
  const long long pairs = c.npix / 2;
  const int nblk = (int)std::min<long long>((pairs + 255) / 256, 1024);
  return Launch<T>::vec(c.desc, c.ninst, a, nblk, s);
}

template <typename T>
cudaError_t row(fill_plan* p, cudaStream_t s, int op, int sop, bool in_spec, bool out_spec,
                int skip, int ninst = -1, int spec_sel = 0) {
  return row<T>(ctx<T>(p, ninst), s, op, sop, in_spec, out_spec, skip, spec_sel);
}
template <typename T>
cudaError_t col(fill_plan* p, cudaStream_t s, int table, int skip, int ninst = -1,
                int spec_sel = 0) {
  return col<T>(ctx<T>(p, ninst), s, table, skip, spec_sel);
}
template <typename T>
cudaError_t vec(fill_plan* p, cudaStream_t s, int op, int sop, int skip) {
  return vec<T>(ctx<T>(p), s, op, sop, skip);
}

#define CE(expr)                              \
  do {                                        \
    cudaError_t e_ = (expr);                  \
    if (e_ != cudaSuccess) return e_;         \
  } while (0)

// Unconstrained draw and right-hand side (Sects. 2.3, 2.1):
//   y = F^-1 sqrt(P) F xi;  b = -P_x F^-1 (1/P) F [(d - y) on U].
template <typename T>
cudaError_t draw_and_rhs(const Ctx<T>& c, cudaStream_t s, bool plain_cg) {
  CE(row<T>(c, s, OP_XI, SC_NONE, false, true, false));
  CE(col<T>(c, s, 1, false));
  CE(row<T>(c, s, OP_Y_W, SC_NONE, true, true, false));
  CE(col<T>(c, s, 0, false));
  return row<T>(c, s, OP_B, plain_cg ? SC_BB_RHO : SC_BB, true, false, false);
}

// First preconditioned residual z0 = S S r0 and rho0 = r0^T z0.
template <typename T>
cudaError_t pcg_start(const Ctx<T>& c, cudaStream_t s, int load_sop) {
  if (!c.precond) {
    if (load_sop == SC_NONE) return cudaSuccess;
    // plain CG inner solve: rho = bb = ||r||^2, beta = 0
    return row<T>(c, s, OP_LOAD_R, SC_BB_RHO, false, true, true);
  }
  CE(row<T>(c, s, OP_LOAD_R, load_sop, false, true, true));
  CE(col<T>(c, s, 1, true));
  CE(row<T>(c, s, OP_MASK, SC_NONE, true, true, true));
  CE(col<T>(c, s, 1, true));
  return row<T>(c, s, OP_Z, SC_BETA, true, false, true);
}

// One CG iteration (Sect. 2.4).  Preconditioned form with B = S S:
//   p = z + beta p; q = A p; alpha = rho / p^T q; u += alpha p; r -= alpha q;
//   z = S S r; beta = r^T z / rho.
template <typename T>
cudaError_t pcg_iter(const Ctx<T>& c, cudaStream_t s) {
  if (c.precond) {
    CE(row<T>(c, s, OP_P_UPD_Z, SC_NONE, false, true, true));
    CE(col<T>(c, s, 0, true));
    CE(row<T>(c, s, OP_Q, SC_ALPHA, true, false, true));
    CE(row<T>(c, s, OP_R_UPD, SC_RCHECK, false, true, true));
    CE(col<T>(c, s, 1, true));
    CE(row<T>(c, s, OP_MASK, SC_NONE, true, true, true));
    CE(col<T>(c, s, 1, true));
    return row<T>(c, s, OP_Z, SC_BETA, true, false, true);
  }
  CE(row<T>(c, s, OP_P_UPD_R, SC_NONE, false, true, true));
  CE(col<T>(c, s, 0, true));
  CE(row<T>(c, s, OP_Q, SC_ALPHA, true, false, true));
  return vec<T>(c, s, VOP_UPDATE, SC_RCHECK_BETA, true);
}

template <typename T>
cudaError_t draw_and_rhs(fill_plan* p, cudaStream_t s, bool plain_cg, bool ml = false) {
  if (!ml) return draw_and_rhs<T>(ctx<T>(p), s, plain_cg);
  // maximum-likelihood fill (Sect. 2.1): y = 0, b = -P_x F^-1 (1/P) F (d on U)
  const Ctx<T> c = ctx<T>(p);
  CE(cudaMemsetAsync(prec<T>(p).y, 0, size_t(p->batch) * p->npix * sizeof(T), s));
  CE(row<T>(c, s, OP_LOAD_D_U, SC_NONE, false, true, false));
  CE(col<T>(c, s, 0, false));
  return row<T>(c, s, OP_B, plain_cg ? SC_BB_RHO : SC_BB, true, false, false);
}
template <typename T>
cudaError_t pcg_start(fill_plan* p, cudaStream_t s, int load_sop) {
  return pcg_start<T>(ctx<T>(p), s, load_sop);
}
// Lanes: a plan's CG loops run its batch as nlanes sub-batches of
// consecutive instances, each on its own stream (parallel branches of the
// loop graph when captured).  Every pass computes each instance on its own,
// so the results do not depend on the lanes.
template <typename T>
Ctx<T> lane_ctx(fill_plan* p, int first, int count) {
  Ctx<T> c = ctx<T>(p);
  c.desc += first;
  c.ninst = count;
  return c;
}

// body(first, count, stream) for each lane: on s itself with one lane, else
// on the lane streams forked from s and joined back to it.
template <typename F>
cudaError_t on_lanes(fill_plan* p, cudaStream_t s, bool capturing, F body) {
  if (p->nlanes <= 1) return body(0, p->batch, s);
  const cudaEvent_t fork = capturing ? p->lane_fork_cap : p->lane_fork;
  CE(cudaEventRecord(fork, s));
  const int per = (p->batch + p->nlanes - 1) / p->nlanes;
  for (int l = 0; l < p->nlanes; ++l) {
    const int first = l * per, count = std::min(per, p->batch - first);
    if (count <= 0) break;
    CE(cudaStreamWaitEvent(p->lane_s[l], fork, 0));
    CE(body(first, count, p->lane_s[l]));
    CE(cudaEventRecord(p->lane_join[l], p->lane_s[l]));
    CE(cudaStreamWaitEvent(s, p->lane_join[l], 0));
  }
  return cudaSuccess;
}

// Lanes that hold instances (the IF nodes of a mixed loop body).
int active_lanes(const fill_plan* p) {
  const int per = (p->batch + p->nlanes - 1) / p->nlanes;
  return (p->batch + per - 1) / per;
}

template <typename T>
cudaError_t pcg_iter(fill_plan* p, cudaStream_t s, bool capturing = false) {
  return on_lanes(p, s, capturing, [&](int first, int count, cudaStream_t ls) {
    return pcg_iter<T>(lane_ctx<T>(p, first, count), ls);
  });
}

// ----------------------------------------------------------------- device-side CG loop
// A CG loop is one graph launch: a reset node, then a conditional WHILE node
// whose body is one iteration followed by k_loop_ctl, which keeps the loop
// going while any instance is not done -- and stops it after `limit` bodies
// whatever the states say, so the loop always ends.
// counter[0]: loop bodies run; counter[1]: IF bodies run (update passes).
__global__ void k_loop_reset(int* counter) {
  counter[0] = 0;
  counter[1] = 0;
}

__global__ void k_loop_ctl(cudaGraphConditionalHandle h, CgState* const* sts, int n, int* counter,
                           int limit) {
  __shared__ int running;
  if (threadIdx.x == 0) running = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (!*(volatile int*)&sts[i]->done) running = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int c = ++*counter;
    cudaGraphSetConditional(h, (running && c < limit) ? 1u : 0u);
  }
}

template <typename Body>
fill_status build_loop_graph(cudaStream_t cap, Body body, CgState* const* sts, int n,
                             int* counter, int limit, long long* launches,
                             cudaGraphExec_t* exec_out, long long* body_kernels) {
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  auto fail = [&](cudaError_t e, const char* where) {
    cudaGraphDestroy(g);
    return cuda_fail(e, where);
  };
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return fail(e, "cudaGraphConditionalHandleCreate");
  cudaKernelNodeParams kp{};
  void* args[] = {&counter};
  kp.func = reinterpret_cast<void*>(k_loop_reset);
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(1);
  kp.kernelParams = args;
  cudaGraphNode_t reset;
  e = cudaGraphAddKernelNode(&reset, g, nullptr, 0, &kp);
  if (e != cudaSuccess) return fail(e, "cudaGraphAddKernelNode");
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  e = cudaGraphAddNode(&wnode, g, &reset, nullptr, 1, &cp);
  if (e != cudaSuccess) return fail(e, "cudaGraphAddNode(while)");
  cudaGraph_t bg = cp.conditional.phGraph_out[0];
  const long long before = *launches;
  e = cudaStreamBeginCaptureToGraph(cap, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(e, "cudaStreamBeginCaptureToGraph");
  e = body(cap);
  if (e == cudaSuccess) {
    k_loop_ctl<<<1, 256, 0, cap>>>(h, sts, n, counter, limit);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaStreamEndCapture(cap, &bg);
  *body_kernels = *launches - before + 1;
  *launches = before;
  if (e != cudaSuccess) return fail(e, "capture loop body");
  if (e2 != cudaSuccess) return fail(e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(exec_out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(loop)");
  return FILL_OK;
}

// Launches a loop graph on the plan's stream and accounts for its kernels
// (if_kernels of each body run only when its IF node fires).
fill_status run_loop_graph(fill_plan* p, cudaGraphExec_t exec, long long body_kernels,
                           long long if_kernels = 0, int n_if = 1) {
  CK(cudaGraphLaunch(exec, p->s));
  CK(cudaMemcpyAsync(p->hloop, p->loop_counter, 2 * sizeof(int), cudaMemcpyDeviceToHost, p->s));
  CK(cudaStreamSynchronize(p->s));
  p->launches += 1 + (long long)p->hloop[0] * (body_kernels - n_if * if_kernels) +
                 (long long)p->hloop[1] * if_kernels;
  return FILL_OK;
}

// Host-driven form of a loop graph (opts.host_loops = 1): the body's kernels
// are launched from the host and the instances' done flags are read back
// every kHostCheck bodies; bodies past the last convergence cost only the
// kernels' early exits.  For profilers that cannot see kernels inside
// conditional graph nodes.
constexpr int kHostCheck = 8;

__global__ void k_any_running(CgState* const* sts, int n, int* flag) {
  __shared__ int running;
  if (threadIdx.x == 0) running = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (!*(volatile int*)&sts[i]->done) running = 1;
  __syncthreads();
  if (threadIdx.x == 0) *flag = running;
}

template <typename Body>
fill_status run_loop_host(cudaStream_t s, Body body, CgState* const* sts, int n, int* dflag,
                          int* hflag, int limit, long long* launches) {
  for (int it = 0; it < limit;) {
    for (int k = 0; k < kHostCheck && it < limit; ++k, ++it) CK(body(s));
    ++*launches;
    k_any_running<<<1, 256, 0, s>>>(sts, n, dflag);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!*hflag) break;
  }
  return FILL_OK;
}

template <typename T>
fill_status build_iter_graph(fill_plan* p) {
  Precision<T>& P = prec<T>(p);
  if (P.iter_graph) return FILL_OK;
  return build_loop_graph(
      p->cap, [&](cudaStream_t s) { return pcg_iter<T>(p, s, true); }, P.stp, p->batch,
      p->loop_counter, p->o.max_iter + 4, &p->launches, &P.iter_graph, &P.iter_graph_kernels);
}

// Runs CG iterations until every instance's state is done: one launch of the
// plan's loop graph.
template <typename T>
fill_status run_pcg(fill_plan* p) {
  Precision<T>& P = prec<T>(p);
  if (p->o.host_loops)
    return run_loop_host(
        p->s, [&](cudaStream_t s) { return pcg_iter<T>(p, s); }, P.stp, p->batch,
        p->loop_counter, p->hloop, p->o.max_iter + 4, &p->launches);
  fill_status fs = build_iter_graph<T>(p);
  if (fs != FILL_OK) return fs;
  return run_loop_graph(p, P.iter_graph, P.iter_graph_kernels);
}

// Mixed-precision solve of A u = b: b, r (double-float) and r32 are set and the high-precision
// state holds ||b||^2.  Each step runs an FP32 PCG on A delta = r32 to the
// tolerance the outer target still needs, then u += delta and the true
// residual r = b - A u in double-float (iterative refinement).
fill_status mixed_refine(fill_plan* p, double tol) {
  const int B = p->batch;
  const int nb = (B + 127) / 128;
  for (int outer = 0; outer < p->o.max_refine; ++outer) {
    ++p->launches;
    k_inner_reset<<<nb, 128, 0, p->s>>>(p->f.desc, p->h.desc, B, tol, p->o.inner_tol, p->o.max_iter);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(p->f.u, 0, B * p->nv * sizeof(float), p->s));
    CK(cudaMemsetAsync(p->f.p, 0, B * p->nv * sizeof(float), p->s));
    CK(pcg_start<float>(p, p->s, SC_BB));
    fill_status fs = run_pcg<float>(p);
    if (fs != FILL_OK) return fs;
    CK(row<df>(p, p->s, OP_U64_UPD, SC_NONE, false, true, true));
    CK(col<df>(p, p->s, 0, true));
    CK(row<df>(p, p->s, OP_RES, SC_RES, true, false, true));
    CK(cudaMemcpyAsync(p->h.hst, p->h.st, sizeof(CgState) * B, cudaMemcpyDeviceToHost, p->s));
    CK(cudaStreamSynchronize(p->s));
    bool all = true;
    for (int i = 0; i < B; ++i) all = all && p->h.hst[i].done;
    if (all) break;
  }
  ++p->launches;
  k_inner_collect<<<nb, 128, 0, p->s>>>(p->f.desc, p->h.desc, B);
  CK(cudaGetLastError());
  return FILL_OK;
}

// Links the FP32 and high-precision states of each instance and sets the reliable-update
// threshold on the FP32 state.
__global__ void k_link_states(const InstDesc<float>* lo, const InstDesc<df>* hi, int n,
                              double delta2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  CgState* a = lo[i].st;
  CgState* g = hi[i].st;
  a->peer = g;
  g->peer = a;
  a->delta2 = delta2;
  a->tol2 = g->tol2;
}

// Sets an IF condition to 1 iff some instance's state has an update due.
__global__ void k_if_any_upd(cudaGraphConditionalHandle h, CgState* const* sts, int n,
                             int* counter) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (*(volatile int*)&sts[i]->upd) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (any) counter[1] += 1;
    cudaGraphSetConditional(h, any ? 1u : 0u);
  }
}

// Inside a stream capture on s: adds an IF node (on handle h of the captured
// graph) whose body is body(s2), captured on stream s2; capture on s resumes
// after the node.
template <typename Body>
cudaError_t capture_if(cudaStream_t s, cudaStream_t s2, cudaGraphConditionalHandle h, Body body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  CE(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, &ed, &nd));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CE(cudaGraphAddNode(&node, g, deps, ed, nd, &cp));
  CE(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t bg = cp.conditional.phGraph_out[0];
  CE(cudaStreamBeginCaptureToGraph(s2, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = body(s2);
  cudaError_t e2 = cudaStreamEndCapture(s2, &bg);
  return e != cudaSuccess ? e : e2;
}

// One iteration of the mixed reliable-update PCG: an FP32 CG step; if the
// FP32 residual has dropped by update_delta since the last update (or looks
// converged), fold the FP32 correction into the double-float solution, recompute
// the true residual r = b - A u in double-float, restart the FP32 residual from it and
// keep the search direction; then the preconditioned residual.  The update
// passes skip every instance without a pending update.
// The update passes sit in an IF node that runs only when some instance of
// the contexts has an update due (kernels inside still skip the instances
// without one).  The contexts lo (FP32) and hi (double-float) cover the same
// instances: a plan's batch, or a size class of a group.

// What a mixed loop body needs beyond its two launch contexts.
struct MixedLoop {
  CgState* const* st_hi;   // device: the high-precision state of every instance
  int n;
  int* counter;            // device loop counters ([1]: IF bodies run)
  cudaStream_t cap2;       // stream that captures the IF bodies
  bool host_loops;
  long long* if_kernels;   // kernels inside one IF body
};

cudaError_t mixed_update_passes(const Ctx<float>& lo, const Ctx<df>& hi, cudaStream_t s,
                                bool reload) {
  CE(row<df>(hi, s, OP_U64_UPD, SC_NONE, false, true, SKIP_UNLESS_UPD));
  CE(col<df>(hi, s, 0, SKIP_UNLESS_UPD));
  CE(row<df>(hi, s, OP_RES, SC_RES_UPD, true, false, SKIP_UNLESS_UPD));
  if (!reload) return cudaSuccess;
  return row<float>(lo, s, OP_LOAD_R, SC_CLEAR_UPD, false, true, SKIP_UNLESS_UPD);
}

cudaError_t update_if(const Ctx<float>& lo, const Ctx<df>& hi, cudaStream_t s, bool reload,
                      const MixedLoop& m) {
  // no graph: the update passes run every iteration and skip the instances
  // without an update due
  if (m.host_loops) return mixed_update_passes(lo, hi, s, reload);
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  CE(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr));
  cudaGraphConditionalHandle h;
  CE(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
  ++*lo.launches;
  k_if_any_upd<<<1, 256, 0, s>>>(h, m.st_hi, m.n, m.counter);
  CE(cudaGetLastError());
  const long long before = *lo.launches;
  cudaError_t e = capture_if(s, m.cap2, h, [&](cudaStream_t s2) -> cudaError_t {
    return mixed_update_passes(lo, hi, s2, reload);
  });
  *m.if_kernels = *lo.launches - before;
  return e;
}

cudaError_t mixed_iter(const Ctx<float>& lo, const Ctx<df>& hi, cudaStream_t s,
                       const MixedLoop& m) {
  if (!lo.precond) {
    CE(row<float>(lo, s, OP_P_UPD_R, SC_NONE, false, true, SKIP_DONE));
    CE(col<float>(lo, s, 0, SKIP_DONE));
    CE(row<float>(lo, s, OP_Q, SC_ALPHA, true, false, SKIP_DONE));
    CE(vec<float>(lo, s, VOP_UPDATE, SC_RCHECK_UPD, SKIP_DONE));
    CE(update_if(lo, hi, s, false, m));
    // plain CG: z = r, so beta = r^T r / rho (the reload pass also reduces ||r||^2)
    return row<float>(lo, s, OP_LOAD_R, SC_BETA, false, true, SKIP_DONE);
  }
  CE(row<float>(lo, s, OP_P_UPD_Z, SC_NONE, false, true, SKIP_DONE));
  CE(col<float>(lo, s, 0, SKIP_DONE));
  CE(row<float>(lo, s, OP_Q, SC_ALPHA, true, false, SKIP_DONE));
  CE(row<float>(lo, s, OP_R_UPD, SC_RCHECK_UPD, false, true, SKIP_DONE));
  CE(update_if(lo, hi, s, true, m));
  CE(col<float>(lo, s, 1, SKIP_DONE));
  CE(row<float>(lo, s, OP_MASK, SC_NONE, true, true, SKIP_DONE));
  CE(col<float>(lo, s, 1, SKIP_DONE));
  return row<float>(lo, s, OP_Z, SC_BETA, true, false, SKIP_DONE);
}

// Before a mixed loop (b, r and r32 set, the high-precision states holding
// ||b||^2, u = 0 in double-float): link the two precisions' states, set the
// reliable-update threshold, mirror the instances already done (b = 0) into
// the FP32 states, and start the FP32 PCG from r32.
cudaError_t mixed_start(const Ctx<float>& lo, const Ctx<df>& hi, cudaStream_t s, double tol,
                        double delta, int max_iter) {
  const int nb = (lo.ninst + 127) / 128;
  ++*lo.launches;
  k_link_states<<<nb, 128, 0, s>>>(lo.desc, hi.desc, lo.ninst, delta * delta);
  CE(cudaGetLastError());
  CE(vec<float>(lo, s, VOP_ZERO_UP, SC_NONE, false));
  ++*lo.launches;
  k_inner_reset<<<nb, 128, 0, s>>>(lo.desc, hi.desc, lo.ninst, tol, 0.0, max_iter);
  CE(cudaGetLastError());
  ++*lo.launches;
  k_link_states<<<nb, 128, 0, s>>>(lo.desc, hi.desc, lo.ninst, delta * delta);
  CE(cudaGetLastError());
  return pcg_start<float>(lo, s, SC_BB);
}

// After a mixed loop: fold anything left (breakdown / limits), report the
// true residual, and add the FP32 iterations to the high-precision counts.
cudaError_t mixed_finish(const Ctx<float>& lo, const Ctx<df>& hi, cudaStream_t s) {
  CE(row<df>(hi, s, OP_U64_UPD, SC_NONE, false, true, SKIP_DONE));
  CE(col<df>(hi, s, 0, SKIP_DONE));
  CE(row<df>(hi, s, OP_RES, SC_RES, true, false, SKIP_DONE));
  ++*lo.launches;
  k_inner_collect<<<(lo.ninst + 127) / 128, 128, 0, s>>>(lo.desc, hi.desc, lo.ninst);
  return cudaGetLastError();
}

cudaError_t mixed_iter(fill_plan* p, cudaStream_t s, bool capturing) {
  return on_lanes(p, s, capturing, [&](int first, int count, cudaStream_t ls) {
    const MixedLoop m{p->h.stp + first, count, p->loop_counter, p->cap2, p->o.host_loops != 0,
                      &p->if_kernels};
    return mixed_iter(lane_ctx<float>(p, first, count), lane_ctx<df>(p, first, count), ls, m);
  });
}

fill_status build_mixed_graph(fill_plan* p) {
  if (p->mixed_graph) return FILL_OK;
  return build_loop_graph(
      p->cap, [&](cudaStream_t s) { return mixed_iter(p, s, true); }, p->f.stp, p->batch,
      p->loop_counter, p->o.max_iter + 4, &p->launches, &p->mixed_graph, &p->mixed_graph_kernels);
}

// Mixed-precision solve with reliable updates (b, r, r32 and the high-precision state
// with ||b||^2 are set; u64 = 0).
fill_status mixed_reliable(fill_plan* p, double tol) {
  CK(mixed_start(ctx<float>(p), ctx<df>(p), p->s, tol, p->o.update_delta, p->o.max_iter));
  fill_status fs;
  if (p->o.host_loops) {
    fs = run_loop_host(
        p->s, [&](cudaStream_t s) { return mixed_iter(p, s, false); }, p->f.stp, p->batch,
        p->loop_counter, p->hloop, p->o.max_iter + 4, &p->launches);
  } else {
    fs = build_mixed_graph(p);
    if (fs != FILL_OK) return fs;
    fs = run_loop_graph(p, p->mixed_graph, p->mixed_graph_kernels, p->if_kernels,
                        active_lanes(p));
  }
  if (fs != FILL_OK) return fs;
  CK(mixed_finish(ctx<float>(p), ctx<df>(p), p->s));
  return FILL_OK;
}

fill_status mixed_solve(fill_plan* p, double tol) {
  return p->o.update_delta > 0.0 ? mixed_reliable(p, tol) : mixed_refine(p, tol);
}

// Sums the band partials of every CTA in order: out[i][b] (+)= sum_c part[i][c][b].
__global__ void k_band_sum(const double* part, int ninst, int nctas, int nbands, double* out,
                           int accumulate) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ninst * nbands) return;
  const int i = t / nbands, b = t % nbands;
  double s = 0.0;
  for (int c = 0; c < nctas; ++c) s += part[((long long)i * nctas + c) * nbands + b];
  out[t] = accumulate ? out[t] + s : s;
}

template <typename T>
cudaError_t init_states(fill_plan* p, double tol);
template <typename T>
void fill_desc(fill_plan* p, const void* d, long long d_stride, const uint64_t* seeds, void* out,
               const void* gx);
template <typename T>
cudaError_t upload_desc(fill_plan* p);

template <typename T>
cudaError_t band_term(fill_plan* p, int src1, int src2, const T* coef, bool accumulate) {
  Precision<T>& P = prec<T>(p);
  CE(row<T>(p, p->s, src1, SC_NONE, false, true, false, -1, 0));
  CE(row<T>(p, p->s, src2, SC_NONE, false, true, false, -1, 1));
  CE(col<T>(p, p->s, -1, false, -1, 0));
  CE(col<T>(p, p->s, -1, false, -1, 1));
  DotArgs a{(long long)(p->nx / 2 + 1) * p->ny, P.nbands, P.band, coef, P.bpart};
  ++p->launches;
  CE(Launch<T>::band_dot(P.desc, p->batch, a, p->s));
  const int tot = p->batch * P.nbands;
  ++p->launches;
  k_band_sum<<<(tot + 127) / 128, 128, 0, p->s>>>(P.bpart, p->batch, kDotCtas, P.nbands, P.bsum,
                                                 accumulate ? 1 : 0);
  return cudaGetLastError();
}

// Adjoint gradients (differentiation of the realization; the paper is silent):
// with g = dL/dx, lam = A^-1 g_M (same operator and preconditioner),
// dL/dd = g_U - (C^-1 lam)_U on U (0 on M), h = dL/dy = g on M, (C^-1 lam)_U
// on U, and for P = sum_b a_b T_b + N, T_b = 1[k in b] S(k):
//   dL/da_b = sum_k T_b [ Re(conj(F h) F xi) / (2 n sqrt P) + Re(conj(F lam) F w) / (n P^2) ]
// with w = d - y on U and u on M, xi the seed's white noise.
template <typename T>
fill_status backward_t(fill_plan* p, const void* d, long long d_stride, const void* gx,
                       double tol, void* grad_d, double* grad_bands) {
  Precision<T>& P = prec<T>(p);
  const int B = p->batch;
  fill_desc<T>(p, d, d_stride, nullptr, grad_d, gx);
  CK(upload_desc<T>(p));
  CK(vec<T>(p, p->s, VOP_MAKE_W, SC_NONE, false));
  const bool mixed = p->o.mode == FILL_MODE_MIXED;
  CK(init_states<T>(p, tol));
  CK(cudaMemsetAsync(P.u, 0, B * p->nv * sizeof(T), p->s));
  if (mixed) {
    fill_desc<float>(p, nullptr, 0, nullptr, nullptr, nullptr);
    CK(upload_desc<float>(p));
    CK(init_states<float>(p, p->o.inner_tol));
    CK(vec<T>(p, p->s, VOP_LOAD_G, SC_BB, false));
    fill_status fs = mixed_solve(p, tol);
    if (fs != FILL_OK) return fs;
  } else {
    CK(cudaMemsetAsync(P.p, 0, B * p->nv * sizeof(T), p->s));
    CK(vec<T>(p, p->s, VOP_LOAD_G, p->o.precond ? SC_BB : SC_BB_RHO, false));
    CK(pcg_start<T>(p, p->s, SC_NONE));
    fill_status fs = run_pcg<T>(p);
    if (fs != FILL_OK) return fs;
  }
  // lam is in u.  C^-1 lam -> dL/dd and h (into y).
  CK(row<T>(p, p->s, OP_LOAD_U, SC_NONE, false, true, false));
  CK(col<T>(p, p->s, 0, false));
  CK(row<T>(p, p->s, OP_GRAD, SC_NONE, true, false, false));
  if (grad_bands) {
    CK(band_term<T>(p, OP_XI, OP_LOAD_Y, P.coef1, false));
    CK(band_term<T>(p, OP_LOAD_U, OP_LOAD_W, P.coef2, true));
    CK(cudaMemcpyAsync(grad_bands, P.bsum, sizeof(double) * B * P.nbands,
                       cudaMemcpyDeviceToHost, p->s));
  }
  return FILL_OK;
}

template <typename T>
void fill_desc(fill_plan* p, const void* d, long long d_stride, const uint64_t* seeds, void* out,
               const void* gx) {
  Precision<T>& P = prec<T>(p);
  for (int i = 0; i < p->batch; ++i) {
    InstDesc<T>& D = P.hdesc[i];
    const size_t off = size_t(i) * p->npix;
    using M = typename MapOf<T>::type;
    D.d = d ? reinterpret_cast<const M*>(d) + size_t(d_stride) * i : nullptr;
    D.out = out ? reinterpret_cast<M*>(out) + off : nullptr;
    D.gx = gx ? reinterpret_cast<const M*>(gx) + off : nullptr;
    if (seeds) D.seed = (unsigned long long)seeds[i];
  }
}

template <typename T>
cudaError_t upload_desc(fill_plan* p) {
  Precision<T>& P = prec<T>(p);
  return cudaMemcpyAsync(P.desc, P.hdesc, sizeof(InstDesc<T>) * p->batch, cudaMemcpyHostToDevice,
                         p->s);
}

// W_n^t = exp(-2 pi i t / n), t < count, from angles reduced to [0, pi/4]
// (octant symmetry), so every entry carries the FP64 cos / sin accuracy.
void twiddles_len(int n, int count, std::vector<double>& w) {
  w.resize(2 * size_t(count));
  for (int t = 0; t < count; ++t) {
    // 8 t / n = o + f: angle 2 pi t / n = (pi/4) (o + f)
    const long long m = (long long)8 * (t % n);
    const int o = (int)(m / n);
    const double f = double(m % n) / double(n);
    double c, sn;   // cos, sin of the angle
    const double th = (o & 1) ? (1.0 - f) * M_PI / 4.0 : f * M_PI / 4.0;
    const double c0 = std::cos(th), s0 = std::sin(th);
    switch (o) {
      case 0: c = c0; sn = s0; break;
      case 1: c = s0; sn = c0; break;
      case 2: c = -s0; sn = c0; break;
      case 3: c = -c0; sn = s0; break;
      case 4: c = -c0; sn = -s0; break;
      case 5: c = -s0; sn = -c0; break;
      case 6: c = s0; sn = -c0; break;
      default: c = c0; sn = -s0; break;
    }
    w[2 * size_t(t)] = c;
    w[2 * size_t(t) + 1] = -sn;
  }
}

// The table of a factored mixed-radix length (complex entries, interleaved,
// FP64: the stage twiddles in the layout of GenLen::twoff; at least one entry)
// and its digit-reversal maps.
void gen_tables(const GenLen& g, std::vector<double>& tw, std::vector<unsigned short>& rev,
                std::vector<unsigned short>& pos) {
  const int n = g.n, S = g.nst;
  std::vector<double> w;   // W_n^t, t < n
  twiddles_len(n, n, w);
  tw.clear();
  auto push = [&](const std::vector<double>& src, int t) {
    tw.push_back(src[2 * size_t(t)]);
    tw.push_back(src[2 * size_t(t) + 1]);
  };
  // W_ns^{q j} = W_n^{q j (n / ns)}
  int ns = n;
  for (int s = 0; s < S - 1; ++s) {
    const int R = g.radix[s], h = ns / R, step = n / ns;
    for (int j = 0; j < h; ++j)
      for (int q = 1; q < R; ++q) push(w, (int)(((long long)q * j * step) % n));
    ns = h;
  }
  // position p = sum_s q_s h_s holds frequency k = sum_s q_s R_0 ... R_{s-1}
  rev.assign(n, 0);
  pos.assign(n, 0);
  for (int p = 0; p < n; ++p) {
    int rem = p, k = 0, wgt = 1, nss = n;
    for (int s = 0; s < S; ++s) {
      const int h = nss / g.radix[s], q = rem / h;
      rem -= q * h;
      k += q * wgt;
      wgt *= g.radix[s];
      nss = h;
    }
    rev[p] = (unsigned short)k;
    pos[k] = (unsigned short)p;
  }
}

// Threads per group of V mixed-radix transforms (a multiple of 32, at most
// 512).  A stage of radix R has n/R butterflies, shared round-robin by the
// group's threads; the last round leaves threads idle.  Among the
// candidates, take the one with the best product of stage efficiency
// (butterflies / thread slots over all stages) and SM occupancy (groups
// resident per SM by shared memory -- V n complex values each -- times
// threads, against the threads an SM runs at the kernels' register counts:
// kGenThreads x gen_minb).
void gen_threads(GenLen* g, int V, bool wide) {
  const double tmax = double(kGenThreads) * (wide ? gen_minb<double>() : gen_minb<float>());
  const size_t bytes = size_t(V) * g->n * (wide ? 16 : 8);
  const size_t per_sm = std::max<size_t>(1, size_t(225) * 1024 / bytes);
  double best = -1.0;
  for (int nt = 32; nt <= kGenThreads; nt += 32) {
    long long slots_used = 0, work = 0;
    for (int s = 0; s < g->nst; ++s) {
      const int nb = g->n / g->radix[s];
      work += nb;
      slots_used += (long long)((nb + nt - 1) / nt) * nt;
    }
    const double eff = double(work) / double(slots_used);
    const double resident = std::min<double>(double(per_sm), std::floor(tmax / nt));
    const double score = eff * std::min(1.0, resident * nt / tmax);
    if (score > best + 1e-9 || (score > best - 1e-9 && nt > g->nt)) {
      best = std::max(best, score);
      g->nt = nt;
    }
  }
}

// Whether precision T carries the plan's CG loop (FP64 in FP64 mode, FP32
// otherwise): the schedule options rows_per_cta / ffts_per_cta set its CTA
// shapes; the double-float passes of the mixed mode keep their defaults.
template <typename T>
bool loop_precision(const fill_plan* p) {
  return p->o.mode == FILL_MODE_FP64 ? std::is_same<T, double>::value
                                     : std::is_same<T, float>::value;
}

// Validity of a mixed-radix CTA shape for precision T: rows per CTA and
// column FFTs per CTA are multiples of the group width V = gen_v<T>(), the
// row groups a power of two, within kGenThreads threads, the partial-sum slots
// and 200 KB of shared memory.
template <typename T>
bool gen_row_ok(const fill_plan* p, int r) {
  constexpr int V = gen_vrow<T>();
  return r >= V && r % V == 0 && pow2(r / V) && (r / V) * p->grow.nt <= GenLaunch<T>::max_threads() &&
         (p->ny + r - 1) / r <= kMaxPartials && GenLaunch<T>::row_smem(p->nx / 2, r) <= 200 * 1024;
}
template <typename T>
bool gen_col_ok(const fill_plan* p, int f) {
  constexpr int V = gen_v<T>();
  return f >= V && f % V == 0 && (f / V) * p->gcol.nt <= GenLaunch<T>::max_threads() &&
         GenLaunch<T>::col_smem(p->ny, f) <= 200 * 1024;
}

// Twiddle tables of precision T for the plan's current radix schedules, in
// fresh device buffers (launch graphs captured earlier keep the buffers they
// were built with).
template <typename T>
fill_status gen_upload(fill_plan* p) {
  Precision<T>& P = prec<T>(p);
  const int L = p->nx / 2;
  std::vector<double> wl, wx, wn;
  std::vector<unsigned short> rev, pos;
  gen_tables(p->grow, wl, rev, pos);
  twiddles_len(p->nx, L + 1, wx);
  gen_tables(p->gcol, wn, rev, pos);
  auto upload = [&](T** dst, const std::vector<double>& src) -> cudaError_t {
    std::vector<T> h(std::max<size_t>(src.size(), 2));
    for (size_t i = 0; i < src.size(); ++i) h[i] = (T)src[i];
    cudaError_t e = p->dalloc(dst, h.size());
    if (e == cudaSuccess) e = cudaMemcpy(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
  };
  CK(upload(&P.gwl, wl));
  CK(upload(&P.gwx, wx));
  CK(upload(&P.gwn, wn));
  return FILL_OK;
}

// Digit-reversal maps of the current radix schedules (fresh device buffers).
fill_status gen_upload_maps(fill_plan* p) {
  auto upload_map = [&](const unsigned short** dst, const std::vector<unsigned short>& src) {
    unsigned short* d = nullptr;
    cudaError_t e = p->dalloc(&d, src.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(d, src.data(), src.size() * sizeof(unsigned short), cudaMemcpyHostToDevice);
    *dst = d;
    return e;
  };
  std::vector<double> tw;
  std::vector<unsigned short> rev, pos;
  gen_tables(p->grow, tw, rev, pos);
  CK(upload_map(&p->grow.rev, rev));
  CK(upload_map(&p->grow.pos, pos));
  gen_tables(p->gcol, tw, rev, pos);
  CK(upload_map(&p->gcol.rev, rev));
  CK(upload_map(&p->gcol.pos, pos));
  return FILL_OK;
}

// Mixed-radix schedule and twiddle tables of one precision: rows per CTA
// and column FFTs per CTA (one or two groups of g.nt threads, within 75 KB of
// shared memory so that three CTAs share an SM), unless the options fix them;
// the digit-reversal maps once per plan.
template <typename T>
fill_status setup_generic(fill_plan* p) {
  Precision<T>& P = prec<T>(p);
  constexpr int V = gen_v<T>(), VR = gen_vrow<T>();
  const size_t third = 75 * 1024;
  const bool user = loop_precision<T>(p);
  if (user && p->o.rows_per_cta > 0) {
    P.rows = p->o.rows_per_cta;
  } else {
    P.rows = VR;
    if (gen_row_ok<T>(p, 2 * VR) && GenLaunch<T>::row_smem(p->nx / 2, 2 * VR) <= third)
      P.rows = 2 * VR;
  }
  if (user && p->o.ffts_per_cta > 0) {
    P.ffts = p->o.ffts_per_cta;
  } else {
    P.ffts = V;
    while (gen_col_ok<T>(p, 2 * P.ffts) && GenLaunch<T>::col_smem(p->ny, 2 * P.ffts) <= third &&
           2 * P.ffts <= 16)
      P.ffts *= 2;
  }
  if (!gen_row_ok<T>(p, P.rows) || !gen_col_ok<T>(p, P.ffts)) return FILL_EINVAL;
  fill_status fs = gen_upload<T>(p);
  if (fs != FILL_OK) return fs;
  if (!p->grow.rev) {
    fs = gen_upload_maps(p);
    if (fs != FILL_OK) return fs;
  }
  CK(GenLaunch<T>::prepare());
  return FILL_OK;
}

// P must be finite, > 0, and real-symmetric on the two self-conjugate columns
// kx = 0 and kx = nx/2, so that C is a real symmetric operator (Sect. 4).
bool spectrum_valid(int ny, int nx, const double* P_half) {
  const int nkx = nx / 2 + 1;
  for (long long i = 0; i < (long long)ny * nkx; ++i)
    if (!(std::isfinite(P_half[i]) && P_half[i] > 0.0)) return false;
  for (int col : {0, nx / 2})
    for (int my = 0; my < ny; ++my) {
      const double a = P_half[(size_t)my * nkx + col], b = P_half[(size_t)((ny - my) % ny) * nkx + col];
      if (std::fabs(a - b) > 1e-12 * std::fabs(a)) return false;
    }
  return true;
}

// Spectral tables [kx][ky] with the inverse DFT's 1/n folded in: 1/(nP) for
// C^-1 and sqrt(P)/n for C^{1/2} (Sects. 2.1, 2.3, 2.4); *relax_a = max 1/P,
// the white level of C^-1 used by the relaxation of Sect. 5.
void spectral_tables(int ny, int nx, const double* P_half, std::vector<double>& tinv,
                     std::vector<double>& tsqrt, double* relax_a) {
  const int nkx = nx / 2 + 1;
  const double n = double(ny) * double(nx);
  tinv.assign((size_t)nkx * ny, 0.0);
  tsqrt.assign((size_t)nkx * ny, 0.0);
  double a = 0.0;
  for (int ky = 0; ky < ny; ++ky)
    for (int kx = 0; kx < nkx; ++kx) {
      const double P = P_half[(size_t)ky * nkx + kx];
      a = std::max(a, 1.0 / P);
      tinv[(size_t)kx * ny + ky] = 1.0 / (P * n);
      tsqrt[(size_t)kx * ny + ky] = std::sqrt(P) / n;
    }
  *relax_a = a;
}

// Copies the tables into a precision's device buffers (synchronous).
template <typename T>
cudaError_t upload_tables(fill_plan* p, const std::vector<double>& tinv,
                          const std::vector<double>& tsqrt) {
  Precision<T>& P = prec<T>(p);
  const size_t ntab = tinv.size();
  std::vector<T> a(ntab), b(ntab);
  for (size_t i = 0; i < ntab; ++i) {
    a[i] = (T)tinv[i];
    b[i] = (T)tsqrt[i];
  }
  CE(cudaMemcpy(P.t_inv, a.data(), ntab * sizeof(T), cudaMemcpyHostToDevice));
  return cudaMemcpy(P.t_sqrt, b.data(), ntab * sizeof(T), cudaMemcpyHostToDevice);
}

template <typename T>
fill_status setup_precision(fill_plan* p, const std::vector<double>& tinv,
                            const std::vector<double>& tsqrt, const std::vector<double>& tw) {
  Precision<T>& P = prec<T>(p);
  P.used = true;
  const size_t B = p->batch, n = p->npix, nv = p->nv;
  const size_t nspec = 2 * size_t(p->nx / 2 + 1) * p->ny;
  T** cvecs[] = {&P.r, &P.p, &P.q, &P.z, &P.u, &P.b};   // compact CG vectors
  for (T** v : cvecs)
    if (p->dalloc(v, B * nv) != cudaSuccess) return FILL_ENOMEM;
  if (p->dalloc(&P.y, B * n) != cudaSuccess || p->dalloc(&P.w, B * n) != cudaSuccess)
    return FILL_ENOMEM;
  if (p->dalloc(&P.spec, B * nspec) != cudaSuccess) return FILL_ENOMEM;
  if (p->o.backward) {
    if (p->dalloc(&P.spec2, B * nspec) != cudaSuccess) return FILL_ENOMEM;
  }
  const size_t ntab = size_t(p->nx / 2 + 1) * p->ny;
  if (p->dalloc(&P.t_inv, ntab) != cudaSuccess || p->dalloc(&P.t_sqrt, ntab) != cudaSuccess ||
      p->dalloc(&P.tw, 2 * size_t(kTwEntries)) != cudaSuccess)
    return FILL_ENOMEM;
  if (p->dalloc(&P.st, B) != cudaSuccess || p->halloc(&P.hst, B) != cudaSuccess ||
      p->dalloc(&P.partial, B * kMaxPartials) != cudaSuccess ||
      p->dalloc(&P.desc, B) != cudaSuccess || p->halloc(&P.hdesc, B) != cudaSuccess)
    return FILL_ENOMEM;
  const int hc = std::max(p->o.history_cap, 1);
  if (p->dalloc(&P.hist, B * hc) != cudaSuccess) return FILL_ENOMEM;
  if (p->o.history_cap > 0 && p->dalloc(&P.coef, 2 * B * hc) != cudaSuccess) return FILL_ENOMEM;
  if (p->dalloc(&P.stp, B) != cudaSuccess) return FILL_ENOMEM;
  {
    std::vector<CgState*> ptrs(B);
    for (size_t i = 0; i < B; ++i) ptrs[i] = P.st + i;
    CK(cudaMemcpy(P.stp, ptrs.data(), B * sizeof(CgState*), cudaMemcpyHostToDevice));
  }
  std::vector<T> w(2 * size_t(kTwEntries));
  for (size_t i = 0; i < w.size(); ++i) w[i] = (T)tw[i];
  CK(upload_tables<T>(p, tinv, tsqrt));
  CK(cudaMemcpy(P.tw, w.data(), w.size() * sizeof(T), cudaMemcpyHostToDevice));
  CK(cudaMemset(P.u, 0, B * nv * sizeof(T)));
  CK(cudaMemset(P.p, 0, B * nv * sizeof(T)));
  if (p->gen) {
    fill_status gs = setup_generic<T>(p);
    if (gs != FILL_OK) return gs;
  } else {
    const bool user = loop_precision<T>(p);
    P.rows = user && p->o.rows_per_cta > 0 ? std::min(p->o.rows_per_cta, p->ny)
                                           : default_rows<T>(p->log_l, p->ny);
    P.ffts = user && p->o.ffts_per_cta > 0 ? p->o.ffts_per_cta
                                           : default_ffts<T>(p->log_n, p->nx / 2 + 1);
    if (!schedule_valid<T>(p->log_l, p->log_n, p->ny, P.rows, P.ffts)) return FILL_EINVAL;
    P.col_variant = std::is_same<T, float>::value ? p->o.col_kernel : 0;
  }
  CK(Launch<T>::prepare());
  for (size_t i = 0; i < B; ++i) {
    InstDesc<T> D{};
    D.mw = p->mw;
    D.nvec = p->nmasked;
    D.t_inv = P.t_inv;
    D.t_sqrt = P.t_sqrt;
    D.spec = P.spec + i * nspec;
    D.spec2 = P.spec2 ? P.spec2 + i * nspec : nullptr;
    D.w = P.w + i * n;
    D.r = P.r + i * nv;
    D.p = P.p + i * nv;
    D.q = P.q + i * nv;
    D.z = P.z + i * nv;
    D.u = P.u + i * nv;
    D.y = P.y + i * n;
    D.b = P.b + i * nv;
    D.st = P.st + i;
    D.partial = P.partial + i * kMaxPartials;
    D.hist = P.hist + i * hc;
    D.coef = P.coef ? P.coef + 2 * i * hc : nullptr;
    P.hdesc[i] = D;
  }
  return FILL_OK;
}

template <typename T>
cudaError_t init_states(fill_plan* p, double tol) {
  Precision<T>& P = prec<T>(p);
  const int hc = std::max(p->o.history_cap, 1);
  ++p->launches;
  k_state_init<T><<<(p->batch + 127) / 128, 128, 0, p->s>>>(P.desc, p->batch, tol * tol,
                                                           p->o.max_iter, hc);
  return cudaGetLastError();
}

// Severity of a per-realization status: invalid data outranks a breakdown,
// which outranks a solve that ran out of iterations.
int severity(int st) {
  switch (st) {
    case FILL_OK: return 0;
    case FILL_ENOTCONV: return 1;
    case FILL_EBREAKDOWN: return 2;
    default: return 3;
  }
}
void note_status(int st, fill_status* worst) {
  if (severity(st) > severity(*worst)) *worst = (fill_status)st;
}

void collect_stats(fill_plan* p, fill_stats* stats, double ms, fill_status* worst) {
  const bool mixed = p->o.mode == FILL_MODE_MIXED;
  for (int i = 0; i < p->batch; ++i) {
    fill_stats st{};
    if (mixed) {
      const CgState& a = p->f.hst[i];
      const CgState& g = p->h.hst[i];
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
    note_status(st.status, worst);
    if (stats) stats[i] = st;
  }
}

// Queues the read-back of the device error flag on the plan's stream (before
// the call's final synchronisation).
cudaError_t queue_err_readback(fill_plan* p) {
  return cudaMemcpyAsync(&p->hloop[2], p->dev_err, sizeof(int), cudaMemcpyDeviceToHost, p->s);
}

// After the final synchronisation: a kernel whose bounded wait gave up set
// the flag; report it once (FILL_ETIMEOUT) and clear it.
fill_status take_err(fill_plan* p) {
  if (!p->hloop[2]) return FILL_OK;
  p->hloop[2] = 0;
  cudaMemsetAsync(p->dev_err, 0, sizeof(int), p->s);
  cudaStreamSynchronize(p->s);
  g_last_error = "a bounded device wait timed out (a kernel gave up waiting for a copy)";
  return FILL_ETIMEOUT;
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
  o->update_delta = 1e-2;
}

fill_status fill_init(fill_plan** out, int ny, int nx, const double* P_half,
                      const uint8_t* observed, const fill_opts* opts, void* stream) {
  if (!out || !P_half || !observed) return FILL_EINVAL;
  *out = nullptr;
  const bool po2 = pow2(nx) && pow2(ny) && nx >= 32 && nx <= 8192 && ny >= 16 && ny <= 8192;
  cgf::GenLen grow{}, gcol{};
  if (!po2) {
    // mixed-radix grid: nx/2 and ny products of 2, 3, 5, 7, at most 4096
    if (nx % 2 != 0 || nx < 16 || ny < 8 || !gen_factor(nx / 2, &grow) || !gen_factor(ny, &gcol))
      return FILL_EINVAL;
    // threads per transform, for the precision that carries the CG loop
    const bool wide = opts && opts->mode == FILL_MODE_FP64;
    gen_threads(&grow, wide ? 1 : gen_vrow<float>(), wide);
    gen_threads(&gcol, wide ? 1 : gen_v<float>(), wide);
  }
  fill_opts o;
  if (opts)
    o = *opts;
  else
    fill_opts_default(&o);
  if (o.mode < 0 || o.mode > 2 || o.batch < 1 || o.batch > 65535 || o.max_iter < 1 ||
      o.max_refine < 1 || o.host_loops < 0 || o.host_loops > 1 || !(o.inner_tol > 0.0) || o.history_cap < 0 || o.rows_per_cta < 0 ||
      o.ffts_per_cta < 0 || o.backward < 0 || o.backward > 1 || !(o.update_delta >= 0.0) ||
      !(o.update_delta < 1.0) || o.col_kernel < 0 || o.col_kernel > 1 || o.lanes < 0 ||
      o.lanes > kMaxLanes)
    return FILL_EINVAL;
  const int nkx = nx / 2 + 1;
  if (!spectrum_valid(ny, nx, P_half)) return FILL_EINVAL;
  const long long npix = (long long)ny * nx;
  long long nmasked = 0;
  std::vector<uint2> words((npix + 31) / 32, make_uint2(0u, 0u));
  for (long long w = 0; w < (long long)words.size(); ++w) {
    words[w].y = (unsigned int)nmasked;   // compact index of the word's first masked pixel
    for (int b = 0; b < 32; ++b) {
      const long long i = w * 32 + b;
      if (i >= npix) break;
      if (observed[i] > 1) return FILL_EINVAL;
      if (observed[i])
        words[w].x |= 1u << b;
      else
        ++nmasked;
    }
  }
  fill_plan* p = new (std::nothrow) fill_plan();
  if (!p) return FILL_ENOMEM;
  p->ny = ny;
  p->nx = nx;
  p->gen = !po2;
  p->grow = grow;
  p->gcol = gcol;
  p->log_l = po2 ? ilog2(nx / 2) : -1;
  p->log_n = po2 ? ilog2(ny) : -1;
  p->batch = o.batch;
  p->npix = npix;
  p->nmasked = nmasked;
  p->nv = std::max<long long>(64, (nmasked + 63) / 64 * 64);
  p->o = o;
  p->s = reinterpret_cast<cudaStream_t>(stream);
  p->P_half.assign(P_half, P_half + (size_t)ny * nkx);
  {
    static std::atomic<unsigned long long> next_serial{1};
    p->serial = next_serial++;
  }
  fill_status fs = FILL_OK;
  auto fail = [&](fill_status st) {
    delete p;
    return st;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap2, cudaStreamNonBlocking);
  p->nlanes = o.lanes > 0 ? std::min(o.lanes, o.batch)
                          : (o.batch >= 2 && npix >= (1LL << 20) ? 2 : 1);
  if (p->nlanes > 1) {
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->lane_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->lane_fork_cap, cudaEventDisableTiming);
    for (int l = 0; l < p->nlanes && e == cudaSuccess; ++l) {
      e = cudaStreamCreateWithFlags(&p->lane_s[l], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->lane_join[l], cudaEventDisableTiming);
    }
  }
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamCreate"));
  if (p->dalloc(&p->mw, words.size()) != cudaSuccess) return fail(FILL_ENOMEM);
  if (p->dalloc(&p->P_dev, (size_t)ny * nkx) != cudaSuccess) return fail(FILL_ENOMEM);
  e = cudaMemcpy(p->P_dev, P_half, (size_t)ny * nkx * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_fail(e, "upload spectrum"));
  if (p->dalloc(&p->loop_counter, 2) != cudaSuccess || p->halloc(&p->hloop, 3) != cudaSuccess ||
      p->dalloc(&p->dev_err, 1) != cudaSuccess)
    return fail(FILL_ENOMEM);
  e = cudaMemset(p->dev_err, 0, sizeof(int));
  if (e != cudaSuccess) return fail(cuda_fail(e, "fill_init"));
  e = cudaMemcpy(p->mw, words.data(), words.size() * sizeof(uint2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_fail(e, "upload mask"));
  std::vector<double> tinv, tsqrt, tw;
  spectral_tables(ny, nx, P_half, tinv, tsqrt, &p->relax_a);
  twiddles_host(tw);
  if (o.mode == FILL_MODE_FP32 || o.mode == FILL_MODE_MIXED) {
    fs = setup_precision<float>(p, tinv, tsqrt, tw);
    if (fs != FILL_OK) return fail(fs);
  }
  if (o.mode == FILL_MODE_FP64) {
    fs = setup_precision<double>(p, tinv, tsqrt, tw);
    if (fs != FILL_OK) return fail(fs);
  }
  if (o.mode == FILL_MODE_MIXED) {
    fs = setup_precision<df>(p, tinv, tsqrt, tw);
    if (fs != FILL_OK) return fail(fs);
    for (int i = 0; i < p->batch; ++i) {
      p->h.hdesc[i].dlt = p->f.hdesc[i].u;
      p->h.hdesc[i].r32 = p->f.hdesc[i].r;
    }
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(cuda_fail(e, "fill_init"));
  *out = p;
  return FILL_OK;
}

}  // extern "C"

namespace {
// fill_realize (ml = false) and fill_ml (ml = true: no random part, y = 0).
fill_status realize_impl(fill_plan* p, const void* d, long long d_stride, const uint64_t* seeds,
                         double tol, void* out, fill_stats* stats, bool ml) {
  if (!p || !d || (!seeds && !ml) || !out || !(tol >= 0.0) || d_stride < 0) return FILL_EINVAL;
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
      fill_desc<float>(p, d, d_stride, seeds, out, nullptr);
      CK(upload_desc<float>(p));
      CK(init_states<float>(p, tol));
      CK(cudaMemsetAsync(p->f.u, 0, B * p->nv * sizeof(float), p->s));
      CK(cudaMemsetAsync(p->f.p, 0, B * p->nv * sizeof(float), p->s));
      CK(draw_and_rhs<float>(p, p->s, !p->o.precond, ml));
      CK(pcg_start<float>(p, p->s, SC_NONE));
      fs = run_pcg<float>(p);
      if (fs != FILL_OK) return fs;
      CK(vec<float>(p, p->s, VOP_ASSEMBLE, SC_NONE, false));
      CK(cudaMemcpyAsync(p->f.hst, p->f.st, sizeof(CgState) * B, cudaMemcpyDeviceToHost, p->s));
    } else {
      fill_desc<double>(p, d, d_stride, seeds, out, nullptr);
      CK(upload_desc<double>(p));
      CK(init_states<double>(p, tol));
      CK(cudaMemsetAsync(p->g.u, 0, B * p->nv * sizeof(double), p->s));
      CK(cudaMemsetAsync(p->g.p, 0, B * p->nv * sizeof(double), p->s));
      CK(draw_and_rhs<double>(p, p->s, !p->o.precond, ml));
      CK(pcg_start<double>(p, p->s, SC_NONE));
      fs = run_pcg<double>(p);
      if (fs != FILL_OK) return fs;
      CK(vec<double>(p, p->s, VOP_ASSEMBLE, SC_NONE, false));
      CK(cudaMemcpyAsync(p->g.hst, p->g.st, sizeof(CgState) * B, cudaMemcpyDeviceToHost, p->s));
    }
  } else {
    // Mixed: double-float draw / RHS / residuals, FP32 PCG with residual updates.
    fill_desc<df>(p, d, d_stride, seeds, out, nullptr);
    fill_desc<float>(p, nullptr, 0, seeds, nullptr, nullptr);
    CK(upload_desc<df>(p));
    CK(upload_desc<float>(p));
    CK(init_states<df>(p, tol));
    CK(init_states<float>(p, p->o.inner_tol));
    CK(cudaMemsetAsync(p->h.u, 0, B * p->nv * sizeof(df), p->s));
    CK(draw_and_rhs<df>(p, p->s, false, ml));
    fs = mixed_solve(p, tol);
    if (fs != FILL_OK) return fs;
    CK(vec<df>(p, p->s, VOP_ASSEMBLE, SC_NONE, false));
    CK(cudaMemcpyAsync(p->h.hst, p->h.st, sizeof(CgState) * B, cudaMemcpyDeviceToHost, p->s));
    CK(cudaMemcpyAsync(p->f.hst, p->f.st, sizeof(CgState) * B, cudaMemcpyDeviceToHost, p->s));
  }
  CK(queue_err_readback(p));
  CK(cudaStreamSynchronize(p->s));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  collect_stats(p, stats, ms, &worst);
  const fill_status te = take_err(p);
  return te != FILL_OK ? te : worst;
}
}  // namespace

extern "C" {

fill_status fill_realize(fill_plan* p, const void* d, long long d_stride, const uint64_t* seeds,
                         double tol, void* out, fill_stats* stats) {
  return realize_impl(p, d, d_stride, seeds, tol, out, stats, false);
}

fill_status fill_ml(fill_plan* p, const void* d, long long d_stride, double tol, void* out,
                    fill_stats* stats) {
  return realize_impl(p, d, d_stride, nullptr, tol, out, stats, true);
}

}  // extern "C"

namespace {
__global__ void k_set_step(CgState* const* sts, int n, double step) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) sts[i]->alpha = step;
}

// Kernel relaxation (Sect. 5, eq. Algo): w_M <- (K * w)_M = w_M - (C^-1 w)_M / a,
// three passes per sweep, from w = d on U, 0 on M.
template <typename T>
fill_status relax_t(fill_plan* p, const void* d, long long d_stride, int iters, void* out,
                    fill_stats* stats) {
  Precision<T>& P = prec<T>(p);
  const auto t0 = std::chrono::steady_clock::now();
  const int B = p->batch;
  p->launches = 0;
  fill_desc<T>(p, d, d_stride, nullptr, out, nullptr);
  CK(upload_desc<T>(p));
  CK(init_states<T>(p, 0.0));
  ++p->launches;
  k_set_step<<<(B + 127) / 128, 128, 0, p->s>>>(P.stp, B, 1.0 / p->relax_a);
  CK(cudaGetLastError());
  CK(vec<T>(p, p->s, VOP_W_FROM_D, SC_NONE, SKIP_NEVER));
  for (int k = 0; k < iters; ++k) {
    CK(row<T>(p, p->s, OP_LOAD_W, SC_NONE, false, true, SKIP_NEVER));
    CK(col<T>(p, p->s, 0, SKIP_NEVER));
    CK(row<T>(p, p->s, OP_RELAX, k == 0 ? SC_BB : SC_RES, true, false, SKIP_NEVER));
  }
  CK(vec<T>(p, p->s, VOP_W_TO_OUT, SC_NONE, SKIP_NEVER));
  CK(cudaMemcpyAsync(P.hst, P.st, sizeof(CgState) * B, cudaMemcpyDeviceToHost, p->s));
  CK(cudaStreamSynchronize(p->s));
  const double ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats)
    for (int i = 0; i < B; ++i) {
      const CgState& a = P.hst[i];
      fill_stats st{};
      st.iters = iters;
      st.status = a.status == 4 ? FILL_EBREAKDOWN : FILL_OK;
      st.launches = (int)p->launches;
      st.rel_resid = a.bb > 0 ? std::sqrt(a.rr / a.bb) : 0.0;
      st.true_rel_resid = -1.0;
      st.ms = ms;
      stats[i] = st;
    }
  return FILL_OK;
}
}  // namespace

extern "C" {

fill_status fill_relax(fill_plan* p, const void* d, long long d_stride, int iters, void* out,
                       fill_stats* stats) {
  if (!p || !d || !out || iters < 0 || d_stride < 0) return FILL_EINVAL;
  return p->o.mode == FILL_MODE_FP32   ? relax_t<float>(p, d, d_stride, iters, out, stats)
         : p->o.mode == FILL_MODE_FP64 ? relax_t<double>(p, d, d_stride, iters, out, stats)
                                       : relax_t<df>(p, d, d_stride, iters, out, stats);
}

}  // extern "C"

namespace {
// Real part of a transposed spectrum, scaled: the kernel table of one annulus.
template <typename T>
__global__ void k_spec_to_table(const T* spec, T* tab, long long n, double scale) {
  const T sc = (T)scale;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    tab[i] = spec[2 * i] * sc;
}

long long annulus_count(double r_in, double r_out) {
  const int R = (int)std::floor(r_out);
  long long c = 0;
  for (int dy = -R; dy <= R; ++dy)
    for (int dx = -R; dx <= R; ++dx) {
      const double r2 = double(dy) * dy + double(dx) * dx;
      if (r2 > r_in * r_in && r2 <= r_out * r_out && r2 > 0.0) ++c;
    }
  return c;
}

// Kernel tables 1/(count n) Re F(annulus_j) of the Sect. 6.3 solver, from the
// annulus images by the plan's own forward transforms (instance 0's buffers).
template <typename T>
fill_status set_annuli_t(fill_plan* p, int nk, const double* r_in, const double* r_out) {
  Precision<T>& P = prec<T>(p);
  if (!P.used) return FILL_OK;
  const size_t ntab = size_t(p->nx / 2 + 1) * p->ny;
  if (nk > P.nk_cap) {
    if (p->dalloc(&P.kt, size_t(nk) * ntab) != cudaSuccess) return FILL_ENOMEM;
    P.nk_cap = nk;
  }
  const size_t nspec = 2 * ntab;
  if (!P.spec2 && p->dalloc(&P.spec2, size_t(p->batch) * nspec) != cudaSuccess)
    return FILL_ENOMEM;
  P.nk = nk;
  for (int i = 0; i < p->batch; ++i) {
    P.hdesc[i].kt = P.kt;
    P.hdesc[i].spec2 = P.spec2 + size_t(i) * nspec;
  }
  fill_desc<T>(p, nullptr, 0, nullptr, nullptr, nullptr);
  CK(upload_desc<T>(p));
  CK(init_states<T>(p, 0.0));
  const Ctx<T> c1 = ctx<T>(p, 1);
  for (int j = 0; j < nk; ++j) {
    const long long cnt = annulus_count(r_in[j], r_out[j]);
    CK(vec<T>(c1, p->s, VOP_ANNULUS, SC_NONE, SKIP_NEVER, r_in[j] * r_in[j], r_out[j] * r_out[j]));
    CK(row<T>(c1, p->s, OP_LOAD_W, SC_NONE, false, true, SKIP_NEVER));
    CK(col<T>(c1, p->s, -1, SKIP_NEVER));
    ++p->launches;
    k_spec_to_table<T><<<256, 256, 0, p->s>>>(P.spec, P.kt + size_t(j) * ntab, (long long)ntab,
                                            1.0 / (double(cnt) * double(p->npix)));
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(p->s));
  return FILL_OK;
}

// Multi-scale kernel Laplace solver (Sect. 6.3): every sweep averages the map
// over each masked pixel's annulus (class map `cls`), all from the same map.
// One forward transform per sweep (row pass, then the column pass in forward
// mode, into spec); per annulus the column pass multiplies by its table and
// inverts into spec2, from which the inverse row pass writes the pixels of
// that class.
template <typename T>
fill_status laplace_ms_t(fill_plan* p, const void* d, long long d_stride, int iters,
                         const uint8_t* cls, void* out, fill_stats* stats) {
  Precision<T>& P = prec<T>(p);
  if (P.nk < 1) return FILL_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  const int B = p->batch;
  p->launches = 0;
  fill_desc<T>(p, d, d_stride, nullptr, out, nullptr);
  for (int i = 0; i < B; ++i) {
    P.hdesc[i].cls = cls;
    P.hdesc[i].kt = P.kt;
  }
  CK(upload_desc<T>(p));
  CK(init_states<T>(p, 0.0));
  const Ctx<T> c = ctx<T>(p);
  CK(vec<T>(c, p->s, VOP_W_FROM_D, SC_NONE, SKIP_NEVER));
  for (int k = 0; k < iters; ++k) {
    CK(row<T>(c, p->s, OP_LOAD_W, SC_NONE, false, true, SKIP_NEVER));
    CK(col<T>(c, p->s, -1, SKIP_NEVER));
    for (int j = 0; j < P.nk; ++j) {
      CK(col<T>(c, p->s, 2 + j, SKIP_NEVER, 1, 1));
      CK(row<T>(c, p->s, OP_KSEL, SC_NONE, true, false, SKIP_NEVER, 1, j));
    }
    CK(vec<T>(c, p->s, VOP_Y_TO_W_M, k == 0 ? SC_BB : SC_RES, SKIP_NEVER));
  }
  CK(vec<T>(c, p->s, VOP_W_TO_OUT, SC_NONE, SKIP_NEVER));
  CK(cudaMemcpyAsync(P.hst, P.st, sizeof(CgState) * B, cudaMemcpyDeviceToHost, p->s));
  CK(cudaStreamSynchronize(p->s));
  const double ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats)
    for (int i = 0; i < B; ++i) {
      const CgState& a = P.hst[i];
      fill_stats st{};
      st.iters = iters;
      st.status = FILL_OK;
      st.launches = (int)p->launches;
      st.rel_resid = a.bb > 0 ? std::sqrt(a.rr / a.bb) : 0.0;
      st.true_rel_resid = -1.0;
      st.ms = ms;
      stats[i] = st;
    }
  return FILL_OK;
}
}  // namespace

extern "C" {

fill_status fill_set_annuli(fill_plan* p, int nk, const double* r_in, const double* r_out) {
  if (!p || nk < 1 || nk > 250 || !r_in || !r_out) return FILL_EINVAL;
  for (int j = 0; j < nk; ++j)
    if (!(r_in[j] >= 0.0) || !(r_out[j] > r_in[j]) || 2.0 * r_out[j] >= double(p->nx) ||
        2.0 * r_out[j] >= double(p->ny) || annulus_count(r_in[j], r_out[j]) == 0)
      return FILL_EINVAL;
  fill_status fs = set_annuli_t<float>(p, nk, r_in, r_out);
  if (fs == FILL_OK) fs = set_annuli_t<double>(p, nk, r_in, r_out);
  if (fs == FILL_OK) fs = set_annuli_t<df>(p, nk, r_in, r_out);
  return fs;
}

fill_status fill_laplace_ms(fill_plan* p, const void* d, long long d_stride, int iters,
                            const uint8_t* cls, void* out, fill_stats* stats) {
  if (!p || !d || !cls || !out || iters < 0 || d_stride < 0) return FILL_EINVAL;
  return p->o.mode == FILL_MODE_FP32   ? laplace_ms_t<float>(p, d, d_stride, iters, cls, out, stats)
         : p->o.mode == FILL_MODE_FP64 ? laplace_ms_t<double>(p, d, d_stride, iters, cls, out, stats)
                                       : laplace_ms_t<df>(p, d, d_stride, iters, cls, out, stats);
}

fill_status fill_draw(fill_plan* p, const uint64_t* seeds, void* out) {
  if (!p || !seeds || !out) return FILL_EINVAL;
  const size_t n = p->npix;
  if (p->o.mode == FILL_MODE_FP32) {
    fill_desc<float>(p, nullptr, 0, seeds, nullptr, nullptr);
    CK(upload_desc<float>(p));
    CK(init_states<float>(p, 0.0));
    CK(row<float>(p, p->s, OP_XI, SC_NONE, false, true, false));
    CK(col<float>(p, p->s, 1, false));
    CK(row<float>(p, p->s, OP_STORE_Y, SC_NONE, true, false, false));
    CK(cudaMemcpyAsync(out, p->f.y, p->batch * n * sizeof(float), cudaMemcpyDeviceToDevice, p->s));
  } else if (p->o.mode == FILL_MODE_FP64) {
    fill_desc<double>(p, nullptr, 0, seeds, nullptr, nullptr);
    CK(upload_desc<double>(p));
    CK(init_states<double>(p, 0.0));
    CK(row<double>(p, p->s, OP_XI, SC_NONE, false, true, false));
    CK(col<double>(p, p->s, 1, false));
    CK(row<double>(p, p->s, OP_STORE_Y, SC_NONE, true, false, false));
    CK(cudaMemcpyAsync(out, p->g.y, p->batch * n * sizeof(double), cudaMemcpyDeviceToDevice, p->s));
  } else {
    fill_desc<df>(p, nullptr, 0, seeds, out, nullptr);
    CK(upload_desc<df>(p));
    CK(init_states<df>(p, 0.0));
    CK(row<df>(p, p->s, OP_XI, SC_NONE, false, true, false));
    CK(col<df>(p, p->s, 1, false));
    CK(row<df>(p, p->s, OP_STORE_Y, SC_NONE, true, false, false));
    CK(vec<df>(p, p->s, VOP_MAP_OUT, SC_NONE, false));
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
  constexpr bool same = std::is_same<T, typename MapOf<T>::type>::value;
  fill_desc<T>(p, in, 0, nullptr, out, nullptr);
  CK(upload_desc<T>(p));
  CK(init_states<T>(p, 0.0));
  if (same)
    CK(cudaMemcpyAsync(P.w, in, n * sizeof(T), cudaMemcpyDeviceToDevice, p->s));
  else
    CK(vec<T>(ctx<T>(p, 1), p->s, VOP_MAP_IN, SC_NONE, false));
  const bool masked = which >= 2;
  const int table = (which == 0 || which == 2) ? 0 : 1;
  CK(row<T>(p, p->s, masked ? OP_LOAD_W_MASK : OP_LOAD_W, SC_NONE, false, true, false, 1));
  CK(col<T>(p, p->s, table, false, 1));
  CK(row<T>(p, p->s, masked ? OP_STORE_Y_MASK : OP_STORE_Y, SC_NONE, true, false, false, 1));
  if (same)
    CK(cudaMemcpyAsync(out, P.y, n * sizeof(T), cudaMemcpyDeviceToDevice, p->s));
  else
    CK(vec<T>(ctx<T>(p, 1), p->s, VOP_MAP_OUT, SC_NONE, false));
  CK(cudaStreamSynchronize(p->s));
  return FILL_OK;
}
}  // namespace

extern "C" {

fill_status fill_apply(fill_plan* p, int which, const void* in, void* out) {
  if (!p || !in || !out || which < 0 || which > 3 || in == out) return FILL_EINVAL;
  return p->o.mode == FILL_MODE_FP32   ? apply_t<float>(p, which, in, out)
         : p->o.mode == FILL_MODE_FP64 ? apply_t<double>(p, which, in, out)
                                       : apply_t<df>(p, which, in, out);
}

fill_status fill_history(fill_plan* p, int inst, double* hist, int cap, int* count) {
  if (!p || !hist || inst < 0 || inst >= p->batch || cap < 0) return FILL_EINVAL;
  const int hc = std::max(p->o.history_cap, 1);
  int m = 0;
  const double* src = nullptr;
  if (p->o.mode == FILL_MODE_MIXED) {
    m = p->h.hst[inst].refine + 1;  // high-precision true residual after each update
    src = p->h.hist;
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
// Number of eigenvalues below x of the symmetric tridiagonal matrix with
// diagonal d and off-diagonal e (Sturm sequence of the LDL^T pivots).
int sturm_below(const std::vector<double>& d, const std::vector<double>& e, double x) {
  int c = 0;
  double q = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    q = d[i] - x - (i > 0 ? e[i - 1] * e[i - 1] / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++c;
  }
  return c;
}

// The m-th smallest eigenvalue (0-based) of that matrix, by bisection inside
// its Gershgorin interval down to a few ulp.
double tridiag_eig(const std::vector<double>& d, const std::vector<double>& e, int m) {
  double lo = d[0], hi = d[0];
  for (size_t i = 0; i < d.size(); ++i) {
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < d.size() ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 4e-16 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_below(d, e, mid) > m)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}
}  // namespace

extern "C" {

fill_status fill_lanczos(fill_plan* p, int inst, double* alpha, double* beta, int cap, int* count,
                         double* lmin, double* lmax) {
  if (!p || inst < 0 || inst >= p->batch || cap < 0 || p->o.history_cap <= 0) return FILL_EINVAL;
  const bool f32 = p->o.mode != FILL_MODE_FP64;
  const CgState& st = f32 ? p->f.hst[inst] : p->g.hst[inst];
  const double* src = f32 ? p->f.coef : p->g.coef;
  const int hc = p->o.history_cap;
  const int k = std::min(p->o.mode == FILL_MODE_MIXED ? st.last_iter : st.iter, hc);
  if (count) *count = k;
  if (lmin) *lmin = 0.0;
  if (lmax) *lmax = 0.0;
  if (k <= 0) return FILL_OK;
  std::vector<double> c(2 * size_t(k));
  CK(cudaMemcpy(c.data(), src + 2 * size_t(inst) * hc, c.size() * sizeof(double),
                cudaMemcpyDeviceToHost));
  for (int j = 0; j < std::min(k, cap); ++j) {
    if (alpha) alpha[j] = c[2 * j];
    if (beta) beta[j] = j + 1 < k ? c[2 * j + 1] : 0.0;
  }
  // T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j
  std::vector<double> d(k), e(k > 1 ? k - 1 : 0);
  for (int j = 0; j < k; ++j) {
    const double a = c[2 * j];
    if (!(a > 0.0)) return FILL_EBREAKDOWN;
    d[j] = 1.0 / a + (j > 0 ? c[2 * j - 1] / c[2 * j - 2] : 0.0);
    if (j + 1 < k) e[j] = std::sqrt(std::max(c[2 * j + 1], 0.0)) / a;
  }
  if (lmin) *lmin = tridiag_eig(d, e, 0);
  if (lmax) *lmax = tridiag_eig(d, e, k - 1);
  return FILL_OK;
}

}  // extern "C"

namespace {
template <typename T>
fill_status time_pass_t(fill_plan* p, int pass, int reps, double* ms, double* bytes) {
  Precision<T>& P = prec<T>(p);
  if (!P.used) return FILL_EINVAL;
  fill_desc<T>(p, nullptr, 0, nullptr, nullptr, nullptr);
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
  // per instance: compact CG vectors (nM values), spectra; once per launch
  // (shared by the batch): the column table, the mask words (8 bytes per 32 pixels)
  const double nM = double(p->nmasked), MW = n / 4.0;
  double b = 0.0, shared = MW;
  switch (pass) {
    case 0: b = 2.0 * SB; shared = S * t; break;
    case 1: b = 6.0 * nM * t + SB; break;
    case 2: b = 3.0 * nM * t + SB; break;
    case 3: b = SB + 2.0 * nM * t; break;
    default: b = 2.0 * SB; break;
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
  *bytes = b * p->batch + shared;
  return FILL_OK;
}
}  // namespace

extern "C" {

fill_status fill_time_pass(fill_plan* p, int pass, int precision, int reps, double* ms,
                           double* bytes) {
  if (!p || !ms || !bytes || pass < 0 || pass > 4 || reps < 1 || precision < 0 || precision > 1)
    return FILL_EINVAL;
  if (precision == 0) return time_pass_t<float>(p, pass, reps, ms, bytes);
  return p->o.mode == FILL_MODE_MIXED ? time_pass_t<df>(p, pass, reps, ms, bytes)
                                      : time_pass_t<double>(p, pass, reps, ms, bytes);
}

}  // extern "C"

namespace {
template <typename T>
fill_status set_bands_t(fill_plan* p, int nbands, const int32_t* band_of_k, const double* sig) {
  Precision<T>& P = prec<T>(p);
  if (!P.used) return FILL_OK;
  const int nkx = p->nx / 2 + 1, ny = p->ny;
  const size_t nt = (size_t)nkx * ny;
  const double n = double(p->npix);
  std::vector<int> band(nt);
  std::vector<T> c1(nt), c2(nt);
  for (int ky = 0; ky < ny; ++ky)
    for (int kx = 0; kx < nkx; ++kx) {
      const size_t h = (size_t)ky * nkx + kx, t = (size_t)kx * ny + ky;
      const double P_ = p->P_half[h], S = sig[h];
      const double wt = (kx == 0 || kx == p->nx / 2) ? 1.0 : 2.0;
      band[t] = band_of_k[h];
      c1[t] = (T)(wt * S / (2.0 * n * std::sqrt(P_)));
      c2[t] = (T)(wt * S / (n * P_ * P_));
    }
  if (!P.band) {
    if (p->dalloc(&P.band, nt) != cudaSuccess || p->dalloc(&P.coef1, nt) != cudaSuccess ||
        p->dalloc(&P.coef2, nt) != cudaSuccess ||
        p->dalloc(&P.bpart, (size_t)p->batch * kDotCtas * kMaxBands) != cudaSuccess ||
        p->dalloc(&P.bsum, (size_t)p->batch * kMaxBands) != cudaSuccess)
      return FILL_ENOMEM;
  }
  CK(cudaMemcpy(P.band, band.data(), nt * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(P.coef1, c1.data(), nt * sizeof(T), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(P.coef2, c2.data(), nt * sizeof(T), cudaMemcpyHostToDevice));
  P.nbands = nbands;
  return FILL_OK;
}
}  // namespace

extern "C" {

fill_status fill_set_bands(fill_plan* p, int nbands, const int32_t* band_of_k,
                           const double* sig_half) {
  if (!p || !band_of_k || !sig_half || nbands < 1 || nbands > kMaxBands) return FILL_EINVAL;
  const size_t nh = (size_t)p->ny * (p->nx / 2 + 1);
  for (size_t i = 0; i < nh; ++i)
    if (band_of_k[i] < 0 || band_of_k[i] >= nbands || !std::isfinite(sig_half[i])) return FILL_EINVAL;
  fill_status fs = set_bands_t<float>(p, nbands, band_of_k, sig_half);
  if (fs == FILL_OK) fs = set_bands_t<double>(p, nbands, band_of_k, sig_half);
  if (fs == FILL_OK) fs = set_bands_t<df>(p, nbands, band_of_k, sig_half);
  if (fs == FILL_OK) {
    p->band_idx.assign(band_of_k, band_of_k + nh);
    p->band_sig.assign(sig_half, sig_half + nh);
    p->nbands = nbands;
    if (!p->sig_dev && p->dalloc(&p->sig_dev, nh) != cudaSuccess) return FILL_ENOMEM;
    CK(cudaMemcpy(p->sig_dev, sig_half, nh * sizeof(double), cudaMemcpyHostToDevice));
  }
  return fs;
}

fill_status fill_set_spectrum(fill_plan* p, const double* P_half) {
  if (!p || !P_half) return FILL_EINVAL;
  if (!spectrum_valid(p->ny, p->nx, P_half)) {
    cgf_set_last_error("fill_set_spectrum: P must be finite, > 0 and Hermitian-consistent");
    return FILL_EINVAL;
  }
  const size_t nh = (size_t)p->ny * (p->nx / 2 + 1);
  double a = 0.0;
  for (size_t i = 0; i < nh; ++i) a = std::max(a, 1.0 / P_half[i]);
  // the plan's stream may still run work that reads the tables
  CK(cudaStreamSynchronize(p->s));
  CK(cudaMemcpyAsync(p->P_dev, P_half, nh * sizeof(double), cudaMemcpyHostToDevice, p->s));
  // the tables of every precision the plan holds, and the band-gradient
  // weights at the new P (they depend on it), built on the device
  const int nkx = p->nx / 2 + 1, blocks = (int)std::min<size_t>((nh + 255) / 256, 4096);
  const bool bands = p->nbands > 0;
  if (p->f.used)
    k_spectral_tables<float><<<blocks, 256, 0, p->s>>>(p->P_dev, p->sig_dev, p->ny, nkx, p->nx,
        p->f.t_inv, p->f.t_sqrt, bands ? p->f.coef1 : nullptr, bands ? p->f.coef2 : nullptr);
  if (p->g.used)
    k_spectral_tables<double><<<blocks, 256, 0, p->s>>>(p->P_dev, p->sig_dev, p->ny, nkx, p->nx,
        p->g.t_inv, p->g.t_sqrt, bands ? p->g.coef1 : nullptr, bands ? p->g.coef2 : nullptr);
  if (p->h.used)
    k_spectral_tables<df><<<blocks, 256, 0, p->s>>>(p->P_dev, p->sig_dev, p->ny, nkx, p->nx,
        p->h.t_inv, p->h.t_sqrt, bands ? p->h.coef1 : nullptr, bands ? p->h.coef2 : nullptr);
  CK(cudaGetLastError());
  p->relax_a = a;
  p->P_half.assign(P_half, P_half + nh);
  CK(cudaStreamSynchronize(p->s));
  return FILL_OK;
}

fill_status fill_backward(fill_plan* p, const void* d, long long d_stride, const void* grad_x,
                          double tol, void* grad_d, double* grad_bands, fill_stats* stats) {
  if (!p || !d || !grad_x || !grad_d || !(tol >= 0.0) || d_stride < 0) return FILL_EINVAL;
  if (!p->o.backward) return FILL_EINVAL;
  const bool f32 = p->o.mode == FILL_MODE_FP32, mixed = p->o.mode == FILL_MODE_MIXED;
  if (grad_bands && (f32 ? p->f.nbands : mixed ? p->h.nbands : p->g.nbands) == 0)
    return FILL_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  p->launches = 0;
  fill_status fs = f32     ? backward_t<float>(p, d, d_stride, grad_x, tol, grad_d, grad_bands)
                   : mixed ? backward_t<df>(p, d, d_stride, grad_x, tol, grad_d, grad_bands)
                           : backward_t<double>(p, d, d_stride, grad_x, tol, grad_d, grad_bands);
  if (fs != FILL_OK) return fs;
  if (mixed) {
    CK(cudaMemcpyAsync(p->h.hst, p->h.st, sizeof(CgState) * p->batch, cudaMemcpyDeviceToHost, p->s));
    CK(cudaMemcpyAsync(p->f.hst, p->f.st, sizeof(CgState) * p->batch, cudaMemcpyDeviceToHost, p->s));
  } else if (f32) {
    CK(cudaMemcpyAsync(p->f.hst, p->f.st, sizeof(CgState) * p->batch, cudaMemcpyDeviceToHost, p->s));
  } else {
    CK(cudaMemcpyAsync(p->g.hst, p->g.st, sizeof(CgState) * p->batch, cudaMemcpyDeviceToHost, p->s));
  }
  CK(queue_err_readback(p));
  CK(cudaStreamSynchronize(p->s));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  fill_status worst = FILL_OK;
  collect_stats(p, stats, ms, &worst);
  const fill_status te = take_err(p);
  return te != FILL_OK ? te : worst;
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

// =================================================================== tuning
namespace {

// Times `reps` launches of f(stream) with CUDA events (after one warm-up).
template <typename F>
cudaError_t time_launches(cudaStream_t s, int reps, F f, float* ms) {
  cudaEvent_t e0, e1;
  CE(cudaEventCreate(&e0));
  CE(cudaEventCreate(&e1));
  cudaError_t e = f(s);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int i = 0; i < reps && e == cudaSuccess; ++i) e = f(s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

// The row and column passes of one preconditioned iteration, without scalar
// updates or done checks (schedule timing only; vector contents are scratch).
template <typename T>
cudaError_t tune_rows_once(const Ctx<T>& c, cudaStream_t s) {
  CE(row<T>(c, s, OP_P_UPD_Z, SC_NONE, false, true, false));
  CE(row<T>(c, s, OP_Q, SC_NONE, true, false, false));
  CE(row<T>(c, s, OP_R_UPD, SC_NONE, false, true, false));
  CE(row<T>(c, s, OP_MASK, SC_NONE, true, true, false));
  return row<T>(c, s, OP_Z, SC_NONE, true, false, false);
}

// Chooses rows per CTA (row passes) and FFTs per CTA (column pass) for a
// launch context by timing every valid candidate.
template <typename T>
cudaError_t autotune_ctx(Ctx<T> c, cudaStream_t s, int* best_rows, int* best_ffts) {
  int optin = 0, dev = 0;
  CE(cudaGetDevice(&dev));
  CE(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t limit = size_t(optin) - 1024;
  const int TT = (1 << c.log_l) / 16, TN = (1 << c.log_n) / 16, nkx = c.nx / 2 + 1;
  float best = 1e30f;
  for (int r = 1; r <= c.ny && r <= 256; r *= 2) {
    if (r * TT > Launch<T>::max_threads() || r * TT < 32 || c.ny / r > kMaxPartials ||
        Launch<T>::row_smem(c.log_l, r) > limit)
      continue;
    c.rows = r;
    float ms = 0.f;
    CE(time_launches(s, 3, [&](cudaStream_t st) { return tune_rows_once<T>(c, st); }, &ms));
    if (ms < best) {
      best = ms;
      *best_rows = r;
    }
  }
  best = 1e30f;
  c.col_variant = 0;
  for (int f = 1; f <= nkx && f <= 64; f *= 2) {
    if (f * TN > Launch<T>::max_threads() || Launch<T>::col_smem(c.log_n, f) > limit) continue;
    c.ffts = f;
    float ms = 0.f;
    CE(time_launches(s, 3, [&](cudaStream_t st) { return col<T>(c, st, 0, false); }, &ms));
    if (ms < best) {
      best = ms;
      *best_ffts = f;
    }
  }
  if (std::is_same<T, float>::value) {
    // the persistent bulk-copy-fed column kernel (its own column blocking):
    // recorded as ffts = -1
    c.col_variant = 1;
    float ms = 0.f;
    CE(time_launches(s, 3, [&](cudaStream_t st) { return col<T>(c, st, 0, false); }, &ms));
    if (ms < best) *best_ffts = -1;
  }
  return cudaSuccess;
}

// Applies a tuned column choice: ffts > 0 register-fed kernel with that many
// FFTs per CTA, ffts = -1 the bulk-copy-fed kernel (the CTA shape stays).
void apply_col_choice(int tuned, int* ffts, int* variant) {
  if (tuned < 0) {
    *variant = 1;
  } else {
    *variant = 0;
    *ffts = tuned;
  }
}

// Autotune cache: lines "prec ny nx ninst rows ffts".
// Precision code of the tuning cache: 0 FP32, 1 FP64, 2 double-float.
template <typename T>
int prec_code() {
  return std::is_same<T, float>::value ? 0 : std::is_same<T, double>::value ? 1 : 2;
}

bool cache_lookup(const char* path, int prec, int ny, int nx, int ninst, int* rows, int* ffts) {
  if (!path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[256];
  int a, b, c, d, r, q;
  bool found = false;
  while (std::fgets(line, sizeof line, f))
    if (std::sscanf(line, "%d %d %d %d %d %d", &a, &b, &c, &d, &r, &q) == 6 && a == prec &&
        b == ny && c == nx && d == ninst) {
      *rows = r;
      *ffts = q;
      found = true;
    }
  std::fclose(f);
  return found;
}

void cache_store(const char* path, int prec, int ny, int nx, int ninst, int rows, int ffts) {
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%d %d %d %d %d %d\n", prec, ny, nx, ninst, rows, ffts);
  std::fclose(f);
}

// Mixed-radix plans: lines "g prec ny nx ninst rows ffts row_code col_code".
bool cache_lookup_gen(const char* path, int prec, int ny, int nx, int ninst, int* rows, int* ffts,
                      int* rcode, int* ccode) {
  if (!path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[256];
  int a, b, c, d, r, q, x, y;
  bool found = false;
  while (std::fgets(line, sizeof line, f))
    if (std::sscanf(line, "g %d %d %d %d %d %d %d %d", &a, &b, &c, &d, &r, &q, &x, &y) == 8 &&
        a == prec && b == ny && c == nx && d == ninst && x >= 0 && x < kGenCodes && y >= 0 &&
        y < kGenCodes) {
      *rows = r;
      *ffts = q;
      *rcode = x;
      *ccode = y;
      found = true;
    }
  std::fclose(f);
  return found;
}

void cache_store_gen(const char* path, int prec, int ny, int nx, int ninst, int rows, int ffts,
                     int rcode, int ccode) {
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "g %d %d %d %d %d %d %d %d\n", prec, ny, nx, ninst, rows, ffts, rcode, ccode);
  std::fclose(f);
}

template <typename T>
fill_status tune_plan_t(fill_plan* p, const char* path) {
  Precision<T>& P = prec<T>(p);
  if (!P.used) return FILL_OK;
  const int pr = prec_code<T>();
  int rows = P.rows, ffts = P.col_variant ? -1 : P.ffts;
  if (!cache_lookup(path, pr, p->ny, p->nx, p->batch, &rows, &ffts)) {
    fill_desc<T>(p, nullptr, 0, nullptr, nullptr, nullptr);
    CK(upload_desc<T>(p));
    CK(init_states<T>(p, 0.0));
    CK(autotune_ctx<T>(ctx<T>(p), p->s, &rows, &ffts));
    cache_store(path, pr, p->ny, p->nx, p->batch, rows, ffts);
  }
  int nf = P.ffts, nv = P.col_variant;
  apply_col_choice(ffts, &nf, &nv);
  if (rows != P.rows || nf != P.ffts || nv != P.col_variant) {
    P.rows = rows;
    P.ffts = nf;
    P.col_variant = nv;
    if (P.iter_graph) {
      cudaGraphExecDestroy(P.iter_graph);
      P.iter_graph = nullptr;
    }
    if (p->mixed_graph) {
      cudaGraphExecDestroy(p->mixed_graph);
      p->mixed_graph = nullptr;
    }
  }
  return FILL_OK;
}

// Destroys the plan's captured CG-loop graphs (after a schedule change).
void drop_graphs(fill_plan* p) {
  auto drop = [](cudaGraphExec_t& g) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  };
  drop(p->f.iter_graph);
  drop(p->g.iter_graph);
  drop(p->h.iter_graph);
  drop(p->mixed_graph);
}

// Switches one transform length (rows: nx / 2, else ny) of a mixed-radix plan
// to radix schedule `code`: new tables for every precision in use and new
// digit-reversal maps; the threads per group stay, so every CTA shape stays
// valid.
fill_status apply_gen_code(fill_plan* p, bool rows, int code) {
  GenLen& g = rows ? p->grow : p->gcol;
  if (g.code == code) return FILL_OK;
  GenLen t = g;
  if (!gen_factor(g.n, &t, code)) return FILL_EINVAL;
  g = t;
  fill_status fs = FILL_OK;
  if (p->f.used) fs = gen_upload<float>(p);
  if (fs == FILL_OK && p->g.used) fs = gen_upload<double>(p);
  if (fs == FILL_OK && p->h.used) fs = gen_upload<df>(p);
  if (fs == FILL_OK) fs = gen_upload_maps(p);
  return fs;
}

// The radix schedules of a length that differ from one another.
std::vector<int> gen_candidates(int n) {
  std::vector<int> out;
  std::vector<std::vector<int>> seen;
  for (int code = 0; code < kGenCodes; ++code) {
    GenLen g{};
    if (!gen_factor(n, &g, code)) continue;
    std::vector<int> r(g.radix, g.radix + g.nst);
    if (std::find(seen.begin(), seen.end(), r) == seen.end()) {
      seen.push_back(r);
      out.push_back(code);
    }
  }
  return out;
}

// Mixed-radix plans: the radix schedule of each transform length and the CTA
// shapes, timed on the precision T that carries the CG loop; the other
// precisions follow the chosen schedules and keep their CTA shapes.
template <typename T>
fill_status tune_gen_t(fill_plan* p, const char* path) {
  Precision<T>& P = prec<T>(p);
  constexpr int V = gen_v<T>();
  const int pr = prec_code<T>();
  int rows = P.rows, ffts = P.ffts, rcode = p->grow.code, ccode = p->gcol.code;
  if (!cache_lookup_gen(path, pr, p->ny, p->nx, p->batch, &rows, &ffts, &rcode, &ccode)) {
    fill_desc<T>(p, nullptr, 0, nullptr, nullptr, nullptr);
    CK(upload_desc<T>(p));
    CK(init_states<T>(p, 0.0));
    float best = 1e30f;
    for (int code : gen_candidates(p->grow.n)) {
      fill_status fs = apply_gen_code(p, true, code);
      if (fs != FILL_OK) return fs;
      for (int r = gen_vrow<T>(); r <= 4 * gen_vrow<T>(); r *= 2) {
        if (!gen_row_ok<T>(p, r)) continue;
        Ctx<T> c = ctx<T>(p);
        c.rows = r;
        float ms = 0.f;
        CK(time_launches(p->s, 3, [&](cudaStream_t st) { return tune_rows_once<T>(c, st); }, &ms));
        if (ms < best) {
          best = ms;
          rows = r;
          rcode = code;
        }
      }
    }
    best = 1e30f;
    for (int code : gen_candidates(p->gcol.n)) {
      fill_status fs = apply_gen_code(p, false, code);
      if (fs != FILL_OK) return fs;
      for (int f = V; f <= 16; f *= 2) {
        if (!gen_col_ok<T>(p, f)) continue;
        Ctx<T> c = ctx<T>(p);
        c.ffts = f;
        float ms = 0.f;
        CK(time_launches(p->s, 3, [&](cudaStream_t st) { return col<T>(c, st, 0, false); }, &ms));
        if (ms < best) {
          best = ms;
          ffts = f;
          ccode = code;
        }
      }
    }
    cache_store_gen(path, pr, p->ny, p->nx, p->batch, rows, ffts, rcode, ccode);
  }
  if (!gen_row_ok<T>(p, rows) || !gen_col_ok<T>(p, ffts)) return FILL_EINVAL;
  fill_status fs = apply_gen_code(p, true, rcode);
  if (fs == FILL_OK) fs = apply_gen_code(p, false, ccode);
  if (fs != FILL_OK) return fs;
  P.rows = rows;
  P.ffts = ffts;
  drop_graphs(p);
  return FILL_OK;
}

}  // namespace

// =================================================================== groups
namespace {

struct GroupClass {
  int ny = 0, nx = 0, log_l = 0, log_n = 0, rows = 0, ffts = 0, ninst = 0, col_variant = 0;
  long long npix = 0;
  std::vector<int> plans;       // group indices of the plans in this class
  void* desc = nullptr;         // device InstDesc<T>[ninst] (T: FP32 in mixed mode)
  void* hdesc = nullptr;        // pinned mirror
  CgState* st = nullptr;        // device gather buffer
  CgState* hst = nullptr;       // pinned
  cudaStream_t cs = nullptr;    // class stream
  cudaEvent_t join = nullptr;
  // mixed mode: the double-float descriptors, schedule and states of the
  // same instances
  void* desc_hi = nullptr;
  void* hdesc_hi = nullptr;
  int rows_hi = 0, ffts_hi = 0, col_variant_hi = 0;
  CgState* st_hi = nullptr;
  CgState* hst_hi = nullptr;
  CgState** stp_hi = nullptr;   // device: the double-float state of every instance
};

}  // namespace

struct fill_group {
  std::vector<fill_plan*> plans;
  std::vector<int> first;       // first flat instance of each plan
  std::vector<GroupClass> cls;
  int mode = 1, precond = 1, max_iter = 10000, ntot = 0, host_loops = 0;
  double update_delta = 1e-2;   // mixed mode (reliable updates)
  long long if_kernels = 0;     // mixed mode: kernels inside one update IF body
  cudaStream_t s = nullptr, cap = nullptr, cap2 = nullptr;
  cudaEvent_t fork = nullptr, fork_cap = nullptr;
  CgState** stp = nullptr;      // device: state pointer of every instance
  int* counter = nullptr;       // device: loop bodies run by the last launch
  int* hloop = nullptr;         // pinned
  cudaGraphExec_t graph = nullptr;
  long long graph_kernels = 0, launches = 0;
  std::vector<void*> dev, host;
  ~fill_group() {
    if (graph) cudaGraphExecDestroy(graph);
    if (cap2) cudaStreamDestroy(cap2);
    for (auto& c : cls) {
      if (c.cs) cudaStreamDestroy(c.cs);
      if (c.join) cudaEventDestroy(c.join);
    }
    if (fork) cudaEventDestroy(fork);
    if (fork_cap) cudaEventDestroy(fork_cap);
    if (cap) cudaStreamDestroy(cap);
    for (void* v : dev) cudaFree(v);
    for (void* v : host) cudaFreeHost(v);
  }
};

namespace {

// Launch context of a size class (hi: the double-float side of a mixed
// group).
template <typename T>
Ctx<T> gctx(fill_group* g, GroupClass& c, bool hi = false) {
  fill_plan* p0 = g->plans[c.plans[0]];
  Ctx<T> x{c.ny, c.nx, c.log_l, c.log_n, hi ? c.rows_hi : c.rows, hi ? c.ffts_hi : c.ffts,
           c.ninst, g->precond, hi ? c.col_variant_hi : c.col_variant, c.npix,
           reinterpret_cast<const InstDesc<T>*>(hi ? c.desc_hi : c.desc), prec<T>(p0).tw,
           &g->launches, p0->dev_err};
  if (p0->gen) {   // mixed-radix grid: the class shares the first plan's transforms
    x.grow = &p0->grow;
    x.gcol = &p0->gcol;
    x.gwl = prec<T>(p0).gwl;
    x.gwx = prec<T>(p0).gwx;
    x.gwn = prec<T>(p0).gwn;
  }
  return x;
}

template <typename T>
fill_status group_setup(fill_group* g, int autotune, const char* path) {
  for (auto& c : g->cls) {
    const size_t nb = sizeof(InstDesc<T>) * c.ninst;
    if (cudaMalloc(&c.desc, nb) != cudaSuccess) return FILL_ENOMEM;
    g->dev.push_back(c.desc);
    if (cudaMallocHost(&c.hdesc, nb) != cudaSuccess) return FILL_ENOMEM;
    g->host.push_back(c.hdesc);
    InstDesc<T>* h = reinterpret_cast<InstDesc<T>*>(c.hdesc);
    int k = 0;
    for (int pi : c.plans) {
      fill_plan* p = g->plans[pi];
      for (int i = 0; i < p->batch; ++i) h[k++] = prec<T>(p).hdesc[i];
    }
    fill_plan* p0 = g->plans[c.plans[0]];
    c.rows = prec<T>(p0).rows;
    c.ffts = prec<T>(p0).ffts;
    c.col_variant = prec<T>(p0).col_variant;
    CK(cudaMemcpy(c.desc, c.hdesc, nb, cudaMemcpyHostToDevice));
    if (autotune && !p0->gen) {   // mixed-radix classes keep their fixed schedule
      const int pr = prec_code<T>();
      int tuned = c.col_variant ? -1 : c.ffts;
      if (cache_lookup(path, pr, c.ny, c.nx, c.ninst, &c.rows, &tuned)) {
        apply_col_choice(tuned, &c.ffts, &c.col_variant);
      } else {
        Ctx<T> cx_ = gctx<T>(g, c);
        k_state_init<T><<<(c.ninst + 127) / 128, 128, 0, g->s>>>(
            reinterpret_cast<const InstDesc<T>*>(c.desc), c.ninst, 0.0, 1, 1);
        CK(cudaGetLastError());
        int rows = c.rows;
        tuned = c.ffts;
        CK(autotune_ctx<T>(cx_, g->s, &rows, &tuned));
        cache_store(path, pr, c.ny, c.nx, c.ninst, rows, tuned);
        c.rows = rows;
        apply_col_choice(tuned, &c.ffts, &c.col_variant);
      }
    }
  }
  return FILL_OK;
}

// Mixed groups: the double-float descriptors (each plan's, copied per
// class), their schedule (the first plan's) and the state buffers.
fill_status group_setup_hi(fill_group* g) {
  for (auto& c : g->cls) {
    const size_t nb = sizeof(InstDesc<df>) * c.ninst;
    if (cudaMalloc(&c.desc_hi, nb) != cudaSuccess) return FILL_ENOMEM;
    g->dev.push_back(c.desc_hi);
    if (cudaMallocHost(&c.hdesc_hi, nb) != cudaSuccess) return FILL_ENOMEM;
    g->host.push_back(c.hdesc_hi);
    if (cudaMalloc(&c.st_hi, sizeof(CgState) * c.ninst) != cudaSuccess) return FILL_ENOMEM;
    g->dev.push_back(c.st_hi);
    if (cudaMallocHost(&c.hst_hi, sizeof(CgState) * c.ninst) != cudaSuccess) return FILL_ENOMEM;
    g->host.push_back(c.hst_hi);
    if (cudaMalloc(&c.stp_hi, sizeof(CgState*) * c.ninst) != cudaSuccess) return FILL_ENOMEM;
    g->dev.push_back(c.stp_hi);
    InstDesc<df>* h = reinterpret_cast<InstDesc<df>*>(c.hdesc_hi);
    std::vector<CgState*> ptrs;
    int k = 0;
    for (int pi : c.plans) {
      fill_plan* p = g->plans[pi];
      for (int i = 0; i < p->batch; ++i) {
        h[k++] = p->h.hdesc[i];
        ptrs.push_back(p->h.st + i);
      }
    }
    fill_plan* p0 = g->plans[c.plans[0]];
    c.rows_hi = p0->h.rows;
    c.ffts_hi = p0->h.ffts;
    c.col_variant_hi = p0->h.col_variant;
    CK(cudaMemcpy(c.desc_hi, c.hdesc_hi, nb, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.stp_hi, ptrs.data(), sizeof(CgState*) * ptrs.size(), cudaMemcpyHostToDevice));
  }
  return FILL_OK;
}

MixedLoop group_mixed_loop(fill_group* g, GroupClass& c, bool host_loops) {
  return MixedLoop{c.stp_hi, c.ninst, g->counter, g->cap2, host_loops, &g->if_kernels};
}

// One iteration of every class of a mixed group (class streams forked from
// and joined back to s).
cudaError_t group_mixed_iter(fill_group* g, cudaStream_t s, cudaEvent_t fork, bool host_loops) {
  CE(cudaEventRecord(fork, s));
  for (auto& c : g->cls) {
    CE(cudaStreamWaitEvent(c.cs, fork, 0));
    CE(mixed_iter(gctx<float>(g, c), gctx<df>(g, c, true), c.cs, group_mixed_loop(g, c, host_loops)));
    CE(cudaEventRecord(c.join, c.cs));
    CE(cudaStreamWaitEvent(s, c.join, 0));
  }
  return cudaSuccess;
}

// The group's CG loop graph: every loop body forks the size classes onto
// their streams (parallel branches), runs one iteration of each, and joins.
template <typename T>
fill_status group_build_graph(fill_group* g) {
  if (g->graph) return FILL_OK;
  return build_loop_graph(
      g->cap,
      [&](cudaStream_t cap) -> cudaError_t {
        CE(cudaEventRecord(g->fork_cap, cap));
        for (auto& c : g->cls) {
          CE(cudaStreamWaitEvent(c.cs, g->fork_cap, 0));
          CE(pcg_iter<T>(gctx<T>(g, c), c.cs));
          CE(cudaEventRecord(c.join, c.cs));
          CE(cudaStreamWaitEvent(cap, c.join, 0));
        }
        return cudaSuccess;
      },
      g->stp, g->ntot, g->counter, g->max_iter + 4, &g->launches, &g->graph, &g->graph_kernels);
}

// The same for a mixed group: each class's body is the reliable-update
// iteration, with its own update IF node.
fill_status group_build_mixed_graph(fill_group* g) {
  if (g->graph) return FILL_OK;
  return build_loop_graph(
      g->cap, [&](cudaStream_t cap) { return group_mixed_iter(g, cap, g->fork_cap, false); },
      g->stp, g->ntot, g->counter, g->max_iter + 4, &g->launches, &g->graph, &g->graph_kernels);
}

// Starts every class on its own stream after `s` reaches this point, and
// makes `s` wait for all of them at the end of the enclosed work.
template <typename T, typename F>
fill_status group_fork_join(fill_group* g, F body) {
  CK(cudaEventRecord(g->fork, g->s));
  for (auto& c : g->cls) {
    CK(cudaStreamWaitEvent(c.cs, g->fork, 0));
    CK(body(c));
    CK(cudaEventRecord(c.join, c.cs));
    CK(cudaStreamWaitEvent(g->s, c.join, 0));
  }
  return FILL_OK;
}

template <typename T>
fill_status group_realize_t(fill_group* g, const void* const* d, const uint64_t* seeds,
                            double tol, void* const* out, fill_stats* stats) {
  // per-call descriptor fields
  for (auto& c : g->cls) {
    InstDesc<T>* h = reinterpret_cast<InstDesc<T>*>(c.hdesc);
    int k = 0;
    for (int pi : c.plans) {
      fill_plan* p = g->plans[pi];
      for (int i = 0; i < p->batch; ++i, ++k) {
        h[k].d = reinterpret_cast<const T*>(d[pi]);
        h[k].out = reinterpret_cast<T*>(out[pi]) + size_t(i) * p->npix;
        h[k].seed = (unsigned long long)seeds[g->first[pi] + i];
      }
    }
    CK(cudaMemcpyAsync(c.desc, c.hdesc, sizeof(InstDesc<T>) * c.ninst, cudaMemcpyHostToDevice, g->s));
  }
  const int hc = 1;
  fill_status fs = group_fork_join<T>(g, [&](GroupClass& c) -> cudaError_t {
    Ctx<T> cx_ = gctx<T>(g, c);
    ++g->launches;
    k_state_init<T><<<(c.ninst + 127) / 128, 128, 0, c.cs>>>(cx_.desc, c.ninst, tol * tol,
                                                            g->max_iter, hc);
    CE(cudaGetLastError());
    CE(vec<T>(cx_, c.cs, VOP_ZERO_UP, SC_NONE, false));
    CE(draw_and_rhs<T>(cx_, c.cs, !g->precond));
    return pcg_start<T>(cx_, c.cs, SC_NONE);
  });
  if (fs != FILL_OK) return fs;
  if (g->host_loops) {
    fs = run_loop_host(
        g->s,
        [&](cudaStream_t s) -> cudaError_t {
          CE(cudaEventRecord(g->fork, s));
          for (auto& c : g->cls) {
            CE(cudaStreamWaitEvent(c.cs, g->fork, 0));
            CE(pcg_iter<T>(gctx<T>(g, c), c.cs));
            CE(cudaEventRecord(c.join, c.cs));
            CE(cudaStreamWaitEvent(s, c.join, 0));
          }
          return cudaSuccess;
        },
        g->stp, g->ntot, g->counter, g->hloop, g->max_iter + 4, &g->launches);
    if (fs != FILL_OK) return fs;
  } else {
    fs = group_build_graph<T>(g);
    if (fs != FILL_OK) return fs;
    CK(cudaGraphLaunch(g->graph, g->s));
    CK(cudaMemcpyAsync(g->hloop, g->counter, sizeof(int), cudaMemcpyDeviceToHost, g->s));
  }
  fs = group_fork_join<T>(g, [&](GroupClass& c) -> cudaError_t {
    Ctx<T> cx_ = gctx<T>(g, c);
    CE(vec<T>(cx_, c.cs, VOP_ASSEMBLE, SC_NONE, false));
    ++g->launches;
    k_gather_states<T><<<(c.ninst + 127) / 128, 128, 0, c.cs>>>(cx_.desc, c.ninst, c.st);
    CE(cudaGetLastError());
    return cudaMemcpyAsync(c.hst, c.st, sizeof(CgState) * c.ninst, cudaMemcpyDeviceToHost, c.cs);
  });
  if (fs != FILL_OK) return fs;
  fill_plan* p0 = g->plans[0];   // its stream is the group's
  CK(queue_err_readback(p0));
  CK(cudaStreamSynchronize(g->s));
  if (!g->host_loops) g->launches += 1 + (long long)(*g->hloop) * g->graph_kernels;
  fill_status worst = FILL_OK;
  if (take_err(p0) != FILL_OK) return FILL_ETIMEOUT;
  for (auto& c : g->cls) {
    int k = 0;
    for (int pi : c.plans) {
      fill_plan* p = g->plans[pi];
      for (int i = 0; i < p->batch; ++i, ++k) {
        const CgState& a = c.hst[k];
        note_status(a.status, &worst);
        if (!stats) continue;
        fill_stats st{};
        st.iters = a.iter;
        st.status = a.status;
        st.rel_resid = a.bb > 0 ? std::sqrt(a.rr / a.bb) : 0.0;
        st.true_rel_resid = -1.0;
        stats[g->first[pi] + i] = st;
      }
    }
  }
  return worst;
}

// Mixed groups (Sects. 2.1-2.4 as in a mixed plan): the double-float draw and
// right-hand side per class, one FP32 PCG loop with reliable updates over all
// classes (one graph, classes as parallel branches, an update IF node per
// class), then per class the final fold, true residual and assembly.
fill_status group_realize_mixed(fill_group* g, const void* const* d, const uint64_t* seeds,
                                double tol, void* const* out, fill_stats* stats) {
  for (auto& c : g->cls) {
    InstDesc<df>* h = reinterpret_cast<InstDesc<df>*>(c.hdesc_hi);
    InstDesc<float>* f = reinterpret_cast<InstDesc<float>*>(c.hdesc);
    int k = 0;
    for (int pi : c.plans) {
      fill_plan* p = g->plans[pi];
      for (int i = 0; i < p->batch; ++i, ++k) {
        const unsigned long long seed = (unsigned long long)seeds[g->first[pi] + i];
        h[k].d = reinterpret_cast<const double*>(d[pi]);
        h[k].out = reinterpret_cast<double*>(out[pi]) + size_t(i) * p->npix;
        h[k].seed = seed;
        f[k].d = nullptr;
        f[k].out = nullptr;
        f[k].seed = seed;
      }
    }
    CK(cudaMemcpyAsync(c.desc_hi, c.hdesc_hi, sizeof(InstDesc<df>) * c.ninst,
                       cudaMemcpyHostToDevice, g->s));
    CK(cudaMemcpyAsync(c.desc, c.hdesc, sizeof(InstDesc<float>) * c.ninst,
                       cudaMemcpyHostToDevice, g->s));
  }
  fill_status fs = group_fork_join<df>(g, [&](GroupClass& c) -> cudaError_t {
    const Ctx<float> lo = gctx<float>(g, c);
    const Ctx<df> hi = gctx<df>(g, c, true);
    const int nb = (c.ninst + 127) / 128;
    g->launches += 2;
    k_state_init<df><<<nb, 128, 0, c.cs>>>(hi.desc, c.ninst, tol * tol, g->max_iter, 1);
    CE(cudaGetLastError());
    k_state_init<float><<<nb, 128, 0, c.cs>>>(lo.desc, c.ninst, 0.0, g->max_iter, 1);
    CE(cudaGetLastError());
    CE(vec<df>(hi, c.cs, VOP_ZERO_UP, SC_NONE, false));
    CE(draw_and_rhs<df>(hi, c.cs, false));
    return mixed_start(lo, hi, c.cs, tol, g->update_delta, g->max_iter);
  });
  if (fs != FILL_OK) return fs;
  if (g->host_loops) {
    fs = run_loop_host(
        g->s, [&](cudaStream_t s) { return group_mixed_iter(g, s, g->fork, true); }, g->stp,
        g->ntot, g->counter, g->hloop, g->max_iter + 4, &g->launches);
    if (fs != FILL_OK) return fs;
  } else {
    fs = group_build_mixed_graph(g);
    if (fs != FILL_OK) return fs;
    CK(cudaGraphLaunch(g->graph, g->s));
    CK(cudaMemcpyAsync(g->hloop, g->counter, 2 * sizeof(int), cudaMemcpyDeviceToHost, g->s));
  }
  fs = group_fork_join<df>(g, [&](GroupClass& c) -> cudaError_t {
    const Ctx<float> lo = gctx<float>(g, c);
    const Ctx<df> hi = gctx<df>(g, c, true);
    CE(mixed_finish(lo, hi, c.cs));
    CE(vec<df>(hi, c.cs, VOP_ASSEMBLE, SC_NONE, false));
    const int nb = (c.ninst + 127) / 128;
    g->launches += 2;
    k_gather_states<df><<<nb, 128, 0, c.cs>>>(hi.desc, c.ninst, c.st_hi);
    CE(cudaGetLastError());
    k_gather_states<float><<<nb, 128, 0, c.cs>>>(lo.desc, c.ninst, c.st);
    CE(cudaGetLastError());
    CE(cudaMemcpyAsync(c.hst_hi, c.st_hi, sizeof(CgState) * c.ninst, cudaMemcpyDeviceToHost, c.cs));
    return cudaMemcpyAsync(c.hst, c.st, sizeof(CgState) * c.ninst, cudaMemcpyDeviceToHost, c.cs);
  });
  if (fs != FILL_OK) return fs;
  fill_plan* p0 = g->plans[0];   // its stream is the group's
  CK(queue_err_readback(p0));
  CK(cudaStreamSynchronize(g->s));
  if (!g->host_loops) {
    const long long ifk = g->if_kernels, ncls = (long long)g->cls.size();
    g->launches += 1 + (long long)g->hloop[0] * (g->graph_kernels - ncls * ifk) +
                   (long long)g->hloop[1] * ifk;
  }
  fill_status worst = FILL_OK;
  if (take_err(p0) != FILL_OK) return FILL_ETIMEOUT;
  for (auto& c : g->cls) {
    int k = 0;
    for (int pi : c.plans) {
      fill_plan* p = g->plans[pi];
      for (int i = 0; i < p->batch; ++i, ++k) {
        const CgState& a = c.hst[k];
        const CgState& h = c.hst_hi[k];
        fill_stats st{};
        st.iters = h.total_iter;
        st.refine_steps = h.refine;
        const bool conv = h.rr <= h.tol2 * h.bb;
        st.status = h.status ? h.status : (conv ? FILL_OK : FILL_ENOTCONV);
        st.rel_resid = a.bb > 0 ? std::sqrt(a.rr / a.bb) : 0.0;
        st.true_rel_resid = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
        note_status(st.status, &worst);
        if (stats) stats[g->first[pi] + i] = st;
      }
    }
  }
  return worst;
}

}  // namespace

extern "C" {

fill_status fill_autotune(fill_plan* p, const char* cache_path) {
  if (!p) return FILL_EINVAL;
  if (p->gen) {   // mixed-radix grids: radix schedules and CTA shapes
    fill_status fs = p->o.mode == FILL_MODE_FP64 ? tune_gen_t<double>(p, cache_path)
                                                 : tune_gen_t<float>(p, cache_path);
    if (fs == FILL_OK) CK(cudaStreamSynchronize(p->s));
    return fs;
  }
  fill_status fs = tune_plan_t<float>(p, cache_path);
  if (fs == FILL_OK) fs = tune_plan_t<double>(p, cache_path);
  if (fs == FILL_OK) fs = tune_plan_t<df>(p, cache_path);
  if (fs == FILL_OK) CK(cudaStreamSynchronize(p->s));
  return fs;
}

fill_status fill_group_init(fill_group** out, fill_plan* const* plans, int count, int autotune,
                            const char* cache_path) {
  if (!out || !plans || count < 1) return FILL_EINVAL;
  *out = nullptr;
  const int mode = plans[0] ? plans[0]->o.mode : -1;
  if (mode != FILL_MODE_FP32 && mode != FILL_MODE_FP64 && mode != FILL_MODE_MIXED)
    return FILL_EINVAL;
  fill_group* g = new (std::nothrow) fill_group();
  if (!g) return FILL_ENOMEM;
  auto fail = [&](fill_status st) {
    delete g;
    return st;
  };
  g->mode = mode;
  g->precond = plans[0]->o.precond;
  g->max_iter = plans[0]->o.max_iter;
  g->host_loops = plans[0]->o.host_loops;
  g->update_delta = plans[0]->o.update_delta;
  g->s = plans[0]->s;
  int flat = 0;
  for (int i = 0; i < count; ++i) {
    fill_plan* p = plans[i];
    if (!p || p->o.mode != mode || p->o.precond != g->precond || p->s != g->s)
      return fail(FILL_EINVAL);
    // mixed groups run the reliable-update loop (update_delta > 0), one
    // threshold for all
    if (mode == FILL_MODE_MIXED && (!(p->o.update_delta > 0.0) || p->o.update_delta != g->update_delta))
      return fail(FILL_EINVAL);
    g->plans.push_back(p);
    g->first.push_back(flat);
    flat += p->batch;
    g->max_iter = std::max(g->max_iter, p->o.max_iter);
    size_t ci = 0;
    for (; ci < g->cls.size(); ++ci)
      if (g->cls[ci].ny == p->ny && g->cls[ci].nx == p->nx) break;
    if (ci == g->cls.size()) {
      GroupClass c;
      c.ny = p->ny;
      c.nx = p->nx;
      c.log_l = p->log_l;
      c.log_n = p->log_n;
      c.npix = p->npix;
      g->cls.push_back(c);
    }
    g->cls[ci].plans.push_back(i);
    g->cls[ci].ninst += p->batch;
  }
  g->ntot = flat;
  cudaError_t e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess && mode == FILL_MODE_MIXED)
    e = cudaStreamCreateWithFlags(&g->cap2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->fork_cap, cudaEventDisableTiming);
  for (auto& c : g->cls) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&c.st, sizeof(CgState) * c.ninst);
    if (e == cudaSuccess) g->dev.push_back(c.st);
    if (e == cudaSuccess) e = cudaMallocHost(&c.hst, sizeof(CgState) * c.ninst);
    if (e == cudaSuccess) g->host.push_back(c.hst);
  }
  if (e == cudaSuccess) e = cudaMalloc(&g->counter, 2 * sizeof(int));
  if (e == cudaSuccess) g->dev.push_back(g->counter);
  if (e == cudaSuccess) e = cudaMallocHost(&g->hloop, 2 * sizeof(int));
  if (e == cudaSuccess) g->host.push_back(g->hloop);
  if (e == cudaSuccess) e = cudaMalloc(&g->stp, sizeof(CgState*) * g->ntot);
  if (e == cudaSuccess) g->dev.push_back(g->stp);
  if (e == cudaSuccess) {
    std::vector<CgState*> ptrs;
    for (auto& c : g->cls)
      for (int pi : c.plans) {
        fill_plan* p = g->plans[pi];
        CgState* st = mode == FILL_MODE_FP64 ? p->g.st : p->f.st;   // the CG loop's states
        for (int i = 0; i < p->batch; ++i) ptrs.push_back(st + i);
      }
    e = cudaMemcpy(g->stp, ptrs.data(), sizeof(CgState*) * ptrs.size(), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return fail(cuda_fail(e, "fill_group_init"));
  fill_status fs = mode == FILL_MODE_FP64 ? group_setup<double>(g, autotune, cache_path)
                                          : group_setup<float>(g, autotune, cache_path);
  if (fs == FILL_OK && mode == FILL_MODE_MIXED) fs = group_setup_hi(g);
  if (fs != FILL_OK) return fail(fs);
  e = cudaStreamSynchronize(g->s);
  if (e != cudaSuccess) return fail(cuda_fail(e, "fill_group_init"));
  *out = g;
  return FILL_OK;
}

fill_status fill_group_realize(fill_group* g, const void* const* d, const uint64_t* seeds,
                               double tol, void* const* out, fill_stats* stats) {
  if (!g || !d || !seeds || !out || !(tol >= 0.0)) return FILL_EINVAL;
  for (size_t i = 0; i < g->plans.size(); ++i)
    if (!d[i] || !out[i]) return FILL_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  g->launches = 0;
  const fill_status worst =
      g->mode == FILL_MODE_MIXED  ? group_realize_mixed(g, d, seeds, tol, out, stats)
      : g->mode == FILL_MODE_FP32 ? group_realize_t<float>(g, d, seeds, tol, out, stats)
                                  : group_realize_t<double>(g, d, seeds, tol, out, stats);
  if (worst == FILL_ECUDA) return worst;
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats)
    for (int i = 0; i < g->ntot; ++i) {
      stats[i].ms = ms;
      stats[i].launches = (int)g->launches;
    }
  return worst;
}

int fill_group_size(const fill_group* g) { return g ? g->ntot : -1; }

fill_status fill_realize_batch(fill_plan* const* plans, int count, const void* const* d,
                               const uint64_t* seeds, double tol, void* const* out,
                               fill_stats* stats) {
  if (!plans || count < 1 || !d || !seeds || !out || !(tol >= 0.0)) return FILL_EINVAL;
  std::vector<unsigned long long> key(count);
  bool groupable = true;
  for (int i = 0; i < count; ++i) {
    fill_plan* p = plans[i];
    if (!p || !d[i] || !out[i]) return FILL_EINVAL;
    key[i] = p->serial;
    groupable = groupable && p->o.mode == plans[0]->o.mode &&
                p->o.precond == plans[0]->o.precond && p->s == plans[0]->s &&
                (p->o.mode != FILL_MODE_MIXED ||
                 (p->o.update_delta > 0.0 && p->o.update_delta == plans[0]->o.update_delta));
  }
  if (!groupable) {
    // one plan after another, each with its own data map shared by its batch
    fill_status worst = FILL_OK;
    int first = 0;
    for (int i = 0; i < count; ++i) {
      fill_status fs = fill_realize(plans[i], d[i], 0, seeds + first, tol, out[i],
                                    stats ? stats + first : nullptr);
      if (fs == FILL_ECUDA) return fs;
      note_status(fs, &worst);
      first += plans[i]->batch;
    }
    return worst;
  }
  fill_plan* p0 = plans[0];
  if (!p0->batch_group || p0->batch_key != key) {
    fill_group_destroy(p0->batch_group);
    p0->batch_group = nullptr;
    p0->batch_key.clear();
    fill_status fs = fill_group_init(&p0->batch_group, plans, count, 0, nullptr);
    if (fs != FILL_OK) return fs;
    p0->batch_key = key;
  }
  return fill_group_realize(p0->batch_group, d, seeds, tol, out, stats);
}

void fill_group_destroy(fill_group* g) {
  if (!g) return;
  cudaStreamSynchronize(g->s);
  delete g;
}

}  // extern "C"
