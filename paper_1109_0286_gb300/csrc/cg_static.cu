// fill_apply_static: the operator application of fill_apply for callers that
// cannot allocate device memory (for example code running inside a memory
// pool or arena owned by someone else, or a process whose allocator is locked
// down).  Instead of a plan's buffers it uses one file-scope device array as
// scratch, so the call itself performs no cudaMalloc / cudaFree and calls no
// allocating library routine.
//
// The scratch lives in g_static_scratch (kStaticScratchBytes per device that
// loads this library, held until the process exits).  It holds the twiddle
// table, the spectral table, the transposed half spectrum, the mask bits and
// one instance descriptor with its CG state.  Host code may not use the
// array's name as a device address: the address comes from
// cudaGetSymbolAddress, taken once per device (with that device current) on
// the first call, which also raises the kernels' shared-memory limits; make
// that first call before any stream capture.  Every call shares the array and
// overwrites it, so calls that overlap on the GPU (different streams, or
// threads without ordering) race; order them on one stream.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/cgfill.h"
#include "cg_launch.h"
#include "cg_schedule.h"
#include "cg_types.h"

namespace {

using namespace cgf;

constexpr size_t kStaticScratchBytes = size_t(8) << 20;   // 8 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_mutex;

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

// Records the reason of a rejected call for fill_last_error (cgfill.cu).
void cgf_set_last_error(const char* msg);

namespace {

// Scratch layout for an ny x nx FP32 problem.
struct Layout {
  size_t tw, tab, spec, bits, desc, st, part, total;
};

Layout layout(int ny, int nx) {
  const size_t nkx = size_t(nx) / 2 + 1, npix = size_t(ny) * nx;
  Layout L{};
  size_t o = 0;
  L.tw = o;   o = align256(o + 2 * sizeof(float) * kTwEntries);
  L.tab = o;  o = align256(o + sizeof(float) * nkx * ny);
  L.spec = o; o = align256(o + 2 * sizeof(float) * nkx * ny);
  L.bits = o; o = align256(o + sizeof(uint2) * ((npix + 31) / 32));
  L.desc = o; o = align256(o + sizeof(InstDesc<float>));
  L.st = o;   o = align256(o + sizeof(CgState));
  L.part = o; o = align256(o + sizeof(double) * kMaxPartials);
  L.total = o;
  return L;
}

// Builds everything a call needs inside the scratch: twiddles W_8192^m and
// the FFT stage tables, the
// table (1/(nP) or sqrt(P)/n in the transposed [kx][ky] layout), the mask
// bits, a zeroed CG state and the instance descriptor.
__global__ void k_static_setup(unsigned char* base, Layout L, int ny, int nx, const double* P,
                               const uint8_t* observed, int sqrt_table, const float* in,
                               float* out) {
  const int nkx = nx / 2 + 1;
  const long long npix = (long long)ny * nx;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nthr = (long long)gridDim.x * blockDim.x;
  float* tw = reinterpret_cast<float*>(base + L.tw);
  float* tab = reinterpret_cast<float*>(base + L.tab);
  uint2* bits = reinterpret_cast<uint2*>(base + L.bits);
  for (long long m = tid; m < kLmax; m += nthr) {
    double s, c;
    sincospi(2.0 * double(m) / double(kLmax), &s, &c);
    tw[2 * m] = (float)c;
    tw[2 * m + 1] = (float)-s;
  }
  // the per-stage tables of every power-of-two length (layout in cg_types.h)
  for (long long e = tid; e < kStwEntries; e += nthr) {
    int l = 4;
    while (l < 13 && e >= stw_base(l + 1)) ++l;
    int rem = (int)(e - stw_base(l));
    int st = stw_first(l);
    while (st + 1 < l / 4 && rem >= stw_stage_off(l, st + 1)) ++st;
    rem -= stw_stage_off(l, st);
    const int ns = stw_ns(l, st);
    const int r = 1 + rem / ns, jm = rem % ns;
    double s, c;
    sincospi(2.0 * double((long long)jm * r) / double(16LL * ns), &s, &c);
    tw[2 * (kLmax + e)] = (float)c;
    tw[2 * (kLmax + e) + 1] = (float)-s;
  }
  for (long long t = tid; t < (long long)nkx * ny; t += nthr) {
    const int kx = (int)(t / ny), ky = (int)(t % ny);
    const double p = P[(long long)ky * nkx + kx];
    tab[t] = (float)(sqrt_table ? sqrt(p) / double(npix) : 1.0 / (p * double(npix)));
  }
  for (long long w = tid; w < (npix + 31) / 32; w += nthr) {
    uint32_t word = 0;
    for (int b = 0; b < 32; ++b) {
      const long long i = w * 32 + b;
      if (i < npix && (observed == nullptr || observed[i])) word |= 1u << b;
    }
    bits[w] = make_uint2(word, 0u);   // compact offsets unused by these passes
  }
  if (tid == 0) {
    CgState* st = reinterpret_cast<CgState*>(base + L.st);
    *st = CgState{};
    InstDesc<float> D{};
    D.mw = bits;
    D.t_inv = tab;
    D.t_sqrt = tab;
    D.spec = reinterpret_cast<float*>(base + L.spec);
    D.w = const_cast<float*>(in);   // read only (the source pass)
    D.y = out;                      // the sink
    D.st = st;
    D.partial = reinterpret_cast<double*>(base + L.part);
    *reinterpret_cast<InstDesc<float>*>(base + L.desc) = D;
  }
}

int pow2_log(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return (1 << l) == v ? l : -1;
}

// Rejected call: records the reason for fill_last_error.
fill_status reject(const char* why) {
  cgf_set_last_error((std::string("fill_apply_static: ") + why).c_str());
  return FILL_EINVAL;
}

fill_status cuda_error(cudaError_t e, const char* where) {
  cgf_set_last_error((std::string("fill_apply_static: ") + where + ": " + cudaGetErrorString(e)).c_str());
  return FILL_ECUDA;
}

}  // namespace

extern "C" fill_status fill_apply_static(int ny, int nx, const double* P_half,
                                         const uint8_t* observed, int which, const float* in,
                                         float* out, void* stream) {
  cgf_set_last_error("");
  if (!P_half || !in || !out) return reject("null pointer");
  if (in == out) return reject("in and out may not alias");
  if (which < 0 || which > 3) return reject("which must be 0, 1, 2 or 3");
  if (which >= 2 && !observed) return reject("which >= 2 needs the observed mask");
  const int log_l = pow2_log(nx / 2), log_n = pow2_log(ny);
  if (log_l < 4 || log_l > 12 || log_n < 4 || log_n > 13)
    return reject("grid must be powers of two with 32 <= nx <= 8192 and 16 <= ny <= 8192");
  const Layout L = layout(ny, nx);
  if (L.total > kStaticScratchBytes)
    return reject("grid too large for the 8 MiB static scratch (at most about 1024 x 1024 pixels)");
  // the launch schedule of a plan with default options on this grid
  const int rows = default_rows<float>(log_l, ny), ffts = default_ffts<float>(log_n, nx / 2 + 1);
  if (!schedule_valid<float>(log_l, log_n, ny, rows, ffts))
    return reject("no valid launch schedule for this grid");
  // an error left pending by earlier, unrelated work would otherwise be
  // reported by the launch checks below as if this call had caused it
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "a CUDA error was pending before this call");
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return reject("device index beyond the supported 64");
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress");
      if (!ptr) return cuda_error(cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
      e = Launch<float>::prepare();
      if (e != cudaSuccess) return cuda_error(e, "kernel attributes");
      g_scratch_addr[dev] = ptr;
    }
  }
  unsigned char* base = static_cast<unsigned char*>(g_scratch_addr[dev]);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool masked = which >= 2;
  k_static_setup<<<256, 256, 0, s>>>(base, L, ny, nx, P_half, masked ? observed : nullptr,
                                     (which == 1 || which == 3) ? 1 : 0, in, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "set-up kernel launch");
  const InstDesc<float>* desc = reinterpret_cast<const InstDesc<float>*>(base + L.desc);
  const float* tw = reinterpret_cast<const float*>(base + L.tw);
  const int lr = pow2_log(rows);
  RowArgs ra{ny, nx, rows, lr, masked ? OP_LOAD_W_MASK : OP_LOAD_W, SC_NONE, SKIP_NEVER, 0};
  e = Launch<float>::row(log_l, false, true, desc, 1, ra, tw, s);
  if (e != cudaSuccess) return cuda_error(e, "forward row pass");
  ColArgs ca{ny, nx / 2 + 1, ffts, 0, SKIP_NEVER, 0};
  e = Launch<float>::col(log_n, desc, 1, ca, tw, s);
  if (e != cudaSuccess) return cuda_error(e, "column pass");
  RowArgs rb{ny, nx, rows, lr, masked ? OP_STORE_Y_MASK : OP_STORE_Y, SC_NONE, SKIP_NEVER, 0};
  e = Launch<float>::row(log_l, true, false, desc, 1, rb, tw, s);
  if (e != cudaSuccess) return cuda_error(e, "inverse row pass");
  return FILL_OK;
}
