// Shared host/device data structures of the constrained-realization solver.
//
// Layout on the device, per realization ("instance"):
//   * full maps (d, y, w, out, gx): row-major ny x nx;
//   * CG vectors (r, p, q, z, u, b and the mixed-mode r32 / dlt): COMPACT,
//     one value per masked pixel in row-major order (the masked system of
//     Sect. 2.4 lives on M only; the vectors are zero on U);
//   * half spectrum "spec": transposed, (nx/2+1) rows of ny complex values,
//     spec[kx * ny + y]; the column pass runs along contiguous rows;
//   * spectral tables [kx][ky] (same transposed layout), real, with the
//     1/n of the inverse DFT folded in;
//   * mask words: for each 32 pixels, the observed bits (1 = constraint) and
//     the compact index of the word's first masked pixel.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define CGF_HD __host__ __device__
#else
#define CGF_HD
#endif

namespace cgf {

// Scalar state of one CG solve (Sect. 2.4), kept on the device so the
// iteration runs without host round trips.
struct CgState {
  double rho;      // r^T z of the current iterate
  double alpha;    // step length
  double beta;     // direction update
  double bb;       // ||b||^2
  double rr;       // ||r||^2 after the last update
  double tol2;     // tol^2 (stop when rr <= tol2 * bb)
  double pq;       // last p^T A p
  double rrmax;    // ||r||^2 at the last true-residual update (reliable updates)
  double delta2;   // update when rr <= delta2 * rrmax (reliable updates)
  int iter;        // completed operator applications
  int max_iter;
  int done;        // 1 once converged / stopped; later passes skip the instance
  int status;      // 0 ok, 1 invalid data (non-finite), 3 not converged, 4 breakdown
  int first;       // 1 before the first z: beta = 0
  int hist_cap;
  unsigned int ticket;  // last-CTA counter for the grid reductions
  int refine;      // true-residual recomputations (mixed mode)
  int total_iter;  // inner iterations summed over refinement steps
  int upd;         // reliable updates: update (high-precision state) / reload (FP32 state) due
  int last_iter;   // mixed mode, FP32 state: iterations of the last inner solve
  CgState* peer;   // the other precision's state of the same instance (mixed mode)
  double* hist;    // ||r_k|| / ||b||, k = 0..iter
  double* coef;    // CG coefficients: alpha_j at [2j], beta_j at [2j+1], j < hist_cap
};


// Double-float number hi + lo (|lo| <= ulp(hi) / 2, about 48 significant
// bits): the high-precision type of the mixed mode, whose arithmetic runs on
// the FP32 pipes (GB300's FP64 rate is 1/58 of its FP32 rate).
struct df {
  float hi, lo;
  df() = default;
  CGF_HD constexpr df(float h, float l) : hi(h), lo(l) {}
  CGF_HD constexpr df(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  CGF_HD constexpr df(float x) : hi(x), lo(0.f) {}
  CGF_HD constexpr df(int x) : df((double)x) {}
  CGF_HD explicit operator float() const { return hi + lo; }
  CGF_HD explicit operator double() const { return (double)hi + (double)lo; }
};
struct alignas(16) df2 {
  df x, y;
};

// Element type of the caller's maps (d, out, dL/dx) for a pass element type.
template <typename T>
struct MapOf {
  using type = T;
};
template <>
struct MapOf<df> {
  using type = double;
};

// Per-instance pointers handed to every kernel (element type T of the pass).
template <typename T>
struct InstDesc {
  const uint2* mw;         // mask words: x = observed bits, y = compact offset
  const T* t_inv;          // 1 / (n P)     [kx][ky]
  const T* t_sqrt;         // sqrt(P) / n   [kx][ky]
  T* spec;                 // interleaved complex half spectrum, transposed
  T* spec2;                // second spectrum (gradient products), or null
  T* r;
  T* p;
  T* q;
  T* z;
  T* u;
  T* y;
  T* b;
  const typename MapOf<T>::type* d;    // caller's data map
  typename MapOf<T>::type* out;        // caller's output map (dL/dd in the backward pass)
  const typename MapOf<T>::type* gx;   // caller's dL/dx (backward pass)
  T* w;                    // w = d - y on U, u on M (backward pass)
  float* dlt;              // FP32 correction (mixed mode, high-precision passes)
  float* r32;              // FP32 residual target (mixed mode, high-precision passes)
  CgState* st;
  double* partial;         // per-CTA partial sums
  double* hist;            // residual history (hist_cap entries), or null
  double* coef;            // CG coefficients (2 hist_cap entries), or null
  const T* kt;             // kernel tables [j][kx][ky] of the Sect. 6.3 solver, or null
  const uint8_t* cls;      // kernel class of every pixel (Sect. 6.3 solver), or null
  long long nvec;          // compact CG-vector length: masked pixels of this instance
  unsigned long long seed;
};

// Elementwise operations fused into the row passes (runtime-uniform switch).
enum RowOp : int {
  // sources (row pass without an input spectrum)
  OP_XI = 1,        // v = unit white noise (Philox4x32-10 + Box-Muller)
  OP_LOAD_R = 2,    // v = r
  OP_P_UPD_Z = 3,   // p = z + beta p; store p; v = p
  OP_P_UPD_R = 4,   // p = r + beta p; store p; v = p   (no preconditioner)
  OP_R_UPD = 5,     // r -= alpha q; u += alpha p; store; acc ||r||^2; v = r
  OP_U64_UPD = 6,   // u += dlt (FP32 correction); store; v = u  (mixed mode)
  OP_LOAD_W_MASK = 7,  // v = P_x w (full maps; operator checks)
  OP_LOAD_U = 8,    // v = u
  OP_LOAD_Y = 9,    // v = y
  OP_LOAD_D_U = 28, // v = d on U, 0 on M (maximum-likelihood right-hand side)
  // middles (input spectrum -> output spectrum)
  OP_MASK = 10,     // v = P_x v
  OP_Y_W = 11,      // store y = v; v = (d - y) on U, 0 on M
  // sinks (input spectrum, no output spectrum)
  OP_STORE_Y = 20,  // store y = v
  OP_STORE_Y_MASK = 27,  // store y = P_x v (full maps; operator checks)
  OP_Q = 21,        // q = P_x v; store; acc p^T q
  OP_Z = 22,        // z = P_x v; store; acc r^T z
  OP_B = 23,        // b = -P_x v; store r = b (and b); acc ||b||^2
  OP_RES = 24,      // r = b - P_x v; store; acc ||r||^2; r32 = (float) r
  OP_GRAD = 25,     // v = C^-1 lam: out = (g - v) on U, 0 on M; y = h = g on M, v on U
  OP_RELAX = 29,    // v = C^-1 w: w -= alpha v on M (alpha = 1/a, Sect. 5 relaxation);
                    // acc ||v_M||^2
  OP_KSEL = 30,     // v = kernel j * w: y = v on the masked pixels of class j (Sect. 6.3)
  OP_LOAD_W = 26,   // (source) v = w
};

// Scalar updates run by the last CTA of a reducing pass.
enum ScalarOp : int {
  SC_NONE = 0,
  SC_BB = 1,          // bb = sum; rr = bb; done if bb == 0
  SC_BB_RHO = 2,      // as SC_BB, plus rho = bb, beta = 0 (no preconditioner)
  SC_ALPHA = 3,       // pq = sum; alpha = rho / pq (breakdown if pq <= 0)
  SC_RCHECK = 4,      // rr = sum; iter++; convergence / iteration limit
  SC_RCHECK_BETA = 5, // SC_RCHECK, then beta = rr / rho; rho = rr
  SC_BETA = 6,        // rz = sum; beta = rz / rho (0 on the first); rho = rz
  SC_RES = 7,         // rr = sum (true residual); refine++; done if rr <= tol2 bb
  SC_RCHECK_UPD = 8,  // reliable updates, FP32 state: rr = sum; iter++; request an
                      // update when rr <= delta2 rrmax or rr <= tol2 bb or at max_iter
  SC_RES_UPD = 9,     // reliable updates, high-precision state: true residual; converged -> both
                      // done; else FP32 residual replaced, reload of its spectrum due
  SC_CLEAR_UPD = 10,  // upd = 0 (after the reload)
};

// Instance skipping of a pass: 0 never; 1 once the state is done;
// 2 unless an update is due (and the state is not done).
enum SkipMode : int { SKIP_NEVER = 0, SKIP_DONE = 1, SKIP_UNLESS_UPD = 2 };

enum VecOp : int {
  VOP_UPDATE = 1,     // r -= alpha q; u += alpha p; acc ||r||^2
  VOP_ASSEMBLE = 2,   // out = d on U, y + u on M
  VOP_COPY_D = 3,     // out = d
  VOP_MAKE_W = 5,     // w = d - y on U, u on M
  VOP_LOAD_G = 6,     // r = b = P_x g (r32 = (float) r if set); acc ||r||^2
  VOP_ZERO_UP = 7,    // u = 0, p = 0
  VOP_MAP_IN = 8,     // w = d (caller's map -> pass element type)
  VOP_MAP_OUT = 9,    // out = y (pass element type -> caller's map)
  VOP_W_FROM_D = 10,  // w = d on U, 0 on M
  VOP_W_TO_OUT = 11,  // out = w (pass element type -> caller's map)
  VOP_ANNULUS = 12,   // w = 1 where r_in^2 < |offset|^2 <= r_out^2 (offset from pixel 0), else 0
  VOP_Y_TO_W_M = 13,  // w = y on M; acc ||y - w||^2 over M
};

// Launch arguments of the pass kernels.
struct RowArgs {
  int ny, nx;       // grid (nx = 2 L)
  int rows;         // rows per CTA (power of two)
  int log_rows;     // log2(rows)
  int op;           // RowOp
  int sop;          // ScalarOp (SC_NONE: no reduction)
  int check_done;   // skip instances whose CG state is done
  int spec_sel;     // 0: spec, 1: spec2
  int param;        // op parameter (OP_KSEL: the kernel class)
};

struct ColArgs {
  int ny;           // column length (FFT size)
  int nkx;          // nx/2 + 1 spectrum rows
  int ffts;         // column FFTs per CTA
  int table;        // 0: 1/(nP), 1: sqrt(P)/n; j + 2: kernel table j; -1: forward only
  int check_done;
  int spec_sel;     // 0: spec, 1: spec2
  int pre;          // 1: the input is spec, already column-transformed (table >= 0; the
                    // forward FFT is skipped and the result goes to spec_sel's buffer)
  int* err;         // device error flag (set to 1 when a bounded wait gave up), or null
  int variant;      // FP32 table passes: 0 register-fed kernel, 1 persistent bulk-copy-fed
                    // kernel (chosen per grid by the autotuner)
};

// Band-binned spectral products for the band-power gradient.
struct DotArgs {
  long long nmodes;     // (nx/2+1) * ny half-plane modes per instance
  int nbands;
  const int* band;      // [kx][ky] band of every mode
  const void* coef;     // [kx][ky] weight (element type of the pass)
  double* part;         // [inst][cta][nbands] partial sums
};

struct VecArgs {
  long long npix;   // pixels per instance
  int op;           // VecOp
  int sop;
  int check_done;
  double p0, p1;    // op parameters (VOP_ANNULUS: r_in^2, r_out^2)
  int nx;           // row length (VOP_ANNULUS)
};

constexpr int kLmax = 8192;        // twiddle master table: W_8192^m

// Per-stage twiddle tables of the register-resident FFT (cg_fft.cuh), stored
// after the master table.  A transform of length 2^log (4 <= log <= 13) has
// one leading stage of radix 2^(log mod 4) (if nonzero) and log/4 radix-16
// stages; the radix-16 stage s runs on sub-transforms of size
// ns = 2^(log mod 4) 16^s and needs W_{16 ns}^(jm r), jm < ns, r = 1..15
// (none for the very first stage, ns = 1).  Its table holds them as
// [r - 1][jm], so that the threads of a warp (consecutive jm) read
// consecutive entries.
CGF_HD constexpr int stw_ns0(int log) { return (log % 4) ? (1 << (log % 4)) : 1; }
CGF_HD constexpr int stw_first(int log) { return (log % 4) ? 0 : 1; }   // first twiddled stage
CGF_HD constexpr int stw_ns(int log, int s) {
  int ns = stw_ns0(log);
  for (int t = 0; t < s; ++t) ns *= 16;
  return ns;
}
// entries of the stages before s of length 2^log
CGF_HD constexpr int stw_stage_off(int log, int s) {
  int o = 0;
  for (int t = stw_first(log); t < s; ++t) o += 15 * stw_ns(log, t);
  return o;
}
CGF_HD constexpr int stw_size(int log) { return stw_stage_off(log, log / 4); }
// entries of the lengths 2^4 .. 2^(log-1) (the tables of length 2^log start here)
CGF_HD constexpr int stw_base(int log) {
  int o = 0;
  for (int l = 4; l < log; ++l) o += stw_size(l);
  return o;
}
constexpr int kStwEntries = stw_base(14);   // all lengths 2^4 .. 2^13
constexpr int kTwEntries = kLmax + kStwEntries;   // complex entries of a twiddle buffer
constexpr int kMaxPartials = 4096; // CTAs per instance per reducing pass
constexpr int kMaxBands = 64;      // band-power gradient bins
constexpr int kDotCtas = 256;      // CTAs per instance of the band-binned product

}  // namespace cgf
