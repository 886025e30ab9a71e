// Mixed-radix grids: the pass kernels for nx / 2 and ny with prime factors
// 2, 3, 5 and 7 (for example 7000 x 600 = 2^3 5^3 7 x 2^3 3 5^2), which the
// power-of-two register FFTs of cg_kernels.cuh do not cover.
//
// Same passes, same operations and the same transposed half-spectrum layout
// as the power-of-two path (the CG loops in cgfill.cu call either through the
// same helpers): a ROW pass (real row <-> half spectrum, R2C / C2R by a
// half-length complex FFT, the elementwise operation of the pass fused in),
// a COLUMN pass (forward FFT, x real table, inverse FFT) and the inverse ROW
// pass.
//
// The transforms run in place in shared memory.  The forward transform is a
// decimation-in-frequency (Gentleman-Sande) factorisation n = R_0 R_1 ...
// R_{S-1}: stage s splits every block of n_s = R_s ... R_{S-1} points into R_s
// interleaved sub-blocks with butterflies of radix R_s, each thread reading
// and writing the same R_s positions, so no second buffer is needed.  Its
// output sits in digit-reversed order: position p = sum_s q_s h_s
// (h_s = n_{s+1}) holds frequency k = sum_s q_s R_0 ... R_{s-1}.  The inverse
// is the transposed factorisation (decimation in time, stages in reverse
// order, conjugate twiddles), which takes digit-reversed input to natural
// output.  The column pass chains the two with the spectral table applied at
// the digit-reversed positions, fusing the last forward stage, the table and
// the first inverse stage into one step; the row passes permute once, when
// they read or write the half spectrum (frequency k <-> position pos[k]).
//
// A thread group of g.nt threads works on V transforms at once (V rows, or V
// columns), their values interleaved in shared memory as [position][V]: a
// butterfly's index arithmetic and twiddles serve all V, and a position's V
// values move as one 16-byte access in FP32.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "cg_types.h"

namespace cgf {

constexpr int kGenMaxStages = 16;
constexpr int kGenMaxLen = 4096;   // nx / 2 and ny at most 4096

// One transform length: its stage radices (applied in this order by the
// forward transform), the offsets of the stages' twiddles in its table, the
// threads that share one group of V transforms, and the digit-reversal maps.
struct GenLen {
  int n;
  int nst;
  int nt;
  int code;   // radix schedule (gen_factor)
  int radix[kGenMaxStages];
  // Stage s < nst - 1: twiddles W_{n_s}^{q j} (j < h_s, q = 1 .. R_s - 1) at
  // complex entry twoff[s] + j (R_s - 1) + q - 1 of the table.  The last stage
  // (h = 1) has none.
  int twoff[kGenMaxStages];
  const unsigned short* rev;   // device, n entries: position -> frequency
  const unsigned short* pos;   // device, n entries: frequency -> position
};

// Factor n into stages and lay out the stage twiddles; false if n has a prime
// factor above 7.  The radix schedule `code`: radix-8 stages first unless bit
// 0 is set, then 4, 2, and the odd radices ascending (3, 5, 7), or descending
// with bit 1.  (The tables themselves and the digit-reversal maps are built
// with the plan; the threads per group, nt, are left as they are.)
bool gen_factor(int n, GenLen* g, int code = 0);
constexpr int kGenCodes = 4;

// Columns per thread group of the column pass: 2 in FP32 (a build-time
// width), 1 in FP64 and double-float (their butterflies already hold twice
// the registers).
#ifndef CGF_GEN_VCOL
#define CGF_GEN_VCOL 2
#endif
template <typename T>
constexpr int gen_v() { return std::is_same<T, float>::value ? CGF_GEN_VCOL : 1; }
// Rows per thread group of the row passes (FP32; FP64 and double-float 1).
#ifndef CGF_GEN_VROW
#define CGF_GEN_VROW 2
#endif
template <typename T>
constexpr int gen_vrow() { return std::is_same<T, float>::value ? CGF_GEN_VROW : 1; }
#ifndef CGF_GEN_THREADS
#define CGF_GEN_THREADS 256
#endif
#ifndef CGF_GEN_MINB
#define CGF_GEN_MINB 3
#endif
#ifndef CGF_GEN_COL_MINB
#define CGF_GEN_COL_MINB CGF_GEN_MINB
#endif
constexpr int kGenThreads = CGF_GEN_THREADS;   // most threads in one CTA
// CTAs per SM the row kernels are compiled for (registers per thread
// 65536 / (kGenThreads x this)): FP32, then FP64 and double-float; and the
// column kernels.
template <typename T>
constexpr int gen_minb() { return std::is_same<T, float>::value ? CGF_GEN_MINB : 2; }
template <typename T>
constexpr int gen_col_minb() { return std::is_same<T, float>::value ? CGF_GEN_COL_MINB : 2; }

template <typename T>
struct GenLaunch {
  // wl: table of nx / 2, wx: W_nx^k (k <= nx / 2), wn: table of ny.  Rows per
  // CTA (RowArgs::rows) are multiples of gen_vrow<T>(), columns per CTA
  // (ColArgs::ffts) of gen_v<T>().  The white-noise source (op OP_XI) runs its
  // own instantiation.
  static cudaError_t row(bool in_spec, bool out_spec, const InstDesc<T>* d, int ninst,
                         const RowArgs& a, const GenLen& g, const T* wl, const T* wx,
                         cudaStream_t s);
  static cudaError_t col(const InstDesc<T>* d, int ninst, const ColArgs& a, const GenLen& g,
                         const T* wn, cudaStream_t s);
  static size_t row_smem(int L, int rows);
  static size_t col_smem(int ny, int ffts);
  static int max_threads();
  static cudaError_t prepare();
};

}  // namespace cgf
