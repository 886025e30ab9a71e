// Mixed-radix grids: the pass kernels for nx / 2 and ny with prime factors
// 2, 3, 5 and 7 (for example 7000 x 600 = 2^3 5^3 7 x 2^3 3 5^2), which the
// power-of-two register FFTs of cg_kernels.cuh do not cover.
//
// Same passes, same operations and the same transposed half-spectrum layout
// as the power-of-two path (the CG loops in cgfill.cu call either through the
// same helpers): a ROW pass (real row <-> half spectrum, R2C / C2R by a
// half-length complex FFT, the elementwise operation of the pass fused in),
// a COLUMN pass (forward FFT, x real table, inverse FFT) and the inverse ROW
// pass.  The transforms are self-sorting (Stockham) mixed-radix FFTs in shared
// memory: stages of radix 4, 2, 3, 5, 7, each thread taking whole butterflies,
// two buffers ping-ponged between stages, twiddles W_n^t from a table built in
// FP64 on the host.
#pragma once
#include <cuda_runtime.h>

#include "cg_types.h"

namespace cgf {

constexpr int kGenMaxStages = 24;
constexpr int kGenMaxLen = 4096;   // nx / 2 and ny at most 4096

// One transform length: its stage radices (applied in this order) and the
// threads that share one transform.
struct GenLen {
  int n;
  int nst;
  int nt;
  int radix[kGenMaxStages];
};

// Factor n into radix-4, 2, 3, 5, 7 stages; false if n has another prime factor.
bool gen_factor(int n, GenLen* g);

template <typename T>
struct GenLaunch {
  // wl: W_L^t (t < L), wx: W_nx^k (k <= L), wn: W_ny^t (t < ny); complex, interleaved.
  // The white-noise source (op OP_XI) runs its own instantiation.
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
