// Host-side launchers for the pass kernels, one instantiation set per
// precision, each split into a row-pass and a column-pass translation unit
// (cg_launch_{f32,f64,df}_{row,col}.cu) so that they compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "cg_types.h"

namespace cgf {


template <typename T>
struct Launch {
  // log_l = log2(nx/2) in [4, 12]; log_n = log2(ny) in [4, 13].
  static cudaError_t row(int log_l, bool in_spec, bool out_spec, const InstDesc<T>* d, int ninst,
                         const RowArgs& a, const T* tw, cudaStream_t s);
  static cudaError_t col(int log_n, const InstDesc<T>* d, int ninst, const ColArgs& a,
                         const T* tw, cudaStream_t s);
  static cudaError_t vec(const InstDesc<T>* d, int ninst, const VecArgs& a, int nblk, cudaStream_t s);
  static cudaError_t band_dot(const InstDesc<T>* d, int ninst, const DotArgs& a, cudaStream_t s);
  static size_t row_smem(int log_l, int rows);
  static size_t col_smem(int log_n, int ffts);
  static int max_threads();
  // Raise the dynamic shared-memory limit of every kernel once (not a stream op).
  static cudaError_t prepare() {
    cudaError_t e = prepare_rows();
    return e == cudaSuccess ? prepare_cols() : e;
  }
  static cudaError_t prepare_rows();   // the row-pass kernels
  static cudaError_t prepare_cols();   // the column-pass kernels
};

}  // namespace cgf
