// Size dispatch: runtime log2 sizes -> compile-time kernel instantiations.
#pragma once
#include <type_traits>

#include "cg_kernels.cuh"
#include "cg_launch.h"

namespace cgf {

template <typename T>
size_t Launch<T>::row_smem(int log_l, int rows) {
  // FFT areas / transposed tile, then one mask word (8 bytes) per thread
  const size_t tt = (size_t(1) << log_l) / 16;
  return row_main_bytes<T>(log_l, rows) + size_t(rows) * tt * sizeof(uint2);
}

template <typename T>
size_t Launch<T>::col_smem(int log_n, int ffts) {
  const size_t N = size_t(1) << log_n;
  return size_t(ffts) * 2 * (N + N / 16 + 1) * sizeof(T);
}

template <typename T>
int Launch<T>::max_threads() { return KCfg<T>::kMaxThreads; }

namespace detail {

// Opt the kernel in to the largest dynamic shared memory the device allows
// next to its static shared memory.
template <typename K>
inline cudaError_t allow_smem(K kernel) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

template <typename T, int LL>
cudaError_t row_ll(bool in_spec, bool out_spec, const InstDesc<T>* d, int ninst, const RowArgs& a,
                   const T* tw, cudaStream_t s) {
  constexpr int TT = (1 << LL) / 16;
  dim3 grid(a.ny / a.rows, ninst), block(a.rows * TT);
  const size_t sm = Launch<T>::row_smem(LL, a.rows);
  if (in_spec && out_spec)
    k_row<T, LL, true, true><<<grid, block, sm, s>>>(d, a, tw);
  else if (in_spec)
    k_row<T, LL, true, false><<<grid, block, sm, s>>>(d, a, tw);
  else if (a.op == OP_XI)
    k_row<T, LL, false, true, true><<<grid, block, sm, s>>>(d, a, tw);
  else
    k_row<T, LL, false, true><<<grid, block, sm, s>>>(d, a, tw);
  return cudaGetLastError();
}

// Persistent CTAs of the TMA column pass (SMs x resident CTAs), per log2 N;
// set by prepare_cols.
static int g_col_tma_ctas[14] = {};

// Column FFTs per item of the TMA column pass: F N = 4096 complex values
// (256 threads) when N <= 4096, one 8192-point column otherwise.
inline int col_tma_ffts(int log_n) { return log_n >= 12 ? 1 : (4096 >> log_n); }

template <int LN>
cudaError_t prep_col_tma() {
  const int F = col_tma_ffts(LN), threads = F * ((1 << LN) / 16);
  const size_t sm = col_tma_smem(LN, F);
  cudaError_t e = cudaFuncSetAttribute(k_col_tma<LN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  int dev = 0, sms = 0, per = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_col_tma<LN>, threads, sm);
  if (e == cudaSuccess) g_col_tma_ctas[LN] = sms * (per > 0 ? per : 1);
  return e;
}

template <typename T, int LN>
cudaError_t col_ln(const InstDesc<T>* d, int ninst, const ColArgs& a, const T* tw, cudaStream_t s) {
  constexpr int TT = (1 << LN) / 16;
  if constexpr (std::is_same<T, float>::value) {
    // the CG loops' table passes: persistent, bulk-copy fed
    if (a.variant == 1 && (a.table == 0 || a.table == 1) && !a.pre && a.spec_sel == 0 &&
        g_col_tma_ctas[LN] > 0) {
      const int F = col_tma_ffts(LN);
      ColArgs b = a;
      b.ffts = F;
      const long long items = (long long)((a.nkx + F - 1) / F) * ninst;
      const int grid = (int)(items < g_col_tma_ctas[LN] ? items : g_col_tma_ctas[LN]);
      k_col_tma<LN><<<grid, F * TT, col_tma_smem(LN, F), s>>>(d, b, tw, ninst);
      return cudaGetLastError();
    }
  }
  dim3 grid(ninst, (a.nkx + a.ffts - 1) / a.ffts), block(a.ffts * TT);
  const size_t sm = Launch<T>::col_smem(LN, a.ffts);
  if (a.pre)
    k_col<T, LN, true><<<grid, block, sm, s>>>(d, a, tw);
  else
    k_col<T, LN><<<grid, block, sm, s>>>(d, a, tw);
  return cudaGetLastError();
}

template <typename T, int LL>
cudaError_t prep_row() {
  cudaError_t e = allow_smem(k_row<T, LL, true, true>);
  if (e == cudaSuccess) e = allow_smem(k_row<T, LL, true, false>);
  if (e == cudaSuccess) e = allow_smem(k_row<T, LL, false, true>);
  if (e == cudaSuccess) e = allow_smem(k_row<T, LL, false, true, true>);
  return e;
}

}  // namespace detail

#define CGF_ROW_CASE(LL) \
  case LL: return detail::row_ll<T, LL>(in_spec, out_spec, d, ninst, a, tw, s);
template <typename T>
cudaError_t Launch<T>::row(int log_l, bool in_spec, bool out_spec, const InstDesc<T>* d, int ninst,
                           const RowArgs& a, const T* tw, cudaStream_t s) {
  switch (log_l) {
    CGF_ROW_CASE(4) CGF_ROW_CASE(5) CGF_ROW_CASE(6) CGF_ROW_CASE(7) CGF_ROW_CASE(8)
    CGF_ROW_CASE(9) CGF_ROW_CASE(10) CGF_ROW_CASE(11) CGF_ROW_CASE(12)
    default: return cudaErrorInvalidValue;
  }
}
#undef CGF_ROW_CASE

#define CGF_COL_CASE(LN) \
  case LN: return detail::col_ln<T, LN>(d, ninst, a, tw, s);
template <typename T>
cudaError_t Launch<T>::col(int log_n, const InstDesc<T>* d, int ninst, const ColArgs& a,
                           const T* tw, cudaStream_t s) {
  switch (log_n) {
    CGF_COL_CASE(4) CGF_COL_CASE(5) CGF_COL_CASE(6) CGF_COL_CASE(7) CGF_COL_CASE(8)
    CGF_COL_CASE(9) CGF_COL_CASE(10) CGF_COL_CASE(11) CGF_COL_CASE(12) CGF_COL_CASE(13)
    default: return cudaErrorInvalidValue;
  }
}
#undef CGF_COL_CASE

template <typename T>
cudaError_t Launch<T>::vec(const InstDesc<T>* d, int ninst, const VecArgs& a, int nblk, cudaStream_t s) {
  k_vec<T><<<dim3(nblk, ninst), 256, 0, s>>>(d, a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::band_dot(const InstDesc<T>* d, int ninst, const DotArgs& a, cudaStream_t s) {
  k_band_dot<T><<<dim3(kDotCtas, ninst), kDotThreads, 0, s>>>(d, a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::prepare_rows() {
  cudaError_t e = cudaSuccess;
#define CGF_PREP_ROW(LL) if (e == cudaSuccess) e = detail::prep_row<T, LL>();
  CGF_PREP_ROW(4) CGF_PREP_ROW(5) CGF_PREP_ROW(6) CGF_PREP_ROW(7) CGF_PREP_ROW(8)
  CGF_PREP_ROW(9) CGF_PREP_ROW(10) CGF_PREP_ROW(11) CGF_PREP_ROW(12)
#undef CGF_PREP_ROW
  return e;
}

template <typename T>
cudaError_t Launch<T>::prepare_cols() {
  cudaError_t e = cudaSuccess;
  if constexpr (std::is_same<T, float>::value) {
#define CGF_PREP_TMA(LN) if (e == cudaSuccess) e = detail::prep_col_tma<LN>();
    CGF_PREP_TMA(4) CGF_PREP_TMA(5) CGF_PREP_TMA(6) CGF_PREP_TMA(7) CGF_PREP_TMA(8)
    CGF_PREP_TMA(9) CGF_PREP_TMA(10) CGF_PREP_TMA(11) CGF_PREP_TMA(12) CGF_PREP_TMA(13)
#undef CGF_PREP_TMA
  }
#define CGF_PREP_COL(LN)                                             \
  if (e == cudaSuccess) e = detail::allow_smem(k_col<T, LN>);        \
  if (e == cudaSuccess) e = detail::allow_smem(k_col<T, LN, true>);
  CGF_PREP_COL(4) CGF_PREP_COL(5) CGF_PREP_COL(6) CGF_PREP_COL(7) CGF_PREP_COL(8)
  CGF_PREP_COL(9) CGF_PREP_COL(10) CGF_PREP_COL(11) CGF_PREP_COL(12) CGF_PREP_COL(13)
#undef CGF_PREP_COL
  return e;
}

// Row-pass kernels of one transform length LL = log2(nx/2): explicit
// instantiation (EXT empty) in the unit that compiles them, or an extern
// declaration (EXT = extern) where they are only called, so that the lengths
// can be spread over several translation units that compile in parallel.
#define CGF_ROW_LL(EXT, T, LL)                                                              \
  EXT template cudaError_t detail::row_ll<T, LL>(bool, bool, const InstDesc<T>*, int,       \
                                                 const RowArgs&, const T*, cudaStream_t);   \
  EXT template cudaError_t detail::prep_row<T, LL>();
#define CGF_ROW_EXTERN_ALL(T)                                                               \
  CGF_ROW_LL(extern, T, 4) CGF_ROW_LL(extern, T, 5) CGF_ROW_LL(extern, T, 6)                \
  CGF_ROW_LL(extern, T, 7) CGF_ROW_LL(extern, T, 8) CGF_ROW_LL(extern, T, 9)                \
  CGF_ROW_LL(extern, T, 10) CGF_ROW_LL(extern, T, 11) CGF_ROW_LL(extern, T, 12)

// Explicit instantiation of one precision's row-pass dispatch or column-pass
// members.
#define CGF_INSTANTIATE_ROWS(T)                                                             \
  CGF_ROW_EXTERN_ALL(T)                                                                     \
  template cudaError_t Launch<T>::row(int, bool, bool, const InstDesc<T>*, int,             \
                                      const RowArgs&, const T*, cudaStream_t);              \
  template cudaError_t Launch<T>::prepare_rows();                                           \
  template size_t Launch<T>::row_smem(int, int);
#define CGF_INSTANTIATE_COLS(T)                                                             \
  template cudaError_t Launch<T>::col(int, const InstDesc<T>*, int, const ColArgs&,         \
                                      const T*, cudaStream_t);                              \
  template cudaError_t Launch<T>::vec(const InstDesc<T>*, int, const VecArgs&, int,         \
                                      cudaStream_t);                                        \
  template cudaError_t Launch<T>::band_dot(const InstDesc<T>*, int, const DotArgs&,         \
                                           cudaStream_t);                                   \
  template cudaError_t Launch<T>::prepare_cols();                                           \
  template size_t Launch<T>::col_smem(int, int);                                            \
  template int Launch<T>::max_threads();

}  // namespace cgf
