// Default launch schedule of the power-of-two passes, shared by the plans
// (cgfill.cu) and the plan-free operator entry point (cg_static.cu), so the
// two cannot drift apart.
#pragma once
#include <algorithm>

#include "cg_launch.h"
#include "cg_types.h"

namespace cgf {

// Row-pass CTA height: at least 16 rows or 256 threads, at most 512 threads
// (two CTAs per SM) unless that would leave fewer than 4 rows per CTA, and
// within the shared memory of a CTA.
template <typename T>
inline int default_rows(int log_l, int ny) {
  const int TT = (1 << log_l) / 16;
  int rows = std::max(16, 256 / TT);
  const int cap = std::min(512, Launch<T>::max_threads());
  rows = std::min(rows, std::max(cap / TT, std::min(4, Launch<T>::max_threads() / TT)));
  while (rows > 1 && Launch<T>::row_smem(log_l, rows) > 210 * 1024) rows /= 2;
  return std::min(rows, ny);
}

// Column FFTs per CTA: about 256 threads, within the thread and
// shared-memory limits.
template <typename T>
inline int default_ffts(int log_n, int nkx) {
  const int TT = (1 << log_n) / 16;
  int f = std::max(1, 256 / TT);
  f = std::min(f, std::max(1, Launch<T>::max_threads() / TT));
  while (f > 1 && Launch<T>::col_smem(log_n, f) > 100 * 1024) f /= 2;
  return std::min(f, nkx);
}

// Whether a (rows, ffts) schedule can be launched on an ny x nx grid.
template <typename T>
inline bool schedule_valid(int log_l, int log_n, int ny, int rows, int ffts) {
  const int TT = (1 << log_l) / 16, TN = (1 << log_n) / 16;
  return rows >= 1 && ffts >= 1 && rows * TT <= Launch<T>::max_threads() && ny % rows == 0 &&
         ny / rows <= kMaxPartials && Launch<T>::row_smem(log_l, rows) <= 227 * 1024 &&
         ffts * TN <= Launch<T>::max_threads() && Launch<T>::col_smem(log_n, ffts) <= 227 * 1024;
}

}  // namespace cgf
