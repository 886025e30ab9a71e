// Subdivision of the masked region by distance from the observed region
// (Sect. 6.2): the observed indicator convolved with the normalised top hat of
// radius delta/2 (periodic), thresholded on the masked pixels.  The convolution
// at a pixel is the count of observed pixels in the disc around it over the
// disc's pixel count; the count is taken exactly from per-row prefix sums, one
// horizontal chord of the disc per row offset, so the threshold test is exact.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/cgfill.h"

void cgf_set_last_error(const char* msg);

namespace {

// Half-width of the disc's chord at row offset dy: the largest h with
// h^2 + dy^2 <= r^2.
__host__ __device__ inline int chord(double r2, int dy) {
  const double v = r2 - double(dy) * double(dy);
  if (v < 0.0) return -1;
  int h = (int)floor(sqrt(v));
  while (double(h + 1) * double(h + 1) <= v) ++h;
  while (h > 0 && double(h) * double(h) > v) --h;
  return h;
}

// pre[y][x] = number of observed pixels in row y left of column x (nx + 1 per row).
__global__ void k_row_prefix(const uint8_t* __restrict__ obs, int nx, int* __restrict__ pre) {
  __shared__ int part[1024];
  const int y = blockIdx.x, t = threadIdx.x, nt = blockDim.x;
  const int chunk = (nx + nt - 1) / nt, x0 = t * chunk, x1 = min(nx, x0 + chunk);
  const uint8_t* row = obs + (size_t)y * nx;
  int s = 0;
  for (int x = x0; x < x1; ++x) s += row[x] ? 1 : 0;
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {   // inclusive scan of the chunk sums
    const int v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - s;                      // exclusive prefix of this chunk
  int* out = pre + (size_t)y * (nx + 1);
  if (t == 0) out[0] = 0;
  for (int x = x0; x < x1; ++x) {
    run += row[x] ? 1 : 0;
    out[x + 1] = run;
  }
}

__global__ void k_layer(const uint8_t* __restrict__ obs, const int* __restrict__ pre, int ny,
                        int nx, double r2, int R, long long thr100, long long disc,
                        uint8_t* __restrict__ layer) {
  const long long n = (long long)ny * nx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / nx), x = (int)(i % nx);
    if (obs[i]) {
      layer[i] = 0;
      continue;
    }
    long long count = 0;
    for (int dy = -R; dy <= R; ++dy) {
      const int h = chord(r2, dy);
      if (h < 0) continue;
      const int yy = ((y + dy) % ny + ny) % ny;
      const int* p = pre + (size_t)yy * (nx + 1);
      const int a = x - h, b = x + h;   // inclusive, |a|, |b - nx| <= h < nx
      if (a < 0)
        count += p[nx] - p[a + nx] + p[b + 1];
      else if (b >= nx)
        count += p[nx] - p[a] + p[b - nx + 1];
      else
        count += p[b + 1] - p[a];
    }
    layer[i] = count * 100 > thr100 * disc ? 1 : 0;
  }
}

}  // namespace

extern "C" fill_status fill_subdivide(int ny, int nx, const uint8_t* observed, double delta,
                                      double threshold, int32_t* scratch, uint8_t* layer,
                                      void* stream) {
  const double r = delta / 2.0;
  const int R = (int)floor(r);
  if (ny < 1 || nx < 1 || nx > 65536 || !observed || !scratch || !layer || !(delta >= 0.0) ||
      !(threshold >= 0.0) || 2 * R + 1 > ny || 2 * R + 1 > nx) {
    cgf_set_last_error("fill_subdivide: bad sizes or pointers (the disc must fit the grid)");
    return FILL_EINVAL;
  }
  const double r2 = r * r;
  long long disc = 0;
  for (int dy = -R; dy <= R; ++dy) disc += 2 * chord(r2, dy) + 1;
  const long long thr100 = llround(threshold * 100.0);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_row_prefix<<<ny, 1024, 0, s>>>(observed, nx, reinterpret_cast<int*>(scratch));
  if (cudaGetLastError() != cudaSuccess) return FILL_ECUDA;
  k_layer<<<1024, 256, 0, s>>>(observed, reinterpret_cast<const int*>(scratch), ny, nx, r2, R,
                               thr100, disc, layer);
  if (cudaGetLastError() != cudaSuccess) return FILL_ECUDA;
  return FILL_OK;
}
