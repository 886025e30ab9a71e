// Device building blocks: complex arithmetic, the Philox4x32-10 counter-based
// generator with Box-Muller normals, and reductions whose result is accurate
// to FP64 level.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "cg_types.h"

namespace cgf {

template <typename T>
struct cx {
  T r, i;
};

template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.r + b.r, a.i + b.i}; }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.r - b.r, a.i - b.i}; }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return {a.r * b.r + a.i * b.i, a.i * b.r - a.r * b.i};
}
template <typename T>
__device__ __forceinline__ cx<T> conjx(cx<T> a) { return {a.r, -a.i}; }
template <typename T>
__device__ __forceinline__ cx<T> scal(cx<T> a, T s) { return {a.r * s, a.i * s}; }

// Double-float arithmetic (error-free transformations: Knuth's TwoSum for
// the high parts, FMA-exact products; Dekker's renormalisation).  Relative
// error of an operation about 2^-46 of the operands' magnitude.
__device__ __forceinline__ df operator+(df a, df b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  const float e = ((a.hi - (s - v)) + (b.hi - v)) + (a.lo + b.lo);
  const float h = s + e;
  return df(h, e - (h - s));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)));
  const float h = p + e;
  return df(h, e - (h - p));
}

// Vector types for 8- / 16-byte global accesses.
template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };
template <> struct V2<df> { using t = df2; };

template <typename T>
__device__ __forceinline__ cx<T> ldg_cx(const T* p) {
  typename V2<T>::t v = __ldg(reinterpret_cast<const typename V2<T>::t*>(p));
  return {v.x, v.y};
}
// Read-only scalar load.
template <typename T>
__device__ __forceinline__ T ldg1(const T* p) { return __ldg(p); }
template <>
__device__ __forceinline__ df ldg1<df>(const df* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return df(v.x, v.y);
}
template <>
__device__ __forceinline__ cx<df> ldg_cx<df>(const df* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return {df(v.x, v.y), df(v.z, v.w)};
}
template <typename T>
__device__ __forceinline__ cx<T> ld_cx(const T* p) {
  typename V2<T>::t v = *reinterpret_cast<const typename V2<T>::t*>(p);
  return {v.x, v.y};
}
template <typename T>
__device__ __forceinline__ void st_cx(T* p, cx<T> a) {
  typename V2<T>::t v;
  v.x = a.r;
  v.y = a.i;
  *reinterpret_cast<typename V2<T>::t*>(p) = v;
}
// Real pixel pairs (2j, 2j+1) as one vector access.
template <typename T>
__device__ __forceinline__ void ld_pair(const T* p, T& a, T& b) {
  typename V2<T>::t v = *reinterpret_cast<const typename V2<T>::t*>(p);
  a = v.x;
  b = v.y;
}
template <typename T>
__device__ __forceinline__ void st_pair(T* p, T a, T b) {
  typename V2<T>::t v;
  v.x = a;
  v.y = b;
  *reinterpret_cast<typename V2<T>::t*>(p) = v;
}

// Complex load of data read once by this kernel: no allocation in L1, so the
// twiddle table cached there stays resident (coherent path: the kernel may
// write the same address after reading it).
template <typename T>
__device__ __forceinline__ cx<T> ld_stream_cx(const T* p);
template <>
__device__ __forceinline__ cx<float> ld_stream_cx<float>(const float* p) {
  float x, y;
  asm volatile("ld.global.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "l"(p));
  return {x, y};
}
template <>
__device__ __forceinline__ cx<double> ld_stream_cx<double>(const double* p) {
  double x, y;
  asm volatile("ld.global.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(x), "=d"(y) : "l"(p));
  return {x, y};
}
template <>
__device__ __forceinline__ cx<df> ld_stream_cx<df>(const df* p) {
  float a, b, c, d;
  asm volatile("ld.global.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(a), "=f"(b), "=f"(c), "=f"(d)
               : "l"(p));
  return {df(a, b), df(c, d)};
}

// Asks the copy engine to bring elements [c0, c1) of a vector into L2 (one
// instruction for the whole range; rounded out to 16-byte boundaries, which
// stay inside the vector's allocation since its length is padded to a
// multiple of 64 elements).
template <typename S>
__device__ __forceinline__ void prefetch_l2(const S* v, long long c0, long long c1) {
  if (!v || c1 <= c0) return;
  const uintptr_t b = reinterpret_cast<uintptr_t>(v + c0) & ~uintptr_t(15);
  const uintptr_t e = (reinterpret_cast<uintptr_t>(v + c1) + 15) & ~uintptr_t(15);
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b), "r"((uint32_t)(e - b))
               : "memory");
}

// Pixel pairs of the caller's maps, converted to / from the pass element type.
template <typename T>
__device__ __forceinline__ void ld_map_pair(const typename MapOf<T>::type* p, T& a, T& b) {
  using M = typename MapOf<T>::type;
  typename V2<M>::t v = *reinterpret_cast<const typename V2<M>::t*>(p);
  a = (T)v.x;
  b = (T)v.y;
}
template <typename T>
__device__ __forceinline__ void st_map_pair(typename MapOf<T>::type* p, T a, T b) {
  using M = typename MapOf<T>::type;
  typename V2<M>::t v;
  v.x = static_cast<M>(a);
  v.y = static_cast<M>(b);
  *reinterpret_cast<typename V2<M>::t*>(p) = v;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
// multiply/xor bijection on a 128-bit counter under a 64-bit key.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) {
      k.x += W0;
      k.y += W1;
    }
    uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Uniform in (0,1) from 52 random bits: ((a>>6) 2^26 + (b>>6) + 1/2) 2^-52.
__device__ __forceinline__ double uniform52(uint32_t a, uint32_t b) {
  double m = (double)(a >> 6) * 67108864.0 + (double)(b >> 6);
  return (m + 0.5) * 2.220446049250313080847263336181640625e-16;  // 2^-52
}

// Unit normals for pixels 2j and 2j+1 of the instance (row-major), counter
// (j, 0, 0, 0), key (seed lo, seed hi); Box-Muller in FP64.
__device__ __forceinline__ void normal_pair(unsigned long long seed, uint32_t j,
                                            double& x0, double& x1) {
  uint4 w = philox4x32_10(make_uint4(j, 0u, 0u, 0u),
                          make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  double u1 = uniform52(w.x, w.y), u2 = uniform52(w.z, w.w);
  double rad = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  x0 = rad * c;
  x1 = rad * s;
}

// ---------------------------------------------------------------------------
// Inner-product accumulators.  FP32 data: each product is split exactly into
// hi + lo (fma), and the running sum is a compensated FP32 pair, so that a
// thread's partial carries ~44 bits; partials then combine in FP64.  This
// keeps the reductions FP64-accurate without one FP64 instruction per
// element.  FP64 data: plain FP64 accumulation.
// ---------------------------------------------------------------------------
template <typename T> struct Acc;

template <>
struct Acc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    float p = a * b;
    float e = fmaf(a, b, -p);
    float t = hi + p;
    float bp = t - hi;
    float e2 = (hi - (t - bp)) + (p - bp);
    lo += e + e2;
    hi = t;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <>
struct Acc<df> {
  df s = df(0.f, 0.f);
  __device__ __forceinline__ void add_prod(df a, df b) { s = s + a * b; }
  __device__ __forceinline__ double value() const { return (double)s.hi + (double)s.lo; }
};

template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};

// Block-wide FP64 sum (all threads call; result valid in thread 0).
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // lanes present in this warp (the last warp may be partial)
  const int nl = min(32, (int)blockDim.x - (wid << 5));
  const unsigned mask = nl == 32 ? 0xffffffffu : ((1u << nl) - 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_down_sync(mask, v, o);
    if (lane + o < nl) v += t;
  }
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) s += sh[w];
  }
  return s;
}

// CG coefficient record for the Lanczos estimate (Sect. 6.4): alpha_j when
// computed (j = iterations completed so far), beta_j after iteration j.
__device__ __forceinline__ void record_alpha(CgState* st) {
  if (st->coef && st->iter < st->hist_cap) st->coef[2 * st->iter] = st->alpha;
}
__device__ __forceinline__ void record_beta(CgState* st) {
  if (st->coef && st->iter >= 1 && st->iter - 1 < st->hist_cap)
    st->coef[2 * (st->iter - 1) + 1] = st->beta;
}

// Scalar update executed once per instance by the last CTA of a pass, with
// the sum of all CTA partials (fixed order, so results are reproducible).
__device__ __forceinline__ void scalar_update(int sop, CgState* st, double sum) {
  switch (sop) {
    case SC_BB:
    case SC_BB_RHO:
      st->bb = sum;
      st->rr = sum;
      st->rrmax = sum;
      if (st->hist && st->hist_cap > 0) st->hist[0] = sum > 0.0 ? 1.0 : 0.0;
      if (!isfinite(sum)) {
        st->done = 1;
        st->status = 1;  // FILL_EINVAL: NaN / Inf in the data (P is validated on the host)
      } else if (sum == 0.0) {
        st->done = 1;    // nothing to solve: u = 0
      }
      if (sop == SC_BB_RHO) {   // plain CG: z = r, rho = ||r||^2, p = r
        st->rho = sum;
        st->beta = 0.0;
        st->first = 0;
      }
      break;
    case SC_ALPHA:
      st->pq = sum;
      if (!(sum > 0.0) || !isfinite(sum)) {
        st->status = 4;
        st->done = 1;
      } else {
        st->alpha = st->rho / sum;
        record_alpha(st);
      }
      break;
    case SC_RCHECK:
    case SC_RCHECK_BETA: {
      st->rr = sum;
      st->iter += 1;
      if (st->hist && st->iter < st->hist_cap) st->hist[st->iter] = sqrt(sum / st->bb);
      if (!isfinite(sum)) {
        st->status = 4;
        st->done = 1;
      } else if (sum <= st->tol2 * st->bb) {
        st->done = 1;
      } else if (st->iter >= st->max_iter) {
        st->status = 3;
        st->done = 1;
      } else if (sop == SC_RCHECK_BETA) {
        st->beta = sum / st->rho;
        st->rho = sum;
        record_beta(st);
      }
      break;
    }
    case SC_BETA:
      if (!(sum > 0.0) || !isfinite(sum)) {
        st->status = 4;
        st->done = 1;
      } else if (st->first) {
        st->first = 0;
        st->rho = sum;
        st->beta = 0.0;
      } else {
        st->beta = sum / st->rho;
        st->rho = sum;
        record_beta(st);
      }
      break;
    case SC_RCHECK_UPD: {
      st->rr = sum;
      st->iter += 1;
      if (st->hist && st->iter < st->hist_cap) st->hist[st->iter] = sqrt(sum / st->bb);
      if (!isfinite(sum)) {
        st->status = 4;
        st->done = 1;
        st->peer->upd = 1;   // fold what was gained and report the true residual
      } else if (sum <= st->delta2 * st->rrmax || sum <= st->tol2 * st->bb) {
        st->peer->upd = 1;
      } else if (st->iter >= st->max_iter) {
        st->status = 3;
        st->done = 1;
        st->peer->upd = 1;
      }
      break;
    }
    case SC_RES_UPD: {
      CgState* f = st->peer;
      st->rr = sum;
      st->upd = 0;
      st->refine += 1;
      if (st->hist && st->refine < st->hist_cap) st->hist[st->refine] = sqrt(sum / st->bb);
      if (!isfinite(sum)) {
        st->status = 4;
        st->done = 1;
        f->done = 1;
      } else if (sum <= st->tol2 * st->bb) {
        st->done = 1;
        f->done = 1;
      } else if (!f->done) {
        f->rr = sum;
        f->rrmax = sum;
        f->upd = 1;
      }
      break;
    }
    case SC_CLEAR_UPD:
      st->upd = 0;
      break;
    case SC_RES:
      st->rr = sum;
      st->refine += 1;
      if (st->hist && st->refine < st->hist_cap) st->hist[st->refine] = sqrt(sum / st->bb);
      if (!isfinite(sum)) {
        st->status = 4;
        st->done = 1;
      } else if (sum <= st->tol2 * st->bb) {
        st->done = 1;
      }
      break;
    default:
      break;
  }
}

// Whether a pass skips this instance (SkipMode).
__device__ __forceinline__ bool skip_instance(int mode, const CgState* st) {
  if (mode == SKIP_NEVER) return false;
  const int done = *(volatile const int*)&st->done;
  if (mode == SKIP_DONE) return done != 0;
  return done != 0 || *(volatile const int*)&st->upd == 0;
}

// Writes this CTA's partial; the last CTA of the instance sums all partials in
// order and runs the scalar update.  Called by all threads of the CTA.
__device__ __forceinline__ void grid_reduce(double v, double* sh, double* partial,
                                            CgState* st, int sop, int ncta, int cta) {
  double s = block_sum(v, sh);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partial[cta] = s;
    __threadfence();
    unsigned int t = atomicAdd(&st->ticket, 1u);
    last = (t == (unsigned int)(ncta - 1));
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double tot = 0.0;
    volatile double* vp = partial;
    for (int c = 0; c < ncta; ++c) tot += vp[c];
    st->ticket = 0u;
    scalar_update(sop, st, tot);
  }
}

}  // namespace cgf
