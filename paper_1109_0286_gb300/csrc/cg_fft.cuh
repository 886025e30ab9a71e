// Register-resident complex FFT of length L = 2^LOG_L (16 <= L <= 8192) by a
// group of L/16 threads that each hold 16 elements.
//
// Stockham auto-sort formulation: a stage of radix R after sub-transforms of
// size Ns reads element j + r L/R, multiplies it by W_{Ns R}^{(j mod Ns) r},
// applies a length-R DFT and writes element (j div Ns) Ns R + (j mod Ns) + r Ns.
// The plan is one leading stage of radix 2^(LOG_L mod 4) (if nonzero) and then
// radix-16 stages.  On entry thread t holds x[t + e L/16] in v[e]; on exit it
// holds X[t + e L/16] -- the same positions -- so a forward transform, a
// diagonal multiply and an inverse transform chain without a shared-memory
// round trip.  Between stages data goes through shared memory (XBuf).  A
// radix-16 stage needs W^(jm r), r = 1..15: fifteen loads from its own
// table of correctly rounded values (stw_* in cg_types.h), or three master
// table entries and complex products (TAB = false).
#pragma once
#include "cg_common.cuh"

namespace cgf {

// Exchange area of one FFT in shared memory (PADL = L + L/16 + 1 words per
// component).  Element i lives at padded index i + i/16, which keeps every
// stage write (strides 1..16) and the strided stage reads free of bank
// conflicts for 8-byte elements.  FP32: interleaved complex (one 8-byte access
// per element); FP64: split real / imaginary arrays (8-byte accesses).
template <typename T> struct XBuf;

template <>
struct XBuf<float> {
  float2* c;
  __device__ __forceinline__ XBuf(float* base, int padl) : c(reinterpret_cast<float2*>(base)) {}
  __device__ __forceinline__ void st(int i, cx<float> v) const {
    c[i + (i >> 4)] = make_float2(v.r, v.i);
  }
  __device__ __forceinline__ cx<float> ld(int i) const {
    const float2 t = c[i + (i >> 4)];
    return {t.x, t.y};
  }
};

template <>
struct XBuf<double> {
  double* re;
  double* im;
  __device__ __forceinline__ XBuf(double* base, int padl) : re(base), im(base + padl) {}
  __device__ __forceinline__ void st(int i, cx<double> v) const {
    re[i + (i >> 4)] = v.r;
    im[i + (i >> 4)] = v.i;
  }
  __device__ __forceinline__ cx<double> ld(int i) const {
    return {re[i + (i >> 4)], im[i + (i >> 4)]};
  }
};

template <>
struct XBuf<df> {   // same layout as FP64: split real / imaginary arrays of 8-byte elements
  df* re;
  df* im;
  __device__ __forceinline__ XBuf(df* base, int padl) : re(base), im(base + padl) {}
  __device__ __forceinline__ void st(int i, cx<df> v) const {
    re[i + (i >> 4)] = v.r;
    im[i + (i >> 4)] = v.i;
  }
  __device__ __forceinline__ cx<df> ld(int i) const {
    return {re[i + (i >> 4)], im[i + (i >> 4)]};
  }
};

// Unpadded FP32 exchange area of one transform (L interleaved complex
// elements): element i lives at i ^ ((i >> 4) & 15).  The XOR keeps every
// access of fft_regs free of bank conflicts -- the contiguous stage reads,
// the stride-16 writes after the first radix-16 stage, the stride-R0 writes
// after a leading radix-2/4/8 stage -- without the padding of XBuf, so an
// area that received a contiguous TMA copy can serve as the exchange area.
struct XBufSw {
  float2* c;
  __device__ __forceinline__ explicit XBufSw(float2* base) : c(base) {}
  __device__ __forceinline__ void st(int i, cx<float> v) const {
    c[i ^ ((i >> 4) & 15)] = make_float2(v.r, v.i);
  }
  __device__ __forceinline__ cx<float> ld(int i) const {
    const float2 t = c[i ^ ((i >> 4) & 15)];
    return {t.x, t.y};
  }
};

// a * (-i) for the forward transform, a * (+i) for the inverse.
template <typename T, bool INV>
__device__ __forceinline__ cx<T> mul_mi(cx<T> a) {
  return INV ? cx<T>{-a.i, a.r} : cx<T>{a.i, -a.r};
}
// a * (c - i s) forward, a * (c + i s) inverse.
template <typename T, bool INV>
__device__ __forceinline__ cx<T> twc(cx<T> a, T c, T s) {
  return INV ? cx<T>{a.r * c - a.i * s, a.r * s + a.i * c}
             : cx<T>{a.r * c + a.i * s, a.i * c - a.r * s};
}

template <typename T, bool INV>
__device__ __forceinline__ void dft2(cx<T>& a, cx<T>& b) {
  cx<T> t = a;
  a = t + b;
  b = t - b;
}

template <typename T, bool INV>
__device__ __forceinline__ void dft4(cx<T>& a0, cx<T>& a1, cx<T>& a2, cx<T>& a3) {
  cx<T> s02 = a0 + a2, d02 = a0 - a2, s13 = a1 + a3;
  cx<T> d13 = mul_mi<T, INV>(a1 - a3);
  a0 = s02 + s13;
  a2 = s02 - s13;
  a1 = d02 + d13;
  a3 = d02 - d13;
}

// cos(pi/8), sin(pi/8), sqrt(1/2)
#define CGF_C8 0.92387953251128674
#define CGF_S8 0.38268343236508978
#define CGF_R2 0.70710678118654752

// Length-8 DFT, natural order in and out (8 = 2 x 4 split).
template <typename T, bool INV>
__device__ __forceinline__ void dft8(cx<T> (&v)[8]) {
  const T r2 = (T)CGF_R2;
  dft2<T, INV>(v[0], v[4]);
  dft2<T, INV>(v[1], v[5]);
  dft2<T, INV>(v[2], v[6]);
  dft2<T, INV>(v[3], v[7]);
  v[5] = twc<T, INV>(v[5], r2, r2);
  v[6] = mul_mi<T, INV>(v[6]);
  v[7] = twc<T, INV>(v[7], -r2, r2);
  dft4<T, INV>(v[0], v[1], v[2], v[3]);
  dft4<T, INV>(v[4], v[5], v[6], v[7]);
  cx<T> o[8] = {v[0], v[4], v[1], v[5], v[2], v[6], v[3], v[7]};
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = o[i];
}

// Length-16 DFT, natural order in and out (16 = 4 x 4 split:
// n = 4 n1 + n2, k = k1 + 4 k2, inner twiddles W16^(n2 k1)).
template <typename T, bool INV>
__device__ __forceinline__ void dft16(cx<T> (&v)[16]) {
  const T c = (T)CGF_C8, s = (T)CGF_S8, r2 = (T)CGF_R2;
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<T, INV>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
  v[5] = twc<T, INV>(v[5], c, s);      // W^1
  v[9] = twc<T, INV>(v[9], r2, r2);    // W^2
  v[13] = twc<T, INV>(v[13], s, c);    // W^3
  v[6] = twc<T, INV>(v[6], r2, r2);    // W^2
  v[10] = mul_mi<T, INV>(v[10]);       // W^4
  v[14] = twc<T, INV>(v[14], -r2, r2); // W^6
  v[7] = twc<T, INV>(v[7], s, c);      // W^3
  v[11] = twc<T, INV>(v[11], -r2, r2); // W^6
  v[15] = twc<T, INV>(v[15], -c, -s);  // W^9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<T, INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  cx<T> o[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) o[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = o[i];
}

template <typename T, int R, bool INV>
__device__ __forceinline__ void dft_small(cx<T> (&u)[R]) {
  if constexpr (R == 2) {
    dft2<T, INV>(u[0], u[1]);
  } else if constexpr (R == 4) {
    dft4<T, INV>(u[0], u[1], u[2], u[3]);
  } else {
    dft8<T, INV>(u);
  }
}

// W_kLmax^m = exp(-2 pi i m / kLmax), interleaved table.
template <typename T>
__device__ __forceinline__ cx<T> twiddle(const T* __restrict__ tw, int m) {
  return ldg_cx<T>(tw + 2 * m);
}

// W_32^e = exp(-2 pi i e / 32), e = 0..15: the factor W_nx^(e L/16) of the
// real-transform pre/post-processing.  In constant memory, so that with the
// element loops unrolled it is an instruction operand (no shared-memory or
// register traffic).
#define CGF_W32_TABLE(CAST)                                                             \
  {CAST(1.0), CAST(0.0)}, {CAST(0.980785280403230449126), CAST(-0.195090322016128267848)}, \
  {CAST(0.923879532511286756128), CAST(-0.382683432365089771728)},                        \
  {CAST(0.831469612302545237079), CAST(-0.555570233019602224743)},                        \
  {CAST(0.707106781186547524401), CAST(-0.707106781186547524401)},                        \
  {CAST(0.555570233019602224743), CAST(-0.831469612302545237079)},                        \
  {CAST(0.382683432365089771728), CAST(-0.923879532511286756128)},                        \
  {CAST(0.195090322016128267848), CAST(-0.980785280403230449126)},                        \
  {CAST(0.0), CAST(-1.0)}, {CAST(-0.195090322016128267848), CAST(-0.980785280403230449126)}, \
  {CAST(-0.382683432365089771728), CAST(-0.923879532511286756128)},                       \
  {CAST(-0.555570233019602224743), CAST(-0.831469612302545237079)},                       \
  {CAST(-0.707106781186547524401), CAST(-0.707106781186547524401)},                       \
  {CAST(-0.831469612302545237079), CAST(-0.555570233019602224743)},                       \
  {CAST(-0.923879532511286756128), CAST(-0.382683432365089771728)},                       \
  {CAST(-0.980785280403230449126), CAST(-0.195090322016128267848)}
#define CGF_AS_FLOAT(x) ((float)(x))
#define CGF_AS_DOUBLE(x) (x)
#define CGF_AS_DF(x) df(x)
static __constant__ float2 c_w32f[16] = {CGF_W32_TABLE(CGF_AS_FLOAT)};
static __constant__ double2 c_w32d[16] = {CGF_W32_TABLE(CGF_AS_DOUBLE)};
static __constant__ df2 c_w32h[16] = {CGF_W32_TABLE(CGF_AS_DF)};
#undef CGF_AS_DF
#undef CGF_AS_FLOAT
#undef CGF_AS_DOUBLE
#undef CGF_W32_TABLE

template <typename T>
__device__ __forceinline__ cx<T> w32(int e);
template <>
__device__ __forceinline__ cx<float> w32<float>(int e) {
  return {c_w32f[e].x, c_w32f[e].y};
}
template <>
__device__ __forceinline__ cx<double> w32<double>(int e) {
  return {c_w32d[e].x, c_w32d[e].y};
}
template <>
__device__ __forceinline__ cx<df> w32<df>(int e) {
  return {c_w32h[e].x, c_w32h[e].y};
}

// Barrier over the threads of one transform.  When a transform spans whole
// warps and a CTA holds at most 8 of them, each transform syncs on its own
// named barrier (1 + idx), so the transforms of a CTA advance independently;
// otherwise the whole CTA syncs.
struct XBar {
  int id, n;   // id 0: __syncthreads
  __device__ __forceinline__ void sync() const {
    if (id == 0)
      __syncthreads();
    else
      asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
  }
  static __device__ __forceinline__ XBar make(int tpt, int count, int idx) {
    return (tpt >= 32 && count > 1 && count <= 8) ? XBar{1 + idx, tpt} : XBar{0, 0};
  }
};

// TAB: twiddles from the per-stage tables (the row passes: 5-11% faster at
// 4096^2), else from three entries of the master table and complex products
// (the column passes: the tables' loads raise their register pressure into
// spills, 21% slower).
template <typename T, int LOG_L, bool INV, bool TAB = true, typename XB>
__device__ __forceinline__ void fft_regs(cx<T> (&v)[16], const XB& xb, int tid,
                                         const T* __restrict__ tw, XBar first = XBar{0, 0},
                                         XBar bar = XBar{0, 0}) {
  constexpr int TT = (1 << LOG_L) / 16;
  constexpr int S16 = LOG_L / 4;
  constexpr int REM = LOG_L % 4;
  constexpr int NS0 = REM > 0 ? (1 << REM) : 1;
  if constexpr (REM > 0) {
    constexpr int R0 = 1 << REM, NB = 16 / R0;
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      cx<T> u[R0];
#pragma unroll
      for (int r = 0; r < R0; ++r) u[r] = v[q + r * NB];
      dft_small<T, R0, INV>(u);
#pragma unroll
      for (int r = 0; r < R0; ++r) v[q + r * NB] = u[r];
    }
    first.sync();
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        xb.st((tid + q * TT) * R0 + r, v[q + r * NB]);
      }
  }
#pragma unroll
  for (int s = 0; s < S16; ++s) {
    int ns = NS0;
#pragma unroll
    for (int t = 0; t < s; ++t) ns *= 16;
    const bool first_stage = (REM == 0) && (s == 0);
    const bool last = (s == S16 - 1);
    if (!first_stage) {
      bar.sync();
#pragma unroll
      for (int e = 0; e < 16; ++e) v[e] = xb.ld(tid + e * TT);
      const int jm = tid & (ns - 1);
      // W_{16 ns}^(jm r), r = 1..15: correctly rounded entries of the stage's
      // table ([r - 1][jm]; consecutive jm of a warp read consecutive entries)
      if constexpr (TAB) {
        // Loaded in three groups of five, each applied before the next group is
        // issued (the empty asm with a memory clobber keeps the compiler from
        // hoisting all fifteen loads, which would need 30 more registers).
        const T* ts = tw + 2 * (kLmax + stw_base(LOG_L) + stw_stage_off(LOG_L, s) + jm);
#pragma unroll
        for (int g = 0; g < 3; ++g) {
          cx<T> w[5];
#pragma unroll
          for (int k = 0; k < 5; ++k) w[k] = ldg_cx<T>(ts + 2 * (5 * g + k) * ns);
#pragma unroll
          for (int k = 0; k < 5; ++k) {
            const int r = 5 * g + k + 1;
            v[r] = INV ? cmulc(v[r], w[k]) : cmul(v[r], w[k]);
          }
          asm volatile("" ::: "memory");
        }
      } else {
        // W^(jm r) from three master-table entries (W^jm, W^4jm, W^8jm) and at
        // most four complex products each (a few ulp)
        const int stride = kLmax / (ns * 16);
        cx<T> w[16];
        w[1] = twiddle<T>(tw, jm * stride);
        w[4] = twiddle<T>(tw, 4 * jm * stride);
        w[8] = twiddle<T>(tw, 8 * jm * stride);
        w[2] = cmul(w[1], w[1]);
        w[3] = cmul(w[2], w[1]);
        w[5] = cmul(w[4], w[1]);
        w[6] = cmul(w[4], w[2]);
        w[7] = cmul(w[4], w[3]);
#pragma unroll
        for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = INV ? cmulc(v[r], w[r]) : cmul(v[r], w[r]);
      }
    }
    dft16<T, INV>(v);
    if (!last) {
      if (REM == 0 && s == 0)
        first.sync();
      else
        bar.sync();
      const int jm = tid & (ns - 1);
      const int base = (tid - jm) * 16 + jm;
#pragma unroll
      for (int r = 0; r < 16; ++r) xb.st(base + r * ns, v[r]);
    }
  }
}

}  // namespace cgf
