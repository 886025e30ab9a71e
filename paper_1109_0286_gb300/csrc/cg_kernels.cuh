// Fused FFT passes of the masked operator (Sect. 2.4, eq. ModEq):
//
//   C^s v = F^-1 diag(P^s) F v on the periodic grid (exact unitarity, Sect. 4)
//
// is split into a ROW pass (real row <-> half-spectrum row, R2C / C2R by a
// half-length complex FFT), a COLUMN pass (forward column FFT, multiply by the
// real table, inverse column FFT, all in registers), and the inverse ROW pass.
// The row passes write / read the half spectrum transposed (kx-major), so the
// column pass streams contiguous rows.  Everything elementwise -- the mask
// projections P_x, the white-noise draw, the CG vector updates and the inner
// products -- is fused into the row passes.
#pragma once
#include "cg_fft.cuh"

namespace cgf {

template <typename T> struct KCfg;
template <> struct KCfg<float> { static constexpr int kMaxThreads = 1024; };
template <> struct KCfg<double> { static constexpr int kMaxThreads = 512; };

__device__ __forceinline__ bool observed_bit(const uint32_t* __restrict__ obs, long long pix) {
  return (__ldg(obs + (pix >> 5)) >> (pix & 31)) & 1u;
}

// ----------------------------------------------------------------- sources
// A source op produces the real values fed to the forward row transform.
// Loads and compute/stores are split so that a chunk of pixel pairs issues
// all its loads before any of its stores (the loads then overlap).
template <typename T>
struct SrcIn {
  T x0, x1, y0, y1, z0, z1, w0, w1;
};

template <typename T>
__device__ __forceinline__ void src_load(int op, const InstDesc<T>& I, long long pix, SrcIn<T>& in) {
  switch (op) {
    case OP_LOAD_R_MASK:
    case OP_LOAD_R:
      ld_pair(I.r + pix, in.x0, in.x1);
      break;
    case OP_LOAD_U:
      ld_pair(I.u + pix, in.x0, in.x1);
      break;
    case OP_LOAD_Y:
      ld_pair(I.y + pix, in.x0, in.x1);
      break;
    case OP_LOAD_W:
      ld_pair(I.w + pix, in.x0, in.x1);
      break;
    case OP_P_UPD_Z:
    case OP_P_UPD_R:
      ld_pair((op == OP_P_UPD_Z ? I.z : I.r) + pix, in.x0, in.x1);
      ld_pair(I.p + pix, in.y0, in.y1);
      break;
    case OP_R_UPD:
      ld_pair(I.r + pix, in.x0, in.x1);
      ld_pair(I.q + pix, in.y0, in.y1);
      ld_pair(I.u + pix, in.z0, in.z1);
      ld_pair(I.p + pix, in.w0, in.w1);
      break;
    case OP_U64_UPD: {
      ld_pair(I.u + pix, in.x0, in.x1);
      const float2 dl = *reinterpret_cast<const float2*>(I.dlt + pix);
      in.y0 = (T)dl.x;
      in.y1 = (T)dl.y;
      break;
    }
    default:
      break;
  }
}

template <typename T>
__device__ __forceinline__ void src_apply(int op, const InstDesc<T>& I, long long pix,
                                          const SrcIn<T>& in, T alpha, T beta, T& a0, T& a1,
                                          Acc<T>& acc) {
  switch (op) {
    case OP_LOAD_R_MASK: {
      const uint32_t w = __ldg(I.obs + (pix >> 5));
      a0 = ((w >> (pix & 31)) & 1u) ? (T)0 : in.x0;
      a1 = ((w >> ((pix + 1) & 31)) & 1u) ? (T)0 : in.x1;
      break;
    }
    case OP_LOAD_R:
      a0 = in.x0;
      a1 = in.x1;
      acc.add_prod(a0, a0);
      acc.add_prod(a1, a1);
      break;
    case OP_LOAD_U:
    case OP_LOAD_Y:
    case OP_LOAD_W:
      a0 = in.x0;
      a1 = in.x1;
      break;
    case OP_P_UPD_Z:
    case OP_P_UPD_R:
      a0 = in.x0 + beta * in.y0;
      a1 = in.x1 + beta * in.y1;
      st_pair(I.p + pix, a0, a1);
      break;
    case OP_R_UPD:
      a0 = in.x0 - alpha * in.y0;
      a1 = in.x1 - alpha * in.y1;
      st_pair(I.r + pix, a0, a1);
      st_pair(I.u + pix, in.z0 + alpha * in.w0, in.z1 + alpha * in.w1);
      acc.add_prod(a0, a0);
      acc.add_prod(a1, a1);
      break;
    case OP_U64_UPD:
      a0 = in.x0 + in.y0;
      a1 = in.x1 + in.y1;
      st_pair(I.u + pix, a0, a1);
      *reinterpret_cast<float2*>(I.dlt + pix) = make_float2(0.f, 0.f);   // folded
      break;
    default:
      a0 = a1 = (T)0;
  }
}

// ----------------------------------------------------------------- middles / sinks
template <typename T>
struct SinkIn {
  T x0, x1;
  uint32_t w;
};

template <typename T>
__device__ __forceinline__ void sink_load(int op, const InstDesc<T>& I, long long pix, SinkIn<T>& in) {
  in.w = __ldg(I.obs + (pix >> 5));
  switch (op) {
    case OP_Y_W:
      ld_pair(I.d + pix, in.x0, in.x1);
      break;
    case OP_Q:
      ld_pair(I.p + pix, in.x0, in.x1);
      break;
    case OP_Z:
      ld_pair(I.r + pix, in.x0, in.x1);
      break;
    case OP_RES:
      ld_pair(I.b + pix, in.x0, in.x1);
      break;
    case OP_GRAD:
      ld_pair(I.gx + pix, in.x0, in.x1);
      break;
    default:
      break;
  }
}

template <typename T>
__device__ __forceinline__ void sink_apply(int op, const InstDesc<T>& I, long long pix,
                                           const SinkIn<T>& in, T& a0, T& a1, Acc<T>& acc) {
  const bool o0 = (in.w >> (pix & 31)) & 1u, o1 = (in.w >> ((pix + 1) & 31)) & 1u;
  switch (op) {
    case OP_MASK:
      a0 = o0 ? (T)0 : a0;
      a1 = o1 ? (T)0 : a1;
      break;
    case OP_Y_W:
      st_pair(I.y + pix, a0, a1);
      a0 = o0 ? in.x0 - a0 : (T)0;
      a1 = o1 ? in.x1 - a1 : (T)0;
      break;
    case OP_STORE_Y:
      st_pair(I.y + pix, a0, a1);
      break;
    case OP_Q:
    case OP_Z:
      a0 = o0 ? (T)0 : a0;
      a1 = o1 ? (T)0 : a1;
      st_pair((op == OP_Q ? I.q : I.z) + pix, a0, a1);
      acc.add_prod(in.x0, a0);
      acc.add_prod(in.x1, a1);
      break;
    case OP_B:
      a0 = o0 ? (T)0 : -a0;
      a1 = o1 ? (T)0 : -a1;
      st_pair(I.r + pix, a0, a1);
      if (I.b) st_pair(I.b + pix, a0, a1);
      if (I.r32) *reinterpret_cast<float2*>(I.r32 + pix) = make_float2((float)a0, (float)a1);
      acc.add_prod(a0, a0);
      acc.add_prod(a1, a1);
      break;
    case OP_RES:
      a0 = in.x0 - (o0 ? (T)0 : a0);
      a1 = in.x1 - (o1 ? (T)0 : a1);
      st_pair(I.r + pix, a0, a1);
      if (I.r32) *reinterpret_cast<float2*>(I.r32 + pix) = make_float2((float)a0, (float)a1);
      acc.add_prod(a0, a0);
      acc.add_prod(a1, a1);
      break;
    case OP_GRAD:
      // v = C^-1 lam.  dL/dd_U = g_U - (C^-1 lam)_U, dL/dd_M = 0;
      // dL/dy = h = g on M, (C^-1 lam)_U on U (kept in y).
      st_pair(I.out + pix, o0 ? in.x0 - a0 : (T)0, o1 ? in.x1 - a1 : (T)0);
      st_pair(I.y + pix, o0 ? a0 : in.x0, o1 ? a1 : in.x1);
      break;
    default:
      break;
  }
}

// ----------------------------------------------------------------- row pass
// CTA = `rows` consecutive grid rows, L/16 threads per row; blockIdx.y is the
// instance.  Shared memory: per-row FFT exchange areas, aliased with the
// transposed tile [(L+1) x (rows+1)] used for the spectrum load / store.
// XI: the source is the seed's white noise (kept out of the other source
// kernels, whose register allocation it would otherwise burden).
template <typename T, int LOG_L, bool IN_SPEC, bool OUT_SPEC, bool XI = false>
__global__ void __launch_bounds__(KCfg<T>::kMaxThreads)
k_row(const InstDesc<T>* __restrict__ insts, RowArgs a, const T* __restrict__ tw) {
  constexpr int L = 1 << LOG_L, TT = L / 16, PADL = L + L / 16 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  __shared__ double red[32];
  __shared__ cx<T> wcol[16];   // W_nx^(e TT), e = 0..15 (warp-uniform factor)
  const InstDesc<T>& I = insts[blockIdx.y];
  if (skip_instance(a.check_done, I.st)) return;

  const int rows = a.rows;
  const int row = threadIdx.x / TT, tid = threadIdx.x - row * TT;
  const int y0 = blockIdx.x * rows, y = y0 + row;
  const int ny = a.ny, nx = a.nx;
  const int tstride = rows + 1;
  const XBuf<T> xb(sm + row * 2 * PADL, PADL);
  T* tre = sm;
  T* tim = sm + (L + 1) * tstride;
  constexpr int TWS = kLmax / (2 * L);   // W_{nx}^k = table[k * TWS]
  const long long rowpix = (long long)y * nx;

  cx<T> v[16];
  Acc<T> acc;

  if constexpr (IN_SPEC) {
    const T* spec = a.spec_sel ? I.spec2 : I.spec;
    for (int e = threadIdx.x; e < (L + 1) * rows; e += blockDim.x) {
      const int k = e / rows, rr = e - k * rows;
      const cx<T> s = ld_cx<T>(spec + 2 * ((long long)k * ny + y0 + rr));
      tre[k * tstride + rr] = s.r;
      tim[k * tstride + rr] = s.i;
    }
    if (threadIdx.x < 16) wcol[threadIdx.x] = twiddle<T>(tw, threadIdx.x * TT * TWS);
    __syncthreads();
    // C2R: Z[k] = (X[k] + conj X[L-k]) + i e^{+2 pi i k / nx} (X[k] - conj X[L-k])
    const cx<T> wt = twiddle<T>(tw, tid * TWS);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int k = tid + e * TT;
      cx<T> xk{tre[k * tstride + row], tim[k * tstride + row]};
      cx<T> xc{tre[(L - k) * tstride + row], -tim[(L - k) * tstride + row]};
      if (k == 0) {
        xk.i = (T)0;
        xc.i = (T)0;
      }
      const cx<T> w = cmul(wt, wcol[e]);   // W_nx^k, k = tid + e TT
      const cx<T> sum = xk + xc;
      const cx<T> dif = cmulc(xk - xc, w);  // (X - conj X') e^{+i...}
      v[e] = cx<T>{sum.r - dif.i, sum.i + dif.r};
    }
    fft_regs<T, LOG_L, true>(v, xb, tid, tw);
    // v[e] = x[2j] + i x[2j+1], j = tid + e TT
    constexpr int CK = 4;   // pixel pairs whose loads are issued together
#pragma unroll
    for (int h = 0; h < 16; h += CK) {
      SinkIn<T> in[CK];
#pragma unroll
      for (int e = 0; e < CK; ++e) sink_load<T>(a.op, I, rowpix + 2 * (tid + (h + e) * TT), in[e]);
#pragma unroll
      for (int e = 0; e < CK; ++e)
        sink_apply<T>(a.op, I, rowpix + 2 * (tid + (h + e) * TT), in[e], v[h + e].r, v[h + e].i, acc);
    }
  } else if constexpr (XI) {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      double x0, x1;
      normal_pair(I.seed, (uint32_t)((rowpix >> 1) + tid + e * TT), x0, x1);
      v[e] = cx<T>{(T)x0, (T)x1};
    }
  } else {
    const T alpha = (T)I.st->alpha, beta = (T)I.st->beta;
    constexpr int CK = 2;   // pixel pairs whose loads are issued together
#pragma unroll
    for (int h = 0; h < 16; h += CK) {
      SrcIn<T> in[CK];
#pragma unroll
      for (int e = 0; e < CK; ++e) src_load<T>(a.op, I, rowpix + 2 * (tid + (h + e) * TT), in[e]);
#pragma unroll
      for (int e = 0; e < CK; ++e)
        src_apply<T>(a.op, I, rowpix + 2 * (tid + (h + e) * TT), in[e], alpha, beta, v[h + e].r,
                     v[h + e].i, acc);
    }
  }

  if constexpr (OUT_SPEC) {
    if (!IN_SPEC && threadIdx.x < 16) wcol[threadIdx.x] = twiddle<T>(tw, threadIdx.x * TT * TWS);
    fft_regs<T, LOG_L, false>(v, xb, tid, tw);
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) xb.st(tid + e * TT, v[e]);
    __syncthreads();
    const cx<T> wt = twiddle<T>(tw, tid * TWS);
    // R2C: X[k] = (Z[k] + conj Z[L-k]) / 2 - (i/2) e^{-2 pi i k/nx} (Z[k] - conj Z[L-k])
    cx<T> nyq{v[0].r - v[0].i, (T)0};
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int k = tid + e * TT;
      const cx<T> zc = conjx(xb.ld((L - k) & (L - 1)));
      const cx<T> zk = v[e];
      const cx<T> ev = scal(zk + zc, (T)0.5);
      const cx<T> od = scal(mul_mi<T, false>(zk - zc), (T)0.5);
      v[e] = ev + cmul(od, cmul(wt, wcol[e]));
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int k = tid + e * TT;
      tre[k * tstride + row] = v[e].r;
      tim[k * tstride + row] = v[e].i;
    }
    if (tid == 0) {
      tre[L * tstride + row] = nyq.r;
      tim[L * tstride + row] = nyq.i;
    }
    __syncthreads();
    T* spec = a.spec_sel ? I.spec2 : I.spec;
    for (int e = threadIdx.x; e < (L + 1) * rows; e += blockDim.x) {
      const int k = e / rows, rr = e - k * rows;
      st_cx<T>(spec + 2 * ((long long)k * ny + y0 + rr),
               cx<T>{tre[k * tstride + rr], tim[k * tstride + rr]});
    }
  }

  if (a.sop != SC_NONE)
    grid_reduce(acc.value(), red, I.partial, I.st, a.sop, gridDim.x, blockIdx.x);
}

// ----------------------------------------------------------------- column pass
// CTA = `ffts` spectrum rows (one kx each), N/16 threads per row; forward
// column FFT, multiply by the real table, inverse column FFT, in place
// (table < 0: forward transform only).
template <typename T, int LOG_N>
__global__ void __launch_bounds__(KCfg<T>::kMaxThreads)
k_col(const InstDesc<T>* __restrict__ insts, ColArgs a, const T* __restrict__ tw) {
  constexpr int N = 1 << LOG_N, TT = N / 16, PADN = N + N / 16 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const InstDesc<T>& I = insts[blockIdx.y];
  if (skip_instance(a.check_done, I.st)) return;
  const int f = threadIdx.x / TT, tid = threadIdx.x - f * TT;
  const int kx = blockIdx.x * a.ffts + f;
  const bool act = kx < a.nkx;
  const XBuf<T> xb(sm + f * 2 * PADN, PADN);
  T* col = (a.spec_sel ? I.spec2 : I.spec) + 2 * (long long)(act ? kx : 0) * N;
  cx<T> v[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) v[e] = act ? ld_cx<T>(col + 2 * (tid + e * TT)) : cx<T>{(T)0, (T)0};
  fft_regs<T, LOG_N, false>(v, xb, tid, tw);
  if (a.table >= 0) {
    const T* tab = (a.table ? I.t_sqrt : I.t_inv) + (long long)(act ? kx : 0) * N;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const T t = act ? __ldg(tab + tid + e * TT) : (T)0;
      v[e] = scal(v[e], t);
    }
    fft_regs<T, LOG_N, true>(v, xb, tid, tw);
  }
  if (act) {
#pragma unroll
    for (int e = 0; e < 16; ++e) st_cx<T>(col + 2 * (tid + e * TT), v[e]);
  }
}

// ----------------------------------------------------------------- elementwise
template <typename T>
__global__ void __launch_bounds__(256)
k_vec(const InstDesc<T>* __restrict__ insts, VecArgs a) {
  __shared__ double red[32];
  const InstDesc<T>& I = insts[blockIdx.y];
  if (skip_instance(a.check_done, I.st)) return;
  Acc<T> acc;
  const T alpha = (T)I.st->alpha;
  const long long npair = a.npix >> 1;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < npair;
       j += (long long)gridDim.x * blockDim.x) {
    const long long pix = 2 * j;
    switch (a.op) {
      case VOP_UPDATE: {
        T r0, r1, q0, q1, u0, u1, p0, p1;
        ld_pair(I.r + pix, r0, r1);
        ld_pair(I.q + pix, q0, q1);
        ld_pair(I.u + pix, u0, u1);
        ld_pair(I.p + pix, p0, p1);
        r0 -= alpha * q0;
        r1 -= alpha * q1;
        st_pair(I.r + pix, r0, r1);
        st_pair(I.u + pix, u0 + alpha * p0, u1 + alpha * p1);
        acc.add_prod(r0, r0);
        acc.add_prod(r1, r1);
        break;
      }
      case VOP_ASSEMBLE: {
        const uint32_t w = __ldg(I.obs + (pix >> 5));
        const bool o0 = (w >> (pix & 31)) & 1u, o1 = (w >> ((pix + 1) & 31)) & 1u;
        T d0, d1, y0, y1, u0, u1;
        ld_pair(I.d + pix, d0, d1);
        ld_pair(I.y + pix, y0, y1);
        ld_pair(I.u + pix, u0, u1);
        st_pair(I.out + pix, o0 ? d0 : y0 + u0, o1 ? d1 : y1 + u1);
        break;
      }
      case VOP_MAKE_W: {
        const uint32_t w = __ldg(I.obs + (pix >> 5));
        const bool o0 = (w >> (pix & 31)) & 1u, o1 = (w >> ((pix + 1) & 31)) & 1u;
        T d0, d1, y0, y1, u0, u1;
        ld_pair(I.d + pix, d0, d1);
        ld_pair(I.y + pix, y0, y1);
        ld_pair(I.u + pix, u0, u1);
        st_pair(I.w + pix, o0 ? d0 - y0 : u0, o1 ? d1 - y1 : u1);
        break;
      }
      case VOP_LOAD_G: {
        const uint32_t w = __ldg(I.obs + (pix >> 5));
        const bool o0 = (w >> (pix & 31)) & 1u, o1 = (w >> ((pix + 1) & 31)) & 1u;
        T g0, g1;
        ld_pair(I.gx + pix, g0, g1);
        g0 = o0 ? (T)0 : g0;
        g1 = o1 ? (T)0 : g1;
        st_pair(I.r + pix, g0, g1);
        st_pair(I.b + pix, g0, g1);
        if (I.r32) *reinterpret_cast<float2*>(I.r32 + pix) = make_float2((float)g0, (float)g1);
        acc.add_prod(g0, g0);
        acc.add_prod(g1, g1);
        break;
      }
      case VOP_ZERO_UP:
        st_pair(I.u + pix, (T)0, (T)0);
        st_pair(I.p + pix, (T)0, (T)0);
        break;
      case VOP_COPY_D: {
        T d0, d1;
        ld_pair(I.d + pix, d0, d1);
        st_pair(I.out + pix, d0, d1);
        break;
      }
      default:
        break;
    }
  }
  if (a.sop != SC_NONE)
    grid_reduce(acc.value(), red, I.partial, I.st, a.sop, gridDim.x, blockIdx.x);
}

// ----------------------------------------------------------------- band products
// part[inst][cta][b] = sum over the CTA's half-plane modes k with band(k) = b
// of coef(k) Re(conj(spec(k)) spec2(k)); both spectra are full 2D transforms
// in the transposed layout, coef carries the Hermitian weight (1 on the two
// self-conjugate columns, 2 elsewhere).
template <typename T>
__global__ void __launch_bounds__(256)
k_band_dot(const InstDesc<T>* __restrict__ insts, DotArgs a) {
  __shared__ double hist[kMaxBands];
  const InstDesc<T>& I = insts[blockIdx.y];
  for (int b = threadIdx.x; b < a.nbands; b += blockDim.x) hist[b] = 0.0;
  __syncthreads();
  const T* coef = reinterpret_cast<const T*>(a.coef);
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < a.nmodes;
       m += (long long)gridDim.x * blockDim.x) {
    const cx<T> x = ld_cx<T>(I.spec + 2 * m), z = ld_cx<T>(I.spec2 + 2 * m);
    const double v = (double)((x.r * z.r + x.i * z.i) * __ldg(coef + m));
    atomicAdd(&hist[__ldg(a.band + m)], v);
  }
  __syncthreads();
  double* out = a.part + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * a.nbands;
  for (int b = threadIdx.x; b < a.nbands; b += blockDim.x) out[b] = hist[b];
}

}  // namespace cgf
