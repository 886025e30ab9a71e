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

// Masked flags and compact CG-vector indices of the pixel pair (pix, pix+1)
// (pix even): one 8-byte mask-word load and a popcount.
struct PairIdx {
  bool m0, m1;   // pixel masked (to fill)
  int i0, i1;    // compact indices (valid where masked)
};

__device__ __forceinline__ PairIdx pair_from_word(uint2 w, int pix) {
  const int b = (int)(pix & 31);
  const uint32_t mb = ~w.x;
  PairIdx q;
  q.m0 = (mb >> b) & 1u;
  q.m1 = (mb >> (b + 1)) & 1u;
  q.i0 = (int)w.y + __popc(mb & ((1u << b) - 1u));
  q.i1 = q.i0 + (q.m0 ? 1 : 0);
  return q;
}

__device__ __forceinline__ uint2 mask_word(const uint2* __restrict__ mw, int pix) {
  return __ldg(mw + (pix >> 5));
}

__device__ __forceinline__ PairIdx pair_index(const uint2* __restrict__ mw, int pix) {
  return pair_from_word(mask_word(mw, pix), pix);
}

// Compact loads / stores of a pixel pair (zero / nothing on observed pixels).
template <typename T, typename S>
__device__ __forceinline__ void ldc(const S* v, const PairIdx& q, T& a0, T& a1) {
  a0 = q.m0 ? (T)v[q.i0] : (T)0;
  a1 = q.m1 ? (T)v[q.i1] : (T)0;
}
template <typename T, typename S>
__device__ __forceinline__ void stc(S* v, const PairIdx& q, T a0, T a1) {
  if (q.m0) v[q.i0] = (S)a0;
  if (q.m1) v[q.i1] = (S)a1;
}

// ----------------------------------------------------------------- sources
// A source op produces the real values fed to the forward row transform.
// Loads and compute/stores are split so that a chunk of pixel pairs issues
// all its loads before any of its stores (the loads then overlap).
template <typename T>
struct SrcIn {
  uint2 w;   // mask word (indices recomputed where needed)
  T x0, x1, y0, y1, z0, z1, w0, w1;
};

template <typename T>
__device__ __forceinline__ void src_load(int op, const InstDesc<T>& I, int pix, SrcIn<T>& in) {
  switch (op) {
    case OP_LOAD_W_MASK:
      in.w = mask_word(I.mw, pix);
      ld_pair(I.w + pix, in.x0, in.x1);
      break;
    case OP_LOAD_Y:
      ld_pair(I.y + pix, in.x0, in.x1);
      break;
    case OP_LOAD_W:
      ld_pair(I.w + pix, in.x0, in.x1);
      break;
    case OP_LOAD_R:
    case OP_LOAD_U: {
      in.w = mask_word(I.mw, pix);
      const PairIdx q = pair_from_word(in.w, pix);
      ldc(op == OP_LOAD_R ? I.r : I.u, q, in.x0, in.x1);
      break;
    }
    case OP_P_UPD_Z:
    case OP_P_UPD_R: {
      in.w = mask_word(I.mw, pix);
      const PairIdx q = pair_from_word(in.w, pix);
      ldc(op == OP_P_UPD_Z ? I.z : I.r, q, in.x0, in.x1);
      ldc(I.p, q, in.y0, in.y1);
      break;
    }
    case OP_R_UPD: {
      in.w = mask_word(I.mw, pix);
      const PairIdx q = pair_from_word(in.w, pix);
      ldc(I.r, q, in.x0, in.x1);
      ldc(I.q, q, in.y0, in.y1);
      ldc(I.u, q, in.z0, in.z1);
      ldc(I.p, q, in.w0, in.w1);
      break;
    }
    case OP_U64_UPD: {
      in.w = mask_word(I.mw, pix);
      const PairIdx q = pair_from_word(in.w, pix);
      ldc(I.u, q, in.x0, in.x1);
      ldc(I.dlt, q, in.y0, in.y1);
      break;
    }
    default:
      break;
  }
}

template <typename T>
__device__ __forceinline__ void src_apply(int op, const InstDesc<T>& I, int pix,
                                          const SrcIn<T>& in, T alpha, T beta, T& a0, T& a1,
                                          Acc<T>& acc) {
  switch (op) {
    case OP_LOAD_W_MASK: {
      const PairIdx q = pair_from_word(in.w, pix);
      a0 = q.m0 ? in.x0 : (T)0;
      a1 = q.m1 ? in.x1 : (T)0;
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
      stc(I.p, pair_from_word(in.w, pix), a0, a1);
      break;
    case OP_R_UPD: {
      const PairIdx q = pair_from_word(in.w, pix);
      a0 = in.x0 - alpha * in.y0;
      a1 = in.x1 - alpha * in.y1;
      stc(I.r, q, a0, a1);
      stc(I.u, q, in.z0 + alpha * in.w0, in.z1 + alpha * in.w1);
      acc.add_prod(a0, a0);
      acc.add_prod(a1, a1);
      break;
    }
    case OP_U64_UPD: {
      const PairIdx q = pair_from_word(in.w, pix);
      a0 = in.x0 + in.y0;
      a1 = in.x1 + in.y1;
      stc(I.u, q, a0, a1);
      stc(I.dlt, q, 0.f, 0.f);   // folded
      break;
    }
    default:
      a0 = a1 = (T)0;
  }
}

// ----------------------------------------------------------------- middles / sinks
template <typename T>
struct SinkIn {
  uint2 w;   // mask word (indices recomputed where needed)
  T x0, x1;
};

template <typename T>
__device__ __forceinline__ void sink_load(int op, const InstDesc<T>& I, int pix, SinkIn<T>& in) {
  in.w = mask_word(I.mw, pix);
  switch (op) {
    case OP_Y_W:
      ld_pair(I.d + pix, in.x0, in.x1);
      break;
    case OP_Q:
      ldc(I.p, pair_from_word(in.w, pix), in.x0, in.x1);
      break;
    case OP_Z:
      ldc(I.r, pair_from_word(in.w, pix), in.x0, in.x1);
      break;
    case OP_RES:
      ldc(I.b, pair_from_word(in.w, pix), in.x0, in.x1);
      break;
    case OP_GRAD:
      ld_pair(I.gx + pix, in.x0, in.x1);
      break;
    default:
      break;
  }
}

template <typename T>
__device__ __forceinline__ void sink_apply(int op, const InstDesc<T>& I, int pix,
                                           const SinkIn<T>& in, T& a0, T& a1, Acc<T>& acc) {
  const int b = (int)(pix & 31);
  const bool o0 = (in.w.x >> b) & 1u, o1 = (in.w.x >> (b + 1)) & 1u;   // observed
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
    case OP_STORE_Y_MASK:
      st_pair(I.y + pix, o0 ? (T)0 : a0, o1 ? (T)0 : a1);
      break;
    case OP_Q:
    case OP_Z:
      a0 = o0 ? (T)0 : a0;
      a1 = o1 ? (T)0 : a1;
      stc(op == OP_Q ? I.q : I.z, pair_from_word(in.w, pix), a0, a1);
      acc.add_prod(in.x0, a0);
      acc.add_prod(in.x1, a1);
      break;
    case OP_B:
      a0 = o0 ? (T)0 : -a0;
      a1 = o1 ? (T)0 : -a1;
      {
        const PairIdx q = pair_from_word(in.w, pix);
        stc(I.r, q, a0, a1);
        if (I.b) stc(I.b, q, a0, a1);
        if (I.r32) stc(I.r32, q, a0, a1);
      }
      acc.add_prod(a0, a0);
      acc.add_prod(a1, a1);
      break;
    case OP_RES:
      a0 = in.x0 - (o0 ? (T)0 : a0);
      a1 = in.x1 - (o1 ? (T)0 : a1);
      {
        const PairIdx q = pair_from_word(in.w, pix);
        stc(I.r, q, a0, a1);
        if (I.r32) stc(I.r32, q, a0, a1);
      }
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

  const int rows = a.rows, lr = a.log_rows;
  const int row = threadIdx.x / TT, tid = threadIdx.x - row * TT;
  const int y0 = blockIdx.x * rows, y = y0 + row;
  const int ny = a.ny, nx = a.nx;
  const int tstride = rows + 1;
  const XBuf<T> xb(sm + row * 2 * PADL, PADL);
  cx<T>* tile = reinterpret_cast<cx<T>*>(sm);   // [(L+1)][rows+1], aliases the FFT areas
  constexpr int TWS = kLmax / (2 * L);   // W_{nx}^k = table[k * TWS]
  const int rowpix = y * nx;
  cx<T> v[16];
  Acc<T> acc;

  if constexpr (IN_SPEC) {
    const T* spec = (a.spec_sel ? I.spec2 : I.spec) + 2 * y0;
    for (int e = threadIdx.x; e < (L + 1) * rows; e += blockDim.x) {
      const int k = e >> lr, rr = e & (rows - 1);
      tile[k * tstride + rr] = ld_cx<T>(spec + 2 * (k * ny + rr));
    }
    if (threadIdx.x < 16) wcol[threadIdx.x] = twiddle<T>(tw, threadIdx.x * TT * TWS);
    __syncthreads();
    // C2R: Z[k] = (X[k] + conj X[L-k]) + i e^{+2 pi i k / nx} (X[k] - conj X[L-k])
    const cx<T> wt = twiddle<T>(tw, tid * TWS);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int k = tid + e * TT;
      cx<T> xk = tile[k * tstride + row];
      cx<T> xc = conjx(tile[(L - k) * tstride + row]);
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
    if constexpr (OUT_SPEC) {
      // middle of a chain: P_x (OP_MASK) or y = v, v = (d - y) on U (OP_Y_W)
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int pix = rowpix + 2 * (tid + e * TT);
        const uint32_t ob = __ldg(&I.mw[pix >> 5].x);
        const int b = (int)(pix & 31);
        const bool o0 = (ob >> b) & 1u, o1 = (ob >> (b + 1)) & 1u;
        if (a.op == OP_Y_W) {
          T d0, d1;
          ld_pair(I.d + pix, d0, d1);
          st_pair(I.y + pix, v[e].r, v[e].i);
          v[e].r = o0 ? d0 - v[e].r : (T)0;
          v[e].i = o1 ? d1 - v[e].i : (T)0;
        } else {
          v[e].r = o0 ? (T)0 : v[e].r;
          v[e].i = o1 ? (T)0 : v[e].i;
        }
      }
    } else {
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
    for (int e = 0; e < 16; ++e) tile[(tid + e * TT) * tstride + row] = v[e];
    if (tid == 0) tile[L * tstride + row] = nyq;
    __syncthreads();
    T* spec = (a.spec_sel ? I.spec2 : I.spec) + 2 * y0;
    for (int e = threadIdx.x; e < (L + 1) * rows; e += blockDim.x) {
      const int k = e >> lr, rr = e & (rows - 1);
      st_cx<T>(spec + 2 * (k * ny + rr), tile[k * tstride + rr]);
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
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gstride = (long long)gridDim.x * blockDim.x;
  if (a.op == VOP_UPDATE || a.op == VOP_ZERO_UP) {
    // compact CG vectors: one element per masked pixel
    const T alpha = (T)I.st->alpha;
    for (long long i = gid; i < I.nvec; i += gstride) {
      if (a.op == VOP_ZERO_UP) {
        I.u[i] = (T)0;
        I.p[i] = (T)0;
      } else {
        const T r = I.r[i] - alpha * I.q[i];
        I.r[i] = r;
        I.u[i] = I.u[i] + alpha * I.p[i];
        acc.add_prod(r, r);
      }
    }
  } else {
    // pixel pairs of the full maps
    for (long long j = gid; j < (a.npix >> 1); j += gstride) {
      const int pix = 2 * j;
      const PairIdx q = pair_index(I.mw, pix);
      switch (a.op) {
        case VOP_ASSEMBLE: {
          T d0, d1, y0, y1, u0, u1;
          ld_pair(I.d + pix, d0, d1);
          ld_pair(I.y + pix, y0, y1);
          ldc(I.u, q, u0, u1);
          st_pair(I.out + pix, q.m0 ? y0 + u0 : d0, q.m1 ? y1 + u1 : d1);
          break;
        }
        case VOP_COPY_D: {
          T d0, d1;
          ld_pair(I.d + pix, d0, d1);
          st_pair(I.out + pix, d0, d1);
          break;
        }
        case VOP_MAKE_W: {
          T d0, d1, y0, y1, u0, u1;
          ld_pair(I.d + pix, d0, d1);
          ld_pair(I.y + pix, y0, y1);
          ldc(I.u, q, u0, u1);
          st_pair(I.w + pix, q.m0 ? u0 : d0 - y0, q.m1 ? u1 : d1 - y1);
          break;
        }
        case VOP_LOAD_G: {
          T g0, g1;
          ld_pair(I.gx + pix, g0, g1);
          g0 = q.m0 ? g0 : (T)0;
          g1 = q.m1 ? g1 : (T)0;
          stc(I.r, q, g0, g1);
          stc(I.b, q, g0, g1);
          if (I.r32) stc(I.r32, q, g0, g1);
          acc.add_prod(g0, g0);
          acc.add_prod(g1, g1);
          break;
        }
        default:
          break;
      }
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
