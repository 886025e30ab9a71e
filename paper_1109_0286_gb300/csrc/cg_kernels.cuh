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
#include "cg_async.cuh"
#include "cg_fft.cuh"

namespace cgf {
// Pixel pairs whose loads a source / sink issues together (register budget
// of 64 per thread at two 512-thread CTAs per SM).
constexpr int kSrcChunk = 4, kSrcChunkWide = 2, kSinkChunk = 4;

template <typename T> struct KCfg;
template <> struct KCfg<float> { static constexpr int kMaxThreads = 1024; };
template <> struct KCfg<double> { static constexpr int kMaxThreads = 512; };
template <> struct KCfg<df> { static constexpr int kMaxThreads = 512; };

// Masked flags and compact CG-vector indices of the pixel pair (pix, pix+1)
// (pix even) from the pair's mask word: a popcount.
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

__device__ __forceinline__ PairIdx pair_index(const uint2* __restrict__ mw, int pix) {
  return pair_from_word(__ldg(mw + (pix >> 5)), pix);
}

// In-row pixel pair j (pixels 2j, 2j+1) from the row's mask words staged in
// shared memory.
__device__ __forceinline__ PairIdx pair_at(const uint2* mwr, int j) {
  return pair_from_word(mwr[j >> 4], 2 * j);
}
__device__ __forceinline__ void observed_at(const uint2* mwr, int j, bool& o0, bool& o1) {
  const uint32_t ob = mwr[j >> 4].x;
  const int b = (2 * j) & 31;
  o0 = (ob >> b) & 1u;
  o1 = (ob >> (b + 1)) & 1u;
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

// The compact CG-vector elements of a CTA's rows form one contiguous range
// [c0, c1) (vectors are stored in row-major order of the masked pixels): its
// first word's offset, and the last word's offset plus its masked count.
// One thread asks the copy engine to bring the ranges the op will read into
// L2, so that the per-pixel-pair gathers later in the pass hit L2 instead of
// waiting on HBM one chunk after another.
template <typename T>
__device__ __forceinline__ void prefetch_compact(const InstDesc<T>& I, int op, const uint2* mws,
                                                 int nwords) {
  const uint2 w0 = mws[0], w1 = mws[nwords - 1];
  const long long c0 = w0.y, c1 = (long long)w1.y + __popc(~w1.x);
  switch (op) {
    case OP_R_UPD:
      prefetch_l2(I.r, c0, c1);
      prefetch_l2(I.q, c0, c1);
      prefetch_l2(I.u, c0, c1);
      prefetch_l2(I.p, c0, c1);
      break;
    // (not for the p updates: measured 8% slower with it at 4096^2 x 8,
    // against 4% faster for the r update and 1% for the sinks)
    case OP_LOAD_R: prefetch_l2(I.r, c0, c1); break;
    case OP_LOAD_U: prefetch_l2(I.u, c0, c1); break;
    case OP_U64_UPD:
      prefetch_l2(I.u, c0, c1);
      prefetch_l2(I.dlt, c0, c1);
      break;
    case OP_Q: prefetch_l2(I.p, c0, c1); break;
    case OP_Z: prefetch_l2(I.r, c0, c1); break;
    case OP_RES: prefetch_l2(I.b, c0, c1); break;
    default: break;
  }
}

// ----------------------------------------------------------------- sources
// A source fills v[e] = (x[2j], x[2j+1]), j = tid + e TT, with the real row
// values fed to the forward transform.  One instantiation per op: a chunk of
// CK pixel pairs issues all its loads (indices come from shared memory, so
// they do not wait on a global load) before its arithmetic and stores.
template <typename T, int TT, int OP>
__device__ __forceinline__ void src_fill(const InstDesc<T>& I, const uint2* mwr, int rowpix,
                                         int tid, T alpha, T beta, cx<T> (&v)[16], Acc<T>& acc) {
  constexpr int CK = (OP == OP_R_UPD || OP == OP_U64_UPD) ? kSrcChunkWide : kSrcChunk;
#pragma unroll
  for (int h = 0; h < 16; h += CK) {
    PairIdx q[CK];
    T x0[CK], x1[CK], y0[CK], y1[CK], z0[CK], z1[CK], w0[CK], w1[CK];
#pragma unroll
    for (int e = 0; e < CK; ++e) {
      const int j = tid + (h + e) * TT;
      if constexpr (OP == OP_LOAD_W || OP == OP_LOAD_W_MASK || OP == OP_LOAD_Y) {
        ld_pair((OP == OP_LOAD_Y ? I.y : I.w) + rowpix + 2 * j, x0[e], x1[e]);
        if constexpr (OP == OP_LOAD_W_MASK) q[e] = pair_at(mwr, j);
      } else {
        q[e] = pair_at(mwr, j);
        if constexpr (OP == OP_LOAD_D_U) ld_map_pair<T>(I.d + rowpix + 2 * j, x0[e], x1[e]);
        if constexpr (OP == OP_LOAD_R) ldc(I.r, q[e], x0[e], x1[e]);
        if constexpr (OP == OP_LOAD_U) ldc(I.u, q[e], x0[e], x1[e]);
        if constexpr (OP == OP_P_UPD_Z || OP == OP_P_UPD_R) {
          ldc(OP == OP_P_UPD_Z ? I.z : I.r, q[e], x0[e], x1[e]);
          ldc(I.p, q[e], y0[e], y1[e]);
        }
        if constexpr (OP == OP_R_UPD) {
          ldc(I.r, q[e], x0[e], x1[e]);
          ldc(I.q, q[e], y0[e], y1[e]);
          ldc(I.u, q[e], z0[e], z1[e]);
          ldc(I.p, q[e], w0[e], w1[e]);
        }
        if constexpr (OP == OP_U64_UPD) {
          ldc(I.u, q[e], x0[e], x1[e]);
          ldc(I.dlt, q[e], y0[e], y1[e]);
        }
      }
    }
#pragma unroll
    for (int e = 0; e < CK; ++e) {
      T a0, a1;
      if constexpr (OP == OP_LOAD_W_MASK) {
        a0 = q[e].m0 ? x0[e] : (T)0;
        a1 = q[e].m1 ? x1[e] : (T)0;
      } else if constexpr (OP == OP_LOAD_D_U) {
        a0 = q[e].m0 ? (T)0 : x0[e];
        a1 = q[e].m1 ? (T)0 : x1[e];
      } else if constexpr (OP == OP_P_UPD_Z || OP == OP_P_UPD_R) {
        a0 = x0[e] + beta * y0[e];
        a1 = x1[e] + beta * y1[e];
        stc(I.p, q[e], a0, a1);
      } else if constexpr (OP == OP_R_UPD) {
        a0 = x0[e] - alpha * y0[e];
        a1 = x1[e] - alpha * y1[e];
        stc(I.r, q[e], a0, a1);
        stc(I.u, q[e], z0[e] + alpha * w0[e], z1[e] + alpha * w1[e]);
        acc.add_prod(a0, a0);
        acc.add_prod(a1, a1);
      } else if constexpr (OP == OP_U64_UPD) {
        a0 = x0[e] + y0[e];
        a1 = x1[e] + y1[e];
        stc(I.u, q[e], a0, a1);
        stc(I.dlt, q[e], 0.f, 0.f);   // folded
      } else {
        a0 = x0[e];
        a1 = x1[e];
        if constexpr (OP == OP_LOAD_R) {
          acc.add_prod(a0, a0);
          acc.add_prod(a1, a1);
        }
      }
      v[h + e] = cx<T>{a0, a1};
    }
  }
}

// ----------------------------------------------------------------- sinks
// A sink consumes the inverse transform's row values v[e] (pairs j = tid + e
// TT): projection, stores and the inner product of its op.
template <typename T, int TT, int OP>
__device__ __forceinline__ void sink_fill(const InstDesc<T>& I, const uint2* mwr, int rowpix,
                                          int tid, const cx<T> (&v)[16], Acc<T>& acc,
                                          int param = 0) {
  constexpr int CK = kSinkChunk;
#pragma unroll
  for (int h = 0; h < 16; h += CK) {
    PairIdx q[CK];
    T x0[CK], x1[CK];
#pragma unroll
    for (int e = 0; e < CK; ++e) {
      const int j = tid + (h + e) * TT;
      q[e] = pair_at(mwr, j);
      if constexpr (OP == OP_Q) ldc(I.p, q[e], x0[e], x1[e]);
      if constexpr (OP == OP_Z) ldc(I.r, q[e], x0[e], x1[e]);
      if constexpr (OP == OP_RES) ldc(I.b, q[e], x0[e], x1[e]);
      if constexpr (OP == OP_GRAD) ld_map_pair<T>(I.gx + rowpix + 2 * j, x0[e], x1[e]);
      if constexpr (OP == OP_RELAX) ld_pair(I.w + rowpix + 2 * j, x0[e], x1[e]);
    }
#pragma unroll
    for (int e = 0; e < CK; ++e) {
      const int j = tid + (h + e) * TT;
      const bool m0 = q[e].m0, m1 = q[e].m1;   // masked = not observed
      // compact-vector ops: nothing to store or add (exactly) for a pair
      // without a masked pixel
      constexpr bool C = OP == OP_Q || OP == OP_Z || OP == OP_B || OP == OP_RES || OP == OP_KSEL;
      if (C && !(m0 || m1)) continue;
      T a0 = v[h + e].r, a1 = v[h + e].i;
      if constexpr (OP == OP_Q || OP == OP_Z) {
        a0 = m0 ? a0 : (T)0;
        a1 = m1 ? a1 : (T)0;
        stc(OP == OP_Q ? I.q : I.z, q[e], a0, a1);
        acc.add_prod(x0[e], a0);
        acc.add_prod(x1[e], a1);
      } else if constexpr (OP == OP_B) {
        a0 = m0 ? -a0 : (T)0;
        a1 = m1 ? -a1 : (T)0;
        stc(I.r, q[e], a0, a1);
        if (I.b) stc(I.b, q[e], a0, a1);
        if (I.r32) stc(I.r32, q[e], a0, a1);
        acc.add_prod(a0, a0);
        acc.add_prod(a1, a1);
      } else if constexpr (OP == OP_RES) {
        a0 = x0[e] - (m0 ? a0 : (T)0);
        a1 = x1[e] - (m1 ? a1 : (T)0);
        stc(I.r, q[e], a0, a1);
        if (I.r32) stc(I.r32, q[e], a0, a1);
        acc.add_prod(a0, a0);
        acc.add_prod(a1, a1);
      } else if constexpr (OP == OP_GRAD) {
        // v = C^-1 lam.  dL/dd_U = g_U - (C^-1 lam)_U, dL/dd_M = 0;
        // dL/dy = h = g on M, (C^-1 lam)_U on U (kept in y).
        st_map_pair<T>(I.out + rowpix + 2 * j, m0 ? (T)0 : x0[e] - a0, m1 ? (T)0 : x1[e] - a1);
        st_pair(I.y + rowpix + 2 * j, m0 ? x0[e] : a0, m1 ? x1[e] : a1);
      } else if constexpr (OP == OP_RELAX) {
        const T step = (T)I.st->alpha;
        a0 = m0 ? a0 : (T)0;
        a1 = m1 ? a1 : (T)0;
        st_pair(I.w + rowpix + 2 * j, x0[e] - step * a0, x1[e] - step * a1);
        acc.add_prod(a0, a0);
        acc.add_prod(a1, a1);
      } else if constexpr (OP == OP_KSEL) {
        const uchar2 c = *reinterpret_cast<const uchar2*>(I.cls + rowpix + 2 * j);
        if (m0 && c.x == param) I.y[rowpix + 2 * j] = a0;
        if (m1 && c.y == param) I.y[rowpix + 2 * j + 1] = a1;
      } else if constexpr (OP == OP_STORE_Y) {
        st_pair(I.y + rowpix + 2 * j, a0, a1);
      } else if constexpr (OP == OP_STORE_Y_MASK) {
        st_pair(I.y + rowpix + 2 * j, m0 ? a0 : (T)0, m1 ? a1 : (T)0);
      }
    }
  }
}

// Middle of a chain (between the inverse and the forward row transform):
// P_x (OP_MASK), or y = v and v = (d - y) on U, 0 on M (OP_Y_W).
template <typename T, int TT, int OP>
__device__ __forceinline__ void mid_fill(const InstDesc<T>& I, const uint2* mwr, int rowpix,
                                         int tid, cx<T> (&v)[16]) {
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const int j = tid + e * TT;
    bool o0, o1;
    observed_at(mwr, j, o0, o1);
    if constexpr (OP == OP_Y_W) {
      T d0, d1;
      ld_map_pair<T>(I.d + rowpix + 2 * j, d0, d1);
      st_pair(I.y + rowpix + 2 * j, v[e].r, v[e].i);
      v[e].r = o0 ? d0 - v[e].r : (T)0;
      v[e].i = o1 ? d1 - v[e].i : (T)0;
    } else {
      v[e].r = o0 ? (T)0 : v[e].r;
      v[e].i = o1 ? (T)0 : v[e].i;
    }
  }
}

// ----------------------------------------------------------------- row pass
// CTA = `rows` consecutive grid rows, L/16 threads per row; blockIdx.y is the
// instance.  Shared memory: per-row FFT exchange areas, aliased with the
// transposed tile [(L+1) x rows] used for the spectrum load / store,
// then the rows' mask words (nx/32 = L/16 per row: one per thread).
// XI: the source is the seed's white noise (kept out of the other source
// kernels, whose register allocation it would otherwise burden).
template <typename T>
__host__ __device__ __forceinline__ size_t row_main_bytes(int log_l, int rows) {
  const size_t L = size_t(1) << log_l, padl = L + L / 16 + 1;
  const size_t fft = size_t(rows) * 2 * padl, tile = 2 * (L + 1) * size_t(rows);
  return ((fft > tile ? fft : tile) * sizeof(T) + 15) & ~size_t(15);
}

template <typename T, int LOG_L, bool IN_SPEC, bool OUT_SPEC, bool XI = false>
__global__ void __launch_bounds__(KCfg<T>::kMaxThreads)
k_row(const InstDesc<T>* __restrict__ insts, RowArgs a, const T* __restrict__ tw) {
  constexpr int L = 1 << LOG_L, TT = L / 16, PADL = L + L / 16 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  __shared__ double red[32];
  const InstDesc<T>& I = insts[blockIdx.y];
  if (skip_instance(a.check_done, I.st)) return;

  const int rows = a.rows, lr = a.log_rows;
  const int row = threadIdx.x / TT, tid = threadIdx.x - row * TT;
  const int y0 = blockIdx.x * rows, y = y0 + row;
  const int ny = a.ny;
  const XBuf<T> xb(sm + row * 2 * PADL, PADL);
  // transposed tile [(L+1)][rows], aliases the FFT areas; column r of row k at
  // k rows + (r ^ g(k)), g(k) = (k >> gs) & (rows - 1): both the
  // consecutive-k accesses of one row and the (k, r) sweep of the global
  // loads / stores are free of bank conflicts
  cx<T>* tile = reinterpret_cast<cx<T>*>(sm);
  const int gs = lr < 4 ? 4 - lr : 0;
  auto tix = [&](int k, int r) { return (k << lr) + (r ^ ((k >> gs) & (rows - 1))); };
  uint2* mws = reinterpret_cast<uint2*>(smem_raw + row_main_bytes<T>(LOG_L, rows));
  const uint2* mwr = mws + row * TT;            // this row's mask words
  constexpr int TWS = kLmax / (2 * L);          // W_{nx}^k = table[k * TWS]
  const int rowpix = y * a.nx;
  // tile element (kk + i TT, rr) for i = 0..15 belongs to thread (kk, rr); the
  // Nyquist row k = L to threads 0..rows-1
  const int rr = threadIdx.x & (rows - 1), kk = threadIdx.x >> lr;
  const size_t tstep = 2 * (size_t)TT * ny;
  // From L = 512 on, TT is a multiple of 2^max(lr, 4) (rows * TT <= 1024), so
  // adding multiples of TT to k leaves the swizzle bits g(k) unchanged: a
  // thread's tile indices for k0 + i TT are one base plus i (TT rows).
  constexpr bool HOIST = LOG_L >= 9;
  const int ts = TT << lr;
  const XBar cta{0, 0}, rbar = XBar::make(TT, rows, row);   // CTA / this row's barrier
  cx<T> v[16];
  Acc<T> acc;

  if constexpr (!XI) mws[threadIdx.x] = __ldg(I.mw + (size_t)y0 * TT + threadIdx.x);

  if constexpr (IN_SPEC) {
    const T* spec = (a.spec_sel ? I.spec2 : I.spec) + 2 * ((size_t)kk * ny + y0 + rr);
    cx<T> t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[i] = ld_stream_cx<T>(spec + i * tstep);
    cx<T> tn{};
    if (threadIdx.x < rows)
      tn = ldg_cx<T>((a.spec_sel ? I.spec2 : I.spec) + 2 * ((size_t)L * ny + y0 + threadIdx.x));
    const int tb = tix(kk, rr);
#pragma unroll
    for (int i = 0; i < 16; ++i) tile[HOIST ? tb + i * ts : tix(kk + i * TT, rr)] = t[i];
    if (threadIdx.x < rows) tile[tix(L, threadIdx.x)] = tn;
    __syncthreads();
    if (threadIdx.x == 0 && !OUT_SPEC) prefetch_compact(I, a.op, mws, rows * TT);
    // C2R: Z[k] = (X[k] + conj X[L-k]) + i e^{+2 pi i k / nx} (X[k] - conj X[L-k])
    const cx<T> wt = twiddle<T>(tw, tid * TWS);
    const int cb = tix(tid, row), cm = tix(L - tid, row);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int k = tid + e * TT;
      cx<T> xk = tile[HOIST ? cb + e * ts : tix(k, row)];
      cx<T> xc = conjx(tile[HOIST ? cm - e * ts : tix(L - k, row)]);
      if (k == 0) {
        xk.i = (T)0;
        xc.i = (T)0;
      }
      const cx<T> w = cmul(wt, w32<T>(e));   // W_nx^k, k = tid + e TT
      const cx<T> sum = xk + xc;
      const cx<T> dif = cmulc(xk - xc, w);  // (X - conj X') e^{+i...}
      v[e] = cx<T>{sum.r - dif.i, sum.i + dif.r};
    }
    // the first exchange overwrites tile entries other rows still read
    fft_regs<T, LOG_L, true>(v, xb, tid, tw, cta, rbar);
    // v[e] = x[2j] + i x[2j+1], j = tid + e TT
    if constexpr (OUT_SPEC) {
      if (a.op == OP_Y_W)
        mid_fill<T, TT, OP_Y_W>(I, mwr, rowpix, tid, v);
      else
        mid_fill<T, TT, OP_MASK>(I, mwr, rowpix, tid, v);
    } else {
      switch (a.op) {
        case OP_Q: sink_fill<T, TT, OP_Q>(I, mwr, rowpix, tid, v, acc); break;
        case OP_Z: sink_fill<T, TT, OP_Z>(I, mwr, rowpix, tid, v, acc); break;
        case OP_B: sink_fill<T, TT, OP_B>(I, mwr, rowpix, tid, v, acc); break;
        case OP_RES: sink_fill<T, TT, OP_RES>(I, mwr, rowpix, tid, v, acc); break;
        case OP_GRAD: sink_fill<T, TT, OP_GRAD>(I, mwr, rowpix, tid, v, acc); break;
        case OP_RELAX: sink_fill<T, TT, OP_RELAX>(I, mwr, rowpix, tid, v, acc); break;
        case OP_KSEL: sink_fill<T, TT, OP_KSEL>(I, mwr, rowpix, tid, v, acc, a.param); break;
        case OP_STORE_Y: sink_fill<T, TT, OP_STORE_Y>(I, mwr, rowpix, tid, v, acc); break;
        case OP_STORE_Y_MASK:
          sink_fill<T, TT, OP_STORE_Y_MASK>(I, mwr, rowpix, tid, v, acc);
          break;
        default: break;
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
    __syncthreads();   // mask words
    if (threadIdx.x == 0) prefetch_compact(I, a.op, mws, rows * TT);
    const T alpha = (T)I.st->alpha, beta = (T)I.st->beta;
    switch (a.op) {
      case OP_R_UPD: src_fill<T, TT, OP_R_UPD>(I, mwr, rowpix, tid, alpha, beta, v, acc); break;
      case OP_P_UPD_Z:
        src_fill<T, TT, OP_P_UPD_Z>(I, mwr, rowpix, tid, alpha, beta, v, acc);
        break;
      case OP_P_UPD_R:
        src_fill<T, TT, OP_P_UPD_R>(I, mwr, rowpix, tid, alpha, beta, v, acc);
        break;
      case OP_LOAD_R: src_fill<T, TT, OP_LOAD_R>(I, mwr, rowpix, tid, alpha, beta, v, acc); break;
      case OP_LOAD_U: src_fill<T, TT, OP_LOAD_U>(I, mwr, rowpix, tid, alpha, beta, v, acc); break;
      case OP_LOAD_Y: src_fill<T, TT, OP_LOAD_Y>(I, mwr, rowpix, tid, alpha, beta, v, acc); break;
      case OP_LOAD_W: src_fill<T, TT, OP_LOAD_W>(I, mwr, rowpix, tid, alpha, beta, v, acc); break;
      case OP_LOAD_W_MASK:
        src_fill<T, TT, OP_LOAD_W_MASK>(I, mwr, rowpix, tid, alpha, beta, v, acc);
        break;
      case OP_LOAD_D_U:
        src_fill<T, TT, OP_LOAD_D_U>(I, mwr, rowpix, tid, alpha, beta, v, acc);
        break;
      case OP_U64_UPD:
        src_fill<T, TT, OP_U64_UPD>(I, mwr, rowpix, tid, alpha, beta, v, acc);
        break;
      default:
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = cx<T>{(T)0, (T)0};
        break;
    }
  }

  if constexpr (OUT_SPEC) {
    fft_regs<T, LOG_L, false>(v, xb, tid, tw, rbar, rbar);
    // Z (the half-length transform) into the transposed tile; the threads of
    // the global stores form X from Z[k] and Z[L-k]:
    // R2C: X[k] = (Z[k] + conj Z[L-k]) / 2 - (i/2) e^{-2 pi i k/nx} (Z[k] - conj Z[L-k])
    __syncthreads();   // the tile overwrites other rows' exchange areas
    const int cb = tix(tid, row);
#pragma unroll
    for (int e = 0; e < 16; ++e) tile[HOIST ? cb + e * ts : tix(tid + e * TT, row)] = v[e];
    __syncthreads();
    const cx<T> wt = twiddle<T>(tw, kk * TWS);
    T* spec = (a.spec_sel ? I.spec2 : I.spec) + 2 * ((size_t)kk * ny + y0 + rr);
    const int tb = tix(kk, rr), tm = tix(L - kk, rr);   // L - kk: the Nyquist row when kk = 0
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int k = kk + i * TT;
      const cx<T> zk = tile[HOIST ? tb + i * ts : tix(k, rr)];
      const int im = (i == 0 && kk == 0) ? tix(0, rr) : tm - i * ts;
      const cx<T> zc = conjx(tile[HOIST ? im : tix((L - k) & (L - 1), rr)]);
      const cx<T> ev = scal(zk + zc, (T)0.5);
      const cx<T> od = scal(mul_mi<T, false>(zk - zc), (T)0.5);
      st_cx<T>(spec + i * tstep, ev + cmul(od, cmul(wt, w32<T>(i))));
    }
    if (threadIdx.x < rows) {   // Nyquist: X[L] = Re Z[0] - Im Z[0]
      const cx<T> z0 = tile[tix(0, threadIdx.x)];
      st_cx<T>((a.spec_sel ? I.spec2 : I.spec) + 2 * ((size_t)L * ny + y0 + threadIdx.x),
               cx<T>{z0.r - z0.i, (T)0});
    }
  }

  if (a.sop != SC_NONE)
    grid_reduce(acc.value(), red, I.partial, I.st, a.sop, gridDim.x, blockIdx.x);
}

// ----------------------------------------------------------------- column pass
// CTA = `ffts` spectrum rows (one kx each), N/16 threads per row; forward
// column FFT, multiply by the real table, inverse column FFT, in place
// (table < 0: forward transform only; PRE: start from the forward transform
// held in spec and write to the buffer spec_sel names).  blockIdx.x is the instance, so the
// CTAs of all instances for the same kx run together and share the table
// row through L2.
template <typename T, int LOG_N, bool PRE = false>
__global__ void __launch_bounds__(KCfg<T>::kMaxThreads)
k_col(const InstDesc<T>* __restrict__ insts, ColArgs a, const T* __restrict__ tw) {
  constexpr int N = 1 << LOG_N, TT = N / 16, PADN = N + N / 16 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const InstDesc<T>& I = insts[blockIdx.x];
  if (skip_instance(a.check_done, I.st)) return;
  const int f = threadIdx.x / TT, tid = threadIdx.x - f * TT;
  const int kx = blockIdx.y * a.ffts + f;
  const bool act = kx < a.nkx;
  const XBuf<T> xb(sm + f * 2 * PADN, PADN);
  const XBar bar = XBar::make(TT, a.ffts, f);
  T* col = (a.spec_sel ? I.spec2 : I.spec) + 2 * (long long)(act ? kx : 0) * N;
  const T* src = PRE ? I.spec + 2 * (long long)(act ? kx : 0) * N : col;
  cx<T> v[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) v[e] = act ? ld_stream_cx<T>(src + 2 * (tid + e * TT)) : cx<T>{(T)0, (T)0};
  if constexpr (!PRE) fft_regs<T, LOG_N, false, false>(v, xb, tid, tw, bar, bar);
  if (a.table >= 0) {
    const T* tab = (a.table >= 2 ? I.kt + (long long)(a.table - 2) * a.nkx * N
                    : a.table ? I.t_sqrt : I.t_inv) + (long long)(act ? kx : 0) * N;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const T t = act ? ldg1(tab + tid + e * TT) : (T)0;
      v[e] = scal(v[e], t);
    }
    // the inverse transform reloads its twiddles through an opaque copy of
    // the table pointer: sharing the forward transform's loads would keep
    // them live across the table multiply and spill registers
    const T* tw_inv;
    asm("mov.b64 %0, %1;" : "=l"(tw_inv) : "l"(tw));
    fft_regs<T, LOG_N, true, false>(v, xb, tid, tw_inv, bar, bar);
  }
  if (act) {
#pragma unroll
    for (int e = 0; e < 16; ++e) st_cx<T>(col + 2 * (tid + e * TT), v[e]);
  }
}

// ----------------------------------------------------------------- column pass (TMA)
// FP32 column pass of the CG loops (forward column FFT, x 1/(nP) or x sqrt(P)/n,
// inverse FFT) as a persistent kernel fed by bulk copies.  A work item is a
// block of F consecutive spectrum rows (kx .. kx+F-1) of one instance: F N
// contiguous complex values and the matching F N table values.  CTA c takes
// a contiguous run of items (kx-major, instance-minor, so an item's table
// rows were usually just read by the previous item and come from L2).  While
// item j is transformed, one thread has the copy engine bring item j+1 into
// the other of two shared-memory slots (cp.async.bulk, completion on the
// slot's mbarrier), so no thread waits on global loads.  The landing area of
// each column is then its exchange area (XBufSw, unpadded), and the results
// go to global memory straight from registers.  Items of instances that are
// done are skipped.  Every wait is bounded: on a timeout the CTA sets
// *a.err, waits (bounded) for the copies it issued, and returns.
constexpr int kColTmaSlots = 2;

__host__ __device__ __forceinline__ size_t col_tma_smem(int log_n, int ffts) {
  const size_t fn = size_t(ffts) << log_n;
  return kColTmaSlots * fn * (sizeof(float2) + sizeof(float)) + 2 * kColTmaSlots * sizeof(uint64_t);
}

template <int LOG_N>
__global__ void __launch_bounds__(LOG_N >= 13 ? 512 : 256, LOG_N >= 13 ? 1 : 2)
k_col_tma(const InstDesc<float>* __restrict__ insts, ColArgs a, const float* __restrict__ tw,
          int ninst) {
  constexpr int N = 1 << LOG_N, TT = N / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int F = a.ffts;
  const size_t fn = size_t(F) * N;
  float2* slot0 = reinterpret_cast<float2*>(smem_raw);
  float* tab0 = reinterpret_cast<float*>(smem_raw + kColTmaSlots * fn * sizeof(float2));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + kColTmaSlots * fn * (sizeof(float2) + sizeof(float)));
  const int f = threadIdx.x / TT, tid = threadIdx.x - f * TT;
  const XBar fbar = XBar::make(TT, F, f);
  const int nkb = (a.nkx + F - 1) / F;
  const long long total = (long long)nkb * ninst;
  const long long per = (total + gridDim.x - 1) / gridDim.x;
  const long long first = (long long)blockIdx.x * per;
  const long long end = first + per < total ? first + per : total;

  auto next_item = [&](long long i) {
    while (i < end && skip_instance(a.check_done, insts[i % ninst].st)) ++i;
    return i;
  };
  auto issue = [&](long long i, int sl) {   // one thread
    const InstDesc<float>& I = insts[i % ninst];
    const int kx0 = (int)(i / ninst) * F;
    const int nc = a.nkx - kx0 < F ? a.nkx - kx0 : F;
    const uint32_t bs = (uint32_t)nc * N * sizeof(float2), bt = (uint32_t)nc * N * sizeof(float);
    mbar_arrive_expect(&bar[sl], bs + bt);
    bulk_g2s(slot0 + sl * fn, I.spec + 2 * (long long)kx0 * N, bs, &bar[sl]);
    bulk_g2s(tab0 + sl * fn, (a.table ? I.t_sqrt : I.t_inv) + (long long)kx0 * N, bt, &bar[sl]);
  };

  if (threadIdx.x == 0) {
    for (int sl = 0; sl < kColTmaSlots; ++sl) mbar_init(&bar[sl], 1);
    fence_mbar_init();
  }
  __syncthreads();
  long long it = next_item(first);
  if (threadIdx.x == 0 && it < end) issue(it, 0);
  uint32_t phase = 0u;                   // bit sl: parity of slot sl's next completion
  uint32_t pending = it < end ? 1u : 0u;  // bit sl: a copy into slot sl is in flight
  int sl = 0;
  while (it < end) {
    const long long nxt = next_item(it + 1);
    if (nxt < end) {
      // the other slot's previous item is finished (CTA barrier at the end of
      // the last iteration): hand it to the copy engine
      if (threadIdx.x == 0) {
        fence_proxy_async();
        issue(nxt, sl ^ 1);
      }
      pending |= 1u << (sl ^ 1);
    }
    const bool ok = mbar_wait(&bar[sl], (phase >> sl) & 1u);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        if (a.err) atomicExch(a.err, 1);
        for (int q = 0; q < kColTmaSlots; ++q)   // let the copies in flight land (bounded)
          if (((pending >> q) & 1u) && !(q == sl && ok)) mbar_wait(&bar[q], (phase >> q) & 1u);
      }
      __syncthreads();
      return;
    }
    pending &= ~(1u << sl);
    phase ^= 1u << sl;

    const InstDesc<float>& I = insts[it % ninst];
    const int kx = (int)(it / ninst) * F + f;
    const bool act = kx < a.nkx;
    float2* buf = slot0 + sl * fn + size_t(f) * N;
    const float* tb = tab0 + sl * fn + size_t(f) * N;
    cx<float> v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const float2 t = act ? buf[tid + e * TT] : make_float2(0.f, 0.f);
      v[e] = cx<float>{t.x, t.y};
    }
    const XBufSw xb(buf);
    fft_regs<float, LOG_N, false, false>(v, xb, tid, tw, fbar, fbar);
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = scal(v[e], act ? tb[tid + e * TT] : 0.f);
    // the inverse transform reloads its twiddles (an opaque copy of the table
    // pointer): keeping the forward transform's alive across the table
    // multiply would cost some 60 registers and spills
    const float* tw_inv;
    asm("mov.b64 %0, %1;" : "=l"(tw_inv) : "l"(tw));
    fft_regs<float, LOG_N, true, false>(v, xb, tid, tw_inv, fbar, fbar);
    if (act) {
      float* col = I.spec + 2 * (long long)kx * N;
#pragma unroll
      for (int e = 0; e < 16; ++e) st_cx<float>(col + 2 * (tid + e * TT), v[e]);
    }
    __syncthreads();   // slot sl is free again
    it = nxt;
    sl ^= 1;
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
        case VOP_ASSEMBLE: {   // observed pixels: the caller's values, bit for bit
          using M = typename MapOf<T>::type;
          M d0, d1;
          T y0, y1, u0, u1;
          ld_pair(I.d + pix, d0, d1);
          ld_pair(I.y + pix, y0, y1);
          ldc(I.u, q, u0, u1);
          st_pair(I.out + pix, q.m0 ? static_cast<M>(y0 + u0) : d0,
                  q.m1 ? static_cast<M>(y1 + u1) : d1);
          break;
        }
        case VOP_COPY_D: {
          typename MapOf<T>::type d0, d1;
          ld_pair(I.d + pix, d0, d1);
          st_pair(I.out + pix, d0, d1);
          break;
        }
        case VOP_MAKE_W: {
          T d0, d1, y0, y1, u0, u1;
          ld_map_pair<T>(I.d + pix, d0, d1);
          ld_pair(I.y + pix, y0, y1);
          ldc(I.u, q, u0, u1);
          st_pair(I.w + pix, q.m0 ? u0 : d0 - y0, q.m1 ? u1 : d1 - y1);
          break;
        }
        case VOP_MAP_IN: {
          T a0, a1;
          ld_map_pair<T>(I.d + pix, a0, a1);
          st_pair(I.w + pix, a0, a1);
          break;
        }
        case VOP_MAP_OUT: {
          T a0, a1;
          ld_pair(I.y + pix, a0, a1);
          st_map_pair<T>(I.out + pix, a0, a1);
          break;
        }
        case VOP_ANNULUS: {   // offsets by minimum image from pixel 0
          const long long nx = a.nx, ny = a.npix / a.nx;
          T av[2];
          for (int t = 0; t < 2; ++t) {
            const long long pp = pix + t, yy = pp / nx, xx = pp % nx;
            const double dy = (double)(yy <= ny / 2 ? yy : yy - ny);
            const double dx = (double)(xx <= nx / 2 ? xx : xx - nx);
            const double r2 = dy * dy + dx * dx;
            av[t] = (r2 > a.p0 && r2 <= a.p1 && r2 > 0.0) ? (T)1 : (T)0;
          }
          st_pair(I.w + pix, av[0], av[1]);
          break;
        }
        case VOP_Y_TO_W_M: {
          T w0, w1, y0, y1;
          ld_pair(I.w + pix, w0, w1);
          ld_pair(I.y + pix, y0, y1);
          const T d0 = q.m0 ? y0 - w0 : (T)0, d1 = q.m1 ? y1 - w1 : (T)0;
          st_pair(I.w + pix, q.m0 ? y0 : w0, q.m1 ? y1 : w1);
          acc.add_prod(d0, d0);
          acc.add_prod(d1, d1);
          break;
        }
        case VOP_W_FROM_D: {
          T a0, a1;
          ld_map_pair<T>(I.d + pix, a0, a1);
          st_pair(I.w + pix, q.m0 ? (T)0 : a0, q.m1 ? (T)0 : a1);
          break;
        }
        case VOP_W_TO_OUT: {   // observed pixels: the caller's values, bit for bit
          using M = typename MapOf<T>::type;
          M d0, d1;
          T a0, a1;
          ld_pair(I.d + pix, d0, d1);
          ld_pair(I.w + pix, a0, a1);
          st_pair(I.out + pix, q.m0 ? static_cast<M>(a0) : d0, q.m1 ? static_cast<M>(a1) : d1);
          break;
        }
        case VOP_LOAD_G: {
          T g0, g1;
          ld_map_pair<T>(I.gx + pix, g0, g1);
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
// self-conjugate columns, 2 elsewhere).  The sums are reproducible bit for
// bit: each warp takes fixed runs of 32 modes, the lanes of one band are
// added in lane order by the band's lowest lane into the warp's own row of
// partial sums, and the rows are added in warp order at the end.
constexpr int kDotThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kDotThreads)
k_band_dot(const InstDesc<T>* __restrict__ insts, DotArgs a) {
  constexpr int NW = kDotThreads / 32;
  __shared__ double hist[NW][kMaxBands];
  __shared__ double vals[NW][32];
  const InstDesc<T>& I = insts[blockIdx.y];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int b = lane; b < a.nbands; b += 32) hist[warp][b] = 0.0;
  __syncwarp();
  const T* coef = reinterpret_cast<const T*>(a.coef);
  const long long stride = (long long)gridDim.x * NW * 32;
  for (long long base = ((long long)blockIdx.x * NW + warp) * 32; base < a.nmodes; base += stride) {
    const long long m = base + lane;
    const bool valid = m < a.nmodes;
    double v = 0.0;
    int b = -1;
    if (valid) {
      const cx<T> x = ld_cx<T>(I.spec + 2 * m), z = ld_cx<T>(I.spec2 + 2 * m);
      v = (double)((x.r * z.r + x.i * z.i) * ldg1(coef + m));
      b = __ldg(a.band + m);
    }
    vals[warp][lane] = v;
    const unsigned g = __match_any_sync(0xffffffffu, b);
    __syncwarp();
    if (valid && lane == __ffs(g) - 1) {
      double sum = 0.0;
      for (unsigned r = g; r; r &= r - 1) sum += vals[warp][__ffs(r) - 1];
      hist[warp][b] += sum;
    }
    __syncwarp();
  }
  __syncthreads();
  double* out = a.part + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * a.nbands;
  for (int b = threadIdx.x; b < a.nbands; b += blockDim.x) {
    double sum = 0.0;
    for (int w = 0; w < NW; ++w) sum += hist[w][b];
    out[b] = sum;
  }
}

}  // namespace cgf
