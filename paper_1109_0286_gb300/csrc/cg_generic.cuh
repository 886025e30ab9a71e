// Mixed-radix pass kernels (radix 2, 3, 4, 5, 7) and their launchers; see
// cg_generic.h.  The fused operations are those of cg_kernels.cuh, applied
// per pixel pair; mask flags and compact indices come from the global mask
// words (a row need not start on a word boundary here).
#pragma once
#include "cg_generic.h"
#include "cg_launch.cuh"

namespace cgf {
namespace gen {

template <typename T>
__device__ __forceinline__ cx<T> tw_at(const T* w, int t) {
  return ldg_cx<T>(w + 2 * t);
}

// In-register DFT of R points, y_q = sum_m v_m W_R^{qm} (forward sign).  For
// odd R the terms m and R - m pair up: with S_m = v_m + v_{R-m},
// D_m = v_m - v_{R-m} (m = 1..H, H = (R-1)/2) and theta = 2 pi q m / R,
//   y_q = v_0 + sum_m cos(theta) S_m - i sum_m sin(theta) D_m,
//   y_{R-q} = the same with +i,
// so each half-pair costs real-by-complex products only.  cs[j] = W_R^j
// (j = 1..H) = (cos 2 pi j/R, -sin 2 pi j/R).
template <typename T, int R>
__device__ __forceinline__ void dft(cx<T> (&v)[R], const cx<T>* cs) {
  if constexpr (R == 2) {
    const cx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  } else if constexpr (R == 4) {
    const cx<T> s02 = v[0] + v[2], d02 = v[0] - v[2];
    const cx<T> s13 = v[1] + v[3], d13 = mul_mi<T, false>(v[1] - v[3]);
    v[0] = s02 + s13;
    v[2] = s02 - s13;
    v[1] = d02 + d13;
    v[3] = d02 - d13;
  } else {
    constexpr int H = (R - 1) / 2;
    cx<T> S[H + 1], D[H + 1];
    cx<T> y0 = v[0];
#pragma unroll
    for (int m = 1; m <= H; ++m) {
      S[m] = v[m] + v[R - m];
      D[m] = v[m] - v[R - m];
      y0 = y0 + S[m];
    }
    cx<T> y[R];
    y[0] = y0;
#pragma unroll
    for (int q = 1; q <= H; ++q) {
      cx<T> a = v[0], b{(T)0, (T)0};
#pragma unroll
      for (int m = 1; m <= H; ++m) {
        const int j = (q * m) % R, jj = j <= H ? j : R - j;
        const T c = cs[jj].r, sn = j <= H ? -cs[jj].i : cs[jj].i;   // cos, sin of 2 pi j / R
        a = a + scal(S[m], c);
        b = b + scal(D[m], sn);
      }
      y[q] = cx<T>{a.r + b.i, a.i - b.r};       // a - i b
      y[R - q] = cx<T>{a.r - b.i, a.i + b.r};   // a + i b
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = y[q];
  }
}

// One self-sorting stage: butterfly b takes in[b + m n/R] (m < R), scales by
// W_{ns R}^{m k} (k = b mod ns), transforms, and writes
// out[(b - k) R + k + m ns].  cin / cout conjugate inputs / outputs (the
// inverse transform as conj F conj).
template <typename T, int R>
__device__ __forceinline__ void stage(const cx<T>* in, cx<T>* out, int n, int ns, const T* w,
                                      int t, int nt, bool cin, bool cout) {
  const int nb = n / R, step = n / (ns * R);
  cx<T> cs[R / 2 + 1];   // W_R^j, j = 1..(R-1)/2, for the odd radices
  if constexpr (R % 2 == 1) {
#pragma unroll
    for (int j = 1; j <= R / 2; ++j) cs[j] = tw_at(w, j * nb);
  }
  // b = j ns + k, stepped by nt without a division per butterfly
  int j = t / ns, k = t - j * ns;
  const int dj = nt / ns, dk = nt - dj * ns, nsr = ns * R;
  for (int b = t; b < nb; b += nt) {
    cx<T> v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      v[m] = in[b + m * nb];
      if (cin) v[m] = conjx(v[m]);
    }
    if (ns > 1) {
#pragma unroll
      for (int m = 1; m < R; ++m) v[m] = cmul(v[m], tw_at(w, m * k * step));
    }
    dft<T, R>(v, cs);
    const int base = j * nsr + k;   // (b - k) R + k
#pragma unroll
    for (int m = 0; m < R; ++m) out[base + m * ns] = cout ? conjx(v[m]) : v[m];
    k += dk;
    j += dj;
    if (k >= ns) {
      k -= ns;
      ++j;
    }
  }
}

// Unnormalised transform of the n values in `a` (forward: W_n = e^{-2 pi i/n};
// inverse: the conjugate).  Every thread of the CTA calls it (CTA barriers);
// threads t < nt of each transform share its butterflies.  Returns the buffer
// that holds the result (a or b).
template <typename T>
__device__ cx<T>* fft(cx<T>* a, cx<T>* b, const GenLen& g, const T* w, int t, bool inv) {
  int ns = 1;
  for (int s = 0; s < g.nst; ++s) {
    const int r = g.radix[s];
    const bool cin = inv && s == 0, cout = inv && s == g.nst - 1;
    switch (r) {
      case 2: stage<T, 2>(a, b, g.n, ns, w, t, g.nt, cin, cout); break;
      case 3: stage<T, 3>(a, b, g.n, ns, w, t, g.nt, cin, cout); break;
      case 4: stage<T, 4>(a, b, g.n, ns, w, t, g.nt, cin, cout); break;
      case 5: stage<T, 5>(a, b, g.n, ns, w, t, g.nt, cin, cout); break;
      default: stage<T, 7>(a, b, g.n, ns, w, t, g.nt, cin, cout); break;
    }
    ns *= r;
    __syncthreads();
    cx<T>* c = a;
    a = b;
    b = c;
  }
  return a;
}

// ----------------------------------------------------------------- per-pair operations
// Each row loop takes kGenChunk pixel pairs per thread at a time: their mask
// words first, then every operand load, then the arithmetic and stores, so
// the loads of a chunk are in flight together.
constexpr int kGenChunk = 4;

struct Opnd {   // one pixel pair: mask flags, compact indices, pixel index
  PairIdx q;
  int pix;
  bool ok;
};

template <typename T, int OP>
__device__ __forceinline__ void src_load(const InstDesc<T>& I, const Opnd& o, T (&x)[8]) {
  if constexpr (OP == OP_LOAD_W || OP == OP_LOAD_Y || OP == OP_LOAD_W_MASK) {
    ld_pair((OP == OP_LOAD_Y ? I.y : I.w) + o.pix, x[0], x[1]);
  } else if constexpr (OP == OP_LOAD_D_U) {
    ld_map_pair<T>(I.d + o.pix, x[0], x[1]);
  } else if constexpr (OP == OP_LOAD_R || OP == OP_LOAD_U) {
    ldc(OP == OP_LOAD_R ? I.r : I.u, o.q, x[0], x[1]);
  } else if constexpr (OP == OP_P_UPD_Z || OP == OP_P_UPD_R) {
    ldc(OP == OP_P_UPD_Z ? I.z : I.r, o.q, x[0], x[1]);
    ldc(I.p, o.q, x[2], x[3]);
  } else if constexpr (OP == OP_R_UPD) {
    ldc(I.r, o.q, x[0], x[1]);
    ldc(I.q, o.q, x[2], x[3]);
    ldc(I.u, o.q, x[4], x[5]);
    ldc(I.p, o.q, x[6], x[7]);
  } else if constexpr (OP == OP_U64_UPD) {
    ldc(I.u, o.q, x[0], x[1]);
    ldc(I.dlt, o.q, x[2], x[3]);
  }
}

template <typename T, int OP>
__device__ __forceinline__ cx<T> src_op(const InstDesc<T>& I, const Opnd& o, const T (&x)[8],
                                        T alpha, T beta, Acc<T>& acc) {
  const PairIdx& q = o.q;
  T a0 = x[0], a1 = x[1];
  if constexpr (OP == OP_LOAD_W_MASK) {
    a0 = q.m0 ? a0 : (T)0;
    a1 = q.m1 ? a1 : (T)0;
  } else if constexpr (OP == OP_LOAD_D_U) {
    a0 = q.m0 ? (T)0 : a0;
    a1 = q.m1 ? (T)0 : a1;
  } else if constexpr (OP == OP_LOAD_R) {
    acc.add_prod(a0, a0);
    acc.add_prod(a1, a1);
  } else if constexpr (OP == OP_P_UPD_Z || OP == OP_P_UPD_R) {
    a0 = x[0] + beta * x[2];
    a1 = x[1] + beta * x[3];
    stc(I.p, q, a0, a1);
  } else if constexpr (OP == OP_R_UPD) {
    a0 = x[0] - alpha * x[2];
    a1 = x[1] - alpha * x[3];
    stc(I.r, q, a0, a1);
    stc(I.u, q, x[4] + alpha * x[6], x[5] + alpha * x[7]);
    acc.add_prod(a0, a0);
    acc.add_prod(a1, a1);
  } else if constexpr (OP == OP_U64_UPD) {
    a0 = x[0] + x[2];
    a1 = x[1] + x[3];
    stc(I.u, q, a0, a1);
    stc(I.dlt, q, 0.f, 0.f);
  }
  return cx<T>{a0, a1};
}

template <typename T, int OP>
__device__ __forceinline__ void sink_load(const InstDesc<T>& I, const Opnd& o, T (&x)[2]) {
  if constexpr (OP == OP_Q || OP == OP_Z || OP == OP_RES) {
    ldc(OP == OP_Q ? I.p : OP == OP_Z ? I.r : I.b, o.q, x[0], x[1]);
  } else if constexpr (OP == OP_GRAD) {
    ld_map_pair<T>(I.gx + o.pix, x[0], x[1]);
  } else if constexpr (OP == OP_RELAX) {
    ld_pair(I.w + o.pix, x[0], x[1]);
  }
}

template <typename T, int OP>
__device__ __forceinline__ void sink_op(const InstDesc<T>& I, const Opnd& o, const T (&x)[2],
                                        cx<T> v, Acc<T>& acc, int param) {
  const PairIdx& q = o.q;
  const int pix = o.pix;
  const bool m0 = q.m0, m1 = q.m1;   // masked = not observed
  T a0 = v.r, a1 = v.i;
  if constexpr (OP == OP_Q || OP == OP_Z) {
    a0 = m0 ? a0 : (T)0;
    a1 = m1 ? a1 : (T)0;
    stc(OP == OP_Q ? I.q : I.z, q, a0, a1);
    acc.add_prod(x[0], a0);
    acc.add_prod(x[1], a1);
  } else if constexpr (OP == OP_B) {
    a0 = m0 ? -a0 : (T)0;
    a1 = m1 ? -a1 : (T)0;
    stc(I.r, q, a0, a1);
    if (I.b) stc(I.b, q, a0, a1);
    if (I.r32) stc(I.r32, q, a0, a1);
    acc.add_prod(a0, a0);
    acc.add_prod(a1, a1);
  } else if constexpr (OP == OP_RES) {
    a0 = x[0] - (m0 ? a0 : (T)0);
    a1 = x[1] - (m1 ? a1 : (T)0);
    stc(I.r, q, a0, a1);
    if (I.r32) stc(I.r32, q, a0, a1);
    acc.add_prod(a0, a0);
    acc.add_prod(a1, a1);
  } else if constexpr (OP == OP_GRAD) {
    st_map_pair<T>(I.out + pix, m0 ? (T)0 : x[0] - a0, m1 ? (T)0 : x[1] - a1);
    st_pair(I.y + pix, m0 ? x[0] : a0, m1 ? x[1] : a1);
  } else if constexpr (OP == OP_RELAX) {
    const T step = (T)I.st->alpha;
    a0 = m0 ? a0 : (T)0;
    a1 = m1 ? a1 : (T)0;
    st_pair(I.w + pix, x[0] - step * a0, x[1] - step * a1);
    acc.add_prod(a0, a0);
    acc.add_prod(a1, a1);
  } else if constexpr (OP == OP_KSEL) {
    const uchar2 c = *reinterpret_cast<const uchar2*>(I.cls + pix);
    if (m0 && c.x == param) I.y[pix] = a0;
    if (m1 && c.y == param) I.y[pix + 1] = a1;
  } else if constexpr (OP == OP_STORE_Y) {
    st_pair(I.y + pix, a0, a1);
  } else if constexpr (OP == OP_STORE_Y_MASK) {
    st_pair(I.y + pix, m0 ? a0 : (T)0, m1 ? a1 : (T)0);
  }
}

template <typename T, int OP>
__device__ __forceinline__ cx<T> mid_op(const InstDesc<T>& I, const Opnd& o, T d0, T d1, cx<T> v) {
  if constexpr (OP == OP_Y_W) {
    st_pair(I.y + o.pix, v.r, v.i);
    return cx<T>{o.q.m0 ? (T)0 : d0 - v.r, o.q.m1 ? (T)0 : d1 - v.i};
  } else {
    return cx<T>{o.q.m0 ? v.r : (T)0, o.q.m1 ? v.i : (T)0};
  }
}

// Operands of the chunk's pixel pairs j = j0 + u nt: mask words first.
template <int OP_NEEDS_WORD>
__device__ __forceinline__ void chunk_words(const uint2* mw, int rowpix, int j0, int nt, int L,
                                            Opnd (&o)[kGenChunk]) {
#pragma unroll
  for (int u = 0; u < kGenChunk; ++u) {
    const int j = j0 + u * nt;
    o[u].ok = j < L;
    o[u].pix = rowpix + 2 * (o[u].ok ? j : 0);
    if (OP_NEEDS_WORD) o[u].q = pair_index(mw, o[u].pix);
  }
}

template <typename T, int OP>
__device__ __forceinline__ void src_row(const InstDesc<T>& I, int rowpix, cx<T>* z, int L, int t,
                                        int nt, T alpha, T beta, Acc<T>& acc) {
  constexpr bool W = !(OP == OP_LOAD_W || OP == OP_LOAD_Y);
  for (int j0 = t; j0 < L; j0 += kGenChunk * nt) {
    Opnd o[kGenChunk];
    chunk_words<W>(I.mw, rowpix, j0, nt, L, o);
    T x[kGenChunk][8];
#pragma unroll
    for (int u = 0; u < kGenChunk; ++u)
      if (o[u].ok) src_load<T, OP>(I, o[u], x[u]);
#pragma unroll
    for (int u = 0; u < kGenChunk; ++u)
      if (o[u].ok) z[j0 + u * nt] = src_op<T, OP>(I, o[u], x[u], alpha, beta, acc);
  }
}

template <typename T, int OP>
__device__ __forceinline__ void sink_row(const InstDesc<T>& I, int rowpix, const cx<T>* z, int L,
                                         int t, int nt, Acc<T>& acc, int param) {
  for (int j0 = t; j0 < L; j0 += kGenChunk * nt) {
    Opnd o[kGenChunk];
    chunk_words<1>(I.mw, rowpix, j0, nt, L, o);
    T x[kGenChunk][2];
#pragma unroll
    for (int u = 0; u < kGenChunk; ++u)
      if (o[u].ok) sink_load<T, OP>(I, o[u], x[u]);
#pragma unroll
    for (int u = 0; u < kGenChunk; ++u)
      if (o[u].ok) sink_op<T, OP>(I, o[u], x[u], z[j0 + u * nt], acc, param);
  }
}

template <typename T, int OP>
__device__ __forceinline__ void mid_row(const InstDesc<T>& I, int rowpix, cx<T>* z, int L, int t,
                                        int nt) {
  for (int j0 = t; j0 < L; j0 += kGenChunk * nt) {
    Opnd o[kGenChunk];
    chunk_words<1>(I.mw, rowpix, j0, nt, L, o);
    T d[kGenChunk][2];
#pragma unroll
    for (int u = 0; u < kGenChunk; ++u)
      if (o[u].ok && OP == OP_Y_W) ld_map_pair<T>(I.d + o[u].pix, d[u][0], d[u][1]);
#pragma unroll
    for (int u = 0; u < kGenChunk; ++u)
      if (o[u].ok) z[j0 + u * nt] = mid_op<T, OP>(I, o[u], d[u][0], d[u][1], z[j0 + u * nt]);
  }
}

}  // namespace gen

// ----------------------------------------------------------------- row pass
// CTA = `rows` consecutive grid rows, g.nt threads per row; blockIdx.y is the
// instance.  Shared memory: two buffers of L + 1 complex values per row.
template <typename T, bool IN_SPEC, bool OUT_SPEC, bool XI = false>
__global__ void __launch_bounds__(KCfg<T>::kMaxThreads)
k_row_gen(const InstDesc<T>* __restrict__ insts, RowArgs a, GenLen g, const T* __restrict__ wl,
          const T* __restrict__ wx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const InstDesc<T>& I = insts[blockIdx.y];
  if (skip_instance(a.check_done, I.st)) return;
  const int L = g.n, nt = g.nt, rows = a.rows, ny = a.ny, stride = 2 * (L + 1);
  const int row = threadIdx.x / nt, t = threadIdx.x - row * nt;
  const int y0 = blockIdx.x * rows;
  const int rowpix = (y0 + row) * a.nx;
  cx<T>* base = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* A = base + row * stride;
  cx<T>* B = A + (L + 1);
  cx<T>* Z = A;   // the buffer holding the row's values
  Acc<T> acc;

  if constexpr (IN_SPEC) {
    const T* spec = a.spec_sel ? I.spec2 : I.spec;
    // X[k] of the `rows` rows: consecutive threads take consecutive rows of one k
    const int total = (L + 1) * rows;
    for (int f0 = threadIdx.x; f0 < total; f0 += gen::kGenChunk * blockDim.x) {
      cx<T> tv[gen::kGenChunk];
#pragma unroll
      for (int u = 0; u < gen::kGenChunk; ++u) {
        const int f = f0 + u * blockDim.x;
        if (f < total)
          tv[u] = ldg_cx<T>(spec + 2 * ((size_t)(f >> a.log_rows) * ny + y0 + (f & (rows - 1))));
      }
#pragma unroll
      for (int u = 0; u < gen::kGenChunk; ++u) {
        const int f = f0 + u * blockDim.x;
        if (f < total) base[(f & (rows - 1)) * stride + (f >> a.log_rows)] = tv[u];
      }
    }
    __syncthreads();
    // C2R: Z[k] = (X[k] + conj X[L-k]) + i e^{+2 pi i k/nx} (X[k] - conj X[L-k])
    for (int k = t; k < L; k += nt) {
      cx<T> xk = A[k], xc = conjx(A[L - k]);
      if (k == 0) {
        xk.i = (T)0;
        xc.i = (T)0;
      }
      const cx<T> sum = xk + xc;
      const cx<T> dif = cmulc(xk - xc, gen::tw_at(wx, k));
      B[k] = cx<T>{sum.r - dif.i, sum.i + dif.r};
    }
    __syncthreads();
    Z = gen::fft<T>(B, A, g, wl, t, true);   // Z[j] = x[2j] + i x[2j+1] (scaled)
    if constexpr (OUT_SPEC) {
      if (a.op == OP_Y_W)
        gen::mid_row<T, OP_Y_W>(I, rowpix, Z, L, t, nt);
      else
        gen::mid_row<T, OP_MASK>(I, rowpix, Z, L, t, nt);
    } else {
      switch (a.op) {
        case OP_Q: gen::sink_row<T, OP_Q>(I, rowpix, Z, L, t, nt, acc, 0); break;
        case OP_Z: gen::sink_row<T, OP_Z>(I, rowpix, Z, L, t, nt, acc, 0); break;
        case OP_B: gen::sink_row<T, OP_B>(I, rowpix, Z, L, t, nt, acc, 0); break;
        case OP_RES: gen::sink_row<T, OP_RES>(I, rowpix, Z, L, t, nt, acc, 0); break;
        case OP_GRAD: gen::sink_row<T, OP_GRAD>(I, rowpix, Z, L, t, nt, acc, 0); break;
        case OP_RELAX: gen::sink_row<T, OP_RELAX>(I, rowpix, Z, L, t, nt, acc, 0); break;
        case OP_KSEL: gen::sink_row<T, OP_KSEL>(I, rowpix, Z, L, t, nt, acc, a.param); break;
        case OP_STORE_Y: gen::sink_row<T, OP_STORE_Y>(I, rowpix, Z, L, t, nt, acc, 0); break;
        case OP_STORE_Y_MASK:
          gen::sink_row<T, OP_STORE_Y_MASK>(I, rowpix, Z, L, t, nt, acc, 0);
          break;
        default: break;
      }
    }
  } else if constexpr (XI) {
    for (int j = t; j < L; j += nt) {
      double x0, x1;
      normal_pair(I.seed, (uint32_t)((rowpix >> 1) + j), x0, x1);
      A[j] = cx<T>{(T)x0, (T)x1};
    }
  } else {
    const T alpha = (T)I.st->alpha, beta = (T)I.st->beta;
    switch (a.op) {
      case OP_R_UPD: gen::src_row<T, OP_R_UPD>(I, rowpix, A, L, t, nt, alpha, beta, acc); break;
      case OP_P_UPD_Z:
        gen::src_row<T, OP_P_UPD_Z>(I, rowpix, A, L, t, nt, alpha, beta, acc);
        break;
      case OP_P_UPD_R:
        gen::src_row<T, OP_P_UPD_R>(I, rowpix, A, L, t, nt, alpha, beta, acc);
        break;
      case OP_LOAD_R: gen::src_row<T, OP_LOAD_R>(I, rowpix, A, L, t, nt, alpha, beta, acc); break;
      case OP_LOAD_U: gen::src_row<T, OP_LOAD_U>(I, rowpix, A, L, t, nt, alpha, beta, acc); break;
      case OP_LOAD_Y: gen::src_row<T, OP_LOAD_Y>(I, rowpix, A, L, t, nt, alpha, beta, acc); break;
      case OP_LOAD_W: gen::src_row<T, OP_LOAD_W>(I, rowpix, A, L, t, nt, alpha, beta, acc); break;
      case OP_LOAD_W_MASK:
        gen::src_row<T, OP_LOAD_W_MASK>(I, rowpix, A, L, t, nt, alpha, beta, acc);
        break;
      case OP_LOAD_D_U:
        gen::src_row<T, OP_LOAD_D_U>(I, rowpix, A, L, t, nt, alpha, beta, acc);
        break;
      case OP_U64_UPD:
        gen::src_row<T, OP_U64_UPD>(I, rowpix, A, L, t, nt, alpha, beta, acc);
        break;
      default:
        for (int j = t; j < L; j += nt) A[j] = cx<T>{(T)0, (T)0};
        break;
    }
  }

  if constexpr (OUT_SPEC) {
    __syncthreads();
    Z = gen::fft<T>(Z, Z == A ? B : A, g, wl, t, false);
    const int off = (Z == A) ? 0 : L + 1;   // the same buffer in every row
    // R2C: X[k] = (Z[k] + conj Z[L-k]) / 2 - (i/2) e^{-2 pi i k/nx} (Z[k] - conj Z[L-k]),
    // X[L] = Re Z[0] - Im Z[0]; stored transposed, consecutive threads on consecutive rows
    T* spec = a.spec_sel ? I.spec2 : I.spec;
    for (int f = threadIdx.x; f < (L + 1) * rows; f += blockDim.x) {
      const int k = f >> a.log_rows, r = f & (rows - 1);
      const cx<T>* Zr = base + r * stride + off;
      cx<T> X;
      if (k < L) {
        const cx<T> zk = Zr[k], zc = conjx(Zr[k == 0 ? 0 : L - k]);
        const cx<T> ev = scal(zk + zc, (T)0.5);
        const cx<T> od = scal(mul_mi<T, false>(zk - zc), (T)0.5);
        X = ev + cmul(od, gen::tw_at(wx, k));
      } else {
        const cx<T> z0 = Zr[0];
        X = cx<T>{z0.r - z0.i, (T)0};
      }
      st_cx<T>(spec + 2 * ((size_t)k * ny + y0 + r), X);
    }
  }

  if (a.sop != SC_NONE)
    grid_reduce(acc.value(), red, I.partial, I.st, a.sop, gridDim.x, blockIdx.x);
}

// ----------------------------------------------------------------- column pass
// CTA = `ffts` spectrum rows (one kx each), g.nt threads per column; forward
// FFT, x table, inverse FFT, in place (table < 0: forward only; PRE: input
// already transformed in spec, output to spec_sel's buffer).  Shared memory:
// two buffers of ny complex values per column.
template <typename T, bool PRE = false>
__global__ void __launch_bounds__(KCfg<T>::kMaxThreads)
k_col_gen(const InstDesc<T>* __restrict__ insts, ColArgs a, GenLen g, const T* __restrict__ wn) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const InstDesc<T>& I = insts[blockIdx.x];
  if (skip_instance(a.check_done, I.st)) return;
  const int N = g.n;
  const int f = threadIdx.x / g.nt, t = threadIdx.x - f * g.nt;
  const int kx = blockIdx.y * a.ffts + f;
  const bool act = kx < a.nkx;
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw) + f * 2 * N;
  cx<T>* B = A + N;
  T* col = (a.spec_sel ? I.spec2 : I.spec) + 2 * (long long)(act ? kx : 0) * N;
  const T* srcp = PRE ? I.spec + 2 * (long long)(act ? kx : 0) * N : col;
  for (int j = t; j < N; j += g.nt) A[j] = act ? ld_cx<T>(srcp + 2 * j) : cx<T>{(T)0, (T)0};
  __syncthreads();
  cx<T>* Z = A;
  if constexpr (!PRE) Z = gen::fft<T>(A, B, g, wn, t, false);
  if (a.table >= 0) {
    const T* tab = (a.table >= 2 ? I.kt + (long long)(a.table - 2) * a.nkx * N
                    : a.table ? I.t_sqrt : I.t_inv) + (long long)(act ? kx : 0) * N;
    for (int j = t; j < N; j += g.nt) Z[j] = scal(Z[j], act ? ldg1(tab + j) : (T)0);
    __syncthreads();
    Z = gen::fft<T>(Z, Z == A ? B : A, g, wn, t, true);
  }
  if (act)
    for (int j = t; j < N; j += g.nt) st_cx<T>(col + 2 * j, Z[j]);
}

// ----------------------------------------------------------------- launchers
template <typename T>
size_t GenLaunch<T>::row_smem(int L, int rows) {
  return size_t(rows) * 2 * (L + 1) * sizeof(cx<T>);
}

template <typename T>
size_t GenLaunch<T>::col_smem(int ny, int ffts) {
  return size_t(ffts) * 2 * ny * sizeof(cx<T>);
}

template <typename T>
int GenLaunch<T>::max_threads() { return KCfg<T>::kMaxThreads; }

template <typename T>
cudaError_t GenLaunch<T>::row(bool in_spec, bool out_spec, const InstDesc<T>* d, int ninst,
                              const RowArgs& a, const GenLen& g, const T* wl, const T* wx,
                              cudaStream_t s) {
  const dim3 grid(a.ny / a.rows, ninst), block(a.rows * g.nt);
  const size_t sm = row_smem(g.n, a.rows);
  if (in_spec && out_spec)
    k_row_gen<T, true, true><<<grid, block, sm, s>>>(d, a, g, wl, wx);
  else if (in_spec)
    k_row_gen<T, true, false><<<grid, block, sm, s>>>(d, a, g, wl, wx);
  else if (a.op == OP_XI)
    k_row_gen<T, false, true, true><<<grid, block, sm, s>>>(d, a, g, wl, wx);
  else
    k_row_gen<T, false, true><<<grid, block, sm, s>>>(d, a, g, wl, wx);
  return cudaGetLastError();
}

template <typename T>
cudaError_t GenLaunch<T>::col(const InstDesc<T>* d, int ninst, const ColArgs& a, const GenLen& g,
                              const T* wn, cudaStream_t s) {
  const dim3 grid(ninst, (a.nkx + a.ffts - 1) / a.ffts), block(a.ffts * g.nt);
  const size_t sm = col_smem(g.n, a.ffts);
  if (a.pre)
    k_col_gen<T, true><<<grid, block, sm, s>>>(d, a, g, wn);
  else
    k_col_gen<T><<<grid, block, sm, s>>>(d, a, g, wn);
  return cudaGetLastError();
}

template <typename T>
cudaError_t GenLaunch<T>::prepare() {
  cudaError_t e = detail::allow_smem(k_row_gen<T, true, true>);
  if (e == cudaSuccess) e = detail::allow_smem(k_row_gen<T, true, false>);
  if (e == cudaSuccess) e = detail::allow_smem(k_row_gen<T, false, true>);
  if (e == cudaSuccess) e = detail::allow_smem(k_row_gen<T, false, true, true>);
  if (e == cudaSuccess) e = detail::allow_smem(k_col_gen<T>);
  if (e == cudaSuccess) e = detail::allow_smem(k_col_gen<T, true>);
  return e;
}

}  // namespace cgf
