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
  for (int b = t; b < nb; b += nt) {
    const int k = b % ns;
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
    const int base = (b - k) * R + k;
#pragma unroll
    for (int m = 0; m < R; ++m) out[base + m * ns] = cout ? conjx(v[m]) : v[m];
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
template <typename T, int OP>
__device__ __forceinline__ cx<T> src(const InstDesc<T>& I, int pix, T alpha, T beta, Acc<T>& acc) {
  T a0 = (T)0, a1 = (T)0;
  if constexpr (OP == OP_LOAD_W || OP == OP_LOAD_Y) {
    ld_pair((OP == OP_LOAD_Y ? I.y : I.w) + pix, a0, a1);
  } else {
    const PairIdx q = pair_index(I.mw, pix);
    if constexpr (OP == OP_LOAD_W_MASK) {
      T x0, x1;
      ld_pair(I.w + pix, x0, x1);
      a0 = q.m0 ? x0 : (T)0;
      a1 = q.m1 ? x1 : (T)0;
    } else if constexpr (OP == OP_LOAD_D_U) {
      T x0, x1;
      ld_map_pair<T>(I.d + pix, x0, x1);
      a0 = q.m0 ? (T)0 : x0;
      a1 = q.m1 ? (T)0 : x1;
    } else if constexpr (OP == OP_LOAD_R || OP == OP_LOAD_U) {
      ldc(OP == OP_LOAD_R ? I.r : I.u, q, a0, a1);
      if constexpr (OP == OP_LOAD_R) {
        acc.add_prod(a0, a0);
        acc.add_prod(a1, a1);
      }
    } else if constexpr (OP == OP_P_UPD_Z || OP == OP_P_UPD_R) {
      T x0, x1, y0, y1;
      ldc(OP == OP_P_UPD_Z ? I.z : I.r, q, x0, x1);
      ldc(I.p, q, y0, y1);
      a0 = x0 + beta * y0;
      a1 = x1 + beta * y1;
      stc(I.p, q, a0, a1);
    } else if constexpr (OP == OP_R_UPD) {
      T x0, x1, y0, y1, z0, z1, w0, w1;
      ldc(I.r, q, x0, x1);
      ldc(I.q, q, y0, y1);
      ldc(I.u, q, z0, z1);
      ldc(I.p, q, w0, w1);
      a0 = x0 - alpha * y0;
      a1 = x1 - alpha * y1;
      stc(I.r, q, a0, a1);
      stc(I.u, q, z0 + alpha * w0, z1 + alpha * w1);
      acc.add_prod(a0, a0);
      acc.add_prod(a1, a1);
    } else if constexpr (OP == OP_U64_UPD) {
      T x0, x1, y0, y1;
      ldc(I.u, q, x0, x1);
      ldc(I.dlt, q, y0, y1);
      a0 = x0 + y0;
      a1 = x1 + y1;
      stc(I.u, q, a0, a1);
      stc(I.dlt, q, 0.f, 0.f);
    }
  }
  return cx<T>{a0, a1};
}

template <typename T, int OP>
__device__ __forceinline__ void sink(const InstDesc<T>& I, int pix, cx<T> v, Acc<T>& acc,
                                     int param) {
  const PairIdx q = pair_index(I.mw, pix);
  const bool m0 = q.m0, m1 = q.m1;   // masked = not observed
  T a0 = v.r, a1 = v.i;
  if constexpr (OP == OP_Q || OP == OP_Z) {
    T x0, x1;
    ldc(OP == OP_Q ? I.p : I.r, q, x0, x1);
    a0 = m0 ? a0 : (T)0;
    a1 = m1 ? a1 : (T)0;
    stc(OP == OP_Q ? I.q : I.z, q, a0, a1);
    acc.add_prod(x0, a0);
    acc.add_prod(x1, a1);
  } else if constexpr (OP == OP_B) {
    a0 = m0 ? -a0 : (T)0;
    a1 = m1 ? -a1 : (T)0;
    stc(I.r, q, a0, a1);
    if (I.b) stc(I.b, q, a0, a1);
    if (I.r32) stc(I.r32, q, a0, a1);
    acc.add_prod(a0, a0);
    acc.add_prod(a1, a1);
  } else if constexpr (OP == OP_RES) {
    T x0, x1;
    ldc(I.b, q, x0, x1);
    a0 = x0 - (m0 ? a0 : (T)0);
    a1 = x1 - (m1 ? a1 : (T)0);
    stc(I.r, q, a0, a1);
    if (I.r32) stc(I.r32, q, a0, a1);
    acc.add_prod(a0, a0);
    acc.add_prod(a1, a1);
  } else if constexpr (OP == OP_GRAD) {
    T x0, x1;
    ld_map_pair<T>(I.gx + pix, x0, x1);
    st_map_pair<T>(I.out + pix, m0 ? (T)0 : x0 - a0, m1 ? (T)0 : x1 - a1);
    st_pair(I.y + pix, m0 ? x0 : a0, m1 ? x1 : a1);
  } else if constexpr (OP == OP_RELAX) {
    T x0, x1;
    ld_pair(I.w + pix, x0, x1);
    const T step = (T)I.st->alpha;
    a0 = m0 ? a0 : (T)0;
    a1 = m1 ? a1 : (T)0;
    st_pair(I.w + pix, x0 - step * a0, x1 - step * a1);
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
__device__ __forceinline__ cx<T> mid(const InstDesc<T>& I, int pix, cx<T> v) {
  const PairIdx q = pair_index(I.mw, pix);
  if constexpr (OP == OP_Y_W) {
    T d0, d1;
    ld_map_pair<T>(I.d + pix, d0, d1);
    st_pair(I.y + pix, v.r, v.i);
    return cx<T>{q.m0 ? (T)0 : d0 - v.r, q.m1 ? (T)0 : d1 - v.i};
  } else {
    return cx<T>{q.m0 ? v.r : (T)0, q.m1 ? v.i : (T)0};
  }
}

template <typename T, int OP>
__device__ __forceinline__ void src_row(const InstDesc<T>& I, int rowpix, cx<T>* z, int L, int t,
                                        int nt, T alpha, T beta, Acc<T>& acc) {
  for (int j = t; j < L; j += nt) z[j] = src<T, OP>(I, rowpix + 2 * j, alpha, beta, acc);
}
template <typename T, int OP>
__device__ __forceinline__ void sink_row(const InstDesc<T>& I, int rowpix, const cx<T>* z, int L,
                                         int t, int nt, Acc<T>& acc, int param) {
  for (int j = t; j < L; j += nt) sink<T, OP>(I, rowpix + 2 * j, z[j], acc, param);
}
template <typename T, int OP>
__device__ __forceinline__ void mid_row(const InstDesc<T>& I, int rowpix, cx<T>* z, int L, int t,
                                        int nt) {
  for (int j = t; j < L; j += nt) z[j] = mid<T, OP>(I, rowpix + 2 * j, z[j]);
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
    for (int f = threadIdx.x; f < (L + 1) * rows; f += blockDim.x) {
      const int k = f / rows, r = f - k * rows;
      base[r * stride + k] = ldg_cx<T>(spec + 2 * ((size_t)k * ny + y0 + r));
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
      const int k = f / rows, r = f - k * rows;
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
