// Mixed-radix pass kernels (radix 2, 3, 4, 5, 7, 8, in-place DIF / DIT
// transforms) and their launchers; see cg_generic.h.  The fused operations
// are those of cg_kernels.cuh, applied per pixel pair; mask flags and compact
// indices come from the global mask words (a row need not start on a word
// boundary here).
#pragma once
#include "cg_generic.h"
#include "cg_launch.cuh"

namespace cgf {
namespace gen {

// The V values of one position of a thread group's transforms (one 16-byte
// shared-memory access for two FP32 transforms).
template <typename T, int V>
__device__ __forceinline__ void ld_slot(const cx<T>* p, cx<T> (&v)[V]) {
  if constexpr (V % 2 == 0 && std::is_same<T, float>::value) {
#pragma unroll
    for (int h = 0; h < V; h += 2) {
      const float4 a = *reinterpret_cast<const float4*>(p + h);
      v[h] = cx<float>{a.x, a.y};
      v[h + 1] = cx<float>{a.z, a.w};
    }
  } else {
#pragma unroll
    for (int u = 0; u < V; ++u) v[u] = ld_cx<T>(reinterpret_cast<const T*>(p + u));
  }
}
template <typename T, int V>
__device__ __forceinline__ void st_slot(cx<T>* p, const cx<T> (&v)[V]) {
  if constexpr (V % 2 == 0 && std::is_same<T, float>::value) {
#pragma unroll
    for (int h = 0; h < V; h += 2)
      *reinterpret_cast<float4*>(p + h) = make_float4(v[h].r, v[h].i, v[h + 1].r, v[h + 1].i);
  } else {
#pragma unroll
    for (int u = 0; u < V; ++u) st_cx<T>(reinterpret_cast<T*>(p + u), v[u]);
  }
}

// cos and sin of 2 pi j / R for the odd radices (j = 1 .. (R-1)/2), each the
// double nearest the exact value (from a 50-digit evaluation of the series).
CGF_HD constexpr double radix_cos(int R, int j) {
  return R == 3 ? -0.5
       : R == 5 ? (j == 1 ? 0.30901699437494745 : -0.8090169943749475)
       : (j == 1 ? 0.6234898018587335 : j == 2 ? -0.2225209339563144 : -0.9009688679024191);
}
CGF_HD constexpr double radix_sin(int R, int j) {
  return R == 3 ? 0.8660254037844386
       : R == 5 ? (j == 1 ? 0.9510565162951535 : 0.5877852522924731)
       : (j == 1 ? 0.7818314824680298 : j == 2 ? 0.9749279121818236 : 0.4338837391175581);
}

// In-register DFT of R points, y_q = sum_m v_m W_R^{+-qm} (W_R = e^{-2 pi i/R};
// the inverse takes the conjugate).  For odd R the terms m and R - m pair up:
// with S_m = v_m + v_{R-m}, D_m = v_m - v_{R-m} (m = 1..H, H = (R-1)/2) and
// theta = 2 pi q m / R,
//   y_q = v_0 + sum_m cos(theta) S_m -+ i sum_m sin(theta) D_m,
//   y_{R-q} = the same with the other sign,
// so each half-pair costs real-by-complex products only, with the cosines
// and sines compile-time constants.
template <typename T, int R, bool INV>
__device__ __forceinline__ void dft(cx<T> (&v)[R]) {
  if constexpr (R == 2) {
    const cx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  } else if constexpr (R == 4) {
    const cx<T> s02 = v[0] + v[2], d02 = v[0] - v[2];
    const cx<T> s13 = v[1] + v[3], d13 = mul_mi<T, INV>(v[1] - v[3]);
    v[0] = s02 + s13;
    v[2] = s02 - s13;
    v[1] = d02 + d13;
    v[3] = d02 - d13;
  } else if constexpr (R == 8) {
    // two 4-point DFTs (even, odd inputs), then y_q = E_q + W_8^q O_q and
    // y_{q+4} = E_q - W_8^q O_q
    cx<T> e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft<T, 4, INV>(e);
    dft<T, 4, INV>(o);
    const T h = T(0.70710678118654752);   // 1 / sqrt 2
    // W_8 = (1 - i) / sqrt 2, W_8^3 = (-1 - i) / sqrt 2 (conjugates for the inverse)
    const cx<T> o1 = INV ? cx<T>{(o[1].r - o[1].i) * h, (o[1].i + o[1].r) * h}
                         : cx<T>{(o[1].r + o[1].i) * h, (o[1].i - o[1].r) * h};
    const cx<T> o2 = mul_mi<T, INV>(o[2]);
    const cx<T> o3 = INV ? cx<T>{-(o[3].r + o[3].i) * h, (o[3].r - o[3].i) * h}
                         : cx<T>{(o[3].i - o[3].r) * h, -(o[3].r + o[3].i) * h};
    v[0] = e[0] + o[0];
    v[4] = e[0] - o[0];
    v[1] = e[1] + o1;
    v[5] = e[1] - o1;
    v[2] = e[2] + o2;
    v[6] = e[2] - o2;
    v[3] = e[3] + o3;
    v[7] = e[3] - o3;
  } else {
    constexpr int H = (R - 1) / 2;
    cx<T> S[H + 1], D[H + 1];
    const cx<T> v0 = v[0];
    cx<T> y0 = v0;
#pragma unroll
    for (int m = 1; m <= H; ++m) {
      S[m] = v[m] + v[R - m];
      D[m] = v[m] - v[R - m];
      y0 = y0 + S[m];
    }
    v[0] = y0;
#pragma unroll
    for (int q = 1; q <= H; ++q) {
      cx<T> a = v0, b{(T)0, (T)0};
#pragma unroll
      for (int m = 1; m <= H; ++m) {
        const int j = (q * m) % R, jj = j <= H ? j : R - j;
        const T c = T(radix_cos(R, jj));
        const T sn = T(j <= H ? radix_sin(R, jj) : -radix_sin(R, jj));   // sin 2 pi j / R
        a = a + scal(S[m], c);
        b = b + scal(D[m], sn);
      }
      const cx<T> mib{b.i, -b.r}, pib{-b.i, b.r};   // -i b, +i b
      v[q] = INV ? a + pib : a + mib;
      v[R - q] = INV ? a + mib : a + pib;
    }
  }
}

// One stage of radix R over blocks of ns points (h = ns / R, nb = n / R
// butterflies; butterfly b = blk h + j reads and writes positions
// blk ns + j + m h).  Forward (DIF): DFT, then the twiddles W_ns^{q j} on the
// outputs; inverse (transposed, conjugate): conjugate twiddles on the inputs,
// then the inverse DFT.  `tws` is the stage's twiddle table (unused when
// h = 1).  Thread t of nt takes butterflies t, t + nt, ...
template <typename T, int V, int R, bool INV>
__device__ __forceinline__ void stage(cx<T>* z, int ns, int h, int nb, const T* tws, int t,
                                      int nt) {
  const bool twd = h > 1;
  const int hv = h * V;
  int blk = t / h, j = t - blk * h;
  const int dblk = nt / h, dj = nt - dblk * h;
  for (int b = t; b < nb; b += nt) {
    cx<T>* p = z + (blk * ns + j) * V;
    const T* wj = tws + 2 * (j * (R - 1));
    cx<T> v[V][R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      cx<T> sl[V];
      ld_slot<T, V>(p + m * hv, sl);
#pragma unroll
      for (int u = 0; u < V; ++u) v[u][m] = sl[u];
    }
    if constexpr (INV) {
      if (twd) {
#pragma unroll
        for (int m = 1; m < R; ++m) {
          const cx<T> w = ldg_cx<T>(wj + 2 * (m - 1));
#pragma unroll
          for (int u = 0; u < V; ++u) v[u][m] = cmulc(v[u][m], w);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < V; ++u) dft<T, R, INV>(v[u]);
    if constexpr (!INV) {
      if (twd) {
#pragma unroll
        for (int m = 1; m < R; ++m) {
          const cx<T> w = ldg_cx<T>(wj + 2 * (m - 1));
#pragma unroll
          for (int u = 0; u < V; ++u) v[u][m] = cmul(v[u][m], w);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) {
      cx<T> sl[V];
#pragma unroll
      for (int u = 0; u < V; ++u) sl[u] = v[u][m];
      st_slot<T, V>(p + m * hv, sl);
    }
    j += dj;
    blk += dblk;
    if (j >= h) {
      j -= h;
      ++blk;
    }
  }
}

template <typename T, int V, bool INV>
__device__ __forceinline__ void stage_r(int R, cx<T>* z, int ns, int h, int nb, const T* tws,
                                        int t, int nt) {
  switch (R) {
    case 2: stage<T, V, 2, INV>(z, ns, h, nb, tws, t, nt); break;
    case 3: stage<T, V, 3, INV>(z, ns, h, nb, tws, t, nt); break;
    case 4: stage<T, V, 4, INV>(z, ns, h, nb, tws, t, nt); break;
    case 5: stage<T, V, 5, INV>(z, ns, h, nb, tws, t, nt); break;
    case 8: stage<T, V, 8, INV>(z, ns, h, nb, tws, t, nt); break;
    default: stage<T, V, 7, INV>(z, ns, h, nb, tws, t, nt); break;
  }
}

// Forward stages 0 .. s_end - 1 of the transform in z (natural order in; after
// all stages, digit-reversed order out).  Every thread of the CTA calls it: a
// CTA barrier follows every stage.
template <typename T, int V>
__device__ void dif(cx<T>* z, const GenLen& g, const T* tw, int t, int s_end) {
  int ns = g.n;
  for (int s = 0; s < s_end; ++s) {
    const int R = g.radix[s], h = ns / R;
    stage_r<T, V, false>(R, z, ns, h, g.n / R, tw + 2 * g.twoff[s], t, g.nt);
    __syncthreads();
    ns = h;
  }
}

// Inverse stages s_top - 1 down to 0 (digit-reversed order in, natural order
// out after stage 0), with a CTA barrier after every stage.
template <typename T, int V>
__device__ void dit(cx<T>* z, const GenLen& g, const T* tw, int t, int s_top) {
  int h = g.n;   // n_{s_top}: the points below stage s_top
  for (int s = 0; s < s_top; ++s) h /= g.radix[s];
  for (int s = s_top - 1; s >= 0; --s) {
    const int R = g.radix[s], ns = h * R;
    stage_r<T, V, true>(R, z, ns, h, g.n / R, tw + 2 * g.twoff[s], t, g.nt);
    __syncthreads();
    h = ns;
  }
}

// Half spectrum -> digit-reversed complex row (C2R by a half-length FFT):
// Z[k] = (X[k] + conj X[L-k]) + i e^{+2 pi i k/nx} (X[k] - conj X[L-k]) for
// k < L, the imaginary parts of X[0] and X[L] dropped; stored at position
// pos[k].  A thread takes k and L - k together (one load of each).  Rows at or
// beyond ny (the padding row of an odd ny) read zeros.
template <typename T>
__device__ __forceinline__ cx<T> c2r_one(cx<T> xk, cx<T> xm, cx<T> w) {
  const cx<T> xc = conjx(xm);
  const cx<T> sum = xk + xc;
  const cx<T> dif = cmulc(xk - xc, w);
  return cx<T>{sum.r - dif.i, sum.i + dif.r};
}
template <typename T>
__device__ __forceinline__ cx<T> r2c_one(cx<T> zk, cx<T> zm, cx<T> w) {
  const cx<T> zc = conjx(zm);
  const cx<T> ev = scal(zk + zc, (T)0.5);
  const cx<T> od = scal(mul_mi<T, false>(zk - zc), (T)0.5);
  return ev + cmul(od, w);
}

constexpr int kGenChunk = 4;

// Rows y0 .. y0 + V - 1 of half-spectrum row k (element offset off = k ny + y0):
// one 16-byte access per two FP32 rows when ny is even (off is then even) and
// the group lies inside the grid; rows at or beyond ny (nv < V) read zeros
// and are not written.
template <typename T, int V>
__device__ __forceinline__ void ld_spec(const T* spec, size_t off, int nv, bool vec,
                                        cx<T> (&x)[V]) {
  if constexpr (V % 2 == 0 && std::is_same<T, float>::value) {
    if (vec && nv == V) {
#pragma unroll
      for (int h = 0; h < V; h += 2) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(spec + 2 * (off + h)));
        x[h] = cx<float>{a.x, a.y};
        x[h + 1] = cx<float>{a.z, a.w};
      }
      return;
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v) x[v] = v < nv ? ldg_cx<T>(spec + 2 * (off + v)) : cx<T>{(T)0, (T)0};
}
template <typename T, int V>
__device__ __forceinline__ void st_spec(T* spec, size_t off, int nv, bool vec, const cx<T> (&x)[V]) {
  if constexpr (V % 2 == 0 && std::is_same<T, float>::value) {
    if (vec && nv == V) {
#pragma unroll
      for (int h = 0; h < V; h += 2)
        *reinterpret_cast<float4*>(spec + 2 * (off + h)) =
            make_float4(x[h].r, x[h].i, x[h + 1].r, x[h + 1].i);
      return;
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v)
    if (v < nv) st_cx<T>(spec + 2 * (off + v), x[v]);
}

template <typename T, int V>
__device__ __forceinline__ void c2r(const T* spec, int ny, int y0, const GenLen& g, const T* wx,
                                    cx<T>* z, int t, int nt) {
  const int L = g.n, half = L / 2, nv = min(V, ny - y0);
  const bool vec = (ny & 1) == 0;
  constexpr int CH = 2;
  for (int k0 = t; k0 <= half; k0 += CH * nt) {
    cx<T> xa[CH][V], xb[CH][V], wa[CH], wb[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int k = min(k0 + c * nt, half), kc = L - k;
      ld_spec<T, V>(spec, (size_t)k * ny + y0, nv, vec, xa[c]);
      ld_spec<T, V>(spec, (size_t)kc * ny + y0, nv, vec, xb[c]);
      wa[c] = ldg_cx<T>(wx + 2 * k);
      wb[c] = ldg_cx<T>(wx + 2 * kc);
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int k = k0 + c * nt, kc = L - k;
      if (k > half) break;
      cx<T> za[V], zb[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        cx<T> p = xa[c][v], q = xb[c][v];
        if (k == 0) {
          p.i = (T)0;
          q.i = (T)0;
        }
        za[v] = c2r_one(p, q, wa[c]);
        zb[v] = c2r_one(q, p, wb[c]);
      }
      st_slot<T, V>(z + (int)g.pos[k] * V, za);
      if (k > 0 && kc != k) st_slot<T, V>(z + (int)g.pos[kc] * V, zb);
    }
  }
}

// Digit-reversed complex row -> half spectrum (R2C):
// X[k] = (Z[k] + conj Z[L-k]) / 2 - (i/2) e^{-2 pi i k/nx} (Z[k] - conj Z[L-k])
// (Z[L] = Z[0]), X[L] = Re Z[0] - Im Z[0]; rows at or beyond ny are not stored.
template <typename T, int V>
__device__ __forceinline__ void r2c(T* spec, int ny, int y0, const GenLen& g, const T* wx,
                                    const cx<T>* z, int t, int nt) {
  const int L = g.n, half = L / 2, nv = min(V, ny - y0);
  const bool vec = (ny & 1) == 0;
  for (int k = t; k <= half; k += nt) {
    const int kc = L - k;
    cx<T> za[V], zb[V];
    ld_slot<T, V>(z + (int)g.pos[k] * V, za);
    if (k == 0) {
#pragma unroll
      for (int v = 0; v < V; ++v) zb[v] = za[v];
    } else {
      ld_slot<T, V>(z + (int)g.pos[kc] * V, zb);
    }
    const cx<T> wa = ldg_cx<T>(wx + 2 * k), wb = ldg_cx<T>(wx + 2 * kc);
    cx<T> xa[V], xb[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      xa[v] = r2c_one(za[v], zb[v], wa);
      xb[v] = k == 0 ? cx<T>{za[v].r - za[v].i, (T)0} : r2c_one(zb[v], za[v], wb);
    }
    st_spec<T, V>(spec, (size_t)k * ny + y0, nv, vec, xa);
    if (k == 0 || kc != k) st_spec<T, V>(spec, (size_t)kc * ny + y0, nv, vec, xb);
  }
}

// ----------------------------------------------------------------- per-pair operations
// Each row loop takes kGenChunk pixel pairs per thread at a time: their mask
// words first, then every operand load, then the arithmetic and stores, so
// the loads of a chunk are in flight together.

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

// Operations whose inputs and outputs are all compact CG vectors: a pixel
// pair without a masked pixel reads nothing, writes nothing, adds nothing to
// the reduction and (sources) contributes zeros to the transform.
template <int OP>
struct CompactOnly {
  static constexpr bool value = OP == OP_R_UPD || OP == OP_P_UPD_Z || OP == OP_P_UPD_R ||
                                OP == OP_LOAD_R || OP == OP_LOAD_U || OP == OP_U64_UPD ||
                                OP == OP_LOAD_W_MASK || OP == OP_Q || OP == OP_Z ||
                                OP == OP_B || OP == OP_RES || OP == OP_KSEL;
};

// The elementwise loops take pixel pair j of all V rows of the group in one
// thread (one shared-memory slot), CH = kGenChunk / V pairs at a time: mask
// words first, then every operand load, then the arithmetic and stores.
// Operands of pairs j = j0 + c nt of the group's rows (row v starts at pixel
// pix0 + v nx); rows at or beyond ny (v >= nv) are not ok and read the mask
// word of pixel 0.
template <int V, int CH, bool WORD>
__device__ __forceinline__ void chunk_words(const uint2* mw, int pix0, int nx, int nv, int j0,
                                            int nt, int L, Opnd (&o)[CH][V]) {
#pragma unroll
  for (int c = 0; c < CH; ++c)
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int j = j0 + c * nt;
      o[c][v].ok = j < L && v < nv;
      o[c][v].pix = o[c][v].ok ? pix0 + v * nx + 2 * j : 0;   // pixel 0: a valid dummy
      if (WORD) o[c][v].q = pair_index(mw, o[c][v].pix);
    }
}

template <typename T, int OP, int V>
__device__ __forceinline__ void src_rows(const InstDesc<T>& I, int pix0, int nx, int nv, cx<T>* z,
                                         int L, int t, int nt, T alpha, T beta, Acc<T>& acc) {
  constexpr bool W = !(OP == OP_LOAD_W || OP == OP_LOAD_Y);
  constexpr bool C = CompactOnly<OP>::value;
  constexpr int CH = kGenChunk / V;
  for (int j0 = t; j0 < L; j0 += CH * nt) {
    Opnd o[CH][V];
    chunk_words<V, CH, W>(I.mw, pix0, nx, nv, j0, nt, L, o);
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (C) o[c][v].ok = o[c][v].ok && (o[c][v].q.m0 || o[c][v].q.m1);
    T x[CH][V][8];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (o[c][v].ok) src_load<T, OP>(I, o[c][v], x[c][v]);
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int j = j0 + c * nt;
      if (j >= L) break;
      cx<T> zz[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        zz[v] = cx<T>{(T)0, (T)0};
        if (o[c][v].ok) zz[v] = src_op<T, OP>(I, o[c][v], x[c][v], alpha, beta, acc);
      }
      st_slot<T, V>(z + j * V, zz);
    }
  }
}

template <typename T, int OP, int V>
__device__ __forceinline__ void sink_rows(const InstDesc<T>& I, int pix0, int nx, int nv,
                                          const cx<T>* z, int L, int t, int nt, Acc<T>& acc,
                                          int param) {
  constexpr bool C = CompactOnly<OP>::value;
  constexpr int CH = kGenChunk / V;
  for (int j0 = t; j0 < L; j0 += CH * nt) {
    Opnd o[CH][V];
    chunk_words<V, CH, true>(I.mw, pix0, nx, nv, j0, nt, L, o);
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (C) o[c][v].ok = o[c][v].ok && (o[c][v].q.m0 || o[c][v].q.m1);
    T x[CH][V][2];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (o[c][v].ok) sink_load<T, OP>(I, o[c][v], x[c][v]);
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      bool any = false;
#pragma unroll
      for (int v = 0; v < V; ++v) any = any || o[c][v].ok;
      if (!any) continue;
      cx<T> zz[V];
      ld_slot<T, V>(z + (j0 + c * nt) * V, zz);
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (o[c][v].ok) sink_op<T, OP>(I, o[c][v], x[c][v], zz[v], acc, param);
    }
  }
}

template <typename T, int OP, int V>
__device__ __forceinline__ void mid_rows(const InstDesc<T>& I, int pix0, int nx, int nv, cx<T>* z,
                                         int L, int t, int nt) {
  constexpr int CH = kGenChunk / V;
  for (int j0 = t; j0 < L; j0 += CH * nt) {
    Opnd o[CH][V];
    chunk_words<V, CH, true>(I.mw, pix0, nx, nv, j0, nt, L, o);
    T d[CH][V][2];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (o[c][v].ok && OP == OP_Y_W) ld_map_pair<T>(I.d + o[c][v].pix, d[c][v][0], d[c][v][1]);
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int j = j0 + c * nt;
      if (j >= L) break;
      cx<T> zz[V];
      ld_slot<T, V>(z + j * V, zz);
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (o[c][v].ok) zz[v] = mid_op<T, OP>(I, o[c][v], d[c][v][0], d[c][v][1], zz[v]);
      st_slot<T, V>(z + j * V, zz);
    }
  }
}

}  // namespace gen

// ----------------------------------------------------------------- row pass
// CTA = a.rows consecutive grid rows in groups of V (one group per g.nt
// threads; blockIdx.y is the instance), rows at or beyond ny (odd ny) idle.
// Shared memory: L complex values per row, interleaved [position][V] within a
// group.
template <typename T, int V, bool IN_SPEC, bool OUT_SPEC, bool XI = false>
__global__ void __launch_bounds__(kGenThreads, gen_minb<T>())
k_row_gen(const InstDesc<T>* __restrict__ insts, RowArgs a, GenLen g, const T* __restrict__ wl,
          const T* __restrict__ wx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const InstDesc<T>& I = insts[blockIdx.y];
  if (skip_instance(a.check_done, I.st)) return;
  const int L = g.n, nt = g.nt, ny = a.ny;
  const int grp = threadIdx.x / nt, t = threadIdx.x - grp * nt;
  const int y0 = blockIdx.x * a.rows + grp * V;
  const int nv = min(V, ny - y0);   // rows of this group inside the grid
  cx<T>* Z = reinterpret_cast<cx<T>*>(smem_raw) + grp * L * V;
  Acc<T> acc;

  const int pix0 = y0 * a.nx;
  if constexpr (IN_SPEC) {
    gen::c2r<T, V>(a.spec_sel ? I.spec2 : I.spec, ny, y0, g, wx, Z, t, nt);
    __syncthreads();
    gen::dit<T, V>(Z, g, wl, t, g.nst);   // Z[j] = x[2j] + i x[2j+1] (scaled)
#define CGF_SINK(OPC, PARAM) \
  gen::sink_rows<T, OPC, V>(I, pix0, a.nx, nv, Z, L, t, nt, acc, PARAM)
    if constexpr (OUT_SPEC) {
      if (a.op == OP_Y_W)
        gen::mid_rows<T, OP_Y_W, V>(I, pix0, a.nx, nv, Z, L, t, nt);
      else
        gen::mid_rows<T, OP_MASK, V>(I, pix0, a.nx, nv, Z, L, t, nt);
    } else {
      switch (a.op) {
        case OP_Q: CGF_SINK(OP_Q, 0); break;
        case OP_Z: CGF_SINK(OP_Z, 0); break;
        case OP_B: CGF_SINK(OP_B, 0); break;
        case OP_RES: CGF_SINK(OP_RES, 0); break;
        case OP_GRAD: CGF_SINK(OP_GRAD, 0); break;
        case OP_RELAX: CGF_SINK(OP_RELAX, 0); break;
        case OP_KSEL: CGF_SINK(OP_KSEL, a.param); break;
        case OP_STORE_Y: CGF_SINK(OP_STORE_Y, 0); break;
        case OP_STORE_Y_MASK: CGF_SINK(OP_STORE_Y_MASK, 0); break;
        default: break;
      }
    }
#undef CGF_SINK
  } else if constexpr (XI) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int rowpix = (y0 + (v < nv ? v : 0)) * a.nx;
      for (int j = t; j < L; j += nt) {
        double x0 = 0.0, x1 = 0.0;
        if (v < nv) normal_pair(I.seed, (uint32_t)((rowpix >> 1) + j), x0, x1);
        Z[j * V + v] = cx<T>{(T)x0, (T)x1};
      }
    }
  } else {
    const T alpha = (T)I.st->alpha, beta = (T)I.st->beta;
#define CGF_SRC(OPC) gen::src_rows<T, OPC, V>(I, pix0, a.nx, nv, Z, L, t, nt, alpha, beta, acc)
    switch (a.op) {
      case OP_R_UPD: CGF_SRC(OP_R_UPD); break;
      case OP_P_UPD_Z: CGF_SRC(OP_P_UPD_Z); break;
      case OP_P_UPD_R: CGF_SRC(OP_P_UPD_R); break;
      case OP_LOAD_R: CGF_SRC(OP_LOAD_R); break;
      case OP_LOAD_U: CGF_SRC(OP_LOAD_U); break;
      case OP_LOAD_Y: CGF_SRC(OP_LOAD_Y); break;
      case OP_LOAD_W: CGF_SRC(OP_LOAD_W); break;
      case OP_LOAD_W_MASK: CGF_SRC(OP_LOAD_W_MASK); break;
      case OP_LOAD_D_U: CGF_SRC(OP_LOAD_D_U); break;
      case OP_U64_UPD: CGF_SRC(OP_U64_UPD); break;
      default:
        for (int j = t; j < L * V; j += nt) Z[j] = cx<T>{(T)0, (T)0};
        break;
    }
#undef CGF_SRC
  }

  if constexpr (OUT_SPEC) {
    __syncthreads();
    gen::dif<T, V>(Z, g, wl, t, g.nst);
    gen::r2c<T, V>(a.spec_sel ? I.spec2 : I.spec, ny, y0, g, wx, Z, t, nt);
  }

  if (a.sop != SC_NONE)
    grid_reduce(acc.value(), red, I.partial, I.st, a.sop, gridDim.x, blockIdx.x);
}

// ----------------------------------------------------------------- column pass
// CTA = a.ffts spectrum rows (one kx each) in groups of V; forward FFT (all
// stages but the last), then per butterfly of the last stage: its forward
// DFT, the table at the butterfly's frequencies k0 + q n/R, the inverse DFT;
// then the remaining inverse stages and the store, in natural order
// (table < 0: forward only, the last stage's outputs stored at their
// frequencies; PRE: the input is spec, already transformed, gathered at the
// same frequencies, and the output goes to spec_sel's buffer).  Shared
// memory: ny complex values per column.
namespace gen {

template <typename T, int V, int R, bool PRE>
__device__ __forceinline__ void col_middle(cx<T>* z, const GenLen& g, const T* tab0,
                                           long long tstride, const T* src0, T* dst0,
                                           long long cstride, int nv, int table, int t, int nt) {
  const int N = g.n, nb = N / R;   // the last stage's butterflies; k = k0 + q nb
  for (int blk = t; blk < nb; blk += nt) {
    const int k0 = g.rev[blk * R];
    cx<T> v[V][R];
    if constexpr (PRE) {
#pragma unroll
      for (int u = 0; u < V; ++u)
#pragma unroll
        for (int q = 0; q < R; ++q)
          v[u][q] = u < nv ? ld_cx<T>(src0 + u * cstride + 2 * (k0 + q * nb)) : cx<T>{(T)0, (T)0};
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        cx<T> sl[V];
        ld_slot<T, V>(z + (blk * R + q) * V, sl);
#pragma unroll
        for (int u = 0; u < V; ++u) v[u][q] = sl[u];
      }
#pragma unroll
      for (int u = 0; u < V; ++u) dft<T, R, false>(v[u]);
    }
    if (table < 0) {
#pragma unroll
      for (int u = 0; u < V; ++u)
        if (u < nv)
#pragma unroll
          for (int q = 0; q < R; ++q) st_cx<T>(dst0 + u * cstride + 2 * (k0 + q * nb), v[u][q]);
      continue;
    }
#pragma unroll
    for (int u = 0; u < V; ++u) {
#pragma unroll
      for (int q = 0; q < R; ++q)
        v[u][q] = scal(v[u][q], u < nv ? ldg1(tab0 + u * tstride + k0 + q * nb) : (T)0);
      dft<T, R, true>(v[u]);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      cx<T> sl[V];
#pragma unroll
      for (int u = 0; u < V; ++u) sl[u] = v[u][q];
      st_slot<T, V>(z + (blk * R + q) * V, sl);
    }
  }
}

}  // namespace gen

template <typename T, int V, bool PRE = false>
__global__ void __launch_bounds__(kGenThreads, gen_col_minb<T>())
k_col_gen(const InstDesc<T>* __restrict__ insts, ColArgs a, GenLen g, const T* __restrict__ wn) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const InstDesc<T>& I = insts[blockIdx.x];
  if (skip_instance(a.check_done, I.st)) return;
  const int N = g.n, nt = g.nt;
  const int grp = threadIdx.x / nt, t = threadIdx.x - grp * nt;
  const int kx0 = blockIdx.y * a.ffts + grp * V;
  const int nv = max(0, min(V, a.nkx - kx0));   // columns of this group inside the spectrum
  const int kxa = nv > 0 ? kx0 : 0;
  cx<T>* Z = reinterpret_cast<cx<T>*>(smem_raw) + grp * N * V;
  const long long cstride = 2LL * N;   // T elements between consecutive columns
  T* col = (a.spec_sel ? I.spec2 : I.spec) + cstride * kxa;
  const T* srcp = PRE ? I.spec + cstride * kxa : col;
  const int S = g.nst, R = g.radix[S - 1];

  if constexpr (!PRE) {
    for (int y0 = t; y0 < N; y0 += gen::kGenChunk * nt) {
      cx<T> x[gen::kGenChunk][V];
#pragma unroll
      for (int c = 0; c < gen::kGenChunk; ++c) {
        const int y = min(y0 + c * nt, N - 1);
#pragma unroll
        for (int u = 0; u < V; ++u)
          x[c][u] = u < nv ? ld_stream_cx<T>(srcp + u * cstride + 2 * y) : cx<T>{(T)0, (T)0};
      }
#pragma unroll
      for (int c = 0; c < gen::kGenChunk; ++c)
        if (y0 + c * nt < N) gen::st_slot<T, V>(Z + (y0 + c * nt) * V, x[c]);
    }
    __syncthreads();
    gen::dif<T, V>(Z, g, wn, t, S - 1);
  }
  const T* tab0 = nullptr;
  long long tstride = N;
  if (a.table >= 0)
    tab0 = (a.table >= 2 ? I.kt + (long long)(a.table - 2) * a.nkx * N
            : a.table ? I.t_sqrt : I.t_inv) + (long long)kxa * N;
  switch (R) {
    case 2: gen::col_middle<T, V, 2, PRE>(Z, g, tab0, tstride, srcp, col, cstride, nv, a.table, t, nt); break;
    case 3: gen::col_middle<T, V, 3, PRE>(Z, g, tab0, tstride, srcp, col, cstride, nv, a.table, t, nt); break;
    case 4: gen::col_middle<T, V, 4, PRE>(Z, g, tab0, tstride, srcp, col, cstride, nv, a.table, t, nt); break;
    case 8: gen::col_middle<T, V, 8, PRE>(Z, g, tab0, tstride, srcp, col, cstride, nv, a.table, t, nt); break;
    case 5: gen::col_middle<T, V, 5, PRE>(Z, g, tab0, tstride, srcp, col, cstride, nv, a.table, t, nt); break;
    default: gen::col_middle<T, V, 7, PRE>(Z, g, tab0, tstride, srcp, col, cstride, nv, a.table, t, nt); break;
  }
  if (a.table < 0) return;
  __syncthreads();
  gen::dit<T, V>(Z, g, wn, t, S - 1);
  for (int y0 = t; y0 < N; y0 += gen::kGenChunk * nt) {
#pragma unroll
    for (int c = 0; c < gen::kGenChunk; ++c) {
      const int y = y0 + c * nt;
      if (y >= N) break;
      cx<T> x[V];
      gen::ld_slot<T, V>(Z + y * V, x);
#pragma unroll
      for (int u = 0; u < V; ++u)
        if (u < nv) st_cx<T>(col + u * cstride + 2 * y, x[u]);
    }
  }
}

// ----------------------------------------------------------------- launchers
template <typename T>
size_t GenLaunch<T>::row_smem(int L, int rows) {
  return size_t(rows) * L * sizeof(cx<T>);
}

template <typename T>
size_t GenLaunch<T>::col_smem(int ny, int ffts) {
  return size_t(ffts) * ny * sizeof(cx<T>);
}

template <typename T>
int GenLaunch<T>::max_threads() { return kGenThreads; }

template <typename T>
cudaError_t GenLaunch<T>::row(bool in_spec, bool out_spec, const InstDesc<T>* d, int ninst,
                              const RowArgs& a, const GenLen& g, const T* wl, const T* wx,
                              cudaStream_t s) {
  constexpr int V = gen_vrow<T>();
  const dim3 grid((a.ny + a.rows - 1) / a.rows, ninst), block(a.rows / V * g.nt);
  const size_t sm = row_smem(g.n, a.rows);
  if (in_spec && out_spec)
    k_row_gen<T, V, true, true><<<grid, block, sm, s>>>(d, a, g, wl, wx);
  else if (in_spec)
    k_row_gen<T, V, true, false><<<grid, block, sm, s>>>(d, a, g, wl, wx);
  else if (a.op == OP_XI)
    k_row_gen<T, V, false, true, true><<<grid, block, sm, s>>>(d, a, g, wl, wx);
  else
    k_row_gen<T, V, false, true><<<grid, block, sm, s>>>(d, a, g, wl, wx);
  return cudaGetLastError();
}

template <typename T>
cudaError_t GenLaunch<T>::col(const InstDesc<T>* d, int ninst, const ColArgs& a, const GenLen& g,
                              const T* wn, cudaStream_t s) {
  constexpr int V = gen_v<T>();
  const dim3 grid(ninst, (a.nkx + a.ffts - 1) / a.ffts), block(a.ffts / V * g.nt);
  const size_t sm = col_smem(g.n, a.ffts);
  if (a.pre)
    k_col_gen<T, V, true><<<grid, block, sm, s>>>(d, a, g, wn);
  else
    k_col_gen<T, V><<<grid, block, sm, s>>>(d, a, g, wn);
  return cudaGetLastError();
}

template <typename T>
cudaError_t GenLaunch<T>::prepare() {
  constexpr int V = gen_v<T>(), VR = gen_vrow<T>();
  cudaError_t e = detail::allow_smem(k_row_gen<T, VR, true, true>);
  if (e == cudaSuccess) e = detail::allow_smem(k_row_gen<T, VR, true, false>);
  if (e == cudaSuccess) e = detail::allow_smem(k_row_gen<T, VR, false, true>);
  if (e == cudaSuccess) e = detail::allow_smem(k_row_gen<T, VR, false, true, true>);
  if (e == cudaSuccess) e = detail::allow_smem(k_col_gen<T, V>);
  if (e == cudaSuccess) e = detail::allow_smem(k_col_gen<T, V, true>);
  return e;
}

}  // namespace cgf
