// Instantiations of the mixed-radix pass kernels (FP32, FP64, double-float)
// and the factorisation of a transform length with its twiddle layout.
#include "cg_generic.cuh"

namespace cgf {

bool gen_factor(int n, GenLen* g, int code) {
  if (n < 2 || n > kGenMaxLen) return false;
  int m = n, k = 0;
  auto take = [&](int r) {
    while (m % r == 0 && k < kGenMaxStages) {
      g->radix[k++] = r;
      m /= r;
    }
  };
  if (!(code & 1)) take(8);
  take(4);
  take(2);
  if (code & 2) {
    take(7);
    take(5);
    take(3);
  } else {
    take(3);
    take(5);
    take(7);
  }
  if (m != 1) return false;
  g->n = n;
  g->nst = k;
  g->code = code;
  // stage s (sub-length ns, h = ns / R) holds h (R - 1) twiddles; the last
  // stage (h = 1) none
  int ns = n, off = 0;
  for (int s = 0; s < k; ++s) {
    const int h = ns / g->radix[s];
    g->twoff[s] = off;
    if (s < k - 1) off += h * (g->radix[s] - 1);
    ns = h;
  }
  return true;
}

template struct GenLaunch<float>;
template struct GenLaunch<double>;
template struct GenLaunch<df>;

}  // namespace cgf
