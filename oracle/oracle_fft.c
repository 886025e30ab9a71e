/*
 * oracle_fft.c -- the FP64 oracle's own discrete Fourier transform.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by oracle/cgfill_oracle.py, which only
 * tests/, __graft_entry__.smoke() and the CPU-baseline legs of bench.py use.
 * It shares no code with the CUDA path.
 *
 * What it computes (Sect. 4: on the periodic grid the DFT is exactly unitary,
 * so C^s is the diagonal P(k)^s in Fourier space):
 *
 *     y[k] = sum_{j<n} x[j] exp(sign * 2 pi i j k / n),   sign = -1 forward,
 *                                                          sign = +1 backward
 *
 * unnormalised in both directions (the caller divides by n).  Any length n:
 * plain recursive decimation in time, n = p m with p the smallest prime
 * factor of n, so that
 *
 *     y[k + q m] = sum_{r<p} W_n^(r k) W_p^(r q) Y_r[k],   k < m, q < p,
 *
 * where Y_r is the length-m transform of the decimated sequence
 * x[j p + r], j < m, and W_n = exp(sign 2 pi i / n).  The twiddles W_n^j are
 * cos(2 pi j / n) and sin(2 pi j / n) evaluated directly in FP64 for every j.
 * A prime factor p costs p^2 products per group of p outputs (a direct DFT),
 * so lengths with small factors (2, 3, 5, 7) are fast and any other length is
 * still exact, only slower.
 *
 * The 2D transform of a row-major ny x nx array is the 1D transform of every
 * row, then of every column.  Rows and columns are independent, so they are
 * split over `nthreads` POSIX threads; every element is computed by the same
 * sequence of operations whatever the thread count, so the result does not
 * depend on it.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double kTwoPi = 6.283185307179586476925286766559005768;

static long smallest_factor(long n) {
  for (long p = 2; p * p <= n; ++p)
    if (n % p == 0) return p;
  return n;
}

static long largest_prime_factor(long n) {
  long big = 1;
  while (n > 1) {
    const long p = smallest_factor(n);
    if (p > big) big = p;
    n /= p;
  }
  return big;
}

/* Transform of length n of x[0], x[xs], ..., x[(n-1) xs] into the contiguous
 * y[0..n-1].  w[j * ws] = W_n^j for j < n.  tmp: at least the largest prime
 * factor of n entries, shared by the whole recursion (a level uses it only
 * after its sub-transforms have returned). */
static void dft(long n, const cplx* x, long xs, cplx* y, const cplx* w, long ws, cplx* tmp) {
  if (n == 1) {
    y[0] = x[0];
    return;
  }
  const long p = smallest_factor(n), m = n / p;
  for (long r = 0; r < p; ++r) dft(m, x + r * xs, xs * p, y + r * m, w, ws * p, tmp);
  for (long k = 0; k < m; ++k) {
    for (long r = 0; r < p; ++r) tmp[r] = w[r * k * ws] * y[r * m + k];   /* r k < n */
    for (long q = 0; q < p; ++q) {
      cplx s = 0.0;
      for (long r = 0; r < p; ++r) s += tmp[r] * w[((r * q) % p) * m * ws];   /* W_p^(rq) */
      y[q * m + k] = s;
    }
  }
}

/* W_n^j = cos(2 pi j / n) + sign i sin(2 pi j / n), j < n. */
static cplx* twiddles(long n, int sign) {
  cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  if (!w) return NULL;
  for (long j = 0; j < n; ++j) {
    const double a = kTwoPi * (double)j / (double)n;
    w[j] = cos(a) + (double)sign * sin(a) * I;
  }
  return w;
}

/* Columns are gathered in blocks of this many adjacent columns, so that a
 * gather reads whole cache lines of each row. */
#define COL_BLOCK 8

typedef struct {
  cplx* a;          /* the array, ny x nx row-major */
  long ny, nx;
  int axis;         /* 1: transform the rows (length nx); 0: the columns (length ny) */
  const cplx* w;    /* twiddles of the transformed length */
  long first, last; /* rows [first, last) or column blocks [first, last) */
  int fail;
} job_t;

static void* run_job(void* arg) {
  job_t* J = (job_t*)arg;
  const long n = J->axis ? J->nx : J->ny;
  const long lanes = J->axis ? 1 : COL_BLOCK;
  cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)n * lanes);
  cplx* out = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  cplx* tmp = (cplx*)malloc(sizeof(cplx) * (size_t)largest_prime_factor(n));
  if (!buf || !out || !tmp) {
    J->fail = 1;
    free(buf);
    free(out);
    free(tmp);
    return NULL;
  }
  for (long t = J->first; t < J->last; ++t) {
    if (J->axis) {
      cplx* row = J->a + t * J->nx;
      dft(n, row, 1, out, J->w, 1, tmp);
      memcpy(row, out, sizeof(cplx) * (size_t)n);
    } else {
      const long c0 = t * COL_BLOCK;
      const long nc = (c0 + COL_BLOCK <= J->nx) ? COL_BLOCK : J->nx - c0;
      for (long i = 0; i < n; ++i)
        for (long b = 0; b < nc; ++b) buf[b * n + i] = J->a[i * J->nx + c0 + b];
      for (long b = 0; b < nc; ++b) {
        dft(n, buf + b * n, 1, out, J->w, 1, tmp);
        memcpy(buf + b * n, out, sizeof(cplx) * (size_t)n);
      }
      for (long i = 0; i < n; ++i)
        for (long b = 0; b < nc; ++b) J->a[i * J->nx + c0 + b] = buf[b * n + i];
    }
  }
  free(buf);
  free(out);
  free(tmp);
  return NULL;
}

/* Transforms every row (axis 1) or every column (axis 0) in place. */
static int transform_axis(cplx* a, long ny, long nx, int axis, int sign, int nthreads) {
  const long n = axis ? nx : ny;
  const long units = axis ? ny : (nx + COL_BLOCK - 1) / COL_BLOCK;
  cplx* w = twiddles(n, sign);
  if (!w) return 1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > units) nthreads = (int)units;
  job_t* jobs = (job_t*)calloc((size_t)nthreads, sizeof(job_t));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  int* started = (int*)calloc((size_t)nthreads, sizeof(int));
  int fail = (!jobs || !th || !started);
  for (int t = 0; t < nthreads && !fail; ++t) {
    jobs[t] = (job_t){a, ny, nx, axis, w, units * t / nthreads, units * (t + 1) / nthreads, 0};
    if (t == 0) continue;   /* the calling thread takes the first share */
    started[t] = pthread_create(&th[t], NULL, run_job, &jobs[t]) == 0;
    if (!started[t]) run_job(&jobs[t]);
  }
  if (!fail) run_job(&jobs[0]);
  for (int t = 1; t < nthreads && !fail; ++t)
    if (started[t]) pthread_join(th[t], NULL);
  for (int t = 0; t < nthreads && !fail; ++t) fail |= jobs[t].fail;
  free(jobs);
  free(th);
  free(started);
  free(w);
  return fail;
}

/* 2D transform of the ny x nx complex array a (interleaved re, im; in place):
 * rows, then columns.  Returns 0 on success, 1 if memory ran out. */
int oracle_fft2(long ny, long nx, double* a, int sign, int nthreads) {
  if (ny < 1 || nx < 1 || (sign != 1 && sign != -1)) return 1;
  if (transform_axis((cplx*)a, ny, nx, 1, sign, nthreads)) return 1;
  return transform_axis((cplx*)a, ny, nx, 0, sign, nthreads);
}

/* 1D transform of each of the `rows` contiguous sequences of length n. */
int oracle_fft_rows(long rows, long n, double* a, int sign, int nthreads) {
  if (rows < 1 || n < 1 || (sign != 1 && sign != -1)) return 1;
  return transform_axis((cplx*)a, rows, n, 1, sign, nthreads);
}
