/*
 * Plain FP64 C restatement of Algorithm 1 (Hi-DFT) for a batch of instances
 * that share one homogeneous support, parallel over instances with OpenMP.
 *
 * TEST INFRASTRUCTURE ONLY (the oracle): used by the tests and by the bench's
 * CPU baseline and reference arm; never by the library, and it shares no code
 * with it.
 *
 * Inputs are in the oracle's conventions (oracle/fp64.py): Jc is the support in
 * canonical order, r the pivots (ascending), f the samples at I_r in sample
 * order (interleaved re, im). Algorithm 1's recursion, unrolled bottom-up: at
 * depth m (1..s) every block of 2^m values is [f1 + w f2, f1 - w f2] of its two
 * halves, w_u = exp(-2 pi i (Jc[u] mod 2^{r_m}) / 2^{r_m + 1}) for u < 2^{m-1}
 * (Lemma "rec-hom-tree-split"); the result is scaled by N/k (the normalisation
 * reading of eq. "hom-implies-spectral").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const double kPi = 3.14159265358979323846264338327950288;

/* Twiddle of depth m (1-based) for column u: angle -pi * (Jc[u] mod 2^r) / 2^r. */
static void twiddle(uint64_t j, uint32_t r, double* re, double* im) {
  const uint64_t rho = (r >= 64) ? j : (j & ((r == 0) ? 0ull : ((1ull << r) - 1ull)));
  const double x = ldexp((double)rho, -(int)r);
  *re = cos(kPi * x);
  *im = -sin(kPi * x);
}

/* Returns the number of threads used, or -1 on a bad argument. */
int oracle_alg1_batch(uint32_t M, uint32_t s, const uint32_t* r, const uint64_t* Jc, const double* f, double* c,
                      int64_t batch, int threads) {
  if (s > 30 || (s > 0 && (!r || !Jc)) || !f || !c || batch < 0) return -1;
  const uint64_t k = 1ull << s;
  /* twiddles of every depth: entry (2^{m-1} - 1) + u */
  double* tw = (double*)malloc(sizeof(double) * 2 * (k > 1 ? k - 1 : 1));
  if (!tw) return -1;
  for (uint32_t m = 1; m <= s; ++m) {
    const uint64_t half = 1ull << (m - 1);
    for (uint64_t u = 0; u < half; ++u) twiddle(Jc[u], r[m - 1], &tw[2 * (half - 1 + u)], &tw[2 * (half - 1 + u) + 1]);
  }
  const double scale = ldexp(1.0, (int)M - (int)s);
  int used = 1;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
  {
#pragma omp single
    used = omp_get_num_threads();
  }
#pragma omp parallel for schedule(static)
#endif
  for (int64_t b = 0; b < batch; ++b) {
    double* x = c + (uint64_t)b * 2 * k;
    const double* in = f + (uint64_t)b * 2 * k;
    for (uint64_t i = 0; i < 2 * k; ++i) x[i] = in[i];
    for (uint32_t m = 1; m <= s; ++m) {
      const uint64_t half = 1ull << (m - 1);
      const double* w = tw + 2 * (half - 1);
      for (uint64_t blk = 0; blk < k; blk += 2 * half) {
        for (uint64_t u = 0; u < half; ++u) {
          double* a = x + 2 * (blk + u);
          double* d = x + 2 * (blk + u + half);
          const double tr = w[2 * u] * d[0] - w[2 * u + 1] * d[1];
          const double ti = w[2 * u] * d[1] + w[2 * u + 1] * d[0];
          d[0] = a[0] - tr;
          d[1] = a[1] - ti;
          a[0] = a[0] + tr;
          a[1] = a[1] + ti;
        }
      }
    }
    for (uint64_t i = 0; i < 2 * k; ++i) x[i] *= scale;
  }
  free(tw);
  return used;
}
