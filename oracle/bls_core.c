/*
 * Oracle: binned Box Least Squares signal residue for one star, plain FP64.
 * TEST INFRASTRUCTURE ONLY -- used by tests, the smoke check and the CPU
 * baseline; never linked into the product library.
 *
 * Method (Sec. 2.1 and Sec. 2.2 item 1 of arXiv:2302.01293; BLS of Kovacs et
 * al. 2002 with the Keplerian duration range of Sec. 2.1):
 *   for every trial frequency f
 *     fold:       x = t' f,  phase = x - floor(x),
 *                 bin b = min(nbins-1, floor(phase * nbins))
 *     histogram:  Hw[b] += w_i,  Hy[b] += w_i d_i    (w normalised, d = y - ybar)
 *     boxes:      for every duration j (m_j bins) and every start bin k, the
 *                 cyclic window k .. k+m_j-1 gives r = sum Hw, s = sum Hy and,
 *                 when 0 < r < 1, the residue v = s^2 / (r (1 - r))
 *     SR(f) = max v over (j, k); ties go to the lowest j, then the lowest k;
 *     no valid window: SR = 0, j = k = -1.
 * Build with -ffp-contract=off so that every product and sum is rounded once.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int oracle_bls_star(int64_t n, const double* tp, const double* w, const double* wd,
                    int64_t nf, const double* freq, const int32_t* nbins,
                    const int32_t* m, int32_t nq,
                    double* sr, int32_t* jbest, int32_t* kbest, double* sbest, double* rbest)
{
  int32_t nbmax = 1;
  for (int64_t k = 0; k < nf; ++k)
    if (nbins[k] > nbmax) nbmax = nbins[k];
  double* hw = (double*)malloc(sizeof(double) * (size_t)nbmax);
  double* hy = (double*)malloc(sizeof(double) * (size_t)nbmax);
  if (!hw || !hy) { free(hw); free(hy); return -1; }

  for (int64_t k = 0; k < nf; ++k) {
    const double f = freq[k];
    const int32_t nb = nbins[k];
    memset(hw, 0, sizeof(double) * (size_t)nb);
    memset(hy, 0, sizeof(double) * (size_t)nb);

    /* fold and histogram */
    for (int64_t i = 0; i < n; ++i) {
      const double x = tp[i] * f;
      const double phase = x - floor(x);
      int32_t b = (int32_t)floor(phase * (double)nb);
      if (b > nb - 1) b = nb - 1;
      hw[b] += w[i];
      hy[b] += wd[i];
    }

    /* every duration, every start bin, direct cyclic window sums */
    double best = 0.0, bs = 0.0, br = 0.0;
    int32_t bj = -1, bk = -1;
    for (int32_t j = 0; j < nq; ++j) {
      const int32_t mj = m[k * nq + j];
      for (int32_t kk = 0; kk < nb; ++kk) {
        double r = 0.0, s = 0.0;
        for (int32_t o = 0; o < mj; ++o) {
          const int32_t idx = (kk + o) % nb;
          r += hw[idx];
          s += hy[idx];
        }
        if (r > 0.0 && r < 1.0) {
          const double v = s * s / (r * (1.0 - r));
          if (bj < 0 || v > best) { best = v; bj = j; bk = kk; bs = s; br = r; }
        }
      }
    }
    sr[k] = (bj < 0) ? 0.0 : best;
    jbest[k] = bj;
    kbest[k] = bk;
    sbest[k] = bs;
    rbest[k] = br;
  }
  free(hw);
  free(hy);
  return 0;
}

/* Residue of one box (j, k) at one frequency: the value the search above takes
 * the maximum of; -1 when the window is not valid. Used to check near-ties. */
double oracle_bls_box(int64_t n, const double* tp, const double* w, const double* wd,
                      double f, int32_t nb, int32_t mj, int32_t k0)
{
  double r = 0.0, s = 0.0;
  double* hw = (double*)calloc((size_t)nb, sizeof(double));
  double* hy = (double*)calloc((size_t)nb, sizeof(double));
  if (!hw || !hy) { free(hw); free(hy); return -2.0; }
  for (int64_t i = 0; i < n; ++i) {
    const double x = tp[i] * f;
    const double phase = x - floor(x);
    int32_t b = (int32_t)floor(phase * (double)nb);
    if (b > nb - 1) b = nb - 1;
    hw[b] += w[i];
    hy[b] += wd[i];
  }
  for (int32_t o = 0; o < mj; ++o) {
    const int32_t idx = (k0 + o) % nb;
    r += hw[idx];
    s += hy[idx];
  }
  free(hw);
  free(hy);
  if (r > 0.0 && r < 1.0) return s * s / (r * (1.0 - r));
  return -1.0;
}
