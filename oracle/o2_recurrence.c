/*
 * o2_recurrence.c -- oracle, test and baseline only: a plain FP64 block-sparse Chebyshev
 * recurrence on the host (OpenMP over block rows), written independently of the CUDA library.
 *
 * Sec. II.B.1, Eq. poly_PQ with S = I: y_0 = r, y_1 = H^ r, y_{k+1} = 2 H^ y_k - y_{k-1} with
 * H^ = (2H - (emax + emin) I)/(emax - emin), applied to s Rademacher probes r_i; the moments of
 * Sec. II.C.2 are mu_k = (1/s) sum_i r_i . y_k (direct: order - 1 block products).  With
 * doubled != 0 the same moments come from the Chebyshev product rule C_m C_n = (C_{m+n} +
 * C_{|m-n|})/2: mu_2k = 2 <y_k, y_k>/s - mu_0, mu_2k-1 = 2 <y_k, y_{k-1}>/s - mu_1 (order/2
 * block products), the amount of work the GPU path does per moment.
 *
 * Probe entry (row, j): the sign of the top bit of SplitMix64 output number (row 2^32 + j + 1)
 * of a stream seeded with `seed` (Steele, Lea & Flood, OOPSLA 2014), +1 when the bit is clear.
 *
 * Sums over rows are formed per block of rows in a fixed order and added in row order, so the
 * result does not depend on the number of threads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static double probe_sign(uint64_t seed, uint64_t row, uint64_t j) {
  uint64_t z = seed + ((row << 32) + j + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (z >> 63) ? -1.0 : 1.0;
}

#define ROWS_PER_SUM 64  /* atoms per fixed-order partial sum */

/* y_out = c1 * H^ y_in - y_prev (y_prev may be NULL); partial sums per block of ROWS_PER_SUM atoms:
   part[2 blk] = sum y_out . w, part[2 blk + 1] = sum y_out . y_out, where w = y_in (or r). */
static void step(int n_atoms, int B, const int32_t* rp, const int32_t* col, const double* hv, double shift,
                 double scale, int s, const double* y_in, const double* y_prev, double* y_out, double c1,
                 const double* w, double* part) {
  const int nblk = (n_atoms + ROWS_PER_SUM - 1) / ROWS_PER_SUM;
#pragma omp parallel for schedule(dynamic, 1)
  for (int blk = 0; blk < nblk; ++blk) {
    double p0 = 0.0, p1 = 0.0;
    const int a1 = (blk + 1) * ROWS_PER_SUM < n_atoms ? (blk + 1) * ROWS_PER_SUM : n_atoms;
    double* acc = (double*)malloc(sizeof(double) * (size_t)B * s);
    for (int a = blk * ROWS_PER_SUM; a < a1; ++a) {
      memset(acc, 0, sizeof(double) * (size_t)B * s);
      for (int k = rp[a]; k < rp[a + 1]; ++k) {
        const int b = col[k];
        const double* h = hv + (size_t)k * B * B;
        for (int i = 0; i < B; ++i)
          for (int l = 0; l < B; ++l) {
            const double hil = h[i * B + l];
            if (hil == 0.0) continue;
            const double* x = y_in + ((size_t)b * B + l) * s;
            double* o = acc + (size_t)i * s;
            for (int j = 0; j < s; ++j) o[j] += hil * x[j];
          }
      }
      for (int i = 0; i < B; ++i) {
        const size_t row = (size_t)a * B + i;
        for (int j = 0; j < s; ++j) {
          /* H^ y = (2 H y - (emax + emin) y) / W */
          double v = c1 * scale * (2.0 * acc[(size_t)i * s + j] - shift * y_in[row * s + j]);
          if (y_prev) v -= y_prev[row * s + j];
          y_out[row * s + j] = v;
          p0 += v * w[row * s + j];
          p1 += v * v;
        }
      }
    }
    free(acc);
    part[2 * blk] = p0;
    part[2 * blk + 1] = p1;
  }
}

/* moments[k], k < order, of the s probes (seed) on the BSR H (n_atoms block rows of B x B
   row-major FP64 blocks).  Returns the number of block products, or -1 on an argument error. */
int o2_moments(int n_atoms, int B, const int32_t* rp, const int32_t* col, const double* val, double emin,
               double emax, uint64_t seed, int s, int order, int doubled, double* moments) {
  if (n_atoms < 1 || (B != 1 && B != 9) || s < 1 || order < 1 || !(emax > emin)) return -1;
  const size_t n = (size_t)n_atoms * B, ps = n * (size_t)s;
  const double scale = 1.0 / (emax - emin), shift = emax + emin;
  double* r = (double*)malloc(sizeof(double) * ps);
  double* y0 = (double*)malloc(sizeof(double) * ps);
  double* y1 = (double*)malloc(sizeof(double) * ps);
  const int nblk = (n_atoms + ROWS_PER_SUM - 1) / ROWS_PER_SUM;
  double* part = (double*)malloc(sizeof(double) * 2 * (size_t)nblk);
  if (!r || !y0 || !y1 || !part) return -1;
#pragma omp parallel for
  for (long long i = 0; i < (long long)n; ++i)
    for (int j = 0; j < s; ++j) r[(size_t)i * s + j] = probe_sign(seed, (uint64_t)i, (uint64_t)j);
  for (int k = 0; k < order; ++k) moments[k] = 0.0;
  moments[0] = (double)n;
  int products = 0;
  const int K = doubled ? order / 2 : order - 1;
  double mu1 = 0.0;
  /* y1 = H^ r */
  double *ycur = y1, *yprev = r, *yspare = y0;
  for (int t = 1; t <= K; ++t) {
    double* out = t == 1 ? y1 : (t == 2 ? y0 : yprev);
    const double* in = t == 1 ? r : ycur;
    const double* prev = t == 1 ? NULL : (t == 2 ? r : yprev);
    step(n_atoms, B, rp, col, val, shift, scale, s, in, prev, out, t == 1 ? 1.0 : 2.0, doubled ? in : r, part);
    ++products;
    double d0 = 0.0, d1 = 0.0;
    for (int b = 0; b < nblk; ++b) {
      d0 += part[2 * b];
      d1 += part[2 * b + 1];
    }
    if (doubled) {
      /* d0 = <y_t, y_{t-1}>, d1 = <y_t, y_t> */
      if (t == 1) mu1 = d0 / s;
      if (t == 1 && 1 < order) moments[1] = mu1;
      if (2 * t < order) moments[2 * t] = 2.0 * d1 / s - moments[0];
      if (t >= 2 && 2 * t - 1 < order) moments[2 * t - 1] = 2.0 * d0 / s - mu1;
    } else {
      /* d0 = <y_t, r> */
      moments[t] = d0 / s;
    }
    if (t == 1) {
      ycur = y1;
      yprev = r;
    } else if (t == 2) {
      yprev = y1;
      ycur = y0;
    } else {
      double* tmp = ycur;
      ycur = out;
      yprev = tmp;
    }
  }
  (void)yspare;
  free(r);
  free(y0);
  free(y1);
  free(part);
  return products;
}
