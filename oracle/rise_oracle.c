/*
 * rise_oracle.c -- plain FP64 CPU oracle of the RISE IQ -> boxes path.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this file's library.  It shares no code, header,
 * table or constant generator with the CUDA library: every step below is
 * written out from the paper's description (and, where the paper is silent,
 * from the documented reading of it), with plain loops, in double precision.
 *
 * Steps and the passages they follow (RISE, arXiv 2603.20481):
 *   STFT of consecutive N-point segments ........ Sec. III-A-1 (extended by a hop)
 *   |X|^2 "without explicit normalization" ...... Sec. VI (evaluation setup)
 *   8-bit image (max-anchored 0.25 dB levels) ... not in the paper (reading)
 *   PSD along time, Savitzky-Golay, lowest local
 *   minimum N0, theta_PSD column pruning ........ Sec. IV-B, "Noise floor estimation"
 *   per-column Otsu, argmax sigma_b^2 ........... Sec. IV-B, Eq. (4)
 *   closing, opening, horizontal 1D opening ..... Sec. IV-B, Eq. (5), 3x3 / 1x3 SEs
 *   4-connected CCL, visited marks, min/max box . Sec. IV-B, "Bounding box generation",
 *                                                 box tuple of Eq. (1)
 *
 * Parity unpinned: the offsets behind theta_PSD and theta_Power.  The paper
 * gives neither their formula nor their values; ro_column_thresholds follows a
 * stated reading whose closed forms are pinned, but how its defaults compare
 * with the paper's own thresholds is not.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no fast-math), so
 * x86-64 and aarch64 give the same doubles.  With -fopenmp the independent
 * loops run on several host threads (frames of the STFT, column groups of
 * the histogram, columns of Otsu, rows of the mask and of each morphological
 * operation; the flood fill stays sequential), small images on one thread.
 * Each thread computes whole frames, columns or rows exactly as one thread
 * would, and the only reduction is a maximum, so the results do not depend
 * on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads the parallel loops use (n < 1: every core); returns the
 * count in effect, 1 when the library was built without OpenMP. */
int ro_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n >= 1 ? n : omp_get_num_procs());
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

#define RO_OK 0
#define RO_EINVAL -1
#define RO_ENOMEM -2
#define RO_ETRUNC -3

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Detection parameters, by meaning (the oracle's own definition). */
typedef struct {
  int range_mode;          /* 0: anchor the 8-bit range on the capture's max dB; 1: on hi_db */
  double hi_db;            /* anchor for range_mode 1 */
  double level_db;         /* width of one 8-bit level, dB */
  double psd_offset_db;    /* theta_PSD = N0 + offset; -inf: no column pruning */
  double power_offset_db;  /* theta_Power = N0 + offset; -inf: no power floor */
  int sg_half_window;      /* Savitzky-Golay half window m (window 2m+1), quadratic */
  int morph_order;         /* 0: close3, open3, open1x3 (paper order); 1: open1x3, close3, open3 */
} ro_params;

typedef struct {
  int32_t t0, t1, f0, f1;  /* inclusive time (row) and frequency (column) extent */
  int64_t anchor;          /* raster index t*F+f of the component's first pixel */
  int64_t area;            /* pixels */
  uint64_t sum_q;          /* sum of 8-bit levels */
  uint64_t energy_fx;      /* sum of round(2^32 * 10^((q-255)*level_db/10)) */
} ro_box;

/* ------------------------------------------------------------------------ */
/* STFT                                                                      */
/* ------------------------------------------------------------------------ */

static int is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

/* In-place forward DFT X[k] = sum_n x[n] exp(-2 pi i n k / n_len), by the
 * iterative radix-2 decimation-in-time Cooley-Tukey algorithm.  Twiddles are
 * evaluated directly with cos/sin (no recurrences). */
int ro_fft(double *re, double *im, int n) {
  if (!is_pow2(n)) return RO_EINVAL;
  /* bit-reversal permutation */
  for (int i = 1, j = 0; i < n; i++) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      double t = re[i]; re[i] = re[j]; re[j] = t;
      t = im[i]; im[i] = im[j]; im[j] = t;
    }
  }
  for (int len = 2; len <= n; len <<= 1) {
    int half = len >> 1;
    for (int j = 0; j < half; j++) {
      double ang = -2.0 * M_PI * (double)j / (double)len;
      double wr = cos(ang), wi = sin(ang);
      for (int s = 0; s < n; s += len) {
        int a = s + j, b = a + half;
        double xr = re[b] * wr - im[b] * wi;
        double xi = re[b] * wi + im[b] * wr;
        re[b] = re[a] - xr; im[b] = im[a] - xi;
        re[a] += xr;        im[a] += xi;
      }
    }
  }
  return RO_OK;
}

/* Periodic Hann window w[m] = 0.5 - 0.5 cos(2 pi m / N). */
void ro_hann(int N, double *w) {
  for (int m = 0; m < N; m++) w[m] = 0.5 - 0.5 * cos(2.0 * M_PI * (double)m / (double)N);
}

/* Number of frames T = floor((n - N) / hop) + 1 (0 when n < N). */
int64_t ro_num_frames(int64_t n, int N, int hop) {
  if (n < N || hop < 1) return 0;
  return (n - N) / hop + 1;
}

/* Power |X_t[k]|^2 of frames t0 .. t0+nt-1, written as rows of N columns with
 * column f holding bin k = (f + N/2) mod N (DC in the middle column).
 * iq is interleaved complex64 (re, im floats). */
int ro_stft_power(const float *iq, int64_t n, int N, int hop, int64_t t0, int64_t nt,
                  double *P) {
  if (!is_pow2(N) || hop < 1) return RO_EINVAL;
  int64_t T = ro_num_frames(n, N, hop);
  if (t0 < 0 || nt < 0 || t0 + nt > T) return RO_EINVAL;
  double *w = malloc(sizeof(double) * N), *re = malloc(sizeof(double) * N),
         *im = malloc(sizeof(double) * N);
  if (!w || !re || !im) { free(w); free(re); free(im); return RO_ENOMEM; }
  ro_hann(N, w);
  for (int64_t t = t0; t < t0 + nt; t++) {
    const float *x = iq + 2 * (t * (int64_t)hop);
    for (int m = 0; m < N; m++) {
      re[m] = w[m] * (double)x[2 * m];
      im[m] = w[m] * (double)x[2 * m + 1];
    }
    ro_fft(re, im, N);
    double *row = P + (t - t0) * (int64_t)N;
    for (int f = 0; f < N; f++) {
      int k = (f + N / 2) % N;
      row[f] = re[k] * re[k] + im[k] * im[k];
    }
  }
  free(w); free(re); free(im);
  return RO_OK;
}

/* Largest |X_t[k]|^2 over every frame and bin of the capture. */
int ro_max_power(const float *iq, int64_t n, int N, int hop, double *out_max) {
  int64_t T = ro_num_frames(n, N, hop);
  if (T < 1) return RO_EINVAL;
  double mx = 0.0;
  int err = RO_OK;
#pragma omp parallel if (T * (int64_t)N > 65536)
  {
    double *row = malloc(sizeof(double) * N);
#pragma omp for reduction(max : mx) schedule(static)
    for (int64_t t = 0; t < T; t++) {
      int rc = row ? ro_stft_power(iq, n, N, hop, t, 1, row) : RO_ENOMEM;
      if (rc) {
#pragma omp atomic write
        err = rc;
        continue;
      }
      for (int f = 0; f < N; f++) if (row[f] > mx) mx = row[f];
    }
    free(row);
  }
  if (err) return err;
  *out_max = mx;
  return RO_OK;
}

/* ------------------------------------------------------------------------ */
/* 8-bit image                                                               */
/* ------------------------------------------------------------------------ */

/* q = clamp(floor((dB - lo) / level + 0.5), 0, 255), dB = 10 log10 P,
 * lo = hi_db - 255 * level.  P = 0 gives q = 0. */
void ro_quantize(const double *P, int64_t npx, double hi_db, double level_db, uint8_t *q) {
  double lo = hi_db - 255.0 * level_db;
#pragma omp parallel for schedule(static) if (npx > 65536)
  for (int64_t i = 0; i < npx; i++) {
    if (!(P[i] > 0.0)) { q[i] = 0; continue; }
    double db = 10.0 * log10(P[i]);
    double v = floor((db - lo) / level_db + 0.5);
    if (v < 0.0) v = 0.0;
    if (v > 255.0) v = 255.0;
    q[i] = (uint8_t)v;
  }
}

/* Per-level energy in 2^-32 units of the top level: round(2^32 * 10^((q-255) level/10)). */
void ro_energy_table(double level_db, uint64_t *E) {
  for (int q = 0; q < 256; q++) {
    double v = ldexp(pow(10.0, (double)(q - 255) * level_db / 10.0), 32);
    E[q] = (uint64_t)llround(v);
  }
}

/* ------------------------------------------------------------------------ */
/* Column statistics: PSD, Savitzky-Golay, N0, theta_PSD, Otsu, theta_Power   */
/* ------------------------------------------------------------------------ */

/* hist[f*256 + v] = number of rows t with q[t][f] == v. */
void ro_column_hist(const uint8_t *q, int64_t T, int F, uint32_t *hist) {
  memset(hist, 0, sizeof(uint32_t) * 256 * (size_t)F);
  /* groups of 64 columns, each counted by one thread over every row */
#pragma omp parallel for schedule(dynamic, 1) if (T * (int64_t)F > 65536)
  for (int g = 0; g < F; g += 64) {
    const int ge = g + 64 < F ? g + 64 : F;
    for (int64_t t = 0; t < T; t++)
      for (int f = g; f < ge; f++) hist[(size_t)f * 256 + q[t * F + f]]++;
  }
}

/* Quadratic Savitzky-Golay smoothing weights for a 2m+1 window, scaled to
 * integers: c_i = 3(3m^2+3m-1) - 15 i^2 (i = -m..m), sum c_i = D =
 * (2m-1)(2m+1)(2m+3).  Writes c[0..m] (c[i] = c_{+-i}). */
int ro_sg_coeffs(int m, int64_t *c, int64_t *D) {
  if (m < 1) return RO_EINVAL;
  for (int i = 0; i <= m; i++) c[i] = 3LL * (3LL * m * m + 3LL * m - 1) - 15LL * i * i;
  *D = (int64_t)(2 * m - 1) * (2 * m + 1) * (2 * m + 3);
  return RO_OK;
}

/* Otsu's threshold of a 256-bin histogram: the theta in 0..254 maximising
 * the between-class variance sigma_b^2(theta) of the split {v <= theta} |
 * {v > theta}.  sigma_b^2 = n0 n1 (mu0 - mu1)^2 / n^2 = d^2 / (n0 n1 n^2) with
 * d = s0 n1 - s1 n0; candidates are compared exactly by cross-multiplying
 * d^2 / (n0 n1) in 128-bit integers.  Thetas with an empty class are not
 * candidates; the smallest maximiser wins.  Returns -1 if there is none. */
int ro_otsu(const uint32_t *h) {
  int64_t n = 0, s = 0;
  for (int v = 0; v < 256; v++) { n += h[v]; s += (int64_t)v * h[v]; }
  int best = -1;
  unsigned __int128 best_num = 0, best_den = 1;
  int64_t n0 = 0, s0 = 0;
  for (int th = 0; th < 255; th++) {
    n0 += h[th];
    s0 += (int64_t)th * h[th];
    int64_t n1 = n - n0, s1 = s - s0;
    if (n0 == 0 || n1 == 0) continue;
    __int128 d = (__int128)s0 * n1 - (__int128)s1 * n0;
    unsigned __int128 ad = (unsigned __int128)(d < 0 ? -d : d);
    unsigned __int128 num = ad * ad;
    unsigned __int128 den = (unsigned __int128)n0 * (unsigned __int128)n1;
    /* num/den > best_num/best_den ? */
    if (best < 0 || num * best_den > best_num * den) {
      best = th; best_num = num; best_den = den;
    }
  }
  return best;
}

static int64_t floor_div(int64_t a, int64_t b) {  /* b > 0 */
  int64_t q = a / b;
  if ((a % b != 0) && (a < 0)) q -= 1;
  return q;
}

/* Column thresholds of one image (T rows, F columns, histogram given).
 * Outputs (any may be NULL): S[F] column PSD = sum_t q[t][f];
 * Shat[F] = D * SG-smoothed S on f in [m, F-1-m] (0 elsewhere);
 * keep[F] (1 = column survives theta_PSD); otsu[F] (-1 = none);
 * eff[F] = smallest level counted as foreground (256 = none);
 * info[5] = {N0, delta_psd, delta_pow, P_q, D}. */
int ro_column_thresholds(const uint32_t *hist, int64_t T, int F, const ro_params *p,
                         uint64_t *S_out, int64_t *Shat_out, uint8_t *keep_out,
                         int32_t *otsu_out, int32_t *eff_out, int64_t *info) {
  int m = p->sg_half_window;
  if (F < 2 * m + 3 || m < 1 || T < 1) return RO_EINVAL;
  int64_t c[64], D;
  if (m > 63 || ro_sg_coeffs(m, c, &D)) return RO_EINVAL;
  int64_t *S = malloc(sizeof(int64_t) * F), *Sh = malloc(sizeof(int64_t) * F);
  if (!S || !Sh) { free(S); free(Sh); return RO_ENOMEM; }
  /* PSD: aggregate the TF plot along time (column sums of the levels) */
  for (int f = 0; f < F; f++) {
    int64_t acc = 0;
    for (int v = 0; v < 256; v++) acc += (int64_t)v * hist[(size_t)f * 256 + v];
    S[f] = acc;
  }
  /* Savitzky-Golay smoothing on the interior */
  for (int f = 0; f < F; f++) Sh[f] = 0;
  for (int f = m; f <= F - 1 - m; f++) {
    int64_t acc = 0;
    for (int i = -m; i <= m; i++) acc += c[i < 0 ? -i : i] * S[f + i];
    Sh[f] = acc;
  }
  /* lowest local minimum (strictly below the left neighbour, not above the right) */
  int found = 0;
  int64_t N0 = 0;
  for (int f = m + 1; f <= F - 2 - m; f++) {
    if (Sh[f] < Sh[f - 1] && Sh[f] <= Sh[f + 1]) {
      if (!found || Sh[f] < N0) N0 = Sh[f];
      found = 1;
    }
  }
  if (!found) {
    N0 = Sh[m];
    for (int f = m; f <= F - 1 - m; f++) if (Sh[f] < N0) N0 = Sh[f];
  }
  int64_t DT = D * T;
  int psd_on = !(isinf(p->psd_offset_db) && p->psd_offset_db < 0);
  int pow_on = !(isinf(p->power_offset_db) && p->power_offset_db < 0);
  int64_t dpsd = psd_on ? (int64_t)llround(p->psd_offset_db / p->level_db * (double)DT) : 0;
  int64_t dpow = pow_on ? (int64_t)llround(p->power_offset_db / p->level_db * (double)DT) : 0;
  int64_t Pq = 0;
  if (pow_on) {
    int64_t num = N0 + dpow;
    Pq = -floor_div(-num, DT);  /* ceil(num / DT) */
    if (Pq < 0) Pq = 0;
    if (Pq > 256) Pq = 256;
  }
#pragma omp parallel for schedule(static) if (F > 256)
  for (int f = 0; f < F; f++) {
    int keep = psd_on ? (D * S[f] >= N0 + dpsd) : 1;
    int th = ro_otsu(hist + (size_t)f * 256);
    int eff = 256;
    if (keep && th >= 0) {
      eff = th + 1;
      if (Pq > eff) eff = (int)Pq;
    }
    if (S_out) S_out[f] = (uint64_t)S[f];
    if (Shat_out) Shat_out[f] = Sh[f];
    if (keep_out) keep_out[f] = (uint8_t)keep;
    if (otsu_out) otsu_out[f] = th;
    if (eff_out) eff_out[f] = eff;
  }
  if (info) { info[0] = N0; info[1] = dpsd; info[2] = dpow; info[3] = Pq; info[4] = D; }
  free(S); free(Sh);
  return RO_OK;
}

/* ------------------------------------------------------------------------ */
/* Binary mask and morphology                                               */
/* ------------------------------------------------------------------------ */

/* Foreground: q[t][f] >= eff[f]  (eff = 256 -> none). Masks hold 0/1 bytes. */
void ro_threshold(const uint8_t *q, int64_t T, int F, const int32_t *eff, uint8_t *mask) {
#pragma omp parallel for schedule(static) if (T * (int64_t)F > 65536)
  for (int64_t t = 0; t < T; t++)
    for (int f = 0; f < F; f++) mask[t * F + f] = (int32_t)q[t * F + f] >= eff[f];
}

#define RO_DILATE3 0
#define RO_ERODE3 1
#define RO_DILATE1x3 2
#define RO_ERODE1x3 3

/* Binary dilation (max) or erosion (min) with an all-ones 3x3 (rows t-1..t+1,
 * columns f-1..f+1) or 1x3 (columns only, "horizontal" = along frequency)
 * structuring element.  The window is clipped to the image: pixels outside
 * the image take no part. */
int ro_morph(const uint8_t *in, uint8_t *out, int64_t T, int F, int op) {
  int rt = (op == RO_DILATE3 || op == RO_ERODE3) ? 1 : 0;
  int erode = (op == RO_ERODE3 || op == RO_ERODE1x3);
  if (op < 0 || op > 3) return RO_EINVAL;
#pragma omp parallel for schedule(static) if (T * (int64_t)F > 65536)
  for (int64_t t = 0; t < T; t++) {
    for (int f = 0; f < F; f++) {
      int v = erode ? 1 : 0;
      for (int64_t dt = -rt; dt <= rt; dt++) {
        int64_t tt = t + dt;
        if (tt < 0 || tt >= T) continue;
        for (int df = -1; df <= 1; df++) {
          int ff = f + df;
          if (ff < 0 || ff >= F) continue;
          if (erode) v &= in[tt * F + ff] ? 1 : 0;
          else v |= in[tt * F + ff] ? 1 : 0;
        }
      }
      out[t * F + f] = (uint8_t)v;
    }
  }
  return RO_OK;
}

/* closing = erode(dilate(A)), opening = dilate(erode(A)) -- Eq. (5).
 * order 0 (the order the paper lists): M1 = close3(M0), M2 = open3(M1),
 *   M3 = open1x3(M2).
 * order 1: M1 = open1x3(M0), M2 = close3(M1), M3 = open3(M2).
 * M1, M2 may be NULL. */
int ro_morph_chain(const uint8_t *M0, int64_t T, int F, int order, uint8_t *M1, uint8_t *M2,
                   uint8_t *M3) {
  size_t npx = (size_t)T * F;
  uint8_t *a = malloc(npx ? npx : 1), *b = malloc(npx ? npx : 1);
  if (!a || !b) { free(a); free(b); return RO_ENOMEM; }
  int ops[6];
  if (order == 0) {
    int o[6] = {RO_DILATE3, RO_ERODE3, RO_ERODE3, RO_DILATE3, RO_ERODE1x3, RO_DILATE1x3};
    memcpy(ops, o, sizeof ops);
  } else if (order == 1) {
    int o[6] = {RO_ERODE1x3, RO_DILATE1x3, RO_DILATE3, RO_ERODE3, RO_ERODE3, RO_DILATE3};
    memcpy(ops, o, sizeof ops);
  } else {
    free(a); free(b);
    return RO_EINVAL;
  }
  memcpy(a, M0, npx);
  for (int s = 0; s < 6; s++) {
    ro_morph(a, b, T, F, ops[s]);
    memcpy(a, b, npx);
    if (s == 1 && M1) memcpy(M1, a, npx);
    if (s == 3 && M2) memcpy(M2, a, npx);
  }
  memcpy(M3, a, npx);
  free(a); free(b);
  return RO_OK;
}

/* ------------------------------------------------------------------------ */
/* Connected components and boxes                                           */
/* ------------------------------------------------------------------------ */

/* 4-connected components of the mask, found by one raster scan with
 * breadth-first flood fill; visited pixels are marked (the mask copy is
 * set to 2).  Each component yields its inclusive row/column extent, area,
 * level sum and fixed-point energy; components come out in raster order of
 * their first pixel (the anchor).  Returns RO_ETRUNC when more than cap
 * components exist (*n_out is still the full count). */
int ro_ccl_boxes(const uint8_t *mask, const uint8_t *q, int64_t T, int F, double level_db,
                 ro_box *out, int64_t cap, int64_t *n_out) {
  size_t npx = (size_t)T * F;
  uint8_t *m = malloc(npx ? npx : 1);
  int64_t qcap = 1024, *queue = malloc(sizeof(int64_t) * qcap);
  if (!m || !queue) { free(m); free(queue); return RO_ENOMEM; }
  memcpy(m, mask, npx);
  uint64_t E[256];
  ro_energy_table(level_db, E);
  int64_t count = 0;
  for (int64_t i = 0; i < (int64_t)npx; i++) {
    if (m[i] != 1) continue;
    ro_box b;
    b.t0 = b.t1 = (int32_t)(i / F);
    b.f0 = b.f1 = (int32_t)(i % F);
    b.anchor = i; b.area = 0; b.sum_q = 0; b.energy_fx = 0;
    int64_t head = 0, tail = 0;
    queue[tail++] = i;
    m[i] = 2;
    while (head < tail) {
      int64_t p = queue[head++];
      int32_t t = (int32_t)(p / F), f = (int32_t)(p % F);
      if (t < b.t0) b.t0 = t;
      if (t > b.t1) b.t1 = t;
      if (f < b.f0) b.f0 = f;
      if (f > b.f1) b.f1 = f;
      b.area += 1;
      b.sum_q += q[p];
      b.energy_fx += E[q[p]];
      int64_t nb[4];
      int nn = 0;
      if (t > 0) nb[nn++] = p - F;
      if (t < T - 1) nb[nn++] = p + F;
      if (f > 0) nb[nn++] = p - 1;
      if (f < F - 1) nb[nn++] = p + 1;
      for (int k = 0; k < nn; k++) {
        if (m[nb[k]] != 1) continue;
        m[nb[k]] = 2;
        if (tail == qcap) {
          /* compact the consumed prefix, then grow */
          memmove(queue, queue + head, sizeof(int64_t) * (tail - head));
          tail -= head; head = 0;
          if (tail == qcap) {
            int64_t *nq = realloc(queue, sizeof(int64_t) * qcap * 2);
            if (!nq) { free(m); free(queue); return RO_ENOMEM; }
            queue = nq; qcap *= 2;
          }
        }
        queue[tail++] = nb[k];
      }
    }
    if (count < cap && out) out[count] = b;
    count++;
  }
  free(m); free(queue);
  *n_out = count;
  return count > cap ? RO_ETRUNC : RO_OK;
}

/* ------------------------------------------------------------------------ */
/* Whole path                                                               */
/* ------------------------------------------------------------------------ */

/* From an 8-bit image to boxes: column histogram, PSD pruning, per-column
 * Otsu, power floor, threshold, morphology, CCL.  Optional outputs: hist
 * [F*256], eff [F], info [5], final mask [T*F]. */
int ro_detect_image(const uint8_t *q, int64_t T, int F, const ro_params *p, ro_box *out,
                    int64_t cap, int64_t *n_out, uint32_t *hist_out, int32_t *eff_out,
                    int64_t *info_out, uint8_t *mask_out) {
  size_t npx = (size_t)T * F;
  uint32_t *hist = malloc(sizeof(uint32_t) * 256 * (size_t)F);
  int32_t *eff = malloc(sizeof(int32_t) * F);
  uint8_t *M0 = malloc(npx ? npx : 1), *M3 = malloc(npx ? npx : 1);
  int rc = RO_ENOMEM;
  if (!hist || !eff || !M0 || !M3) goto done;
  ro_column_hist(q, T, F, hist);
  rc = ro_column_thresholds(hist, T, F, p, NULL, NULL, NULL, NULL, eff, info_out);
  if (rc) goto done;
  ro_threshold(q, T, F, eff, M0);
  rc = ro_morph_chain(M0, T, F, p->morph_order, NULL, NULL, M3);
  if (rc) goto done;
  rc = ro_ccl_boxes(M3, q, T, F, p->level_db, out, cap, n_out);
  if (hist_out) memcpy(hist_out, hist, sizeof(uint32_t) * 256 * (size_t)F);
  if (eff_out) memcpy(eff_out, eff, sizeof(int32_t) * F);
  if (mask_out) memcpy(mask_out, M3, npx);
done:
  free(hist); free(eff); free(M0); free(M3);
  return rc;
}

/* From complex64 IQ to boxes.  The 8-bit image is anchored on the capture's
 * largest power (range_mode 0) or on hi_db (range_mode 1).  image_out
 * [T*N] and max_out (largest |X|^2) are optional. */
int ro_detect(const float *iq, int64_t n, int N, int hop, const ro_params *p, ro_box *out,
              int64_t cap, int64_t *n_out, uint8_t *image_out, double *max_out) {
  int64_t T = ro_num_frames(n, N, hop);
  if (T < 1 || !is_pow2(N)) return RO_EINVAL;
  double hi_db, mx = 0.0;
  int rc = ro_max_power(iq, n, N, hop, &mx);
  if (rc) return rc;
  if (max_out) *max_out = mx;
  hi_db = p->range_mode == 1 ? p->hi_db : 10.0 * log10(mx);
  uint8_t *q = image_out ? image_out : malloc((size_t)T * N);
  if (!q) return RO_ENOMEM;
  int err = RO_OK;
#pragma omp parallel if (T * (int64_t)N > 65536)
  {
    double *row = malloc(sizeof(double) * N);
#pragma omp for schedule(static)
    for (int64_t t = 0; t < T; t++) {
      if (!row) {
#pragma omp atomic write
        err = RO_ENOMEM;
        continue;
      }
      ro_stft_power(iq, n, N, hop, t, 1, row);
      ro_quantize(row, N, hi_db, p->level_db, q + t * (int64_t)N);
    }
    free(row);
  }
  rc = err ? err : ro_detect_image(q, T, N, p, out, cap, n_out, NULL, NULL, NULL, NULL);
  if (!image_out) free(q);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Detection quality (Sec. III-A-2, Eqs. 2 and 3): IoU of two boxes over TF  */
/* cells; every ground-truth box's best IoU over the detections and every   */
/* detection's best IoU over the ground truth, by exhaustive pairs; N_t =    */
/* boxes of the ground truth whose best IoU exceeds theta, N_f = detections  */
/* whose best IoU is below theta (IoU equal to theta counts as neither).     */
/* ------------------------------------------------------------------------ */

/* Boxes are int32 quadruples (t0, t1, f0, f1), inclusive cell ranges. */
static int64_t ro_area(const int32_t *b) {
  return ((int64_t)b[1] - b[0] + 1) * ((int64_t)b[3] - b[2] + 1);
}

static int64_t ro_overlap(const int32_t *a, const int32_t *b) {
  int64_t t = (int64_t)(a[1] < b[1] ? a[1] : b[1]) - (a[0] > b[0] ? a[0] : b[0]) + 1;
  int64_t f = (int64_t)(a[3] < b[3] ? a[3] : b[3]) - (a[2] > b[2] ? a[2] : b[2]) + 1;
  return (t > 0 && f > 0) ? t * f : 0;
}

/* best[2 i], best[2 i + 1] = (intersection, union) of box i of A with the
 * box of B of largest IoU (exact comparison of the fractions); (0, 1) when B
 * is empty. */
static void ro_best(const int32_t *A, int64_t na, const int32_t *B, int64_t nb, int64_t *best) {
  for (int64_t i = 0; i < na; i++) {
    int64_t bi = 0, bu = 1;
    const int64_t aa = ro_area(A + 4 * i);
    for (int64_t j = 0; j < nb; j++) {
      const int64_t in = ro_overlap(A + 4 * i, B + 4 * j);
      const int64_t un = aa + ro_area(B + 4 * j) - in;
      if ((__int128)in * bu > (__int128)bi * un) {
        bi = in;
        bu = un;
      }
    }
    best[2 * i] = bi;
    best[2 * i + 1] = bu;
  }
}

/* n_t[k], n_f[k] for the IoU thresholds theta[k] (Eq. 2); gt_best and
 * det_best (optional) receive the best (intersection, union) pairs.  The
 * decisions compare the intersection with theta * union in double. */
int ro_match(const int32_t *gt, int64_t ng, const int32_t *det, int64_t nd, const double *theta,
             int nth, int64_t *n_t, int64_t *n_f, int64_t *gt_best, int64_t *det_best) {
  int64_t *gb = gt_best ? gt_best : malloc(sizeof(int64_t) * 2 * (ng > 0 ? ng : 1));
  int64_t *db = det_best ? det_best : malloc(sizeof(int64_t) * 2 * (nd > 0 ? nd : 1));
  if (!gb || !db) {
    if (!gt_best) free(gb);
    if (!det_best) free(db);
    return RO_ENOMEM;
  }
  ro_best(gt, ng, det, nd, gb);
  ro_best(det, nd, gt, ng, db);
  for (int k = 0; k < nth; k++) {
    int64_t t = 0, f = 0;
    for (int64_t i = 0; i < ng; i++)
      if ((double)gb[2 * i] > theta[k] * (double)gb[2 * i + 1]) t++;
    for (int64_t j = 0; j < nd; j++)
      if ((double)db[2 * j] < theta[k] * (double)db[2 * j + 1]) f++;
    n_t[k] = t;
    n_f[k] = f;
  }
  if (!gt_best) free(gb);
  if (!det_best) free(db);
  return RO_OK;
}

/* ------------------------------------------------------------------------ */
/* Block shapes (Sec. IV-B, bounding-box paragraph: the labelling stage can  */
/* also give the blocks' boundaries): every foreground run with its         */
/* component, and the boundary pixels.                                       */
/* ------------------------------------------------------------------------ */

/* label[p] = component of pixel p, numbered by first pixel in raster order
 * (the box order), -1 for background; BFS flood fill with 4-neighbours. */
int ro_label(const uint8_t *mask, int64_t T, int F, int64_t *label) {
  const int64_t npx = T * (int64_t)F;
  int64_t qcap = 1024, *queue = malloc(sizeof(int64_t) * qcap);
  if (!queue) return RO_ENOMEM;
  for (int64_t i = 0; i < npx; i++) label[i] = -1;
  int64_t comp = 0;
  for (int64_t i = 0; i < npx; i++) {
    if (!mask[i] || label[i] >= 0) continue;
    int64_t head = 0, tail = 0;
    queue[tail++] = i;
    label[i] = comp;
    while (head < tail) {
      const int64_t p = queue[head++];
      const int64_t t = p / F, f = p % F;
      int64_t nb[4];
      int nn = 0;
      if (t > 0) nb[nn++] = p - F;
      if (t < T - 1) nb[nn++] = p + F;
      if (f > 0) nb[nn++] = p - 1;
      if (f < F - 1) nb[nn++] = p + 1;
      for (int k = 0; k < nn; k++) {
        if (!mask[nb[k]] || label[nb[k]] >= 0) continue;
        label[nb[k]] = comp;
        if (tail == qcap) {
          memmove(queue, queue + head, sizeof(int64_t) * (tail - head));
          tail -= head;
          head = 0;
          if (tail == qcap) {
            int64_t *nq = realloc(queue, sizeof(int64_t) * qcap * 2);
            if (!nq) { free(queue); return RO_ENOMEM; }
            queue = nq;
            qcap *= 2;
          }
        }
        queue[tail++] = nb[k];
      }
    }
    comp++;
  }
  free(queue);
  return RO_OK;
}

/* Every maximal horizontal run of foreground, in raster order of its first
 * pixel: runs[4 k .. 4 k + 3] = component, row t, first and last column. */
int ro_component_runs(const uint8_t *mask, int64_t T, int F, int32_t *runs, int64_t cap,
                      int64_t *n_out) {
  int64_t *label = malloc(sizeof(int64_t) * (size_t)(T * F > 0 ? T * F : 1));
  if (!label) return RO_ENOMEM;
  int rc = ro_label(mask, T, F, label);
  if (rc) { free(label); return rc; }
  int64_t n = 0;
  for (int64_t t = 0; t < T; t++) {
    for (int f = 0; f < F; f++) {
      if (!mask[t * F + f] || (f > 0 && mask[t * F + f - 1])) continue;
      int g = f;
      while (g + 1 < F && mask[t * F + g + 1]) g++;
      if (n < cap) {
        runs[4 * n] = (int32_t)label[t * F + f];
        runs[4 * n + 1] = (int32_t)t;
        runs[4 * n + 2] = f;
        runs[4 * n + 3] = g;
      }
      n++;
    }
  }
  free(label);
  *n_out = n;
  return n > cap ? RO_ETRUNC : RO_OK;
}

/* out[p] = 1 for a foreground pixel with a background 4-neighbour, pixels
 * outside the image counting as background. */
void ro_boundary(const uint8_t *mask, int64_t T, int F, uint8_t *out) {
  for (int64_t t = 0; t < T; t++)
    for (int f = 0; f < F; f++) {
      const int64_t p = t * F + f;
      if (!mask[p]) { out[p] = 0; continue; }
      const int up = t > 0 && mask[p - F], dn = t < T - 1 && mask[p + F];
      const int lf = f > 0 && mask[p - 1], rt = f < F - 1 && mask[p + 1];
      out[p] = (uint8_t)!(up && dn && lf && rt);
    }
}
