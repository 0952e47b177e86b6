/*
 * tp_oracle.c -- plain CPU oracle for the hot path of the multibeam transient
 * search of Magro, Hickish & Zarb Adami, "Multibeam GPU Transient Pipeline
 * for the Medicina BEST-2 Array" (arXiv:1307.5700).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the tests, the
 * package smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never does.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Every function follows a definition of the paper (section / equation given
 * in its comment) in the most direct loop form: floating point in IEEE binary64,
 * 8-bit samples in exact 64-bit integers.  It must be compiled with
 * -ffp-contract=off so that no multiply-add is fused.
 *
 * Readings of the paper that are not fixed by its text (each one is also listed
 * with its reason in the design notes):
 *   R1  channel c has centre frequency f_lo + (c + 1/2) * bw / nchan (MHz);
 *       bw < 0 describes a band that descends with channel index.
 *   R2  the reference frequency is the highest channel centre, so every delay
 *       is >= 0 and the top channel has delay 0.
 *   R3  Eq. 1 is evaluated with the constant 4148.808 s MHz^2 and rounded to the
 *       nearest sample, halves upward: floor(v + 0.5).
 *   R4  the bandpass of a block is the per-channel mean of the block's window
 *       (the whole buffer the block processes, overlap included); its spread is
 *       the population standard deviation.
 *   R5  channel thresholding (Sec. 2.2.1): chunk k of channel c is the samples
 *       [kW, min((k+1)W, N)); it exceeds when sum(x - mu_c) > tau_c sigma_c
 *       sqrt(n_k); a chunk is flagged when it or a time-adjacent chunk of the
 *       same channel exceeds (optionally also the same chunk of the adjacent
 *       channels).
 *   R6  spectrum thresholding (Sec. 2.2.1) looks at the bandpass-corrected
 *       spectrum after the channel stage has substituted its chunks: the sum
 *       over the channels unflagged at t of (x - mu_c) is compared with
 *       tau_s sqrt(sum of sigma_c^2 over the same channels), i.e. the mean
 *       over the unflagged band against tau_s times its standard deviation.
 *       The unflagged set changes only at chunk boundaries, so the threshold
 *       is one value per chunk.
 *   R7  a flagged sample is replaced by the channel's bandpass value b_c and b_c
 *       is subtracted from every sample, so a flagged sample contributes
 *       exactly 0.  b_c is mu_c expressed in the data's storage format: the
 *       integer floor(mu_c + 1/2) for 8-bit data, mu_c rounded to nearest even
 *       for binary16 / bfloat16 data, mu_c itself for binary32 data.
 *   R8  the detection threshold of Sec. 2.3 is (D - mu_d) >= nsigma * sigma_d
 *       on each dedispersed series, with sigma_d the population standard
 *       deviation of the series; a series with sigma_d = 0 yields nothing.
 *   R12 complex voltages (Sec. 1.1: 16 bits per complex component) are detected
 *       as power |v|^2 = re^2 + im^2 ("power calculation", Sec. 2); the power
 *       series then takes the binary32 path (bandpass value mu_c itself).
 *   R13 optional fitted bandpass (Sec. 2.2.1 "Bandpass Correction"): the block
 *       means mu_c with high-power channels replaced by their unmasked
 *       neighbours' mean are fitted by least squares with a polynomial of
 *       order p; b_c is the fit, and the channel stage compares chunk means
 *       with b_c + tau_c * RMSE of the fit (see orc_channel_mask_fit).
 *   R11 post-processing (Sec. 2.2.3), optional: the median filter of Eq. 2
 *       replaces y_m by the median of the w = 2h + 1 values centred on m
 *       (odd w; positions beyond the ends of the block's series take the end
 *       value); detrending fits a least-squares line in t to each series and
 *       normalises the residual by its population standard deviation, and the
 *       detection test becomes residual >= nsigma * that deviation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_U8 0
#define ORC_F16 1
#define ORC_BF16 2
#define ORC_F32 3
#define ORC_C16 4 /* complex voltage, int16 real and imaginary parts */

#define ORC_STATS_BLOCK 0
#define ORC_STATS_EXTERNAL 1

/* Dispersion constant of Eq. 1 in s MHz^2 (the printed 4.15e6 ms rounded). */
static const double ORC_KDM = 4148.808;

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }

int orc_get_threads(void) { return g_threads; }

int orc_has_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}

/* IEEE binary16 -> binary64, from the format's definition (exact). */
static double half_bits_to_double(uint16_t h) {
  int sign = (h >> 15) & 1;
  int e = (h >> 10) & 0x1f;
  int m = h & 0x3ff;
  double v;
  if (e == 0)
    v = ldexp((double)m, -24);
  else if (e == 31)
    v = m ? NAN : INFINITY;
  else
    v = ldexp((double)(1024 + m), e - 25);
  return sign ? -v : v;
}

/* bfloat16 is the upper half of a binary32. */
static double bf16_bits_to_double(uint16_t h) {
  uint32_t b = (uint32_t)h << 16;
  float f;
  memcpy(&f, &b, sizeof f);
  return (double)f;
}

/* Stored sample i of a channel-major buffer, converted exactly to binary64. */
static double sample(const void *x, int dtype, int64_t i) {
  switch (dtype) {
  case ORC_U8:
    return (double)((const uint8_t *)x)[i];
  case ORC_F16:
    return half_bits_to_double(((const uint16_t *)x)[i]);
  case ORC_BF16:
    return bf16_bits_to_double(((const uint16_t *)x)[i]);
  case ORC_C16: {
    /* power of the complex voltage (R12), exact in binary64 */
    const double re = (double)((const int16_t *)x)[2 * i];
    const double im = (double)((const int16_t *)x)[2 * i + 1];
    return re * re + im * im;
  }
  default:
    return (double)((const float *)x)[i];
  }
}

static int64_t sample_u8(const void *x, int64_t i) { return (int64_t)((const uint8_t *)x)[i]; }

/* ---- Plan: channel frequencies and the delay table (Eq. 1, R1-R3) ---------- */

void orc_channel_freqs(int nchan, double f_lo, double bw, double *f) {
  double df = bw / (double)nchan;
  for (int c = 0; c < nchan; ++c) f[c] = f_lo + ((double)c + 0.5) * df;
}

/* Delay before rounding, in samples: K * DM * (f_c^-2 - f_ref^-2) / t_samp. */
void orc_delay_exact(int nchan, double f_lo, double bw, double t_samp, const double *dm, int ndm,
                     double *out) {
  double *f = (double *)malloc(sizeof(double) * (size_t)nchan);
  orc_channel_freqs(nchan, f_lo, bw, f);
  double f_ref = f[0];
  for (int c = 1; c < nchan; ++c)
    if (f[c] > f_ref) f_ref = f[c];
  for (int d = 0; d < ndm; ++d)
    for (int c = 0; c < nchan; ++c) {
      double inv_c = 1.0 / (f[c] * f[c]);
      double inv_ref = 1.0 / (f_ref * f_ref);
      out[(int64_t)d * nchan + c] = ORC_KDM * dm[d] * (inv_c - inv_ref) / t_samp;
    }
  free(f);
}

/* Integer delay table delay[d][c]; returns the largest delay, or -1 if the
 * arguments are invalid (nchan, ndm or t_samp not positive, a DM negative or
 * not finite, a channel frequency not positive). */
int64_t orc_delay_table(int nchan, double f_lo, double bw, double t_samp, const double *dm, int ndm,
                        int32_t *delay) {
  if (nchan <= 0 || ndm <= 0 || !(t_samp > 0.0) || !isfinite(t_samp) || !isfinite(f_lo) ||
      !isfinite(bw) || bw == 0.0)
    return -1;
  for (int d = 0; d < ndm; ++d)
    if (!isfinite(dm[d]) || dm[d] < 0.0) return -1;
  double *f = (double *)malloc(sizeof(double) * (size_t)nchan);
  orc_channel_freqs(nchan, f_lo, bw, f);
  for (int c = 0; c < nchan; ++c)
    if (!(f[c] > 0.0)) {
      free(f);
      return -1;
    }
  free(f);
  double *v = (double *)malloc(sizeof(double) * (size_t)nchan * (size_t)ndm);
  orc_delay_exact(nchan, f_lo, bw, t_samp, dm, ndm, v);
  int64_t dmax = 0;
  for (int64_t i = 0; i < (int64_t)nchan * ndm; ++i) {
    double r = floor(v[i] + 0.5);
    if (r > 2147483647.0) {
      free(v);
      return -1;
    }
    delay[i] = (int32_t)r;
    if (delay[i] > dmax) dmax = delay[i];
  }
  free(v);
  return dmax;
}

/* Tie log of the rounding in Eq. 1 (R3): the (d, c) pairs whose unrounded
 * delay v lies within eps of a half-integer, i.e. |v - floor(v) - 1/2| <= eps,
 * where floor(v + 1/2) could go either way under a different rounding of v.
 * Writes up to cap entries (d, c, v) in (d, c) order and returns how many pairs
 * there are (all of them, also beyond cap); -1 for invalid arguments. */
int64_t orc_delay_ties(int nchan, double f_lo, double bw, double t_samp, const double *dm, int ndm,
                       double eps, int32_t *out_d, int32_t *out_c, double *out_v, int64_t cap) {
  if (nchan <= 0 || ndm <= 0 || !(t_samp > 0.0) || !(eps >= 0.0)) return -1;
  double *v = (double *)malloc(sizeof(double) * (size_t)nchan * (size_t)ndm);
  orc_delay_exact(nchan, f_lo, bw, t_samp, dm, ndm, v);
  int64_t n = 0;
  for (int d = 0; d < ndm; ++d)
    for (int c = 0; c < nchan; ++c) {
      const double x = v[(int64_t)d * nchan + c];
      if (fabs(x - floor(x) - 0.5) <= eps) {
        if (n < cap) {
          out_d[n] = d;
          out_c[n] = c;
          out_v[n] = x;
        }
        ++n;
      }
    }
  free(v);
  return n;
}

/* ---- A1: bandpass statistics (Sec. 2.2.1 "Bandpass Correction", R4) --------- */

/* Float samples: mu_c = sum x / N, sigma_c = sqrt(sum (x - mu_c)^2 / N). */
void orc_bandpass_float(const void *x, int dtype, int nchan, int64_t nsamp, int64_t pitch,
                        double *mu, double *sigma) {
  for (int c = 0; c < nchan; ++c) {
    const int64_t row = (int64_t)c * pitch;
    double s = 0.0;
    for (int64_t t = 0; t < nsamp; ++t) s += sample(x, dtype, row + t);
    double m = s / (double)nsamp;
    double q = 0.0;
    for (int64_t t = 0; t < nsamp; ++t) {
      double e = sample(x, dtype, row + t) - m;
      q += e * e;
    }
    mu[c] = m;
    sigma[c] = sqrt(q / (double)nsamp);
  }
}

/* 8-bit samples, exact: S = sum x, Q = sum x^2, V = N Q - S^2 (so that
 * mu = S/N and sigma = sqrt(V)/N), bandpass value b = floor(mu + 1/2)
 * = floor((2S + N) / (2N)). */
void orc_bandpass_u8(const uint8_t *x, int nchan, int64_t nsamp, int64_t pitch, int64_t *S,
                     int64_t *Q, int64_t *V, int64_t *b, double *mu, double *sigma) {
  for (int c = 0; c < nchan; ++c) {
    const int64_t row = (int64_t)c * pitch;
    int64_t s = 0, q = 0;
    for (int64_t t = 0; t < nsamp; ++t) {
      int64_t v = x[row + t];
      s += v;
      q += v * v;
    }
    S[c] = s;
    Q[c] = q;
    V[c] = nsamp * q - s * s;
    b[c] = (2 * s + nsamp) / (2 * nsamp);
    mu[c] = (double)s / (double)nsamp;
    sigma[c] = sqrt((double)V[c]) / (double)nsamp;
  }
}

/* Nearest value of a 16-bit storage format (ties to even), from the format's
 * definition: `sig` significant bits, smallest normal exponent `emin`, largest
 * finite value `maxv`.  Used for the bandpass value of 16-bit data (R7). */
static double round_to_format(double v, int sig, int emin, double maxv) {
  if (v == 0.0 || !isfinite(v)) return v;
  double a = fabs(v);
  int e;
  frexp(a, &e); /* a = m 2^e, m in [1/2, 1) */
  int qexp = e - sig;
  if (qexp < emin - sig + 1) qexp = emin - sig + 1; /* subnormal quantum */
  double q = ldexp(1.0, qexp);
  double r = nearbyint(a / q) * q; /* a / q is exact; default rounding is to nearest even */
  if (r > maxv) r = INFINITY;
  return copysign(r, v);
}

/* Bandpass value of each channel in the storage format of the data (R7):
 * binary16 / bfloat16 round to nearest even, binary32 keeps mu. */
void orc_storage_bandpass(int dtype, const double *mu, int n, double *b) {
  for (int c = 0; c < n; ++c) {
    if (dtype == ORC_F16)
      b[c] = round_to_format(mu[c], 11, -14, 65504.0);
    else if (dtype == ORC_BF16)
      b[c] = round_to_format(mu[c], 8, -126, 3.3895313892515355e38);
    else
      b[c] = mu[c];
  }
}

/* ---- A2: channel thresholding (Sec. 2.2.1 "Channel Thresholding", R5) ------- */

static void dilate(int nchan, int nchunk, const uint8_t *raw, int dilate_channels, uint8_t *flag) {
  for (int c = 0; c < nchan; ++c)
    for (int k = 0; k < nchunk; ++k) {
      int f = raw[(int64_t)c * nchunk + k];
      if (k > 0) f |= raw[(int64_t)c * nchunk + k - 1];
      if (k + 1 < nchunk) f |= raw[(int64_t)c * nchunk + k + 1];
      if (dilate_channels) {
        if (c > 0) f |= raw[(int64_t)(c - 1) * nchunk + k];
        if (c + 1 < nchan) f |= raw[(int64_t)(c + 1) * nchunk + k];
      }
      flag[(int64_t)c * nchunk + k] = (uint8_t)(f != 0);
    }
}

/* Float samples: chunk exceeds when sum_{chunk}(x - mu_c) > tau sigma_c sqrt(n). */
void orc_channel_mask_float(const void *x, int dtype, int nchan, int64_t nsamp, int64_t pitch,
                            int W, double tau, int dilate_channels, const double *mu,
                            const double *sigma, uint8_t *raw, uint8_t *flag) {
  const int nchunk = (int)((nsamp + W - 1) / W);
  for (int c = 0; c < nchan; ++c)
    for (int k = 0; k < nchunk; ++k) {
      int64_t lo = (int64_t)k * W, hi = lo + W < nsamp ? lo + W : nsamp;
      double e = 0.0;
      for (int64_t t = lo; t < hi; ++t) e += sample(x, dtype, (int64_t)c * pitch + t) - mu[c];
      raw[(int64_t)c * nchunk + k] = (uint8_t)(e > tau * sigma[c] * sqrt((double)(hi - lo)));
    }
  dilate(nchan, nchunk, raw, dilate_channels, flag);
}

/* 8-bit samples, block statistics, exact: with mu = S/N and sigma = sqrt(V)/N
 * the test sum(x - mu) > tau sigma sqrt(n) is, multiplied through by N,
 * sum(N x - S) > tau sqrt(V n); the left side is an exact integer. */
void orc_channel_mask_u8(const uint8_t *x, int nchan, int64_t nsamp, int64_t pitch, int W,
                         double tau, int dilate_channels, const int64_t *S, const int64_t *V,
                         uint8_t *raw, uint8_t *flag) {
  const int nchunk = (int)((nsamp + W - 1) / W);
  for (int c = 0; c < nchan; ++c)
    for (int k = 0; k < nchunk; ++k) {
      int64_t lo = (int64_t)k * W, hi = lo + W < nsamp ? lo + W : nsamp;
      int64_t e = 0;
      for (int64_t t = lo; t < hi; ++t) e += nsamp * sample_u8(x, (int64_t)c * pitch + t) - S[c];
      raw[(int64_t)c * nchunk + k] = (uint8_t)((double)e > tau * sqrt((double)V[c] * (double)(hi - lo)));
    }
  dilate(nchan, nchunk, raw, dilate_channels, flag);
}

/* 8-bit samples with an externally supplied integer bandpass b_c and spread
 * sigma_c: sum(x - b_c) is exact and is compared with tau sigma_c sqrt(n). */
void orc_channel_mask_u8_ext(const uint8_t *x, int nchan, int64_t nsamp, int64_t pitch, int W,
                             double tau, int dilate_channels, const int64_t *b,
                             const double *sigma, uint8_t *raw, uint8_t *flag) {
  const int nchunk = (int)((nsamp + W - 1) / W);
  for (int c = 0; c < nchan; ++c)
    for (int k = 0; k < nchunk; ++k) {
      int64_t lo = (int64_t)k * W, hi = lo + W < nsamp ? lo + W : nsamp;
      int64_t e = 0;
      for (int64_t t = lo; t < hi; ++t) e += sample_u8(x, (int64_t)c * pitch + t) - b[c];
      raw[(int64_t)c * nchunk + k] = (uint8_t)((double)e > tau * sigma[c] * sqrt((double)(hi - lo)));
    }
  dilate(nchan, nchunk, raw, dilate_channels, flag);
}

/* Channel thresholding against a fitted bandpass (R13, Sec. 2.2.1 "Bandpass
 * Correction" and Fig. 2): chunk k of channel c exceeds when
 * sum_t (x - b_c) > tau * rmse * n_k, i.e. its mean lies above the fitted
 * bandpass b_c by more than tau times the fit's RMSE; any sample format
 * (8-bit samples are exact in binary64). */
void orc_channel_mask_fit(const void *x, int dtype, int nchan, int64_t nsamp, int64_t pitch, int W,
                          double tau, int dilate_channels, const double *b, double rmse, uint8_t *raw,
                          uint8_t *flag) {
  const int nchunk = (int)((nsamp + W - 1) / W);
  for (int c = 0; c < nchan; ++c)
    for (int k = 0; k < nchunk; ++k) {
      int64_t lo = (int64_t)k * W, hi = lo + W < nsamp ? lo + W : nsamp;
      double e = 0.0;
      for (int64_t t = lo; t < hi; ++t) e += sample(x, dtype, (int64_t)c * pitch + t) - b[c];
      raw[(int64_t)c * nchunk + k] = (uint8_t)(e > tau * rmse * (double)(hi - lo));
    }
  dilate(nchan, nchunk, raw, dilate_channels, flag);
}

/* ---- A3: spectrum thresholding (Sec. 2.2.1 "Spectrum Thresholding", R6) ----- */

/* Per-chunk threshold tau_s sqrt(sum of sigma_c^2 over the channels whose
 * chunk k is not flagged), the sum in channel order. */
static void unflagged_thresholds(int nchan, int nchunk, double tau_s, const double *sigma,
                                 const uint8_t *chunk_flag, double *thr) {
  for (int k = 0; k < nchunk; ++k) {
    double v = 0.0;
    for (int c = 0; c < nchan; ++c)
      if (!chunk_flag[(int64_t)c * nchunk + k]) v += sigma[c] * sigma[c];
    thr[k] = tau_s * sqrt(v);
  }
}

/* Float samples: spectrum t is flagged when the sum over the channels whose
 * chunk is not flagged of (x - mu_c) > tau_s sqrt(sum of their sigma_c^2). */
void orc_spectrum_mask_float(const void *x, int dtype, int nchan, int64_t nsamp, int64_t pitch,
                             int W, double tau_s, const double *mu, const double *sigma,
                             const uint8_t *chunk_flag, uint8_t *spec_flag) {
  const int nchunk = (int)((nsamp + W - 1) / W);
  double *thr = (double *)malloc(sizeof(double) * (size_t)nchunk);
  unflagged_thresholds(nchan, nchunk, tau_s, sigma, chunk_flag, thr);
  /* m[t] accumulates channel c = 0, 1, ... in order for every t */
  double *m = (double *)calloc((size_t)nsamp, sizeof(double));
  for (int c = 0; c < nchan; ++c)
    for (int64_t t = 0; t < nsamp; ++t)
      if (!chunk_flag[(int64_t)c * nchunk + t / W]) m[t] += sample(x, dtype, (int64_t)c * pitch + t) - mu[c];
  for (int64_t t = 0; t < nsamp; ++t) spec_flag[t] = (uint8_t)(m[t] > thr[t / W]);
  free(m);
  free(thr);
}

/* 8-bit samples, block statistics, exact: multiplied through by N the test is
 * sum(N x - S_c) > tau_s sqrt(sum V_c), both sums over the channels unflagged
 * at t.  The sum of V_c can exceed 2^63, so it is kept exactly as a high part
 * (V >> 20) and a low part (V & (2^20 - 1)) and converted as hi * 2^20 + lo. */
void orc_spectrum_mask_u8(const uint8_t *x, int nchan, int64_t nsamp, int64_t pitch, int W,
                          double tau_s, const int64_t *S, const int64_t *V,
                          const uint8_t *chunk_flag, uint8_t *spec_flag) {
  const int nchunk = (int)((nsamp + W - 1) / W);
  double *thr = (double *)malloc(sizeof(double) * (size_t)nchunk);
  for (int k = 0; k < nchunk; ++k) {
    uint64_t vhi = 0, vlo = 0;
    for (int c = 0; c < nchan; ++c)
      if (!chunk_flag[(int64_t)c * nchunk + k]) {
        vhi += (uint64_t)V[c] >> 20;
        vlo += (uint64_t)V[c] & 0xFFFFFu;
      }
    thr[k] = tau_s * sqrt((double)vhi * 1048576.0 + (double)vlo);
  }
  int64_t *m = (int64_t *)calloc((size_t)nsamp, sizeof(int64_t));
  for (int c = 0; c < nchan; ++c)
    for (int64_t t = 0; t < nsamp; ++t)
      if (!chunk_flag[(int64_t)c * nchunk + t / W]) m[t] += nsamp * sample_u8(x, (int64_t)c * pitch + t) - S[c];
  for (int64_t t = 0; t < nsamp; ++t) spec_flag[t] = (uint8_t)((double)m[t] > thr[t / W]);
  free(m);
  free(thr);
}

/* 8-bit samples with external (or fitted) bandpass b_c and spread sigma_c. */
void orc_spectrum_mask_u8_ext(const uint8_t *x, int nchan, int64_t nsamp, int64_t pitch, int W,
                              double tau_s, const int64_t *b, const double *sigma,
                              const uint8_t *chunk_flag, uint8_t *spec_flag) {
  const int nchunk = (int)((nsamp + W - 1) / W);
  double *thr = (double *)malloc(sizeof(double) * (size_t)nchunk);
  unflagged_thresholds(nchan, nchunk, tau_s, sigma, chunk_flag, thr);
  int64_t *m = (int64_t *)calloc((size_t)nsamp, sizeof(int64_t));
  for (int c = 0; c < nchan; ++c)
    for (int64_t t = 0; t < nsamp; ++t)
      if (!chunk_flag[(int64_t)c * nchunk + t / W]) m[t] += sample_u8(x, (int64_t)c * pitch + t) - b[c];
  for (int64_t t = 0; t < nsamp; ++t) spec_flag[t] = (uint8_t)((double)m[t] > thr[t / W]);
  free(m);
  free(thr);
}

/* ---- A4: substitution (R7) --------------------------------------------------- */

static int flagged(const uint8_t *chunk_flag, const uint8_t *spec_flag, int nchunk, int W, int c,
                   int64_t t) {
  if (chunk_flag && chunk_flag[(int64_t)c * nchunk + t / W]) return 1;
  if (spec_flag && spec_flag[t]) return 1;
  return 0;
}

/* Bandpass-corrected, substituted sample x~[c][t] - b_c (floats). */
static double corrected_float(const void *x, int dtype, int64_t pitch, const double *mu,
                              const uint8_t *chunk_flag, const uint8_t *spec_flag, int nchunk, int W,
                              int c, int64_t t) {
  if (flagged(chunk_flag, spec_flag, nchunk, W, c, t)) return 0.0;
  return sample(x, dtype, (int64_t)c * pitch + t) - mu[c];
}

static int64_t corrected_u8(const uint8_t *x, int64_t pitch, const int64_t *b,
                            const uint8_t *chunk_flag, const uint8_t *spec_flag, int nchunk, int W,
                            int c, int64_t t) {
  if (flagged(chunk_flag, spec_flag, nchunk, W, c, t)) return 0;
  return (int64_t)x[(int64_t)c * pitch + t] - b[c];
}

/* Whole substituted, corrected array y[c][t] (float path; for small cases). */
void orc_corrected_float(const void *x, int dtype, int nchan, int64_t nsamp, int64_t pitch,
                         const double *mu, const uint8_t *chunk_flag, const uint8_t *spec_flag,
                         int W, double *y) {
  const int nchunk = (int)((nsamp + W - 1) / W);
  for (int c = 0; c < nchan; ++c)
    for (int64_t t = 0; t < nsamp; ++t)
      y[(int64_t)c * nsamp + t] =
          corrected_float(x, dtype, pitch, mu, chunk_flag, spec_flag, nchunk, W, c, t);
}

/* ---- A5: brute-force dedispersion (Sec. 2.2.2, Eq. 1) --------------------------
 * D[d][t] = sum_{c=0}^{nchan-1} y[c][t + delay[d][c]],  0 <= t < T,
 * T = nsamp - max delay.  Channels are summed in index order. */

void orc_dedisperse_float(const void *x, int dtype, int nchan, int64_t nsamp, int64_t pitch,
                          const double *mu, const uint8_t *chunk_flag, const uint8_t *spec_flag,
                          int W, const int32_t *delay, int ndm, int64_t T, double *D) {
  const int nchunk = W > 0 ? (int)((nsamp + W - 1) / W) : 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
#endif
  for (int d = 0; d < ndm; ++d)
    for (int64_t t = 0; t < T; ++t) {
      double acc = 0.0;
      for (int c = 0; c < nchan; ++c)
        acc += corrected_float(x, dtype, pitch, mu, chunk_flag, spec_flag, nchunk, W, c,
                               t + delay[(int64_t)d * nchan + c]);
      D[(int64_t)d * T + t] = acc;
    }
}

void orc_dedisperse_u8(const uint8_t *x, int nchan, int64_t nsamp, int64_t pitch, const int64_t *b,
                       const uint8_t *chunk_flag, const uint8_t *spec_flag, int W,
                       const int32_t *delay, int ndm, int64_t T, int64_t *D) {
  const int nchunk = W > 0 ? (int)((nsamp + W - 1) / W) : 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
#endif
  for (int d = 0; d < ndm; ++d)
    for (int64_t t = 0; t < T; ++t) {
      int64_t acc = 0;
      for (int c = 0; c < nchan; ++c)
        acc += corrected_u8(x, pitch, b, chunk_flag, spec_flag, nchunk, W, c,
                            t + delay[(int64_t)d * nchan + c]);
      D[(int64_t)d * T + t] = acc;
    }
}

/* Selected outputs D[d_idx[i]][t_idx[i]] only (for checks at full size). */
void orc_dedisperse_points_float(const void *x, int dtype, int nchan, int64_t nsamp, int64_t pitch,
                                 const double *mu, const uint8_t *chunk_flag,
                                 const uint8_t *spec_flag, int W, const int32_t *delay,
                                 const int32_t *d_idx, const int64_t *t_idx, int64_t npts,
                                 double *out) {
  const int nchunk = W > 0 ? (int)((nsamp + W - 1) / W) : 0;
  for (int64_t i = 0; i < npts; ++i) {
    double acc = 0.0;
    for (int c = 0; c < nchan; ++c)
      acc += corrected_float(x, dtype, pitch, mu, chunk_flag, spec_flag, nchunk, W, c,
                             t_idx[i] + delay[(int64_t)d_idx[i] * nchan + c]);
    out[i] = acc;
  }
}

void orc_dedisperse_points_u8(const uint8_t *x, int nchan, int64_t nsamp, int64_t pitch,
                              const int64_t *b, const uint8_t *chunk_flag,
                              const uint8_t *spec_flag, int W, const int32_t *delay,
                              const int32_t *d_idx, const int64_t *t_idx, int64_t npts,
                              int64_t *out) {
  const int nchunk = W > 0 ? (int)((nsamp + W - 1) / W) : 0;
  for (int64_t i = 0; i < npts; ++i) {
    int64_t acc = 0;
    for (int c = 0; c < nchan; ++c)
      acc += corrected_u8(x, pitch, b, chunk_flag, spec_flag, nchunk, W, c,
                          t_idx[i] + delay[(int64_t)d_idx[i] * nchan + c]);
    out[i] = acc;
  }
}

/* Sum over channels of |y| at the delayed positions: the magnitude against
 * which the error of a floating-point D[d][t] is bounded. */
void orc_abs_mass_points_float(const void *x, int dtype, int nchan, int64_t nsamp, int64_t pitch,
                               const double *mu, const uint8_t *chunk_flag,
                               const uint8_t *spec_flag, int W, const int32_t *delay,
                               const int32_t *d_idx, const int64_t *t_idx, int64_t npts,
                               double *out) {
  const int nchunk = W > 0 ? (int)((nsamp + W - 1) / W) : 0;
  for (int64_t i = 0; i < npts; ++i) {
    double acc = 0.0;
    for (int c = 0; c < nchan; ++c)
      acc += fabs(corrected_float(x, dtype, pitch, mu, chunk_flag, spec_flag, nchunk, W, c,
                                  t_idx[i] + delay[(int64_t)d_idx[i] * nchan + c]));
    out[i] = acc;
  }
}

/* Sum over channels of |x~| (the stored, substituted samples) at the delayed
 * positions: the magnitude against which FP32 accumulation of stored 16-bit
 * samples is bounded. */
void orc_stored_mass_points(const void *x, int dtype, int nchan, int64_t nsamp, int64_t pitch,
                            const double *b, const uint8_t *chunk_flag, const uint8_t *spec_flag, int W,
                            const int32_t *delay, const int32_t *d_idx, const int64_t *t_idx,
                            int64_t npts, double *out) {
  const int nchunk = W > 0 ? (int)((nsamp + W - 1) / W) : 0;
  for (int64_t i = 0; i < npts; ++i) {
    double acc = 0.0;
    for (int c = 0; c < nchan; ++c) {
      const int64_t t = t_idx[i] + delay[(int64_t)d_idx[i] * nchan + c];
      acc += flagged(chunk_flag, spec_flag, nchunk, W, c, t) ? fabs(b[c])
                                                              : fabs(sample(x, dtype, (int64_t)c * pitch + t));
    }
    out[i] = acc;
  }
}

/* ---- A6: series statistics (Sec. 2.2.3 normalisation) ---------------------- */

/* Float series: two-pass population mean and standard deviation per DM row. */
void orc_series_stats_float(const double *D, int ndm, int64_t T, double *mu, double *sigma) {
  for (int d = 0; d < ndm; ++d) {
    const double *r = D + (int64_t)d * T;
    double s = 0.0;
    for (int64_t t = 0; t < T; ++t) s += r[t];
    double m = s / (double)T;
    double q = 0.0;
    for (int64_t t = 0; t < T; ++t) q += (r[t] - m) * (r[t] - m);
    mu[d] = m;
    sigma[d] = sqrt(q / (double)T);
  }
}

/* Integer series, exact sums: mu = SD/T, sigma^2 = SD2/T - mu^2 (population),
 * evaluated in binary64 from the exact integer sums. */
void orc_series_stats_int(const int64_t *D, int ndm, int64_t T, int64_t *SD, int64_t *SD2,
                          double *mu, double *sigma) {
  for (int d = 0; d < ndm; ++d) {
    const int64_t *r = D + (int64_t)d * T;
    int64_t s = 0, q = 0;
    for (int64_t t = 0; t < T; ++t) {
      s += r[t];
      q += r[t] * r[t];
    }
    SD[d] = s;
    SD2[d] = q;
    double m = (double)s / (double)T;
    double var = (double)q / (double)T - m * m;
    mu[d] = m;
    sigma[d] = sqrt(var > 0.0 ? var : 0.0);
  }
}

/* ---- A7: detection (Sec. 2.3, R8) ------------------------------------------ */

typedef struct {
  int32_t beam;
  int32_t dm_idx;
  int64_t t_abs;
  float snr;
  float value;
} orc_candidate;

/* Candidates in (d, t) order; writes at most cap records and returns the total. */
int64_t orc_candidates_float(const double *D, int ndm, int64_t T, const double *mu,
                             const double *sigma, double nsigma, int beam, int64_t t0,
                             orc_candidate *out, int64_t cap) {
  int64_t n = 0;
  for (int d = 0; d < ndm; ++d) {
    if (!(sigma[d] > 0.0)) continue;
    for (int64_t t = 0; t < T; ++t) {
      double v = D[(int64_t)d * T + t];
      if (v - mu[d] >= nsigma * sigma[d]) {
        if (n < cap) {
          out[n].beam = beam;
          out[n].dm_idx = d;
          out[n].t_abs = t0 + t;
          out[n].snr = (float)((v - mu[d]) / sigma[d]);
          out[n].value = (float)v;
        }
        ++n;
      }
    }
  }
  return n;
}

int64_t orc_candidates_int(const int64_t *D, int ndm, int64_t T, const double *mu,
                           const double *sigma, double nsigma, int beam, int64_t t0,
                           orc_candidate *out, int64_t cap) {
  int64_t n = 0;
  for (int d = 0; d < ndm; ++d) {
    if (!(sigma[d] > 0.0)) continue;
    for (int64_t t = 0; t < T; ++t) {
      double v = (double)D[(int64_t)d * T + t];
      if (v - mu[d] >= nsigma * sigma[d]) {
        if (n < cap) {
          out[n].beam = beam;
          out[n].dm_idx = d;
          out[n].t_abs = t0 + t;
          out[n].snr = (float)((v - mu[d]) / sigma[d]);
          out[n].value = (float)v;
        }
        ++n;
      }
    }
  }
  return n;
}

/* ---- Post-processing (Sec. 2.2.3) ------------------------------------------- */

/* Median filter, Eq. 2 with the median as the operation (R11): out[d][m] is the
 * median of D[d][clamp(m + i)], i = -h .. h, clamp to [0, T - 1]; the w = 2h + 1
 * values are sorted by insertion and the middle one taken. */
void orc_median_float(const double *D, int ndm, int64_t T, int w, double *out) {
  const int h = w / 2;
  double v[64];
  for (int d = 0; d < ndm; ++d)
    for (int64_t m = 0; m < T; ++m) {
      for (int i = 0; i < w; ++i) {
        int64_t j = m - h + i;
        j = j < 0 ? 0 : (j > T - 1 ? T - 1 : j);
        double x = D[(int64_t)d * T + j];
        int k = i;
        while (k > 0 && v[k - 1] > x) {
          v[k] = v[k - 1];
          --k;
        }
        v[k] = x;
      }
      out[(int64_t)d * T + m] = v[h];
    }
}

void orc_median_int(const int64_t *D, int ndm, int64_t T, int w, int64_t *out) {
  const int h = w / 2;
  int64_t v[64];
  for (int d = 0; d < ndm; ++d)
    for (int64_t m = 0; m < T; ++m) {
      for (int i = 0; i < w; ++i) {
        int64_t j = m - h + i;
        j = j < 0 ? 0 : (j > T - 1 ? T - 1 : j);
        int64_t x = D[(int64_t)d * T + j];
        int k = i;
        while (k > 0 && v[k - 1] > x) {
          v[k] = v[k - 1];
          --k;
        }
        v[k] = x;
      }
      out[(int64_t)d * T + m] = v[h];
    }
}

/* Detrending (R11): least-squares line y ~ mean + beta * u_t with the centred
 * abscissa u_t = 2t - (T - 1) (sum_t u_t = 0, so the intercept is the mean and
 * the slope decouples), from the sums
 *   Sy = sum y,  Suy = sum u y,  Syy = sum y^2,  Suu = sum u^2 = (T-1) T (T+1) / 3,
 *   mean = Sy / T,  beta = Suy / Suu,
 *   RSS = Syy - Sy Sy / T - Suy Suy / Suu  (the least-squares residual identity),
 *   sigma_r = sqrt(max(RSS, 0) / T).
 * Float series: the sums in binary64 in t order.  Integer series: the sums
 * exactly in int64, then the same binary64 formula. */
static void detrend_from_sums(double Sy, double Suy, double Syy, int64_t T, double *mean, double *beta,
                              double *sigma) {
  const double Tn = (double)T;
  const double Suu = (double)(((T - 1) * T * (T + 1)) / 3);
  const double m = Sy / Tn;
  const double b = T > 1 ? Suy / Suu : 0.0;
  double rss = Syy - Sy * Sy / Tn;
  if (T > 1) rss = rss - Suy * Suy / Suu;
  *mean = m;
  *beta = b;
  *sigma = sqrt((rss > 0.0 ? rss : 0.0) / Tn);
}

void orc_detrend_float(const double *D, int ndm, int64_t T, double *mean, double *beta, double *sigma) {
  for (int d = 0; d < ndm; ++d) {
    const double *r = D + (int64_t)d * T;
    double sy = 0.0, suy = 0.0, syy = 0.0;
    for (int64_t t = 0; t < T; ++t) {
      sy += r[t];
      suy += (double)(2 * t - (T - 1)) * r[t];
      syy += r[t] * r[t];
    }
    detrend_from_sums(sy, suy, syy, T, &mean[d], &beta[d], &sigma[d]);
  }
}

void orc_detrend_int(const int64_t *D, int ndm, int64_t T, int64_t *sums, double *mean, double *beta,
                     double *sigma) {
  for (int d = 0; d < ndm; ++d) {
    const int64_t *r = D + (int64_t)d * T;
    int64_t sy = 0, suy = 0, syy = 0;
    for (int64_t t = 0; t < T; ++t) {
      sy += r[t];
      suy += (2 * t - (T - 1)) * r[t];
      syy += r[t] * r[t];
    }
    sums[3 * d] = sy;
    sums[3 * d + 1] = suy;
    sums[3 * d + 2] = syy;
    detrend_from_sums((double)sy, (double)suy, (double)syy, T, &mean[d], &beta[d], &sigma[d]);
  }
}

/* Candidates of detrended series (R11): residual r = y - (mean + beta u_t),
 * a detection when sigma > 0 and r >= nsigma * sigma; snr = r / sigma.  D is
 * binary64 (float data) or int64 (is_int). */
int64_t orc_candidates_detrend(const void *D, int is_int, int ndm, int64_t T, const double *mean,
                               const double *beta, const double *sigma, double nsigma, int beam, int64_t t0,
                               orc_candidate *out, int64_t cap) {
  int64_t n = 0;
  for (int d = 0; d < ndm; ++d) {
    if (!(sigma[d] > 0.0)) continue;
    const double thr = nsigma * sigma[d];
    for (int64_t t = 0; t < T; ++t) {
      const int64_t i = (int64_t)d * T + t;
      const double v = is_int ? (double)((const int64_t *)D)[i] : ((const double *)D)[i];
      const double lin = mean[d] + beta[d] * (double)(2 * t - (T - 1));
      const double r = v - lin;
      if (r >= thr) {
        if (n < cap) {
          out[n].beam = beam;
          out[n].dm_idx = d;
          out[n].t_abs = t0 + t;
          out[n].snr = (float)(r / sigma[d]);
          out[n].value = (float)v;
        }
        ++n;
      }
    }
  }
  return n;
}
