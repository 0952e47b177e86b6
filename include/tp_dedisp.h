/*
 * tp_dedisp.h -- C ABI of the GB300 dedispersion search library.
 *
 * The library runs the data-parallel hot path of the multibeam transient
 * pipeline of Magro, Hickish & Zarb Adami (arXiv:1307.5700) on one GPU:
 *
 *   A0  plan: channel frequencies and the integer delay table of Eq. 1
 *   A1  per-channel bandpass statistics ("Bandpass Correction", Sec. 2.2.1)
 *   A2  channel thresholding ("Channel Thresholding", Sec. 2.2.1)
 *   A3  spectrum thresholding ("Spectrum Thresholding", Sec. 2.2.1)
 *   A4  substitution of flagged samples by the bandpass (Sec. 2.2.1)
 *   A5  brute-force incoherent dedispersion (Sec. 2.2.2)
 *   A6  per-DM series mean / standard deviation (Sec. 2.2.3)
 *   A7  n-sigma thresholding into a candidate list compacted on the device
 *       (Sec. 2.3, first stage of event detection)
 *
 * Conventions shared by every entry point:
 *   - Return value: TP_OK (0) or a negative TP_E* code.  The text of the last
 *     error of the calling thread is available from tp_last_error_string().
 *   - Every GPU operation of an engine is issued on the engine's stream (or on
 *     the beam's stream, see tp_beam_set_stream) and is asynchronous unless the
 *     entry point says it blocks.
 *   - Filterbank blocks are channel-major: sample t of channel c is at element
 *     c * nsamp + t (the paper's beam / channel / time order, Sec. 2.1).
 *   - Pointers are plain host or device addresses, as stated per argument;
 *     the library never keeps a caller pointer after the call returns.
 */
#ifndef TP_DEDISP_H
#define TP_DEDISP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------------- */
#define TP_OK 0
#define TP_EINVAL -1     /* an argument is out of range or inconsistent       */
#define TP_ENOMEM -2     /* a device or host allocation failed                */
#define TP_EADMIT -3     /* the beam does not fit the engine's HBM budget     */
#define TP_EBUSY -4      /* the beam's window still holds an unprocessed block */
#define TP_ENOTREADY -5  /* the step that must come first has not been issued */
#define TP_ETRUNC -6     /* more candidates than the caller's buffer holds    */
#define TP_ECUDA -7      /* a CUDA runtime call failed                         */
#define TP_ETIMEOUT -8   /* a bounded device-side wait gave up                 */
#define TP_EBOUNDS -9    /* a device-side bounds check failed                  */
#define TP_EOVERFLOW -10 /* the candidate buffer of the beam overflowed        */

/* ---- sample formats ---------------------------------------------------------- */
#define TP_U8 0   /* unsigned 8-bit power; exact int32 sums                    */
#define TP_F16 1  /* IEEE binary16; FP32 accumulation                          */
#define TP_BF16 2 /* bfloat16; FP32 accumulation                               */
#define TP_F32 3  /* IEEE binary32; FP32 accumulation                          */
#define TP_C16 4  /* complex voltage, int16 real then int16 imaginary part (4 bytes
                     a sample): detected as power |v|^2 = re^2 + im^2 on load by the
                     statistics and staging kernels (the power stage of Sec. 2;
                     Sec. 1.1: 16 bits per complex component); FP32 accumulation */

/* ---- bandpass statistics modes ---------------------------------------------- */
#define TP_STATS_BLOCK 0    /* measured on each block's window (default)       */
#define TP_STATS_EXTERNAL 1 /* supplied by tp_beam_set_bandpass                */

/* RFI thresholding parameters (Sec. 2.2.1).  The paper gives no numbers; the
 * defaults are W_c = 256 samples, tau_c = 5, tau_s = 6.
 *   channel stage : chunk k of channel c (samples [kW, min((k+1)W, N))) exceeds
 *                   when sum(x - mu_c) > tau_channel * sigma_c * sqrt(n_k); the
 *                   chunk and its time-adjacent chunks (and, with
 *                   dilate_channels, the same chunk of channels c-1, c+1) are
 *                   flagged.
 *   spectrum stage: spectrum t is flagged when the sum of the bandpass-
 *                   corrected samples over the channels whose chunk at t is
 *                   not flagged exceeds tau_spectrum * sqrt(sum of sigma_c^2
 *                   over the same channels) (one threshold per chunk).
 *   A flagged sample is replaced by its channel's bandpass value. */
typedef struct tp_rfi_params {
  int32_t enable_channel;  /* 1: run the channel stage                         */
  int32_t enable_spectrum; /* 1: run the spectrum stage                        */
  int32_t chunk_width;     /* W_c in samples, >= 1                             */
  int32_t dilate_channels; /* 1: also flag adjacent channels' chunks           */
  double tau_channel;      /* tau_c                                            */
  double tau_spectrum;     /* tau_s                                            */
  int32_t stats_mode;      /* TP_STATS_BLOCK or TP_STATS_EXTERNAL              */
  int32_t reserved;        /* must be 0                                        */
} tp_rfi_params;

/* One detection (Sec. 2.3: the (time, DM, intensity) triplet, plus the beam
 * and the dedispersed value).  24 bytes. */
typedef struct tp_candidate {
  int32_t beam;   /* beam id                                                   */
  int32_t dm_idx; /* index into the plan's DM list                              */
  int64_t t_abs;  /* stream sample index (arrival time at the top channel)     */
  float snr;      /* (D - mu_d) / sigma_d                                       */
  float value;    /* D[dm_idx][t]                                               */
} tp_candidate;

/* Clustering of a block's detections (Sec. 2.3), see tp_plan_set_clustering. */
typedef struct tp_cluster_params {
  int32_t t_eps;     /* T_t: neighbourhood half-extent in samples (>= 0)          */
  int32_t dm_eps;    /* DM_t: neighbourhood half-extent in DM trials (>= 0)       */
  double snr_eps;    /* SNR_t: neighbourhood half-extent in SNR (>= 0)            */
  int32_t min_pts;   /* MinPts: neighbours of a core point, itself included (>= 1) */
  int32_t smooth;    /* k of the DM-SNR moving average (odd, >= 1)                */
  double rmse_max;   /* largest RMSE against Eq. 3 of a candidate cluster          */
  double dm_min;     /* clusters peaking below this DM (pc cm^-3) are broadband RFI */
} tp_cluster_params;

/* One cluster of detections and its classification.  48 bytes. */
typedef struct tp_cluster {
  int32_t label;     /* cluster number (clusters numbered by their lowest-index core detection) */
  int32_t n;         /* detections in the cluster                                */
  int32_t d_lo, d_hi; /* DM trial range                                          */
  int32_t d_star;    /* trial with the most detections                           */
  int32_t flags;     /* bit 0: candidate; bit 1: broadband RFI (d_star below dm_min) */
  int64_t t_first, t_last; /* first and last detection (stream sample index)     */
  float snr_max;     /* largest SNR                                              */
  float width_ms;    /* (last - first detection time at d_star + 1) samples, ms  */
  float rmse;        /* RMSE of the normalised DM-SNR signature against Eq. 3    */
  float reserved;
} tp_cluster;

typedef struct tp_engine tp_engine;
typedef struct tp_plan tp_plan;

/* Fill *p with the defaults listed above. */
void tp_rfi_defaults(tp_rfi_params *p);

/* ---- engine ------------------------------------------------------------------- */

/* Create an engine bound to CUDA device `device`.  The engine owns the device
 * memory of its plans and beams and admits beams only while their footprint
 * fits `hbm_budget_bytes` (0 = 90 % of the device memory free at creation).
 * `cuda_stream` is a cudaStream_t borrowed from the caller (NULL = the legacy
 * default stream); it must outlive the engine.  Errors: TP_EINVAL (bad device),
 * TP_ECUDA. */
int tp_engine_create(int device, size_t hbm_budget_bytes, void *cuda_stream, tp_engine **out);

/* Free everything the engine owns (its plans and beams included) after waiting
 * for its streams.  NULL is accepted. */
int tp_engine_destroy(tp_engine *e);

/* Wait until all work the engine issued has finished. */
int tp_sync(tp_engine *e);

/* Device bytes currently held by the engine, and its budget. */
int tp_engine_memory(const tp_engine *e, size_t *used, size_t *budget);

/* ---- A0: plan (Eq. 1) --------------------------------------------------------
 * Channel c has centre frequency f_lo_mhz + (c + 1/2) * bw_mhz / nchan (bw < 0:
 * the band descends with channel index).  The reference frequency is the
 * highest centre.  delay[d][c] = floor(4148.808 * dm_list[d] * (f_c^-2 -
 * f_ref^-2) / t_samp_s + 1/2), evaluated in binary64 on the GPU in exactly
 * that operation order, without fused multiply-adds.
 * dm_list (host, ndm doubles) is copied; it must be finite, >= 0 and
 * non-decreasing.  `rfi` may be NULL for the defaults.  `nsigma` is the
 * detection threshold of A7.  The call blocks until the table is built.
 * Errors: TP_EINVAL (nchan <= 0 or > 65535, ndm <= 0, t_samp <= 0, bw = 0, a
 * channel frequency <= 0, a DM negative / not finite / decreasing, bad rfi params,
 * a delay above 2^31 - 1), TP_ENOMEM, TP_ECUDA. */
int tp_create_plan(tp_engine *e, int nchan, double f_lo_mhz, double bw_mhz, double t_samp_s,
                   const double *dm_list, int ndm, int dtype, const tp_rfi_params *rfi,
                   double nsigma, tp_plan **out);

/* Destroy a plan; fails with TP_EBUSY while an open beam uses it. */
int tp_plan_destroy(tp_plan *p);

/* Sizes of a plan (any pointer may be NULL). */
int tp_plan_info(const tp_plan *p, int *nchan, int *ndm, int *max_delay, int *dtype);

/* Post-processing of the dedispersed series before detection (Sec. 2.2.3,
 * "Post-Processing"), both off by default:
 *   median_width w (odd, 1..9; 1 = off): the median filter of Eq. 2 with the
 *     median as the operation -- each value of a block's series is replaced by
 *     the median of the w values centred on it, positions beyond the ends of
 *     the series taking the end value (an exact selection of a stored value);
 *   detrend (0 or 1): a least-squares line mean + beta u_t, u_t = 2t - (T - 1),
 *     is fitted to each (filtered) series, and a candidate is a sample whose
 *     residual y - (mean + beta u_t) is >= nsigma times the residual's
 *     population standard deviation (snr = residual / deviation); without it
 *     the detection of Sec. 2.3 runs on the (filtered) series as before.
 * Call before any beam of the plan is opened (TP_EBUSY otherwise; the
 * filtered series is part of a beam's footprint).  TP_EINVAL for an even or
 * out-of-range width. */
int tp_plan_set_postprocess(tp_plan *p, int median_width, int detrend);

/* Fitted bandpass (Sec. 2.2.1 "Bandpass Correction", with Fig. 2), in place
 * of the plain block mean: order = p (0..8; -1 turns it off).  Per block the
 * channel means are taken, channels whose mean exceeds the mean of its two
 * neighbours (one at the band edges) by more than tau_mask * 1.4826 * the
 * median absolute excess are masked and replaced by the mean of their
 * nearest unmasked neighbours, the result is fitted by least squares with
 * Legendre polynomials of the normalised channel index, and the fit b_c
 * replaces the mean as the bandpass: a W_c chunk is flagged when its mean
 * exceeds b_c + tau_channel * RMSE (the fit's root-mean-square error against
 * the interpolated means, so tau_channel counts in RMSE units), flagged
 * samples take b_c, and the spectrum stage subtracts b_c (8-bit data: the
 * integer floor(b_c + 1/2); 16-bit data: b_c in the storage format).  Needs
 * block statistics (TP_STATS_BLOCK) and at most 8192 channels (TP_EINVAL);
 * call before any beam of the plan is opened (TP_EBUSY). */
int tp_plan_set_bandpass_fit(tp_plan *p, int order, double tau_mask);

/* Running bandpass statistics across the blocks of a stream (Sec. 2.2.1
 * averages the bandpass per processing iteration; reading R15).  Each beam of the
 * plan folds a block's own mean mu_c and variance sigma_c^2 into an
 * exponential average with weight alpha on the new block,
 *   mu_run = alpha mu + (1 - alpha) mu_run_prev,
 *   var_run = alpha sigma^2 + (1 - alpha) var_run_prev
 * (binary64; the stream's first block starts the average), kept on the device
 * between blocks, and thresholds, substitutes and subtracts with mu_run and
 * sqrt(var_run) as with external statistics (8-bit data: the integer
 * floor(mu_run + 1/2)).  alpha = 1 (the default) is per-block statistics.
 * tp_get_bandpass then returns the running values.  Processing the same
 * window again (tp_beam_rewind) repeats the same update.
 * Errors: TP_EINVAL (alpha outside (0, 1], external statistics, or a fitted
 * bandpass on the plan), TP_EBUSY (the plan has open beams). */
int tp_plan_set_running_stats(tp_plan *p, double alpha);

/* Clustering and classification of every block's detections (Sec. 2.3:
 * DBSCAN of the (time, DM, intensity) triplets, then each cluster's DM-SNR
 * signature against the incorrect-dedispersion model of Eq. 3-4), run on the
 * device after the detection; params = NULL turns it off.
 *   Neighbourhood of a detection p: the detections q with |t_q - t_p| <=
 *   t_eps, |d_q - d_p| <= dm_eps, |snr_q - snr_p| <= snr_eps (p included);
 *   core detections have >= min_pts neighbours; clusters are the connected
 *   groups of core detections; a detection that is not core but has a core
 *   neighbour joins the cluster of its lowest-index core neighbour (records
 *   in (dm_idx, t_abs) order); the rest is noise.  Clusters are numbered in
 *   the order of their lowest-index core detection.  (The paper's FDBSCAN is
 *   an approximation of this clustering for a CPU; the device computes it
 *   exactly.)
 *   Classification of each cluster: the largest SNR per DM trial, its
 *   centred moving average over `smooth` trials (fewer at the ends), d* =
 *   the trial with the most detections (ties: the lowest), broadband RFI
 *   when DM(d*) < dm_min, the width (last - first detection time at d* + 1)
 *   samples, the averaged signature divided by its maximum, Eq. 3 for
 *   dDM = DM(d) - DM(d*) with the band's width and centre frequency, and the
 *   RMSE of the two over the cluster's trials; a candidate when not
 *   broadband RFI and RMSE <= rmse_max.
 * Clustering works on the stored detections (the first cand_capacity in
 * (d, t) order) and keeps at most min(cand_capacity, 65536) clusters.  Call
 * before any beam of the plan is opened (TP_EBUSY).  TP_EINVAL for invalid
 * parameters or a plan of more than 14336 DM trials (the classification
 * keeps one cluster's signature in shared memory). */
int tp_plan_set_clustering(tp_plan *p, const tp_cluster_params *params);

/* Copy the delay table (ndm x nchan int32, row = DM) to host memory `out`
 * holding `count` elements.  Blocks. */
int tp_get_delay_table(const tp_plan *p, int32_t *out, size_t count);

/* ---- beams -----------------------------------------------------------------------
 * A beam is one filterbank stream processed with a plan.  It owns a device
 * window of max_delay + block_nsamp samples per channel (the overlap tail of
 * the previous block followed by the new block), its statistics, masks,
 * dedispersed series (ndm x T) and a candidate buffer of `cand_capacity`
 * records.  Admission is by HBM footprint; on TP_EADMIT nothing is allocated.
 * block_nsamp must exceed the plan's max_delay. */
int tp_beam_open(tp_engine *e, const tp_plan *p, int block_nsamp, int cand_capacity, int *beam_id);
int tp_beam_close(tp_engine *e, int beam);

/* Device bytes beam_open would take for these sizes (no allocation). */
int tp_beam_footprint(const tp_plan *p, int block_nsamp, int cand_capacity, size_t *bytes);

/* Issue this beam's work on `cuda_stream` instead of the engine's (NULL =
 * the engine stream).  The stream is borrowed. */
int tp_beam_set_stream(tp_engine *e, int beam, void *cuda_stream);

/* Statistics for TP_STATS_EXTERNAL plans: mu and sigma (host, nchan doubles
 * each) replace the measured bandpass from the next block on.  For 8-bit data
 * the bandpass value is the integer floor(mu + 1/2). */
int tp_beam_set_bandpass(tp_engine *e, int beam, const double *mu, const double *sigma, int nchan);

/* Append one block of `nsamp` (1..block_nsamp) new samples per channel.
 * `buf` is channel-major [nchan][nsamp] in the plan's dtype, in device memory
 * when buf_is_device, else in host memory (pinned for asynchrony).  The data
 * are copied on the beam's stream: a device buffer may be reused once that
 * stream reaches this point, a pageable host buffer when the call returns.
 * The first block of a stream must be longer than max_delay; it yields
 * nsamp - max_delay outputs, each later block nsamp outputs.
 * Errors: TP_EINVAL (size), TP_EBUSY (the previous block has not been through
 * tp_detect yet).  On a beam stream of its own the copies first wait for the
 * beam's previous detection (which may run on the engine stream). */
int tp_push_block(tp_engine *e, int beam, const void *buf, int nsamp, int buf_is_device);

/* Append a block that a device-side producer wrote into its own buffer, and
 * process it where it lies (no copy of the block).  `buf` is device memory of
 * the engine's device holding nchan rows of `pitch` elements in the plan's
 * dtype; the block's nsamp samples of channel c sit in columns
 * [max_delay, max_delay + nsamp) of row c (max_delay from tp_plan_info).  The
 * engine writes the overlap tail of the previous block (Sec. 2.2.2: the last
 * max_delay samples) into columns [0, max_delay) on the beam's stream, and
 * the statistics and staging kernels then read the window from the buffer.
 * The stream's first block (no overlap yet) is copied into the engine's
 * window instead.  Ownership: the caller keeps the buffer unchanged (apart
 * from the engine's tail) until the beam's next block has been pushed and the
 * beam's stream has passed that push -- the next push copies this block's
 * last max_delay samples out of it; consecutive blocks therefore alternate at
 * least two buffers.  Results equal those of tp_push_block with the same
 * samples.  Errors: TP_EINVAL (NULL, size, pitch < max_delay + nsamp, buf or
 * pitch bytes not a multiple of 16, not device memory of the engine's device,
 * buf holding the previous block), TP_EBUSY as tp_push_block. */
int tp_push_inplace(tp_engine *e, int beam, void *buf, int64_t pitch, int nsamp);

/* Double-buffered ingest (Sec. 2.1: the next GPU buffer is filled while the
 * current one is processed).  tp_prefetch_block starts the host -> device
 * copy of the next block's `nsamp` new samples per channel (`host_buf`,
 * channel-major [nchan][nsamp] in the plan's dtype, pinned host memory for
 * asynchrony) on a copy stream of the beam's own, straight into the window
 * the next block will use, so the copy overlaps the current block's kernels;
 * it may be called while the current block is still being processed.  The
 * caller keeps `host_buf` unchanged until tp_push_prefetched has returned
 * and the beam's stream has passed that point (tp_get_candidates of that
 * block, for instance).  tp_push_prefetched then publishes the block like
 * tp_push_block (its stream waits for the copy and moves the overlap tail);
 * the two calls together are equivalent to tp_push_block with `host_buf`.
 * Errors: tp_prefetch_block TP_EINVAL (size, NULL), TP_EBUSY (a prefetched
 * block is already waiting); tp_push_prefetched TP_ENOTREADY (nothing
 * prefetched), TP_EBUSY (the previous block has not been through
 * tp_detect).  While a prefetched block waits, tp_push_block returns
 * TP_EBUSY. */
int tp_prefetch_block(tp_engine *e, int beam, const void *host_buf, int nsamp);
int tp_push_prefetched(tp_engine *e, int beam);

/* Mark the beam's current window as not yet processed, so that tp_dedisperse
 * runs on it again (for instance after tp_plan_set_shape); the next push
 * still continues the stream from this window.  TP_ENOTREADY if the beam holds
 * no block. */
int tp_beam_rewind(tp_engine *e, int beam);

/* A1-A5 on the beam's current window (async).  beam = -1 processes every beam
 * holding a new block in one batched launch per stage.  TP_ENOTREADY if no
 * block is waiting. */
int tp_dedisperse(tp_engine *e, int beam);

/* A6-A7 on the beam's dedispersed series (async); beam = -1: every beam that
 * was dedispersed and not yet detected.  TP_ENOTREADY if not dedispersed. */
int tp_detect(tp_engine *e, int beam);

/* A1-A7 for every beam holding a new block, as one batch on the engine stream:
 * per-beam statistics / masks / substitution kernels, then ONE dedispersion
 * launch per (kernel shape, sample format) group covering all the group's
 * beams (uneven DM ranges and block lengths included), then per-beam
 * detection.  With use_graph = 1 the whole batch is recorded once into a CUDA
 * graph, cached per batch layout (beams, window parity, block length, kernel
 * shape) and replayed on later calls; this needs a non-default engine
 * stream.  *nbeams (may be NULL) receives the number of beams processed.
 * The batch runs on the engine stream, which first waits for the pushes of
 * beams that have their own stream (tp_beam_set_stream).  TP_ENOTREADY if no
 * beam holds a new block.  Results equal the per-beam tp_dedisperse /
 * tp_detect calls. */
int tp_run_ready(tp_engine *e, int use_graph, int *nbeams);

/* Wait for the beam's detection and copy min(cap, n_total) candidates, sorted
 * by (dm_idx, t_abs), to host memory `out`.  *n_total receives the number
 * found (which can exceed the beam's capacity; only the first
 * cand_capacity in (dm_idx, t) order are kept).  Returns TP_ETRUNC when
 * n_total > cap, TP_EOVERFLOW when n_total exceeded the beam capacity. */
int tp_get_candidates(tp_engine *e, int beam, tp_candidate *out, int cap, int *n_total);

/* The same result without a host wait (Sec. 2.3: the detections handed to the
 * event-detection stage, Table 1's device-to-host copy reduced to the
 * compacted list): enqueues on the beam's stream, after its detection, a
 * kernel that writes the number found to *n_total and the first
 * min(n_total, cand_capacity, cap) records, in the order of
 * tp_get_candidates, to `out`, and the beam's status word (0, TP_ETIMEOUT or
 * TP_EBOUNDS, as tp_get_candidates would report it) to *status (may be NULL),
 * clearing it.  `out`, `n_total` and `status` must be memory the device can
 * write -- page-locked host memory (cudaHostAlloc / cudaHostRegister) or
 * the engine device's memory -- aligned to 8, 8 and 4 bytes; they hold the results once
 * the stream has passed that point (an event, tp_sync), and the caller keeps
 * them until then.  The beam can take its next block at once: the copy runs
 * before the next block's kernels on the same stream.  Errors: TP_EINVAL
 * (pageable or misaligned buffers, cap < 0), TP_ENOTREADY (no detection
 * issued). */
int tp_export_candidates(tp_engine *e, int beam, tp_candidate *out, int cap, unsigned long long *n_total,
                         int *status);

/* ---- inspection (tests, debugging) -------------------------------------------- */

/* Window length, number of outputs, stream index of window sample 0 and the
 * number of W_c chunks of the beam's current block. */
int tp_beam_info(tp_engine *e, int beam, int64_t *nsamp_window, int64_t *nout, int64_t *t0_abs,
                 int *nchunk);

/* Dedispersed series D (ndm x nout, row-major, float32 for float plans, int32
 * for 8-bit plans) into `out` of `bytes` bytes (device memory when
 * out_is_device).  Blocks. */
int tp_get_series(tp_engine *e, int beam, void *out, size_t bytes, int out_is_device);

/* Bandpass statistics of the current block (host, nchan doubles each). */
int tp_get_bandpass(tp_engine *e, int beam, double *mu, double *sigma, int nchan);

/* Masks of the current block: chunk flags (nchan x nchunk bytes, after
 * dilation), the undilated exceedances (same shape), and spectrum flags (one
 * byte per window sample).  Any pointer may be NULL.  Blocks. */
int tp_get_masks(tp_engine *e, int beam, uint8_t *chunk_flag, uint8_t *chunk_raw, uint8_t *spec_flag);

/* Series statistics mu_d, sigma_d (host, ndm doubles each); with detrending
 * the line's mean and the residual deviation. */
int tp_get_series_stats(tp_engine *e, int beam, double *mu, double *sigma, int ndm);

/* The series the detection ran on (ndm x nout, row-major, float32 or int32):
 * the median-filtered series when the plan filters, else D.  Blocks;
 * TP_ENOTREADY before the beam's detection. */
int tp_get_processed_series(tp_engine *e, int beam, void *out, size_t bytes, int out_is_device);

/* Detrending line and residual deviation per series (host, ndm doubles each;
 * any pointer may be NULL): the line is mean + beta (2t - (T - 1)).  Blocks;
 * TP_EINVAL when the plan does not detrend, TP_ENOTREADY before detection. */
int tp_get_detrend(tp_engine *e, int beam, double *mean, double *beta, double *sigma, int ndm);

/* The fitted bandpass of the beam's current block: b_c (nchan doubles), the
 * channels masked before the fit (nchan bytes, 1 = masked) and the fit's RMSE
 * (any pointer may be NULL).  Blocks; TP_EINVAL when the plan does not fit. */
int tp_get_bandpass_fit(tp_engine *e, int beam, double *bfit, uint8_t *masked, double *rmse, int nchan);

/* The clusters of the beam's last detected block (host): min(cap, n) records
 * in cluster order; *n receives the number of clusters, *truncated (may be
 * NULL) 1 when more clusters than the beam keeps were found.  Blocks;
 * TP_EINVAL when the plan does not cluster, TP_ENOTREADY before detection. */
int tp_get_clusters(tp_engine *e, int beam, tp_cluster *out, int cap, int *n, int *truncated);

/* Cluster number of each of the first min(cap, stored) detections of the
 * last detected block (-1: noise), in the order of tp_get_candidates.
 * Blocks; *n receives the number of stored detections. */
int tp_get_candidate_labels(tp_engine *e, int beam, int32_t *labels, int cap, int *n);

/* ---- kernel shapes and autotuning -------------------------------------------------
 * The dedispersion kernel (Sec. 2.2.2) is compiled for several register
 * tilings ("shapes").  A shape fixes:
 *   - the DM trials per warp and the outputs per lane;
 *   - the largest in-window delay offset or step;
 *   - the consumer warps per CTA;
 *   - the consumer scheme: direct shared loads, register windows, or windows
 *     shared by two or four consecutive trials, the latter also with paired
 *     FP32 adds and with or without a producer warp.
 * A plan keeps the shapes its DM list fits.  It starts on the first of them in
 * an order of measured speed on a 1024-channel band. */

/* Number of shapes (return value); the plan's current shape; and, for
 * i < n, feasible[i] = 1 if shape i fits the plan's DM list. */
int tp_plan_shapes(const tp_plan *p, int *shape, int *feasible, int n);

/* Select a feasible shape for every beam of the plan (TP_EINVAL otherwise). */
int tp_plan_set_shape(tp_plan *p, int shape);

/* Time the dedispersion kernel of every feasible shape `reps` times on the
 * beam's current window, select the fastest for the beam's plan, and return
 * it in *best and the mean milliseconds per launch in ms[shape] (-1 for
 * infeasible shapes; n entries).  Blocks.  The beam's series is overwritten:
 * call tp_dedisperse again before tp_detect.  TP_ENOTREADY if the beam never
 * received a block.  Time it on a block of the stream's regular length: the
 * first block of a stream yields block_nsamp - max_delay outputs, and the
 * number of CTA waves (tiles / SMs, rounded up) can then rank the shapes
 * differently. */
int tp_autotune(tp_engine *e, int beam, int reps, int *best, float *ms, int n);

/* Autotuner cache: with a path set, tp_autotune looks up its choice under a
 * key of the device (name, compute capability, SM count), the plan (channels,
 * band, sampling time, sample format, DM list) and the block's output length;
 * a cached shape the plan admits is applied without timing runs (ms holds
 * only that shape's time; as after timing runs, the beam is to be dedispersed
 * again), otherwise the timing
 * runs as usual and the choice is added to the file (a text file, one
 * "key" shape ms entry per line, rewritten through a temporary file).  A
 * missing or unreadable file starts an empty cache; path = NULL turns the
 * cache off.  Errors: TP_EINVAL for a NULL engine. */
int tp_engine_set_tuning_cache(tp_engine *e, const char *path);

/* Batch form of tp_autotune for the batched launch of tp_run_ready: the beams
 * that have received a block are grouped by plan, and for every plan and every
 * shape it admits, `reps` launches of the dedispersion kernel over that plan's
 * beams at once (the layout and grid tp_run_ready uses) are timed; each plan
 * takes its own fastest shape (the batch then launches once per shape).
 * *best = the shape of the plan with the most work (trials x channels x
 * outputs); ms[shape] = the sum over plans of their launch times with that
 * shape where every plan admits it, else -1 (n entries).  A shape's speed on
 * one beam does not predict its speed in a batch (instruction-cache behaviour
 * differs with the number of CTAs in flight), hence a separate tuner.  Blocks;
 * the series are overwritten (run the batch again before detection).
 * TP_ENOTREADY if no beam has received a block. */
int tp_autotune_batch(tp_engine *e, int reps, int *best, float *ms, int n);

/* ---- tracing -------------------------------------------------------------------- */

/* Enable (1) or disable (0) per-stage CUDA-event timing on every beam of the
 * engine.  While enabled each block records events around its stages on the
 * beam's stream. */
int tp_set_profiling(tp_engine *e, int enable);

/* Accumulated stage times of a beam since profiling was enabled, in ms:
 * ms[0] push (window assembly copies), ms[1] A1-A3 (statistics and masks),
 * ms[2] A4-A5 (dedispersion), ms[3] A6-A7 (detection); *count = blocks timed.
 * Blocks until the beam's last timed stage has finished. */
int tp_get_stage_times(tp_engine *e, int beam, double *ms, int64_t *count);

/* Accumulated device time of the batched dedispersion launches (A4-A5 of
 * every beam of a tp_run_ready batch, all kernel-shape groups) issued outside
 * CUDA graphs since profiling was enabled, in ms, and how many batches that
 * covers.  Blocks until the last timed batch has finished.  Batches replayed
 * from graphs are not timed. */
int tp_get_batch_times(tp_engine *e, double *ms, int64_t *count);

/* Attempts (mbarrier try_wait calls) a dedispersion CTA makes while it waits
 * for staged data or for a free stage buffer before it gives up, records
 * TP_ETIMEOUT in the beam's status word (reported by tp_get_candidates) and
 * leaves; before leaving it always lets its own copies in flight land.
 * tries < 0 restores the default (2^24); 0 makes every such wait give up at
 * once, which tests use to exercise the timeout path without a fault or a
 * hang; values above 2^31 - 1 count as 2^31 - 1.  Applies to launches issued
 * after the call (cached batch graphs are dropped).  Errors: TP_EINVAL for a
 * NULL engine. */
int tp_engine_set_wait_limit(tp_engine *e, long long tries);

/* Grid of the batched dedispersion launch (tp_run_ready, tp_dedisperse with
 * beam = -1, tp_autotune_batch).  The kernel drains its work items (every
 * (DM tile, time tile) of every beam of a kernel-shape group) in a loop:
 * ctas = 0 (the default) launches a persistent grid of as many CTAs as are
 * resident on the device at once; ctas > 0 at most that many CTAs (tests use a
 * small grid so that every CTA takes many items); ctas < 0 one CTA per item.
 * Results do not depend on it.  Cached batch graphs are dropped. */
int tp_engine_set_batch_grid(tp_engine *e, int ctas);

/* ---- debugging aids (no compute-sanitizer: nothing here traps a GPU) ---------------
 * Canary padding: with tp_engine_set_canaries(e, 1), every beam opened
 * afterwards gets 256 bytes of the byte 0xA5 before each of its device buffers
 * and after each buffer's nominal size (up to the next 256-byte boundary plus
 * 256 bytes).  tp_engine_check_canaries synchronises the device and stores in
 * *nbad how many of those pads (over the engine's open beams) no longer hold
 * the pattern: a kernel wrote outside its buffer.  Padding costs 512 bytes
 * per buffer, which the footprint (tp_beam_footprint) does not count.
 * Errors: TP_EINVAL (NULL arguments), TP_ECUDA. */
int tp_engine_set_canaries(tp_engine *e, int enable);
int tp_engine_check_canaries(tp_engine *e, int *nbad);

/* 1 when this is the bounds-checking build of the library
 * (libtpdd_debug.so, compiled with TP_DEBUG_BOUNDS), else 0.  Its kernels
 * check the accesses whose indices come from the plan's geometry, the delays
 * or the data (the dedispersion kernel's bulk copies, delay copies, window
 * geometry and D stores; the spectrum/substitution kernel's window loads and
 * staged-series stores; the chunk statistics' window loads; the detection
 * kernels' D reads and candidate writes): a failed check skips the access and
 * records TP_EBOUNDS in the beam's status word, which the block's
 * tp_get_candidates returns.  Nothing traps. */
int tp_debug_bounds(void);

/* Bounds-checking build only: the dedispersion kernel of `beam` treats the
 * staged series as `bytes` long (bytes < 0: its real size), so that copies
 * beyond it fail their check (and are skipped) while every access stays
 * inside the real buffer.  Tests use it to see the checks fire.
 * Errors: TP_EINVAL (no such beam; not the bounds-checking build). */
int tp_debug_limit_staged(tp_engine *e, int beam, int64_t bytes);

/* Kernels launched by the engine since it was created. */
int tp_engine_launches(const tp_engine *e, uint64_t *n);

/* The engine's stream (as given to tp_engine_create) into *stream. */
int tp_engine_stream(const tp_engine *e, void **stream);

/* ---- serving loop ------------------------------------------------------------------
 * Many beam streams (any mix of channel counts, bands, DM lists, sample
 * formats and block lengths) share the engine with continuous batching; the
 * paper runs one processing thread per beam (Sec. 2.2) and drops work when
 * late (Sec. 3); here blocks are queued per stream and batched across
 * streams instead.  A stream's beam is opened when its first block has
 * arrived and its footprint fits the engine's HBM budget (otherwise the
 * stream waits for memory), and closed after its last block once the stream
 * is ended.  Every loop iteration pushes each stream's next arrived block as
 * soon as the stream's previous block is done -- on the stream's own CUDA
 * stream, so copies overlap the batches already running -- and launches one
 * batch (tp_run_ready) for all blocks pushed in that iteration. */
typedef struct tp_server tp_server;

typedef struct tp_stream_desc {
  int32_t nchan;
  int32_t ndm;
  double f_lo_mhz;
  double bw_mhz;
  double t_samp_s;
  const double *dm_list; /* host, ndm values (copied) */
  int32_t dtype;
  int32_t block_nsamp;   /* largest block of the stream */
  int32_t cand_capacity; /* candidate buffer per block */
  int32_t reserved;
} tp_stream_desc;

typedef struct tp_serve_result {
  int32_t stream;
  int32_t seq;          /* block index within its stream */
  double arrival_s;     /* server clock */
  double start_s;       /* block pushed to the GPU */
  double done_s;        /* candidates on the host */
  int64_t n_candidates;
  int32_t status;       /* TP_OK, TP_ETRUNC or TP_EOVERFLOW */
  int32_t reserved;
} tp_serve_result;

/* Create a server on engine `e`; rfi / nsigma apply to every stream (rfi NULL
 * = defaults).  keep_candidates = 1 keeps every block's candidate records on
 * the host for tp_server_candidates. */
int tp_server_create(tp_engine *e, const tp_rfi_params *rfi, double nsigma, int keep_candidates,
                     tp_server **out);

/* Register a stream (no device memory yet); plans are shared between streams
 * with identical band, sampling, DM list and format. */
int tp_server_add_stream(tp_server *s, const tp_stream_desc *d, int *stream_id);

/* Queue one block (host, channel-major [nchan][nsamp]) of a stream, arriving
 * at `arrival_s` on the server clock (seconds since the first tp_server_run).
 * The buffer is read when the block is pushed and must stay valid until the
 * block is done.  Returns the request id (>= 0) or an error. */
int tp_server_submit(tp_server *s, int stream_id, const void *host_block, int nsamp, double arrival_s);

/* No more blocks for this stream: its beam is closed after its last block. */
int tp_server_end_stream(tp_server *s, int stream_id);

/* Run the loop on the calling thread until every block submitted so far is
 * done (TP_OK) or the server clock passes time_limit_s (TP_ETIMEOUT). */
int tp_server_run(tp_server *s, double time_limit_s);

/* Per-request timings and candidate counts, in request order. */
int tp_server_results(tp_server *s, tp_serve_result *out, int cap, int *n);

/* Candidate records of a request (keep_candidates servers only). */
int tp_server_candidates(tp_server *s, int request, tp_candidate *out, int cap, int *n);

/* Wait for the engine, close every stream and free the server's plans. */
int tp_server_destroy(tp_server *s);

/* ---- the same statistics without any allocation ---------------------------------
 * tp_channel_stats_noalloc: A1-A2 (bandpass mean and standard deviation per
 * channel, channel-threshold exceedances and the dilated chunk flags) of one
 * channel-major block, for callers that cannot allocate device memory while
 * they run (pre-partitioned device memory under a real-time scheduler, work
 * recorded into a stream capture that must hold no allocation, runtimes that
 * forbid the CUDA allocator after start-up).  The paper has no counterpart to
 * this entry point: it is a deployment variant of the statistics step that
 * tp_dedisperse runs with beam-owned scratch.
 *
 * x          device, [nchan][pitch] samples of `dtype`, 16-byte aligned, pitch
 *            * element size a multiple of 16 bytes; nsamp samples per row used;
 *            1 <= nchan <= 65535 (else TP_EINVAL)
 * rfi        NULL for the defaults; stats_mode must be TP_STATS_BLOCK (enable_
 *            spectrum and tau_spectrum are ignored)
 * mu, sigma  device, nchan doubles each (outputs)
 * chunk_flag, chunk_raw  device, nchan x ceil(nsamp / W) bytes each (outputs)
 * cuda_stream  cudaStream_t (NULL = legacy default stream); the call is
 *            asynchronous on it
 *
 * Scratch: a 32 MiB array inside the library, held by every device that loads
 * the library until the process exits; TP_EINVAL when nchan * ceil(nsamp / W)
 * * 16 bytes (+ 34 bytes per channel, each of the seven per-channel arrays
 * rounded up to 256 bytes) does not fit.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress), keeps it for the rest of
 * the process and must therefore come before any stream capture on that
 * device; after cudaDeviceReset the kept address is stale, so a process that
 * resets a device must not call this entry point on it again.  No call allocates
 * or frees memory.  All calls share the array and it keeps the contents of the
 * last call: calls that can overlap on the GPU (different streams, or
 * different host threads) race on it and must be ordered by the caller.
 * Results equal those tp_dedisperse computes for the same window. */
int tp_channel_stats_noalloc(const void *x, int dtype, int nchan, int64_t nsamp, int64_t pitch,
                             const tp_rfi_params *rfi, double *mu, double *sigma, uint8_t *chunk_flag,
                             uint8_t *chunk_raw, void *cuda_stream);

/* Stream state of a beam for checkpoint and resume: tp_beam_export writes,
 * between blocks (after tp_detect of the last block, no prefetch pending),
 * everything the next block depends on -- the overlap tail of the window (the
 * last max_delay samples of every channel, in the sample format), the stream
 * position, and the running bandpass statistics when the plan keeps them --
 * to the host buffer `out` (cap bytes; out = NULL only sets *size to the
 * bytes needed).  tp_beam_import loads such a state into a beam that has not
 * received a block, opened on a plan with the same channels, DM list, sample
 * format and running-statistics weight (checked); the next tp_push_block
 * continues the stream, and its results equal those of the stream that was
 * never interrupted.  External statistics (tp_beam_set_bandpass) are not part
 * of the state.  Both block (synchronous copies).  Errors: TP_EINVAL (bad
 * buffer, plan mismatch, malformed state), TP_ENOTREADY (no block yet),
 * TP_EBUSY (export in the middle of a block, import into a used beam). */
int tp_beam_export(tp_engine *e, int beam, void *out, size_t cap, size_t *size);
int tp_beam_import(tp_engine *e, int beam, const void *in, size_t size);

/* Text of the calling thread's last error. */
const char *tp_last_error_string(void);

/* Library version (major * 10000 + minor * 100 + patch). */
int tp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TP_DEDISP_H */
