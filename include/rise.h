/*
 * rise.h -- C ABI of the GB300 RISE library: complex IQ captures in,
 * detected time-frequency boxes out.
 *
 * The calls follow the paper's statement of the problem (RISE, arXiv
 * 2603.20481, Sec. III-A-1): a capture of I/Q samples becomes a T x F
 * time-frequency plot by N_FFT-point FFTs over consecutive segments
 * (F = N_FFT), and every detected energy block is reported as a bounding box
 * B = (f0, f1, t0, t1) (Eq. 1).  The image pipeline between the two is the
 * one of Sec. IV-B: PSD-based column pruning around the noise floor N0,
 * per-column Otsu binarisation (Eq. 4), one 2D closing, one 2D opening and
 * one horizontal 1D opening with 3x3 / 1x3 all-ones elements (Eq. 5), and
 * 4-connected component labelling with min/max boxes.
 *
 * Conventions for every call:
 *  - Return value: RISE_OK (0) or a negative RISE_E* code; rise_strerror()
 *    names it.  Arguments are validated on the host before any launch; a
 *    rejected call changes nothing.
 *  - Pointers named *_dev are device pointers on the context's device; all
 *    other pointers are host pointers.  The caller owns every buffer it
 *    passes; the context owns its device scratch (grown on demand, up to
 *    rise_config.mem_budget) and frees it in rise_destroy().
 *  - Work is issued on the context's stream.  Every call that returns boxes
 *    is synchronous: on return the boxes are in host memory.
 *  - A context is used by one host thread at a time.
 *  - Image layout: row-major [T][F] uint8, row t = frame t (time), column f
 *    = frequency cell; column f holds FFT bin (f + F/2) mod F, so DC sits in
 *    column F/2 and column 0 is the most negative frequency.
 */
#ifndef RISE_H
#define RISE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define RISE_OK 0
#define RISE_EINVAL (-1)    /* bad argument (sizes, pointers, thresholds)      */
#define RISE_ENOMEM (-2)    /* device scratch would exceed mem_budget / OOM     */
#define RISE_ETRUNC (-3)    /* more boxes than `cap`; first `cap` returned      */
#define RISE_ECUDA (-4)     /* a CUDA runtime call failed                       */
#define RISE_ETIMEOUT (-5)  /* a bounded device-side wait gave up               */
#define RISE_EINTERNAL (-6) /* a kernel's own consistency check failed          */
#define RISE_ESCRATCH (-7)  /* size beyond the fixed scratch of an allocation-  *
                            * free entry point                                 */
#define RISE_EAGAIN (-8)    /* server queue full: poll results, then resubmit   */

/* ---- limits ------------------------------------------------------------ */
#define RISE_MIN_FFT 256
#define RISE_MAX_FFT 8192
#define RISE_MAX_ROWS 524288 /* T <= 2^19 keeps the exact Otsu compare in 128 bits */

/* ---- 8-bit range anchoring --------------------------------------------- */
#define RISE_RANGE_AUTO_MAX 0 /* top level = the capture's largest |X|^2      */
#define RISE_RANGE_FIXED 1    /* top level = hi_db (10 log10 |X|^2 units)     */

typedef struct rise_ctx rise_ctx;

/* Context configuration.  Zero fields take the defaults noted. */
typedef struct {
  int device;          /* CUDA device ordinal                                  */
  void *cuda_stream;   /* cudaStream_t for all work; NULL = a stream the ctx   *
                        * creates and owns                                     */
  int64_t max_samples; /* samples to pre-size scratch for (0: grow on demand)  */
  int max_fft;         /* largest FFT to pre-size for (0: grow on demand)      */
  int64_t max_boxes;   /* device box buffer to pre-size (0: grow on demand)    */
  size_t mem_budget;   /* cap on device scratch bytes (0: no cap)              */
} rise_config;

/* Detection parameters.  The paper leaves theta_PSD, theta_Power, the
 * Savitzky-Golay window and the 8-bit image unspecified (Sec. IV-B);
 * rise_thresholds_default() gives the library's reading:
 *   range_mode = RISE_RANGE_AUTO_MAX, level_db = 0.25 (256 levels span
 *   63.75 dB below the top), psd_offset_db = 0.5, power_offset_db = 10,
 *   sg_half_window = 5 (11-point quadratic), morph_order = 0.
 * Column f is kept when D*S_f >= N0 + round(psd_offset_db/level_db*D*T),
 * with S_f the column sum of levels, N0 the lowest local minimum of the
 * D-scaled Savitzky-Golay smoothing of S, D the smoother's integer norm.
 * A kept column's foreground is q > theta_Otsu and q >= P_q, where P_q =
 * ceil((N0 + round(power_offset_db/level_db*D*T)) / (D*T)).
 * -INFINITY for an offset switches that threshold off. */
typedef struct {
  int range_mode;         /* RISE_RANGE_AUTO_MAX | RISE_RANGE_FIXED            */
  double hi_db;           /* top of the 8-bit range for RISE_RANGE_FIXED       */
  double level_db;        /* dB per 8-bit level, 0.01 .. 10                    */
  double psd_offset_db;   /* theta_PSD above N0; -INFINITY: keep every column  */
  double power_offset_db; /* theta_Power above N0; -INFINITY: no power floor   */
  int sg_half_window;     /* Savitzky-Golay half window m, 1..16               */
  int morph_order;        /* 0: close3x3, open3x3, open1x3 (the paper's order) *
                           * 1: open1x3, close3x3, open3x3                     */
} rise_thresholds;

/* One detected energy block (Eq. 1 box plus per-block statistics).
 * t0..t1 are inclusive frame (row) indices, f0..f1 inclusive frequency
 * columns; anchor = t*F + f of the block's first pixel in raster order;
 * area = pixels; sum_q = sum of 8-bit levels; energy_fx = sum over pixels
 * of round(2^32 * 10^((q-255)*level_db/10)), i.e. linear power relative to
 * the top level in 2^-32 units.  Boxes are returned in ascending anchor. */
typedef struct {
  int32_t t0, t1, f0, f1;
  int64_t anchor;
  int64_t area;
  uint64_t sum_q;
  uint64_t energy_fx;
} rise_box;

/* Fills *thr with the defaults listed above. */
void rise_thresholds_default(rise_thresholds *thr);

/* Creates a context on cfg->device.  *out receives the handle.
 * Errors: RISE_EINVAL (NULL out/cfg, bad device), RISE_ECUDA. */
int rise_create(rise_ctx **out, const rise_config *cfg);

/* Frees the context and its device scratch (NULL is a no-op). */
void rise_destroy(rise_ctx *ctx);

/* Static description of a status code. */
const char *rise_strerror(int code);

/* Host-side layout helper for bindings: boxes[i] -> out[8 i .. 8 i + 7] =
 * t0, t1, f0, f1, anchor, area, sum_q, energy_fx as int64 (sum_q and
 * energy_fx stay below 2^63).  in and out are host memory; n >= 0. */
void rise_boxes_widen(const rise_box *in, int64_t n, int64_t *out);

/* Detects energy blocks in one capture (Sec. III-A-1 formulation).
 *  iq_dev    device pointer to n complex64 samples, interleaved (re, im),
 *            8-byte aligned.
 *  n         samples; T = (n - fft_size) / hop + 1 frames; need T >= 1 and
 *            T <= RISE_MAX_ROWS.
 *  fft_size  F = N_FFT, a power of two in [RISE_MIN_FFT, RISE_MAX_FFT].
 *  hop       samples between frame starts, 1..fft_size (hop = fft_size is
 *            the paper's non-overlapping segmentation).
 *  thr       NULL for the defaults.
 *  out       host array of `cap` boxes (may be NULL when cap = 0).
 *  n_boxes   receives the number of boxes found (always, also on ETRUNC).
 * Frame t is samples [t*hop, t*hop + F) times a periodic Hann window; its
 * |X|^2 row is quantised to 8-bit levels of level_db below the anchor
 * (round half up, clamped to 0..255).
 * Errors: RISE_EINVAL, RISE_ENOMEM, RISE_ETRUNC, RISE_ECUDA, RISE_EINTERNAL. */
int rise_detect(rise_ctx *ctx, const void *iq_dev, int64_t n, int fft_size, int hop,
                const rise_thresholds *thr, rise_box *out, int64_t cap, int64_t *n_boxes);

/* As rise_detect, but iq_host is a host pointer (pinned memory gives the
 * fastest copy): the call copies the capture into context-owned device
 * memory on the context's stream, then runs the same path. */
int rise_detect_host(rise_ctx *ctx, const void *iq_host, int64_t n, int fft_size, int hop,
                     const rise_thresholds *thr, rise_box *out, int64_t cap,
                     int64_t *n_boxes);

/* Asynchronous form of rise_detect / rise_detect_host: rise_submit queues
 * one capture's detection and returns; rise_collect waits for the oldest
 * queued call and returns its boxes exactly as the synchronous call would.
 * iq_flags: RISE_IQ_HOST when iq is host memory (else device memory), and
 * RISE_IQ_SC16 when the samples are 16-bit integer I/Q (interleaved int16
 * I, Q, 4-byte aligned; sample = (I + iQ) * 2^-15, exact in float, so the
 * results equal those of the same samples given as complex64) instead of
 * complex64.  At most two calls are queued (RISE_EAGAIN beyond).  Queued
 * calls run one after the other on the context's stream; a host capture is
 * copied into one of two device buffers on a second stream, so the copy
 * of the next capture overlaps the detection of the current one.  The
 * caller's samples must stay valid and unchanged until the call has been
 * collected.  `cap` at submit bounds the boxes the call keeps; rise_collect
 * returns at most min(its cap, that cap) of them (RISE_ETRUNC beyond, with
 * *n_boxes the full count).  While calls are queued, rise_detect,
 * rise_detect_host, rise_detect_image and rise_detect_batch return
 * RISE_EINVAL.  Errors: those of rise_detect; rise_collect with nothing
 * queued: RISE_EINVAL. */
#define RISE_IQ_HOST 1
#define RISE_IQ_SC16 2
int rise_submit(rise_ctx *ctx, const void *iq, int iq_flags, int64_t n, int fft_size, int hop,
                const rise_thresholds *thr, int64_t cap);
int rise_collect(rise_ctx *ctx, rise_box *out, int64_t cap, int64_t *n_boxes);

/* Runs the image part of the path (column histogram onwards, Sec. IV-B) on
 * a given 8-bit image: img_dev device pointer to T*F bytes, layout above,
 * F a power of two in [RISE_MIN_FFT, RISE_MAX_FFT], 1 <= T <= RISE_MAX_ROWS.
 * Same outputs and errors as rise_detect. */
int rise_detect_image(rise_ctx *ctx, const uint8_t *img_dev, int64_t T, int F,
                      const rise_thresholds *thr, rise_box *out, int64_t cap,
                      int64_t *n_boxes);

/* ---- batches ------------------------------------------------------------ */
/* One capture of a batch: iq_dev device pointer to n complex64 samples
 * (8-byte aligned; 16-byte aligned with an even hop lets the STFT stage the
 * frames with bulk copies), FFT size and hop as for rise_detect. */
typedef struct {
  const void *iq_dev;
  int64_t n;
  int fft_size;
  int hop;
} rise_capture;

#define RISE_BATCH_MAX_ROWS 524280 /* frames per capture in a batch (8 x 65535) */

/* Detects the energy blocks of ncap captures in one call, each exactly as
 * rise_detect would (the same thresholds for all; each capture keeps its own
 * 8-bit range anchor, noise floor, Otsu thresholds and components).  The
 * captures share the launches instead: one launch per stage for the whole
 * batch (one STFT launch per FFT size, a persistent grid that takes
 * frame ranges of any capture), so many small captures fill the GPU
 * together.  The first call with a given composition (the list of n,
 * fft_size, hop and alignment) times a few launch shapes and keeps the
 * fastest (RISE_OPT_AUTOTUNE), and records the chain as a CUDA graph that
 * later calls with the same composition replay (RISE_OPT_GRAPH).
 *  caps     ncap captures (host array); ncap >= 0.
 *  out      host array of `cap` boxes: the boxes of capture 0 in anchor
 *           order, then those of capture 1, and so on.
 *  offsets  host array of ncap + 1 entries: capture c's boxes are
 *           [offsets[c], offsets[c+1]) of the full list; offsets[ncap] is
 *           the total, also on RISE_ETRUNC (then `out` holds the first cap).
 * Per capture T = (n - fft_size) / hop + 1 must be in 1..RISE_BATCH_MAX_ROWS.
 * Errors: RISE_EINVAL, RISE_ENOMEM, RISE_ETRUNC, RISE_ECUDA, RISE_ETIMEOUT,
 * RISE_EINTERNAL.  rise_debug_export gives the batch's images, float power
 * and anchors (RISE_DBG_BATCH_*); the single-capture intermediates are not
 * kept for batches. */
int rise_detect_batch(rise_ctx *ctx, const rise_capture *caps, int ncap,
                      const rise_thresholds *thr, rise_box *out, int64_t cap, int64_t *offsets);

/* ---- block shapes ------------------------------------------------------------ */
/* The shapes of the last call's energy blocks (the labelling stage can also
 * give the blocks' boundaries, Sec. IV-B): every foreground run of the final
 * mask, in raster order of its first pixel, as runs[k] = {box index, row t,
 * first column, last column} (int32 x 4; the box index is the run's
 * component in the order boxes are returned), and, if `boundary` is not
 * NULL, the boundary mask: uint32 [T][F/32], bit f%32 of word f/32 set for a
 * foreground pixel with a background 4-neighbour (pixels outside the image
 * count as background).  For the last rise_detect, rise_detect_host,
 * rise_detect_image or collected call, with nothing queued (not after a
 * batch).  *n_runs receives the number of runs; at most cap are written
 * (RISE_ETRUNC beyond).  Errors: RISE_EINVAL, RISE_ETRUNC, RISE_ECUDA. */
int rise_contours(rise_ctx *ctx, int32_t *runs, int64_t cap, int64_t *n_runs, uint32_t *boundary);

/* ---- detection quality ---------------------------------------------------- */
/* Scores detections against ground truth as the paper does (Sec. III-A-2):
 * the IoU of two boxes is |B n B'| / |B u B'| over TF cells; ground-truth box
 * i is detected at threshold theta when its best IoU over the detections
 * exceeds theta, detection j is false when its best IoU over the ground
 * truth is below theta (Eq. 2; IoU equal to theta is neither), and
 * P_d = n_t / n_gt, P_fa = n_f / n_det (Eq. 3).  Runs on the GPU: the best
 * IoU of every box is computed exactly, as an (intersection, union) pair
 * compared by 128-bit cross products; a box with nothing on the other side
 * has (0, 1).  The decisions compare the intersection with theta * union in
 * double.
 *  gt       host int32 [n_gt][4] = t0, t1, f0, f1 (inclusive cell ranges)
 *  det      host rise_box [n_det] (only t0, t1, f0, f1 are read)
 *  thetas   host double [n_theta], each in [0, 1]; n_theta <= 65535
 *  n_t, n_f host int64 [n_theta] outputs
 *  gt_best, det_best  host int64 [n][2] (intersection, union) outputs, or NULL
 * Synchronous, on the context's stream.  Errors: RISE_EINVAL (bad sizes,
 * empty boxes, thresholds outside [0, 1], calls queued), RISE_ENOMEM,
 * RISE_ECUDA. */
int rise_match_boxes(rise_ctx *ctx, const int32_t *gt, int64_t n_gt, const rise_box *det,
                     int64_t n_det, const double *thetas, int n_theta, int64_t *n_t, int64_t *n_f,
                     int64_t *gt_best, int64_t *det_best);

/* ---- serving ------------------------------------------------------------ */
/* A server takes chunks of IQ from many radio streams as they arrive and
 * runs them through the path in batches (continuous batching): lane threads,
 * each with its own context and CUDA stream, take whatever chunks are
 * pending whenever a batch slot and memory are free, so batches overlap on
 * the GPU.  A chunk's result is the same whatever else shares its batch.
 *
 * Streams are continuous: each keeps on the device the samples its last
 * chunk left unused (fewer than fft_size), and its next chunk is processed
 * as those samples followed by the new ones, so every frame t*hop of the
 * stream is transformed exactly once across chunk boundaries.  A chunk
 * whose carried + new samples hold no full frame yields no frames and no
 * boxes and carries everything forward.
 *
 * Window mode (window_frames = W > 0) follows the real-time design of
 * Sec. IV-D: the stream's frames are cut into consecutive TF plots of W
 * frames (plot w = frames [w W, (w + 1) W), samples [w W hop, w W hop +
 * (W - 1) hop + fft_size)), and every plot is detected as soon as the chunk
 * that completes it arrives; chunks may have any length.  Results are one
 * per plot: seq = plot number, first_frame = w W, frames = W, tag and
 * t_submit_ns those of the completing chunk (its latency against the plot
 * deadline W hop / fs is t_done_ns - t_submit_ns); a chunk that completes
 * no plot gives no result.
 *
 * Memory admission: every chunk in flight holds a device slot of
 * (max_chunk + fft_size) samples; the slot pool and the lanes' scratch are
 * sized to fit mem_budget, and chunks wait in the queue until a slot frees.
 * Submitting to a full queue returns RISE_EAGAIN (the chunk is not taken). */
typedef struct rise_server rise_server;

typedef struct {
  int device;
  int fft_size;           /* N of every chunk's STFT                              */
  int hop;                /* 1..fft_size                                          */
  int64_t max_chunk;      /* largest chunk, samples                               */
  int max_streams;        /* stream ids 0 .. max_streams-1                        */
  int lanes;              /* batches in flight at once (0: 2)                     */
  int max_batch;          /* chunks per batch (0: 32)                             */
  int max_pending;        /* queued chunks before RISE_EAGAIN (0: 4096)           */
  size_t mem_budget;      /* device bytes for slots + lane scratch (0: no cap)    */
  const rise_thresholds *thr; /* NULL: defaults; copied at create                 */
  int64_t window_frames;  /* 0: detect each chunk (its complete frames); W > 0:   *
                           * window mode, detect TF plots of W frames             */
  int keep_images;        /* 1: keep every result's 8-bit image on the host for   *
                           * rise_server_result_image (introspection: costs a     *
                           * device-to-host copy per batch and T*F host bytes per *
                           * result until taken); 0: off                          */
  int spin_wait;          /* 1: lanes spin while their batch runs; 0 (default):   *
                           * they sleep (RISE_OPT_BLOCKING_WAIT), leaving host    *
                           * cores to the caller and the other lanes              */
} rise_server_config;

typedef struct {
  int stream;             /* radio stream id                                      */
  int status;             /* RISE_OK or the error of the chunk's batch            */
  uint64_t tag;           /* as given to rise_stream_submit                       */
  int64_t seq;            /* chunk number within its stream, from 0               */
  int64_t first_frame;    /* stream frame index of the chunk's first frame        */
  int64_t frames;         /* frames the chunk completed                           */
  int64_t box_offset;     /* its boxes: arena[box_offset, box_offset + n_boxes)   */
  int64_t n_boxes;        /* box t0/t1 count frames from first_frame              */
  int64_t t_submit_ns;    /* steady-clock times: submitted, batch started, done   */
  int64_t t_start_ns;
  int64_t t_done_ns;
} rise_result;

/* Creates a server and starts its lane threads.  Errors: RISE_EINVAL,
 * RISE_ENOMEM (mem_budget below one slot and one chunk of scratch per lane),
 * RISE_ECUDA. */
int rise_server_create(rise_server **out, const rise_server_config *cfg);

/* Queues n samples (complex64, host memory; pinned memory copies fastest)
 * for stream `stream`.  The buffer must stay valid and unchanged until the
 * chunk's result has been returned by rise_server_poll (window mode, where a
 * chunk may complete no plot: until rise_server_drain has returned).  Chunks of one
 * stream are processed in submission order.  Errors: RISE_EINVAL (bad
 * stream, n < 1 or n > max_chunk), RISE_EAGAIN (queue full). */
int rise_stream_submit(rise_server *s, int stream, const void *iq_host, int64_t n, uint64_t tag);

/* Returns finished chunks, oldest first: up to max_res results into res,
 * their boxes packed into arena (arena_cap boxes; a result whose boxes do
 * not fit stays queued, and a lone result larger than the arena comes back
 * with status RISE_ETRUNC and its first arena_cap boxes).  Waits up to
 * timeout_ms (0: no wait, < 0: until one result is ready) for the first.
 * *n_res receives the count.  Errors: RISE_EINVAL. */
int rise_server_poll(rise_server *s, rise_result *res, int max_res, rise_box *arena,
                     int64_t arena_cap, int *n_res, int timeout_ms);

/* Waits until no chunk is queued or in flight (timeout_ms < 0: no limit).
 * Errors: RISE_ETIMEOUT. */
int rise_server_drain(rise_server *s, int timeout_ms);

/* Copies stream `stream`'s state (its carried samples and counters) to buf,
 * or, with buf NULL, only reports the size in *need; the stream must have
 * nothing queued or in flight.  Import restores such a state into a stream
 * of a server with the same fft_size and hop.  Errors: RISE_EINVAL
 * (busy stream, small buffer, mismatched server). */
int rise_stream_export(rise_server *s, int stream, void *buf, size_t bytes, size_t *need);
int rise_stream_import(rise_server *s, int stream, const void *buf, size_t bytes);

/* Counters: [0] submitted, [1] rejected (RISE_EAGAIN), [2] completed,
 * [3] batches, [4] largest batch, [5] most chunks in flight, [6] slots,
 * [7] lanes, [8] launch chains captured as graphs (all lanes), [9] scratch
 * buffer generations (all lanes; each one drops the lane's graphs),
 * [10] longest batch in microseconds, [11] batches run again with grown
 * run arrays.  Writes min(n, 12) values. */
int rise_server_stats(rise_server *s, int64_t *out, int n);

/* With keep_images set: moves the 8-bit image the result (stream, seq) was
 * detected on (chunk mode: the chunk's frames, carried samples included;
 * window mode: plot seq) into dst, [T][F] with F = fft_size, and drops it
 * from the server.  *T receives its rows; dst may be NULL to ask for T
 * only (the image is then kept).  Valid once the result is ready (polled or
 * not).  Errors: RISE_EINVAL (no such image kept, bytes < T * F). */
int rise_server_result_image(rise_server *s, int stream, int64_t seq, uint8_t *dst, size_t bytes,
                             int64_t *T);

/* Stops the lanes after the chunks in flight and frees everything; queued
 * chunks that never started are dropped. */
void rise_server_destroy(rise_server *s);

/* ---- introspection of the last detect call ----------------------------- */
#define RISE_DBG_POWER_F32 1 /* float [T][F] |X|^2 (needs RISE_OPT_KEEP_POWER)     */
#define RISE_DBG_IMAGE_U8 2  /* uint8 [T][F] levels                                 */
#define RISE_DBG_HIST 3      /* uint32 [F][256] column histograms                   */
#define RISE_DBG_COLSTATS 4  /* rise_colstat [F]                                    */
#define RISE_DBG_FLOOR 5     /* int64 [8]: N0, delta_psd, delta_pow, P_q, D, T, F, 0 */
#define RISE_DBG_MASK0 6     /* uint32 [T][F/32] thresholded mask, bit f%32 of word */
#define RISE_DBG_MASK1 7     /* ... after the first morphological operation pair    */
#define RISE_DBG_MASK2 8     /* ... after the second pair                           */
#define RISE_DBG_MASK3 9     /* ... final mask (always kept)                        */
#define RISE_DBG_MAXPOW 10   /* float [1]: the anchor power (largest |X|^2)          */
#define RISE_DBG_LEVEL_EDGES 11 /* float [257]: smallest power of each level          */
#define RISE_DBG_LAUNCHES 12 /* int64 [1]: kernels launched by this library so far,   *
                              * process-wide (for launch accounting)                */
#define RISE_DBG_GRAPHS 14   /* int64 [4]: [0] the last rise_detect replayed a     *
                              * graph, [1] single-capture graphs kept, [2] batch  *
                              * graphs kept, [3] 0                                */
#define RISE_DBG_CCL 15      /* int64 [4] of the last call's labelling: runs,      *
                              * deferred unions, components, run capacity         */
#define RISE_DBG_BATCH_INFO 13 /* int64 [64] of the last batch: [0] STFT groups G,   *
                                * [1] replayed from a graph (0/1), [2..2+G) frames  *
                                * per STFT item in steps, [2+G] morphology warps    *
                                * per SM, [3+G..3+2G) radix schedule per group,     *
                                * [3+2G..3+3G) FFT size per group, [63] tuned       *
                                * compositions read from the tune cache so far      */
/* Intermediates of the last rise_detect_batch call, kept until the next call
 * of the context (or a buffer growth) overwrites them.  Captures follow one
 * another in call order, capture c taking T_c * F_c entries ([T_c][F_c],
 * row-major, layout above), with no gaps. */
#define RISE_DBG_BATCH_IMAGES 16  /* uint8: every capture's 8-bit image           */
#define RISE_DBG_BATCH_POWER 17   /* float: every capture's |X|^2 (AUTO range only) */
#define RISE_DBG_BATCH_ANCHORS 18 /* float [ncap]: each capture's anchor power     *
                                   * (its largest |X|^2; FIXED: 10^(hi_db/10))     */

typedef struct {
  uint64_t S;    /* column sum of levels                                */
  int64_t Shat;  /* D-scaled Savitzky-Golay smoothing (0 off the interior) */
  int32_t keep;  /* 1: column survives theta_PSD                        */
  int32_t otsu;  /* Otsu threshold, -1 when no split exists             */
  int32_t eff;   /* smallest foreground level, 256 = none               */
  int32_t pad;
} rise_colstat;

/* Copies the named intermediate of the last call into host memory dst
 * (bytes must be at least its size).  Errors: RISE_EINVAL (unknown `what`,
 * too small, nothing kept), RISE_ECUDA. */
int rise_debug_export(rise_ctx *ctx, int what, void *dst, size_t bytes);

/* ---- options -------------------------------------------------------------- */
#define RISE_OPT_KEEP_POWER 1  /* 1: keep the float |X|^2 image of the next calls  */
#define RISE_OPT_KEEP_MASKS 2  /* 1: keep MASK0..MASK2 of the next calls           */
#define RISE_OPT_TIMING 3      /* 1: record per-stage device times                 */
#define RISE_OPT_RANGE_PATH 4  /* 0: auto (2 when the float power image fits     *
                                * mem_budget, else 1); 1: FFT twice (max, then    *
                                * quantise); 2: FFT once, keep float power,       *
                                * quantise after                                  */

#define RISE_OPT_GRAPH 5       /* 1 (default): a call repeating the previous     *
                                * call's arguments (a batch: its composition)     *
                                * replays the launches captured as a CUDA graph   */
#define RISE_OPT_AUTOTUNE 6    /* 1 (default): tune batch launch shapes and radix  *
                                * schedules once per composition (or read them    *
                                * from the tune cache); 0: fixed defaults          */
#define RISE_OPT_RUN_CAPACITY 7 /* runs the labelling arrays hold at the next call *
                                 * (>= 1024; they still grow when a mask needs    *
                                 * more)                                          */
/* Bounds of the labelling stage's device waits.  Every wait gives up after
 * its bound, records the fact in the call's status and lets the kernel
 * return, so the call ends with RISE_ETIMEOUT and the context stays usable.
 * 0 restores the default.  Changing one drops the context's captured graphs. */
#define RISE_OPT_SCAN_WAIT_LIMIT 8 /* polls (32 ns apart) a single-pass scan tile   *
                                    * waits for a predecessor's sum (2^20)          */
#define RISE_OPT_UNION_LIMIT 9     /* steps of one union-find walk (2^26)           */
#define RISE_OPT_TEST_WITHHOLD 10  /* test only: the box-slot scan's tile with this *
                                    * index publishes no sum, so every later tile's *
                                    * wait runs out; -1 (default): none             */
/* The STFT stages each frame group into shared memory with a bulk copy and
 * waits for it on a shared-memory barrier.  That wait gives up after
 * RISE_OPT_COPY_WAIT_LIMIT polls (each suspends the thread for a
 * hardware-defined interval; 0 restores the default 2^22).  Values below
 * 2^12 are rejected: 2^12 polls already last far longer than an issued
 * copy takes to land, and a shorter bound could give up on one on its way.
 * The block then waits, with the same bound, for any copy it still has in
 * flight, records the fact and leaves, and the call returns RISE_ETIMEOUT.
 * Both options act on the float-power STFT (range path 2, the default, and
 * batches without a fixed range), which runs a separate kernel instance
 * while either is away from its default; the other STFT kernels always wait
 * 2^22 polls.  Changing either option drops the context's captured graphs. */
#define RISE_OPT_COPY_WAIT_LIMIT 12
/* How rise_detect_batch waits for its launches: 0 (default) lets the CUDA
 * runtime decide (it spins while the process has few contexts), 1 sleeps on
 * a blocking-sync event, which frees the calling thread's core at the cost of
 * a wake-up delay.  Server lanes use it unless their server was made with
 * spin_wait set. */
#define RISE_OPT_BLOCKING_WAIT 14
#define RISE_OPT_TEST_WITHHOLD_COPY 13  /* test only: block 0 of every STFT launch   *
                                         * issues no copy for its frame group with   *
                                         * this index, so its wait runs out; -1      *
                                         * (default): none                           */
/* Radix schedule of the FFT of single captures.  An N-point transform with
 * N = 16^a * r (r = 2, 4 or 8) runs its radix-r pass last (schedule 0) or
 * first (schedule 1); for r = 2 (N = 512, 8192) schedule 2 splits the
 * frame into two N/2-point transforms run side by side (at N = 8192 by the
 * two halves of the block, which never wait for each other inside the
 * frame loop).  A schedule a size does not have runs schedule 0 (N a power
 * of 16: all are the same).  3 (the default): the library's schedule for
 * N, 2 at N = 8192 and 1 at the other sizes.  -1: the schedule this
 * context's batch tuner (or the tune cache) picked for N, else the
 * library's.  The schedules round differently, so the 8-bit image can
 * differ in a few pixels (all stay within the tolerance of the FP64
 * reference).  The batch tuner times every schedule an FFT size of a new
 * composition has and keeps the fastest; an untuned batch runs the
 * library's schedule.  A batch capture's results equal those of
 * rise_detect run with the batch's schedule. */
#define RISE_OPT_FFT_SCHEDULE 11

/* Tune cache: when the environment variable RISE_TUNE_CACHE names a file,
 * every composition the batch tuner tunes is appended to it as one text
 * line ("rise-tune 1 <device name:SMs> <composition key> <G> <G frames-per-
 * item multipliers> <G radix schedules> <morphology warps per SM>"), and a
 * composition found there for the same device is run without tuning (also
 * in another process). */

/* Sets an option; errors: RISE_EINVAL. */
int rise_set_option(rise_ctx *ctx, int option, int64_t value);

/* Per-stage device milliseconds of the last call with RISE_OPT_TIMING on,
 * from CUDA events recorded on the context's stream:
 * [0] first spectrum pass (anchor max, or float power when kept),
 * [1] level edges + second pass (8-bit image, or quantise + histogram),
 * [2] column histogram, [3] column statistics, [4] threshold + morphology,
 * [5] labelling and box reduction, [6] status and box readback, [7] total.
 * Writes min(nstages, 8) values.  Errors: RISE_EINVAL. */
int rise_stage_times(rise_ctx *ctx, float *ms, int nstages);

/* ---- allocation-free column statistics ----------------------------------- */
/* The paper has no counterpart of this call.  It is for callers that may not
 * allocate device memory: a host framework that owns all device memory and
 * forbids allocation inside its per-frame callbacks, or a real-time loop in
 * which a cudaMalloc / cudaFree (which can synchronise the whole device)
 * would stall the other streams.  It needs no context and allocates nothing;
 * its column histograms live in one fixed device array of
 * RISE_NOALLOC_MAX_COLS x 256 counters (4 MiB), which every GPU that loads
 * the library holds until the process exits.
 *
 * For the 8-bit image img_dev ([T][F] uint8 on the current device, layout
 * above, 2-byte aligned) it writes, per column f, cols_dev[f].S = sum of the
 * column's levels and cols_dev[f].otsu = the exact Otsu threshold, the same
 * value rise_detect_image reports (-1 when no split exists); Shat, keep, eff
 * and pad are set to 0.  cols_dev: device rise_colstat[F],
 * 8-byte aligned.  F a power of two in [RISE_MIN_FFT, RISE_NOALLOC_MAX_COLS],
 * 1 <= T <= RISE_MAX_ROWS.
 *
 * The work is queued on cuda_stream (NULL: the legacy default stream) of the
 * current device and the call returns without waiting; the results are
 * valid once the stream reaches them.  The first call on a device looks up
 * the array's device address (a one-time set-up per device); make that first
 * call before any stream capture.  Later calls made outside a stream capture
 * look the address up again, so a device reset between calls is safe; calls
 * made while their stream is capturing use the address of the last call.
 * Every call, on any stream or thread, shares the one array per device and
 * clears the part it uses before counting: calls whose work overlaps on the
 * GPU race and give wrong results, so order them (one stream, or events).
 * Errors: RISE_EINVAL (NULL or misaligned pointers, pointers not in the
 * current device's memory, bad T or F) and RISE_ESCRATCH
 * (F > RISE_NOALLOC_MAX_COLS) queue nothing; RISE_ECUDA (a CUDA call or
 * launch failed) may come after part of the work was queued, so cols_dev
 * may already have been cleared on the stream. */
#define RISE_NOALLOC_MAX_COLS 4096
int rise_column_stats_noalloc(const uint8_t *img_dev, int64_t T, int F, rise_colstat *cols_dev,
                              void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* RISE_H */
