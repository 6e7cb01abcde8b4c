/*
 * lpf.h -- C ABI of the B300 image-plane dispersed-transient search.
 *
 * Method: Ruhe et al., "Detecting Dispersed Radio Transients in Real Time Using
 * Convolutional Neural Networks" (arXiv 2103.15418).  The library runs, per new
 * frame of F subband images, the brute-force image-plane dedispersion search:
 *
 *   delay table   delay[d][f] = floor(C_DM * DM_d * (nu_f^-2 - nu_ref^-2) / cadence + 1/2)
 *                 with C_DM = 4.148808e3 s MHz^2 cm^3/pc and nu_ref = max_f nu_f
 *                 (Sec. 3.2, dispersion-delay equation);
 *   shift-sum     D_d = sum_f X_f(t0 + delay[d][f]), t0 = T - max_f delay[d][f]
 *                 (App. B.2, "perfect dedispersion" before averaging);
 *   local centre  C = box mean of D over the (2r+1)^2 window clipped to the image
 *                 (Sec. 2.1.1, C := G * X with the uniform kernel, normalised);
 *   local spread  S = box mean of (D - C)^2, the square taken per pixel first
 *                 (Sec. 2.1.1, S := G * (X - C)^2);
 *   detection     snr = (D - C)/sqrt(S); candidate iff snr > kappa, S > 0 and D is
 *                 the maximum of its 3x3 window clipped to the image, ties included
 *                 (Sec. 2.1.1 threshold y, Sec. 2.1.2 max filter q and p = q AND y);
 *   statistics    per DM trial, mean and RMS of snr over pixels with S > 0;
 *   dynspec       per candidate, the F x Tw fluxes of the Tw most recent frames at its
 *                 pixel, optionally the box maximum (Sec. 2.2 flux measurement and
 *                 backward fill), the input of the paper's CNN (Sec. 2.3).
 *
 * All compute runs in CUDA kernels for sm_103a; there is no CPU fallback.  A call
 * that needs the GPU fails with LPF_E_CUDA when no usable device is present.
 *
 * Threading: one host thread per stream handle at a time.  Handles are
 * independent; different handles may be driven from different threads.
 * Errors: every call returns LPF_OK (0) or a negative LPF_E_* code; nothing
 * aborts or throws across the ABI.  lpf_strerror() names a code.
 */
#ifndef LPF_H
#define LPF_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
#define LPF_OK            0
#define LPF_E_ARG        -1   /* invalid argument (null pointer, size out of range, ...) */
#define LPF_E_DEPTH      -2   /* buffer_depth < max delay + 1, or Tw > buffer_depth     */
#define LPF_E_ORDER      -3   /* pushed frame index is not the previous one + 1          */
#define LPF_E_OOM        -4   /* device or pinned-host allocation failed                 */
#define LPF_E_BUDGET     -5   /* server: stream does not fit the HBM budget at all       */
#define LPF_E_TRUNCATED  -6   /* more candidates than the output (or cand_cap) can hold  */
#define LPF_E_STALE      -7   /* frames needed by extract_dynspec left the ring buffer   */
#define LPF_E_TIMEOUT    -8   /* poll: the frame's work did not finish within timeout_ms */
#define LPF_E_CUDA       -9   /* a CUDA runtime call failed (no device, launch failure)  */
#define LPF_E_BUSY      -10   /* all result slots hold unpolled frames; poll first       */
#define LPF_E_NODATA    -11   /* poll with no pushed-and-unpolled frame                  */
#define LPF_E_CAPACITY  -12   /* request larger than a fixed-capacity staging area       */

/* what a stream computes per pushed frame */
#define LPF_MODE_DISPERSED 0   /* the dispersed-transient search over the DM trials (Sec. 2.1, App. B.2) */
#define LPF_MODE_SUBBAND   1   /* the per-subband detector: every band image of the frame (Sec. 2.1.1-2.1.2) */

/* background kernel G of the centre / spread filter (Sec. 2.1.1) */
#define LPF_KERNEL_BOX     0   /* uniform square box of radius box_r                          */
#define LPF_KERNEL_GAUSS   1   /* G(n, m, s) = exp(-(n^2 + m^2) / (2 s^2)) / Z on the (2 box_r + 1)^2
                                  window; per-subband detector only                          */

/* storage type of the ring buffer (arithmetic is always FP32) */
#define LPF_FP32 0
#define LPF_FP16 1
#define LPF_BF16 2

typedef struct lpf_stream lpf_stream;   /* opaque; owns ring buffer, tables, scratch */

typedef struct {
    double cadence_s;     /* frame cadence in seconds (> 0)                     default 1.0   */
    float  kappa;         /* S/N threshold (strict >)                            default 6.0   */
    int    box_r;         /* background box radius r, window (2r+1)^2, 1..16      default 15    */
    int    lmax_r;        /* local-maximum radius: 1 (3x3) for the dispersed search;
                             1..3 for the per-subband detector (3: the paper's 7x7)  default 1 */
    int    dtype;         /* LPF_FP32 / LPF_FP16 / LPF_BF16 ring storage          default FP32  */
    int    cand_cap;      /* device candidate capacity per frame (records)       default 1<<20 */
    int    dyn_box_r;     /* dynspec box radius (0 = the candidate pixel)         default 0     */
    int    result_slots;  /* frames that may be pushed but not yet polled, 1..16  default 2     */
    void*  cuda_stream;   /* cudaStream_t to run on; NULL = a private non-blocking stream    */
    int    filter_impl;   /* 0 = auto (streaming kernel when box_r is 7 or 15, else tiled),
                             1 = tiled kernel, 2 = streaming kernel (box_r 7 or 15 only)      */
    /* Quality control of every pushed frame before it enters the ring (App. A):
     * band image f is imputed with zeros when |z_f| > qc_z, z_f = (b_f - median(b))
     * / MAD(b) over the band-image means b (MAD: median absolute deviation), or
     * when some pixel has |x - mean| > qc_zeta * s under the running per-pixel
     * mean and sample deviation s of the kept band images (Welford; tested once
     * qc_min_frames frames of the band have been kept, where s > 0).             */
    int    qc;            /* 0 = off, 1 = on                                       default 0     */
    float  qc_z;          /* band-score threshold (> 0)                            default 5.0   */
    float  qc_zeta;       /* pixel-score threshold (> 0)                           default 20.0  */
    int    qc_min_frames; /* kept frames before the pixel test applies (>= 2)      default 128   */
    /* LPF_MODE_SUBBAND: each push detects sources in every band image X_f of the
     * frame itself (the one-pass centre/spread filter with box_r 7 or 15, the
     * threshold, the (2 lmax_r + 1)^2 maximum filter on X_f).  n_dm and dm_grid of
     * lpf_stream_open are then ignored (0 and NULL allowed); a candidate's dm_idx
     * is its band f and t0 its frame T; lpf_get_stats has one row per band.     */
    int    mode;          /* LPF_MODE_DISPERSED / LPF_MODE_SUBBAND                 default DISPERSED */
    /* Iterated sigma clipping (Sec. 2.1.1).  Each iteration re-estimates C and S
     * from the window pixels not yet flagged and adds the pixels over the
     * threshold to the flags, until an iteration flags nothing new or clip_iters
     * iterations; candidates are the flagged (2 lmax_r + 1)^2 maxima, with the
     * S/N of the last iteration.  Per-subband detector: of the band images X_f.
     * Dispersed search: of the dedispersed image D_d of every trial, on the
     * direct-form path (D summed from the raw ring per distinct delay row, then
     * the clipping passes over all rows; filter_impl 2 is refused).  1 = one
     * pass.                                                                     */
    int    clip_iters;    /* 1..16                                                 default 1 */
    /* Per-subband detector only: the Gaussian kernel of Sec. 2.1.1 instead of the
     * uniform box, truncated to the (2 box_r + 1)^2 window (box_r 1..16) and
     * normalised per pixel by its weight over the in-image (and, when clipping,
     * unflagged) window pixels.  C, S and the S/N are direct weighted FP32 window
     * sums (rows, then columns) of the stored band image.                        */
    int    kernel;        /* LPF_KERNEL_BOX / LPF_KERNEL_GAUSS                      default BOX */
    float  gauss_sigma;   /* s in pixels (> 0, finite) for LPF_KERNEL_GAUSS          default 0   */
    /* Dispersed search only, opt-in: steady-source suppression.  The paper leaves
     * steady sources to the stages after the search (association with the
     * previous catalogue, Sec. 2.2; the network's DM estimate, Sec. 2.3).  With
     * K = suppress_steady > 0 a pixel is steady once it has been a candidate of a
     * trial whose delay row is all zero (no dispersion, t0 = T) in each of the K
     * most recent pushes, and the candidates of every other trial at a steady
     * pixel are dropped (the zero-delay trials keep theirs).  Persistence, not
     * one frame: the last subband of a bright dispersed pulse can cross the
     * threshold at zero delay in the frame it arrives, but not in K frames in a
     * row for K above the pulse width.  The state (one byte per pixel) is updated
     * by every push in order, from every zero-delay candidate the push finds
     * (stored in the list or not), so it does not depend on cand_cap.  n_out of
     * lpf_poll_candidates counts the kept candidates.  When the list overflowed
     * (cand_cap records stored) the drop is applied to the stored records only,
     * the total is not known, and n_out is the number of kept records among the
     * stored ones (the poll returns LPF_E_TRUNCATED).  0 = off.               */
    int    suppress_steady; /* 0..255                                             default 0   */
} lpf_params;

/* One candidate: pixel (y, x) of DM trial dm_idx (index into dm_grid) whose
 * dispersed sweep arrives at nu_ref in frame t0 (so it is completed by frame
 * t0 + max_f delay[dm_idx][f]), with its S/N.  24 bytes, no padding. */
typedef struct {
    int64_t t0;
    int32_t dm_idx;
    int32_t y;
    int32_t x;
    float   snr;
} lpf_candidate;

typedef struct {
    int     H, W, F, n_dm, depth, dtype;
    int     n_distinct;       /* DM trials with distinct delay rows (computed once each) */
    int     max_delay;        /* max over trials of max_f delay[d][f], frames           */
    size_t  ring_bytes;       /* device bytes of the ring buffer                         */
    size_t  device_bytes;     /* all device bytes owned by the stream                    */
    int64_t frames_pushed;
    int64_t last_T;
} lpf_stream_info_t;

/* Fill *p with the defaults listed above. */
void lpf_default_params(lpf_params* p);

/*
 * Open a stream: H x W images, F subbands with centre frequencies freqs_mhz[F]
 * (MHz, > 0, host), n_dm trial DMs dm_grid[n_dm] (pc cm^-3, >= 0, host), ring
 * of buffer_depth frames.  params may be NULL (defaults).  The library copies
 * every input; the caller keeps nothing alive.  Builds the delay table in FP64
 * on the host (Sec. 3.2) and allocates the ring buffer and scratch on the
 * current CUDA device.
 * F is at most 32, H and W at most 65536, buffer_depth at most 32767.
 * Errors: LPF_E_ARG (sizes <= 0 or above those limits, box_r outside 1..16, lmax_r outside its range
 * for the mode, bad dtype, non-positive frequency or cadence, negative DM, filter_impl 2 with another
 * box_r; an unknown mode or kernel; the Gaussian kernel outside the per-subband detector or with
 * gauss_sigma not positive and finite; the per-subband detector with the box and box_r other than 7 or
 * 15, or with filter_impl 1; clip_iters outside 1..16, or above 1 in the dispersed search with filter_impl 2;
 * quality-control thresholds not positive or qc_min_frames < 2), LPF_E_DEPTH (buffer_depth < max delay
 * + 1), LPF_E_OOM, LPF_E_CUDA (no device).
 */
int lpf_stream_open(lpf_stream** out, int H, int W, int F, const double* freqs_mhz,
                    int n_dm, const double* dm_grid, int buffer_depth, const lpf_params* params);

/*
 * Device bytes lpf_stream_open would request for these arguments, computed on
 * the host without any CUDA call (the same validation and errors as open).
 * The allocator may round each of the stream's ~20 allocations up.
 */
int lpf_stream_footprint(int H, int W, int F, const double* freqs_mhz, int n_dm,
                         const double* dm_grid, int buffer_depth, const lpf_params* params,
                         size_t* bytes);

/*
 * Push frame T: frame_dev is a DEVICE pointer to F*H*W FP32 values laid out
 * [F][H][W] (row-major, subband-major), on the stream's device.  The work is
 * enqueued on the stream's CUDA stream and the call returns at once; the
 * caller keeps frame_dev unchanged until the stream has consumed it (after
 * lpf_poll_candidates returns for T, or lpf_stream_sync).  The first push may
 * use any T >= 0; later pushes must use the previous T + 1.  Push T produces
 * the candidates of every DM trial d with T - max_f delay[d][f] >= first T.
 * Errors: LPF_E_ARG, LPF_E_ORDER, LPF_E_BUSY (result_slots frames unpolled), LPF_E_CUDA.
 */
int lpf_push_frame(lpf_stream* s, const float* frame_dev, int64_t T);

/* Same as lpf_push_frame with a HOST frame (pinned or pageable).  The frame is
 * copied into one of two device staging buffers on a separate upload stream,
 * so the upload of frame T overlaps the search of frame T-1; the search of T
 * starts when its upload is done.  The host buffer may be reused when the call
 * returns if it is pageable, once lpf_poll_candidates has returned T (or after
 * lpf_stream_sync) if it is pinned. */
int lpf_push_frame_host(lpf_stream* s, const float* frame_host, int64_t T);

/*
 * Poll the oldest pushed-and-unpolled frame.  Waits up to timeout_ms (< 0:
 * forever) for its work, then copies its candidates into out_host[cap] (HOST),
 * sorted by (t0, dm_idx, y, x), and sets *n_out to the total number found and
 * *T_out to the frame index.  Returns LPF_E_TRUNCATED (with out_host holding
 * min(cap, cand_cap, *n_out) records of the found set, sorted; which records
 * were dropped beyond cand_cap is unspecified) when *n_out > cap or the device
 * capacity cand_cap overflowed; LPF_E_TIMEOUT (frame stays queued) or
 * LPF_E_NODATA otherwise.  out_host may be NULL when cap == 0.  With
 * suppress_steady, *n_out and the records exclude the dropped candidates, and
 * after an overflow of cand_cap *n_out is the number of kept records stored
 * (see lpf_params).  In every case out_host holds min(cap, cand_cap, *n_out)
 * records.
 */
int lpf_poll_candidates(lpf_stream* s, lpf_candidate* out_host, int cap, int* n_out,
                        int64_t* T_out, int timeout_ms);

/*
 * Gather the dynamic spectra of n candidates c_host[n] (HOST; only y and x are
 * read) for the most recently polled frame T: out_dev (DEVICE, FP32,
 * [n][F][Tw]) receives out[i][f][tau] = X_f(T - Tw + 1 + tau) at (y_i, x_i), or
 * the maximum over the (2 dyn_box_r + 1)^2 box clipped to the image.  Enqueued
 * on the stream; out_dev is valid once the stream reaches it (lpf_stream_sync).
 * The coordinates are staged in page-locked memory the stream owns, so c_host
 * may be reused when the call returns; the call waits only for the previous
 * call's coordinate copy.
 * Errors: LPF_E_ARG (pixel outside the image, n < 0, Tw < 1), LPF_E_DEPTH (Tw >
 * buffer_depth), LPF_E_STALE (a needed frame was overwritten or precedes the
 * first push), LPF_E_NODATA (nothing polled yet).
 */
int lpf_extract_dynspec(lpf_stream* s, const lpf_candidate* c_host, int n, int Tw,
                        float* out_dev);

/*
 * lpf_extract_dynspec_static: the same gather as lpf_extract_dynspec, with the
 * same arguments, results and errors, for callers that must not allocate
 * device memory while they run.  The paper has no counterpart: this is a
 * deployment variant, not a step of the method.
 *
 * Who needs it: lpf_extract_dynspec copies the candidate list into a device
 * buffer that it enlarges with cudaMalloc when a call brings more candidates
 * than any earlier call.  cudaMalloc can block on the whole device and take an
 * unbounded time, and it spends memory outside any budget the caller keeps.
 * A real-time loop that must meet a frame deadline, a server that admits
 * streams against a fixed HBM budget, or a plug-in whose host application owns
 * all device memory cannot have that happen inside a call.  This variant
 * stages the records in a fixed array in device global memory instead and
 * calls no allocating routine (no cudaMalloc, cudaFree or library allocator).
 *
 * Limits and sharing: at most LPF_STATIC_DYNSPEC_MAX candidates per call.
 * Errors are those of lpf_extract_dynspec, checked in the same order, and
 * then LPF_E_CAPACITY for a request above that maximum.  The array (LPF_STATIC_DYNSPEC_MAX records of
 * 24 bytes, 1.5 MiB) is part of the library image: every GPU that loads the
 * library holds it until the process exits.  All calls on a device share it,
 * so calls that overlap on the GPU race; issue them one at a time (from any
 * handle or thread).  Each call writes the records it reads and blocks until
 * its gather has finished (it synchronises the stream's CUDA stream before
 * returning), so nothing carries over between calls and the next call may
 * start as soon as this one returns.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current).
 */
#define LPF_STATIC_DYNSPEC_MAX 65536
int lpf_extract_dynspec_static(lpf_stream* s, const lpf_candidate* c_host, int n, int Tw,
                               float* out_dev);

/* Copy the integer delay table [n_dm][F] (frames) into out (HOST). */
int lpf_get_delay_table(const lpf_stream* s, int32_t* out);

/* Copy [n_dm][2] = (mean, rms) of snr over pixels with S > 0 of every DM trial
 * of the most recently polled frame into out (HOST, FP64); NaN for trials not
 * active at that frame.  Partial sums are FP32 over at most 33 pixels per
 * thread and FP64 above that. */
int lpf_get_stats(const lpf_stream* s, double* out);

int lpf_stream_info(const lpf_stream* s, lpf_stream_info_t* out);

/*
 * Quality control of the most recently polled frame (params.qc = 1): its T, the
 * bands imputed with zeros (bit f) and, if z is not NULL, the F band scores z_f.
 * The paper's quality control (App. A).  Errors: LPF_E_ARG (s NULL),
 * LPF_E_NODATA (qc off, or no frame polled yet).
 */
int lpf_get_qc(const lpf_stream* s, int64_t* T_out, uint32_t* discarded, float* z);

/* Wait (without limit) for all work enqueued on the stream. */
int lpf_stream_sync(lpf_stream* s);

/* Release every resource of the stream after waiting for its work. NULL is OK. */
int lpf_stream_close(lpf_stream* s);

const char* lpf_strerror(int code);

/*
 * Profiling: when on, every push records CUDA events around each kernel stage
 * on the stream it runs on.  lpf_get_kernel_times fills up to n entries of
 * names[] (static strings), total_ms[] and launches[] accumulated since the
 * last reset (reset != 0 clears them after reading) and returns the number of
 * stages.  Reading synchronises the stream.
 */
int lpf_set_profiling(lpf_stream* s, int on);
int lpf_get_kernel_times(lpf_stream* s, const char** names, double* total_ms,
                         int64_t* launches, int n, int reset);

/* ------------------------------------------------------------------ serving
 * A server multiplexes several concurrent streams (different sizes, subbands
 * and DM grids) on the current CUDA device under an HBM budget.  A persistent
 * worker thread owns every stream: it admits requested streams in request
 * order as soon as their device footprint (lpf_stream_footprint) fits the
 * budget left by the admitted ones, moves each stream's submitted frames onto
 * the GPU whenever the stream has a free result slot, and collects finished
 * frames without blocking.  Each stream runs on its own CUDA stream, so work
 * of different streams overlaps on the device; the result of a stream does
 * not depend on what else is being served.  All functions are thread-safe.
 */
typedef struct lpf_server lpf_server;

#define LPF_SERVE_PENDING 0   /* requested, waiting for budget                     */
#define LPF_SERVE_ACTIVE  1   /* admitted: ring buffer and scratch resident         */
#define LPF_SERVE_CLOSED  3   /* drained and released (or failed to open)           */

typedef struct {
    int64_t frames;          /* frames finished                                      */
    double  p50_ms, p99_ms, max_ms;   /* submit -> finished latency                  */
    double  pixel_dm_per_s;  /* H*W*n_dm per finished frame / (first submit -> last finish) */
    size_t  budget_bytes, used_bytes;
} lpf_serve_stats_t;

/* Start a server with an HBM budget (bytes) for its streams' device memory and
 * at most max_streams live (pending or admitted) streams.  Errors: LPF_E_ARG,
 * LPF_E_CUDA (no device), LPF_E_OOM. */
int lpf_server_open(lpf_server** out, size_t hbm_budget_bytes, int max_streams);

/* Request a stream (arguments as lpf_stream_open; params->cuda_stream is
 * ignored).  Returns its id at once; it is admitted when its footprint fits.
 * Frames may be submitted before admission; they queue.  Errors: those of
 * lpf_stream_footprint, LPF_E_BUDGET (larger than the whole budget),
 * LPF_E_BUSY (max_streams live), LPF_E_OOM (pinned frame buffers). */
int lpf_server_open_stream(lpf_server* srv, int H, int W, int F, const double* freqs_mhz,
                           int n_dm, const double* dm_grid, int buffer_depth,
                           const lpf_params* params, int* id_out);

/* Submit frame T ([F][H][W] FP32, HOST) of stream id; copied into the
 * stream's pinned buffers before returning.  Frames of a stream must be
 * submitted in consecutive order.  LPF_E_BUSY when result_slots + 4 frames
 * of the stream are queued or in flight (fetch, then retry). */
int lpf_server_submit(lpf_server* srv, int id, const float* frame_host, int64_t T);

/* Next finished frame of stream id, in submission order: candidates (as
 * lpf_poll_candidates), frame index and submit-to-finish latency.  Waits up
 * to timeout_ms (< 0: until finished or the stream closed).  LPF_E_TIMEOUT,
 * LPF_E_NODATA (stream closed and drained), or the frame's own error code. */
int lpf_server_fetch(lpf_server* srv, int id, lpf_candidate* out_host, int cap, int* n_out,
                     int64_t* T_out, double* latency_ms, int timeout_ms);

/* Close stream id after its queued frames finish; its budget then admits
 * waiting streams.  Unfetched results stay fetchable. */
int lpf_server_close_stream(lpf_server* srv, int id);
int lpf_server_stream_state(lpf_server* srv, int id, int* state);

/* Latency and throughput of stream id, or of all streams (id = -1). */
int lpf_server_stats(lpf_server* srv, int id, lpf_serve_stats_t* out);

/* Stop the worker, wait for all device work and release every stream. */
int lpf_server_close(lpf_server* srv);

/* ------------------------------------------------------------------------
 * Parameter inference on the dynamic-spectrum batch (Sec. 2.3).
 *
 * The paper's network maps a candidate's dynamic spectrum to the mean mu and
 * a Cholesky factor L (lower triangular, positive diagonal) of a Gaussian over
 * its parameters theta, through convolutions with Leaky ReLU hidden states and
 * a final linear layer; it gives the form, not the layers or the weights.
 * This network, with weights the caller supplies, is:
 *   conv1 3x3, 1 -> 16 channels, Leaky ReLU, 2x2 mean;
 *   conv2 3x3, 16 -> 32, Leaky ReLU, 2x2 mean;
 *   conv3 3x3, 32 -> 64, Leaky ReLU, mean over all pixels;
 *   head: linear 64 -> 5, out = (mu0, mu1, exp z2 = L00, z3 = L10, exp z4 = L11);
 * zero padding 1, alpha = 0.01.  conv2 and conv3 run on the tensor cores
 * (BF16 weights and activations, FP32 sums); conv1 and the head in FP32.
 *
 * params: float32, lpf_cnn_param_count() values in this order: conv1.w
 * [16][1][3][3], conv1.b [16], conv2.w [32][16][3][3], conv2.b [32], conv3.w
 * [64][32][3][3], conv3.b [64], head.w [5][64], head.b [5] (HOST, copied).
 */
typedef struct lpf_cnn lpf_cnn;
#define LPF_CNN_OUT 5

size_t lpf_cnn_param_count(void);

/* A network for F x Tw spectra (F subbands by Tw frames, as lpf_extract_dynspec
 * writes them) and batches of at most max_batch; its work is enqueued on
 * cuda_stream (NULL: a stream of its own) on the current device.  F and Tw
 * multiples of 4, (F / 4) (Tw / 4) a power of two <= 128.  Errors: LPF_E_ARG,
 * LPF_E_OOM, LPF_E_CUDA. */
int lpf_cnn_open(lpf_cnn** out, int F, int Tw, const float* params, size_t n_params, int max_batch,
                 void* cuda_stream);

/* out_dev [n][5] (FP32, DEVICE) for the spectra x_dev [n][F][Tw] (FP32, DEVICE),
 * n <= max_batch; asynchronous on the network's stream.  32 x 64 spectra run
 * as one persistent kernel with the activations in shared memory, which copies
 * each spectrum in 16-byte pieces: x_dev must then be 16-byte aligned (LPF_E_ARG
 * otherwise).  Other shapes run as three kernels through global memory.  Both
 * follow the same rounding points (BF16 activations after conv1 and conv2);
 * their FP32 sums may differ in order.  Errors: LPF_E_ARG, LPF_E_CUDA. */
int lpf_cnn_forward(lpf_cnn* net, const float* x_dev, int n, float* out_dev);

/* Wait for the network's work; LPF_E_TIMEOUT if a tensor-core completion wait
 * ran out (its outputs are then not written). */
int lpf_cnn_sync(lpf_cnn* net);
int lpf_cnn_close(lpf_cnn* net);

#ifdef __cplusplus
}
#endif
#endif /* LPF_H */
