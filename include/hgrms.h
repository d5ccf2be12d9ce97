/*
 * hgrms.h - C ABI of the GB300 P-HGRMS salt-and-pepper denoiser.
 *
 * The method (P-HGRMS, Sections 2 and 3 of the paper):
 *   For an 8-bit greyscale image I (rows x cols, row-major I[r*cols + c]),
 *   parameters alpha (grey-level tolerance) and beta (window radius), one
 *   pass computes
 *     card(p)  = #{n in W(p) on the image : I[p]-alpha < I[n] < I[p]+alpha}
 *                (Algorithm 1, the cardinality matrix; W(p) is the
 *                (2 beta + 1)^2 window centred on p, p itself included),
 *     and, for every p with card(p) <= 2 (Algorithm 2),
 *     flag     = #{n in W(p) on the image : NOT (I[p]-alpha < I[n] <= I[p]+alpha)}
 *     sum      = sum of I[n]^2 over those "open" n,
 *     pix_count= (2 beta + 1)^2 (off-image positions included);
 *     if flag > pix_count - 3 the pixel is replaced, in a separate output
 *     image, by floor(sqrt(floor(sum / flag))) - the root mean square of its
 *     open neighbourhood.  Other pixels keep their value.
 *   Passes repeat (Section 2, iteration factor k) until a pass changes no
 *   pixel or max_k passes that changed pixels have run.  k, the number of
 *   passes that changed at least one pixel, is returned.  All arithmetic is
 *   integer; results are exact (bit-identical to a direct evaluation of the
 *   definition).
 *
 * Conventions
 *   - Functions returning int return >= 0 on success and a negative HGRMS_E*
 *     code on failure.  A failed call leaves the image unspecified only for
 *     HGRMS_ECUDA / HGRMS_ETIMEOUT; argument errors are detected before any
 *     device work and leave the image untouched.
 *   - Images are dense: row r starts at img + r*cols.  No alignment is
 *     required.  The pointer may be device memory of the handle's device
 *     (denoised in place on the device), page-locked host memory mapped into
 *     the device's address space (e.g. from cudaHostAlloc: the device reads
 *     it and writes the result back to it directly), or other host memory
 *     (copied to the device and back inside the call).
 *   - Calls are synchronous: when a call returns, the result is in img
 *     (hgrms_denoise_async is the exception: hgrms_wait completes it).
 *     Work is issued on the handle's stream.
 *   - A handle may be used by one host thread at a time.
 *   - Limits: 1 <= rows, cols <= 65536; 0 <= alpha <= 255; 1 <= beta <= 7;
 *     0 <= max_k <= 1000000.
 */
#ifndef HGRMS_H
#define HGRMS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HGRMS_OK        0
#define HGRMS_EINVAL   (-1) /* bad argument (null pointer, size or parameter out of range) */
#define HGRMS_ENOMEM   (-2) /* device or pinned host allocation failed */
#define HGRMS_ECUDA    (-3) /* a CUDA runtime call or kernel failed; see hgrms_last_cuda_error */
#define HGRMS_ETIMEOUT (-4) /* a bounded device wait gave up */
#define HGRMS_ENODEV   (-5) /* no CUDA device, or the device index is out of range */
#define HGRMS_ETOOBIG  (-6) /* image too large for hgrms_denoise_noalloc's fixed scratch */
#define HGRMS_EAGAIN   (-7) /* hgrms_server_wait: the request is not finished yet */
#define HGRMS_EBUSY    (-8) /* the handle has an asynchronous call that hgrms_wait has not finished */

typedef struct hgrms_ctx* hgrms_t;

/* Create a handle on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to issue work on, or NULL for the device's default (legacy) stream.  The
 * handle owns its device buffers and reuses them across calls, growing them on
 * demand: the image buffers that stand for I and the temporary image I' of
 * Section 2 (three padded canvases, so a pass never copies I' back), the
 * change lists and bitmaps that carry the pixels a pass changed to the next
 * pass, and the control block holding the Section 2 iteration state (k, the
 * converged flag, max_k).
 * Writes the handle to *out and returns HGRMS_OK, or a negative code (and
 * *out = NULL). */
int hgrms_create(hgrms_t* out, int device, void* cuda_stream);

/* Release the handle and everything it owns (the buffers above; the
 * iteration state of Section 2 dies with it).  NULL is accepted. */
void hgrms_destroy(hgrms_t h);

/* Denoise one image in place (the full method above).
 * Returns k (0 <= k <= max_k) or a negative error code.  Reaching max_k is
 * not an error; hgrms_converged() tells whether the call ended on a pass
 * that changed nothing.  Images smaller than 2*beta+1 in either dimension
 * are returned unchanged with k = 0 (no pixel can be replaced there). */
int hgrms_denoise(hgrms_t h, uint8_t* img, int rows, int cols,
                  int alpha, int beta, int max_k);

/* Denoise n independent images with the same alpha, beta and max_k, in
 * place: Section 2's iteration of Algorithms 1-2 run on each image, with the
 * stop rule applied per image (image i stops contributing passes once one of
 * its passes changes nothing, or at k_i = max_k).  imgs[i] has rows[i] x cols[i] pixels (each device memory or host
 * memory, as for hgrms_denoise).  k_out[i] receives image i's k, exactly what
 * hgrms_denoise returns for that image alone; image i converged (a further
 * pass would change nothing) exactly when k_out[i] < max_k.  With the
 * default schedule the images are denoised together: one fused launch over
 * the tiles of every image, then one persistent launch that runs the
 * remaining passes for all of them (see HGRMS_OPT_BATCH_MB for how large
 * batches are split).  Returns HGRMS_OK or a negative code; arguments are
 * validated for every image before any work starts.  hgrms_converged() then
 * reports whether every image converged. */
int hgrms_denoise_batch(hgrms_t h, uint8_t* const* imgs, const int* rows,
                        const int* cols, int n, int alpha, int beta, int max_k,
                        int* k_out);

/* Queue the denoising of one image on the handle's stream and return at once
 * (HGRMS_OK or a negative code); hgrms_wait finishes the call and returns k.
 * Same method, arguments, limits and result as hgrms_denoise (Sections 2-3:
 * the passes of Algorithms 1-2 repeated until a pass changes nothing or k =
 * max_k), but `img` must be memory the device reads directly: device memory
 * of the handle's device, or page-locked host memory mapped into its address
 * space (other host memory: HGRMS_EINVAL).  The result is in img once the
 * handle's stream has reached the end of the call (hgrms_wait, or any later
 * work on that stream).  Several handles created on the same stream can each
 * have one call queued, so consecutive calls run back to back on the device
 * with no host round trip between them; the handles' list-pass launches then
 * never overlap.  A handle admits one outstanding call: until hgrms_wait, its
 * other denoising calls return HGRMS_EBUSY.  Options that need the host
 * between launches (HGRMS_OPT_AUTOTUNE, HGRMS_OPT_PREDICT_K, HGRMS_OPT_KERNEL
 * other than 0) make the call run to completion before it returns. */
int hgrms_denoise_async(hgrms_t h, uint8_t* img, int rows, int cols,
                        int alpha, int beta, int max_k);

/* Wait for the call queued by hgrms_denoise_async and return its k (or the
 * negative code of its failure); the statistics, launch times and
 * hgrms_converged then describe it.  HGRMS_EINVAL when no call is
 * outstanding. */
int hgrms_wait(hgrms_t h);

/* The stop rule of Section 2 ("until no noise remains", capped by the
 * iteration factor): 1 if the last hgrms_denoise ended because a pass changed
 * no pixel (the image is a fixed point), 0 if it stopped at max_k, negative
 * on a bad handle.  After hgrms_denoise_batch: 1 only if every image
 * converged. */
int hgrms_converged(hgrms_t h);

/* Human-readable text for a return code (static storage). */
const char* hgrms_strerror(int code);

/* The cudaError_t of the last failing CUDA call on this handle (0 if none). */
int hgrms_last_cuda_error(hgrms_t h);

/* The integer root mean square of Algorithm 2 as the fused and list-pass
 * kernels compute it: out[i] = floor(sqrt(floor(sum[i] / flag[i]))) for n entries,
 * valid for 0 <= sum[i] <= flag[i] * 255^2 and 1 <= flag[i] <= 225 (the
 * range a (2 beta + 1)^2 window of 8-bit pixels produces).  sum, flag and
 * out are device memory of the current device; the call runs on
 * `cuda_stream` (NULL: the default stream) and returns when it is done.
 * Exposed so that the arithmetic can be checked exhaustively against exact
 * integer math.  Returns HGRMS_OK, HGRMS_EINVAL or HGRMS_ECUDA. */
int hgrms_rms(const int* sum, const int* flag, int* out, int n, void* cuda_stream);

/* ---- Denoising without device allocation ------------------------------- */

/* Bytes of the fixed device scratch array behind hgrms_denoise_noalloc. */
#define HGRMS_NOALLOC_SCRATCH_BYTES (16u << 20)

/* The same denoising as hgrms_denoise (fused tile kernel, repeated fused
 * launches), for callers that must not allocate device memory: code whose
 * device memory is owned by a pool or host application it cannot bypass,
 * and latency-critical paths where an allocation may stall or fail.  No
 * handle is needed and the call makes no cudaMalloc/cudaFree (nor any other
 * allocating call): every scratch buffer lives in one file-scope __device__
 * array of HGRMS_NOALLOC_SCRATCH_BYTES that each GPU loading the library
 * keeps until the process exits.  The paper has no counterpart; this is an
 * interface of this library only.
 *
 *   img       device memory of the current CUDA device, rows x cols dense,
 *             denoised in place (host memory is rejected with HGRMS_EINVAL).
 *   cuda_stream  a cudaStream_t, or NULL for the default stream; the call
 *             returns after the work on it finished.
 * Returns k (as hgrms_denoise) or a negative code; HGRMS_ETOOBIG when the
 * scratch the image needs exceeds the array (images with rows, cols <= 2048
 * always fit; larger ones fit while their two padded canvases and change
 * bitmaps do).  There is no handle, so there is no hgrms_converged for this
 * call: a return of k < max_k means it converged (a pass changed nothing),
 * while k == max_k does not tell whether pass max_k happened to leave a fixed
 * point.  The fused launches are queued in groups of 32 passes; after each
 * group (when more are due) the call reads k and the converged flag from the
 * device and stops once it has converged, so a large max_k costs nothing
 * after convergence beyond the group it falls in.  Every call looks up the
 * array's address on the current device (cudaGetSymbolAddress, which
 * allocates nothing); the first call on a device may also load the
 * library's device code there, so make that first call before capturing any
 * stream into a CUDA graph.  All calls on a device share the array (it
 * keeps the last call's contents; each call re-initialises what it reads),
 * so calls whose GPU work overlaps - from two streams or two host threads -
 * race and must be serialised by the caller. */
int hgrms_denoise_noalloc(uint8_t* img, int rows, int cols, int alpha, int beta, int max_k,
                          void* cuda_stream);

/* ---- Serving: continuous batching of requests ------------------------- */

/* A request server on one device.  Requests (one image each, any size, each
 * with its own alpha, beta and max_k) queue up and are served by `slots`
 * worker threads, each with its own handle, CUDA stream and an equal share of
 * `hbm_budget_bytes`.  A slot that becomes free takes, in arrival order,
 * every queued request with the oldest request's (alpha, beta, max_k) while
 * their device memory (resident copies of host images plus the batched
 * schedule's buffers, estimated per pixel) fits its share - the oldest one
 * always, alone if it exceeds the share - and denoises them with one
 * hgrms_denoise_batch call; requests that arrive meanwhile join a later
 * batch, and the batches of different slots run concurrently on the device.
 * A request's output and k are those of hgrms_denoise on its image alone,
 * whatever batch it joins (not a method of the paper: a way of running it
 * for many requests). */
typedef struct hgrms_server* hgrms_server_t;

typedef struct hgrms_request_info {
    int    k;           /* the request's k, or its negative error code */
    double latency_ms;  /* submit -> result ready */
    double queue_ms;    /* submit -> taken by a slot */
    int    batch_size;  /* requests in the batch it was served in */
    int    slot;
} hgrms_request_info_t;

/* Create a server with `slots` (1..64) workers on `device` and a device
 * memory budget of hbm_budget_bytes (>= 64 MiB).  Returns HGRMS_OK and the
 * server in *out, or a negative code. */
int hgrms_server_create(hgrms_server_t* out, int device, long long hbm_budget_bytes, int slots);

/* Queue one request.  `img` is rows x cols bytes, row-major: device memory of
 * the server's device (denoised in place; out must be NULL or img) or host
 * memory (its result is written to `out`, host memory of the same size,
 * which may be img).  Both must stay valid until hgrms_server_wait returns
 * for the request.  Writes the request id to *id.  Returns HGRMS_OK or
 * HGRMS_EINVAL (bad arguments, or the server is shutting down). */
int hgrms_server_submit(hgrms_server_t s, const uint8_t* img, uint8_t* out, int rows, int cols, int alpha,
                        int beta, int max_k, unsigned long long* id);

/* Wait for request `id` (at most timeout_s seconds; negative = no limit),
 * fill *info (if not NULL) and release the request.  Returns its k (>= 0),
 * its error code, HGRMS_EAGAIN (not finished within the timeout; wait again)
 * or HGRMS_EINVAL (unknown id, e.g. already waited for). */
int hgrms_server_wait(hgrms_server_t s, unsigned long long id, double timeout_s, hgrms_request_info_t* info);

/* Counters so far: requests served, batches run, requests queued now, and
 * the most requests on the device at once.  Returns the first error a batch
 * met (0 if none). */
int hgrms_server_stats(hgrms_server_t s, long long* served, long long* batches, long long* queued,
                       long long* max_in_flight);

/* For tests of the failure path (not for production; 0 at creation): the
 * next n allocations of a slot's buffer for host images fail as a failing
 * cudaMalloc would, without calling it.  The requests of each such batch
 * complete with HGRMS_ENOMEM (hgrms_server_wait returns it, and
 * hgrms_server_stats reports it as the first error); later batches allocate
 * again and are served normally.  Replaces any count still pending.  Returns
 * HGRMS_OK, or HGRMS_EINVAL for a NULL server or n < 0. */
int hgrms_server_fail_allocations(hgrms_server_t s, int n);

/* Serve every queued request, stop the workers and free everything.  NULL is
 * accepted. */
void hgrms_server_destroy(hgrms_server_t s);

/* ---- Learned k-predictor (not part of the method) ---------------------- */

/* The paper's concluding section leaves choosing the iteration factor k in
 * advance as future work.  This predictor estimates k from a 64 x 64
 * area-averaged copy of the image and a 16-bin histogram of its grey levels
 * with a 4-layer 3 x 3 convolutional network (16 channels, BF16 operands and
 * FP32 accumulation on the tensor cores) and a linear head; the estimate
 * only chooses the schedule (HGRMS_OPT_PREDICT_K).
 *
 * Load the network for windows of `beta` (one network per beta; a call with
 * HGRMS_OPT_PREDICT_K uses the one of its beta, if loaded): weights[n]
 * holds, in order, conv layer 1 as
 * [tap 0..8][1][16], layers 2..4 as [tap 0..8][16 inputs][16 outputs]
 * (tap = 3 (dy + 1) + (dx + 1)), the 4 x 16 biases, then the head: 16
 * weights on the last layer's channel means, 16 on the histogram and a bias
 * (n = 144 + 3 * 2304 + 64 + 33 = 7153).  Returns HGRMS_OK, or HGRMS_EINVAL
 * for a wrong n. */
int hgrms_predictor_load(hgrms_t h, int beta, const float* weights, int n);

/* Estimate k (windows of `beta`) for n images (device memory or mapped
 * page-locked host memory,
 * as for hgrms_denoise; other host memory is rejected with HGRMS_EINVAL):
 * k_hat[i] >= 0.  Optional outputs (host, NULL to skip): x0 (n x 64 x 64
 * area means / 255), hist (n x 16 bin fractions; bin = value / 16) and gap
 * (n x 16 channel means of the last layer).  Returns HGRMS_OK, HGRMS_EINVAL
 * (no network loaded for beta, bad arguments), HGRMS_ETIMEOUT (a bounded wait for the
 * tensor cores gave up) or another negative code. */
int hgrms_predict_k(hgrms_t h, int beta, uint8_t* const* imgs, const int* rows, const int* cols, int n,
                    float* k_hat, float* x0, float* hist, float* gap);

/* Fit the network on the device (every step on the tensor cores: the
 * forward convolutions, the gradients of their inputs and of their weights,
 * then Adam on CUDA cores).  x0 (n x 64 x 64 area means / 255, as
 * hgrms_predict_k returns them), hist (n x 16) and k (n targets) are host
 * arrays; weights (host, the order of hgrms_predictor_load) holds the
 * initial parameters and receives the fitted ones.  Minimises the mean of
 * (y - k)^2 over minibatches of `batch` images (y: the head before its
 * ReLU), `epochs` passes over a permutation drawn from `seed` (a 64-bit
 * linear congruential generator), learning rate lr (lr / 3 in the last
 * quarter of the epochs).  *loss (if not NULL) receives the last epoch's
 * mean minibatch loss.  Returns HGRMS_OK or a negative code. */
int hgrms_predictor_train(hgrms_t h, float* weights, const float* x0, const float* hist, const float* k, int n,
                          int epochs, int batch, float lr, unsigned long long seed, float* loss);

/* One gradient of that loss over all n images (n <= 4096) for the given
 * weights: grads (host, the weights' order) and *loss.  For tests. */
int hgrms_predictor_grad(hgrms_t h, const float* weights, const float* x0, const float* hist, const float* k, int n,
                         float* grads, float* loss);

/* ---- Tuning and measurement (not part of the method) ------------------ */

/* Options for hgrms_set_option. */
#define HGRMS_OPT_KERNEL   1 /* 0 = fused multi-pass tile launches while many pixels change, then one
                                 persistent launch that runs every remaining pass as a list pass
                                 (default); 1 = unfused one-pass kernel for every pass; 2 = fused tile
                                 launches only */
#define HGRMS_OPT_PASSES   2 /* passes fused per launch; 0 = the built-in choice for beta */
#define HGRMS_OPT_TIMING   3 /* 1 = time every denoising launch with CUDA events (see hgrms_stats) */
#define HGRMS_OPT_LIST_CAP 4 /* capacity of the change lists of list passes (0 = rows*cols/4 + 65536);
                                when a pass changes more pixels, the next pass evaluates every pixel */
#define HGRMS_OPT_BATCH_MB 5 /* hgrms_denoise_batch: device memory (MiB) one batched launch may use for
                                canvases, change lists and bitmaps (0 = 8192); larger batches run as
                                several chunks of consecutive images, with identical results */
#define HGRMS_OPT_RELAUNCH_PPM 6 /* default schedule: after a fused launch, another fused launch runs
                                    (instead of list passes) while a list pass would evaluate more than
                                    this many pixels per million pixels of the call, up to 8 times
                                    (0 = built-in: 25000 for beta 1, up to 3 times, for calls of
                                    at least 4 Mi pixels; never for beta >= 2 or smaller calls;
                                    1000000 or more = never) */
#define HGRMS_OPT_AUTOTUNE 8 /* 1 = choose the fused passes per launch and the in-tile switch point
                                 by timing: the first call of each (beta, single image or batch,
                                 size class = bit length of the pixel count) runs every compiled
                                 passes-per-launch value with switch points 1024..8192 on its own
                                 images, without writing them, and keeps the fastest; the result does
                                 not depend on the choice.  Options 2 and 7, when set, are kept. */
#define HGRMS_OPT_PREDICT_K 9 /* 1 = before the passes, estimate k with the learned predictor (weights
                                  from hgrms_predictor_load; device-readable images only) and run
                                  ceil(k_hat / T) fused launches unconditionally (each stops once a pass
                                  changes nothing) before the list passes; the results and k do not
                                  depend on the estimate */
#define HGRMS_OPT_GRAPH    11 /* 1 = the default schedule records the device work of a call on images
                                   the device reads directly into a CUDA graph and replays it for later
                                   calls with identical arguments (same pointers, sizes, parameters and
                                   options): one graph launch instead of the call's separate launches,
                                   copies and clears; up to 8 graphs per handle, the oldest dropped
                                   first.  Results are identical either way; a call the graph cannot
                                   record runs as usual. */
#define HGRMS_OPT_LIST_CTAS 10 /* CTAs of the list-pass launch (0 = built-in: one per SM below
                                   16 M pixels, else as many as can be co-resident, 2 per SM) */
#define HGRMS_OPT_TILE_EVAL_MAX 7 /* fused kernel: a pass runs as an in-tile list pass while the previous
                                     pass's changes need at most this many evaluations in the tile,
                                     else as a dense pass (0 = built-in: 2048 for beta 2, else
                                     4096, per 64-row tile; twice that with the 128-row tiles of
                                     calls of at least 32 Mi pixels) */

#define HGRMS_OPT_TMA      13 /* 1 = the default schedule's fused launches (beta <= 4) stage each tile
                                   with its halo in shared memory by TMA, the next tile's load running
                                   while the current one computes (default); 0 = ordinary loads.
                                   Results are identical either way. */
#define HGRMS_OPT_WAIT_TEST 12 /* for tests of the bounded device wait (not for production): N > 0 makes
                                   every grid barrier of the list-pass launch wait for one arrival more
                                   than the launch has CTAs - an arrival that never comes - and give up
                                   after N polls (at most 2^22); the call then returns HGRMS_ETIMEOUT once
                                   a list pass runs, its image unspecified, and the handle stays usable.
                                   0 = off (default) */

/* Set an option.  Returns HGRMS_OK or HGRMS_EINVAL (unknown option or value,
 * e.g. a pass count that has no compiled kernel for some beta is rejected at
 * denoise time with HGRMS_EINVAL). */
int hgrms_set_option(hgrms_t h, int option, int value);

/* Statistics of the last hgrms_denoise / hgrms_denoise_batch call. */
typedef struct hgrms_stats {
    int    launches;        /* denoising kernel launches issued */
    int    work_launches;   /* of those, launches that ran at least one pass */
    int    passes;          /* passes needed: k, plus 1 if the call ended on a no-change pass */
    int    passes_executed; /* passes the launches actually ran (a launch runs whole
                               groups of T, so this can exceed `passes`) */
    int    passes_per_launch; /* fused passes per launch (T) */
    int    tile_rows;       /* core tile height of the kernel used */
    int    tile_cols;       /* core tile width of the kernel used */
    long long ctas_per_launch;
    double kernel_ms;       /* HGRMS_OPT_TIMING: summed durations of the launches that ran
                               passes (CUDA events on the handle's stream), else 0 */
    double idle_kernel_ms;  /* HGRMS_OPT_TIMING: summed durations of the launches that found
                               the call already finished and returned at once */
    long long evals_fused;  /* pixel evaluations the passes needed, fused tile launches
                               (every image pixel per dense pass, else the pixels within
                               beta of a change of the previous pass) */
    long long evals_list;   /* the same for list-pass launches */
    int    tile_eval_max;   /* in-tile list/dense switch point used (HGRMS_OPT_TILE_EVAL_MAX) */
    int    autotuned;       /* 1 if the tuning came from the autotuner (HGRMS_OPT_AUTOTUNE) */
    double tune_ms;         /* device time the autotuner's trials took in this call (0 when the
                               choice was already known) */
    double k_pred;          /* HGRMS_OPT_PREDICT_K: the largest predicted k of the call's
                               images, else -1 */
    int    graph;           /* HGRMS_OPT_GRAPH: 1 = the call replayed a recorded graph, 2 = it
                               recorded one (and ran it), 0 = no graph */
} hgrms_stats_t;

int hgrms_stats(hgrms_t h, hgrms_stats_t* out);

/* Per-launch durations (ms) of the last call, recorded when HGRMS_OPT_TIMING
 * is on, in launch order; kind[i] (if kind is not NULL) is 0 for a fused tile
 * launch, 1 for the launch running the list passes, 2 for an unfused pass and
 * 3 for a launch that ran no pass (the call had finished, or the schedule
 * skipped it).  Copies at most n entries and returns the number recorded, or
 * HGRMS_EINVAL. */
int hgrms_launch_times(hgrms_t h, float* ms, int* kind, int n);

/* The passes per launch the built-in choice uses for beta (1..7), or
 * HGRMS_EINVAL. */
int hgrms_default_passes(int beta);

/* Whether a fused kernel with `passes` passes per launch exists for beta. */
int hgrms_has_kernel(int beta, int passes);

#ifdef __cplusplus
}
#endif

#endif /* HGRMS_H */
