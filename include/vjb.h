/*
 * vjb.h -- C ABI of the GB300 (sm_103a) Viola-Jones AdaBoost trainer.
 *
 * The library trains the discrete AdaBoost of Viola and Jones over the full
 * Haar feature set of a window, as restated in Abualkibash, ElSayed and
 * Mahmood, "Highly scalable, parallel and distributed AdaBoost algorithm using
 * light weight threads and web services on a network of multi-core machines"
 * (arXiv 1306.1467), Sec. 2.  Every step of a round runs in the library's own
 * CUDA kernels on one GPU.
 *
 * Conventions for every entry point:
 *   - Return value: VJB_OK (0), a positive VJB_DONE_* status, or a negative
 *     error code.  On a negative code nothing visible to the caller has
 *     changed except where noted, and vjb_last_error() gives a message.
 *   - Pointers named "host" are ordinary host memory owned by the caller; the
 *     library copies from / into them before returning and keeps no
 *     reference.  Pointers named "device" are device memory on the context's
 *     device, owned by the caller, read before the call returns.
 *   - All device memory the library needs is allocated by the context and
 *     released by vjb_destroy().
 *   - Calls on one context must not overlap (one host thread at a time).
 *     Every call is synchronous with respect to the context's stream.
 */
#ifndef VJB_H
#define VJB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define VJB_OK            0
#define VJB_DONE_PERFECT  1   /* eps == 0: stump kept (alpha = +inf), training over   */
#define VJB_DONE_NOGAIN   2   /* eps >= 1/2: stump not kept, training over            */
#define VJB_EINVAL      (-1)  /* bad argument (sizes, labels, ranges)                 */
#define VJB_ESTATE      (-2)  /* call out of order                                    */
#define VJB_ENOMEM      (-3)  /* device allocation failed                             */
#define VJB_ECUDA       (-4)  /* CUDA runtime / driver error                          */
#define VJB_EDEVICE     (-5)  /* a kernel set its error flag (wait timeout, bounds)   */
#define VJB_EFULL       (-6)  /* a batch has no room left (table budget, job slots)   */

/* Limits.  Sample indices are stored in 15 bits and index N marks padding. */
#define VJB_MAX_SAMPLES 32766
#define VJB_MAX_WINDOW  255

/* Haar feature types in canonical order (Sec. 2.2 lists them in this order). */
#define VJB_HAAR_3H 0   /* three rectangles side by side along x, base 3x1 */
#define VJB_HAAR_3V 1   /* three rectangles stacked along y,      base 1x3 */
#define VJB_HAAR_2H 2   /* two rectangles side by side along x,   base 2x1 */
#define VJB_HAAR_2V 3   /* two rectangles stacked along y,        base 1x2 */
#define VJB_HAAR_4  4   /* two by two rectangles,                 base 2x2 */

typedef struct vjb_ctx vjb_ctx;

/* One Haar feature: its top-left corner (x, y) and full size (w, h) in pixels.
 * Value (Sec. 2.2, dark minus white): 2H/2V = S(right|bottom) - S(left|top);
 * 3H/3V = S(middle) - S(first) - S(last); 4 = S(top-right) + S(bottom-left)
 * - S(top-left) - S(bottom-right). */
typedef struct {
    uint8_t type, x, y, w, h;
} vjb_feature;

/* One weak classifier h(x) = 1 iff polarity * f(x) < polarity * threshold
 * (Sec. 2.2), with its round's weighted error (Sec. 2.3 step 2),
 * beta = error / (1 - error) and alpha = log(1 / beta) (Sec. 2.3). */
typedef struct {
    int32_t feature;    /* index into the canonical feature list          */
    int32_t threshold;  /* integer threshold theta                        */
    int32_t polarity;   /* +1 or -1                                       */
    int32_t split;      /* samples on the "below" side in value order     */
    double  error;      /* weighted error, FP64 sum over the samples      */
    double  beta;
    double  alpha;      /* +inf when error == 0                           */
} vjb_stump;

/* What the search saw of one kept round's stump (precision diagnostics),
 * each divided by the round's FP64 weight total so that it compares with the
 * stump record's `error` (the FP64 sum).
 * search_error: the stump's weighted error from the compensated (double-float
 *   FP32) re-scan that chose it.
 * screen_error: the FP32 screened error of the stump's feature.
 * screen_min:   the smallest FP32 screened error of the round.
 * candidates:   features re-scanned compensated in the round.
 * forced:       1 if the round's stump came from vjb_force_stump (the other
 *   fields then repeat the FP64 error and candidates is 0). */
typedef struct {
    double  search_error;
    float   screen_error;
    float   screen_min;
    int32_t candidates;
    int32_t forced;
} vjb_round_diag;

/* Diagnostics of the context and of its last search. */
typedef struct {
    int32_t n, h, w;          /* samples and window size                        */
    int32_t npad;             /* sorted-table row length (samples padded)       */
    int64_t features;         /* F                                              */
    int32_t rounds_done;      /* stumps kept so far                             */
    int32_t status;           /* VJB_OK or VJB_DONE_*                           */
    double  t_pos, t_neg;     /* FP64 class totals of the current weights       */
    double  weight_sum;       /* FP64 sum of the current FP32 weights           */
    float   screen_min;       /* smallest FP32 screened error of the last search */
    int32_t candidates;       /* features re-scanned compensated in that search */
    int32_t device_flags;     /* error flags set by kernels (0 = none)          */
    int32_t kernel_warps;     /* search kernel: consumer warps per CTA          */
    int32_t kernel_stages;    /* search kernel: TMA stages per warp             */
    int32_t kernel_ctas;      /* search kernel: CTAs in the grid                */
    int32_t kernel_unroll;    /* search kernel: 512-entry units a warp works on together */
    int32_t kernel_box_lines; /* search kernel: 128-byte lines per TMA box                */
    int32_t pad0;
    double  search_bytes;     /* algorithmic bytes one search reads: 2 * F * N  */
    int64_t launches;         /* kernels this context has launched so far       */
    int32_t dual_weights;     /* 1: the search gathers from two bank-balanced weight copies */
    int32_t pad;
} vjb_info;

/* Per-launch timing of the rounds run since timing was (re)enabled, from CUDA
 * events recorded on the context's stream around the search kernel and around
 * the whole round (with timing on, vjb_train_strong replays each round as two
 * graphs, the search and the rest, with the events between them). */
typedef struct {
    int32_t rounds;           /* rounds timed                                   */
    int32_t pad;
    double  search_ms_total;  /* sum of search-kernel durations                 */
    double  search_ms_min;
    double  search_ms_max;
    double  round_ms_total;   /* sum of whole-round durations                   */
} vjb_timing;

/* ---- context ----------------------------------------------------------
 * vjb_create: make a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t (may be NULL: the context creates its own non-blocking
 * stream).  *out receives the context.  Errors: VJB_EINVAL (out NULL,
 * device out of range), VJB_ECUDA. */
int vjb_create(vjb_ctx **out, int device, void *cuda_stream);

/* Release every device buffer of the context and the context itself.  NULL is
 * accepted. */
void vjb_destroy(vjb_ctx *ctx);

/* Message of the last failing call on this host thread ("" if none). */
const char *vjb_last_error(void);

/* ---- step 0: training set (Sec. 2.3, Table 1) ---------------------------
 * vjb_load_windows: copy n windows of h x w uint8 pixels, row-major
 * [n][h][w] (host), and n labels (host, 1 = face, 0 = non-face) to the
 * device.  Sets the initial weights of Table 2: 1/(2l) for each of the l
 * faces, 1/(2m) for each of the m non-faces, normalised in FP64 and stored
 * FP32.  Discards any earlier training set and its tables.
 * Errors: VJB_EINVAL if n < 2 or n > VJB_MAX_SAMPLES, h or w outside
 * [1, VJB_MAX_WINDOW], a label not 0/1, or no face or no non-face;
 * VJB_ENOMEM; VJB_ECUDA. */
int vjb_load_windows(vjb_ctx *ctx, const uint8_t *pixels, const uint8_t *labels,
                     int32_t n, int32_t h, int32_t w);

/* Same as vjb_load_windows with `pixels` and `labels` in device memory. */
int vjb_load_windows_device(vjb_ctx *ctx, const uint8_t *pixels, const uint8_t *labels,
                            int32_t n, int32_t h, int32_t w);

/* ---- step 1: integral images (Sec. 2.1) --------------------------------
 * ii(x, y) = sum of pixels at x' < x, y' < y, with a zero first row and
 * column, for every window.  Errors: VJB_ESTATE before load; VJB_ECUDA. */
int vjb_build_integral(vjb_ctx *ctx);

/* ---- step 2: Haar features (Sec. 2.2) ----------------------------------
 * Enumerate every feature of the window in canonical order (types 3H, 3V,
 * 2H, 2V, 4; inside a type by width, height, y, x ascending), evaluate every
 * feature on every window from its integral image (int32, exact), and build
 * the per-feature sample order used by every round: samples sorted by value,
 * ties by sample index.  *count receives F.  If `out` is not NULL it must
 * hold F entries (host) and receives the feature list.  A second call returns
 * the same list without recomputing.  The sort checks every table entry it
 * writes (a word inside the weight array) and counts the rows written; a
 * table that fails the check is not used.  Errors: VJB_ESTATE before
 * vjb_build_integral; VJB_EINVAL (count NULL); VJB_ENOMEM; VJB_EDEVICE (the
 * table check failed); VJB_ECUDA. */
int vjb_enumerate_haar(vjb_ctx *ctx, int64_t *count, vjb_feature *out);

/* ---- step 3: one boosting round (Sec. 2.3 steps 1-4) --------------------
 * Normalised weights -> the stump (f, p, theta) of least weighted error over
 * every feature, polarity and threshold -> beta, alpha -> reweight
 * w <- w * beta^(1 - e) and renormalise (FP64 total, FP32 storage).
 * *out (host, may be NULL) receives the stump.  Returns VJB_OK,
 * VJB_DONE_PERFECT (stump kept, no update) or VJB_DONE_NOGAIN (stump not
 * kept, no update); once training is over further rounds return the same
 * status and do nothing.  Errors: VJB_ESTATE before vjb_enumerate_haar;
 * VJB_EDEVICE; VJB_ECUDA. */
int vjb_train_round(vjb_ctx *ctx, vjb_stump *out);

/* T rounds, replayed as a CUDA graph with one host synchronisation at the
 * end.  out (host, T entries, may be NULL) receives the kept stumps;
 * *rounds_done (may be NULL) how many were kept by this call.  Returns the
 * status of the last round run.  Errors as vjb_train_round, VJB_EINVAL if
 * T < 0. */
int vjb_train_strong(vjb_ctx *ctx, int32_t T, vjb_stump *out, int32_t *rounds_done);

/* ---- state access --------------------------------------------------------
 * vjb_get_weights: copy the n current FP32 weights to `out` (host).
 * vjb_set_weights: replace the weights by `w` (host, n values, finite,
 * >= 0, positive sum), normalised in FP64 and stored FP32, and restart the
 * round status (training may continue after a DONE status).
 * Errors: VJB_ESTATE before load; VJB_EINVAL; VJB_ECUDA. */
int vjb_get_weights(vjb_ctx *ctx, float *out);
int vjb_set_weights(vjb_ctx *ctx, const float *w);

/* Teacher forcing: run steps 3-4 of a round with a given stump instead of the
 * searched one: its error on the current weights (FP64), beta, alpha, and the
 * update.  `feature`, `threshold`, `polarity` as in vjb_stump; *out (host,
 * may be NULL) receives the completed record.  Statuses as
 * vjb_train_round.  Errors: VJB_ESTATE; VJB_EINVAL (feature out of range,
 * polarity not +-1). */
int vjb_force_stump(vjb_ctx *ctx, int32_t feature, int32_t threshold, int32_t polarity,
                    vjb_stump *out);

/* Context and last-search diagnostics.  Errors: VJB_EINVAL (out NULL). */
int vjb_get_info(vjb_ctx *ctx, vjb_info *out);

/* ---- inspection (tests) ----------------------------------------------------
 * vjb_get_integral: copy the integral images, [n][h+1][w+1] int32 (host).
 * vjb_feature_values: evaluate features [f0, f0 + nf) on every window into
 *   out[nf][n] int32 (host).
 * vjb_sorted_rows: copy rows [f0, f0 + nf) of the sorted table into
 *   out[nf][n] uint16 (host).  Entry = sample index (bits 0-14) | bit 15 set
 *   when the value at this position is smaller than the value at the next
 *   position (always set at the last position).
 * vjb_screen_errors: copy the F per-feature FP32 errors of the last search
 *   (host): min over thresholds and polarities of the feature's stump error,
 *   from FP32 prefix sums with a compensated carry.
 * Errors: VJB_ESTATE before the data exists; VJB_EINVAL for a range outside
 * [0, F); VJB_ECUDA. */
int vjb_get_integral(vjb_ctx *ctx, int32_t *out);
int vjb_feature_values(vjb_ctx *ctx, int64_t f0, int64_t nf, int32_t *out);
int vjb_sorted_rows(vjb_ctx *ctx, int64_t f0, int64_t nf, uint16_t *out);
int vjb_screen_errors(vjb_ctx *ctx, float *out);

/* ---- tuning ------------------------------------------------------------------
 * Launch shape of the search kernel.  Fields set to 0 keep their current
 * value.  Shapes whose shared memory does not fit one SM are rejected with
 * VJB_EINVAL.  Takes effect from the next round. */
typedef struct {
    int32_t warps;        /* consumer warps per CTA: 1-20 (1-16 unroll 3, 1-12 unroll 4) */
    int32_t stages;       /* TMA stages per warp: 1-8                              */
    int32_t ctas_per_sm;  /* 1-4                                                   */
    int32_t unroll;       /* 16-entry pieces a lane works on together: 1-4         */
    int32_t box_lines;    /* 128-byte lines per TMA box (stage): 4-32, a multiple of 4 */
} vjb_search_shape;

int vjb_set_search_shape(vjb_ctx *ctx, const vjb_search_shape *shape);
int vjb_get_search_shape(vjb_ctx *ctx, vjb_search_shape *out);

/* Round diagnostics of kept rounds [first, first + count) into out (host).
 * Errors: VJB_EINVAL for a range outside the kept rounds; VJB_ESTATE. */
int vjb_get_round_diag(vjb_ctx *ctx, int32_t first, int32_t count, vjb_round_diag *out);

/* ---- timing ------------------------------------------------------------------
 * vjb_set_timing: enable (1) or disable (0) event timing of rounds; enabling
 * also clears the accumulated figures.  vjb_get_timing: the figures of the
 * rounds run since (host `out`).  Errors: VJB_EINVAL; VJB_ECUDA. */
int vjb_set_timing(vjb_ctx *ctx, int32_t enable);
int vjb_get_timing(vjb_ctx *ctx, vjb_timing *out);

/* ---- the strong classifier ------------------------------------------------------
 * vjb_classify: the final hypothesis of Sec. 2.3 on n windows of the
 * context's size (host pixels [n][h][w], copied):
 *     score(x) = sum_t alpha_t h_t(x),  C(x) = 1 iff score(x) >= 1/2 sum_t alpha_t,
 * h_t(x) = 1 iff p_t f_t(x) < p_t theta_t, f_t feature `stumps[t].feature` of
 * vjb_enumerate_haar's list.  Sums are FP64 in stump order (both of them), so
 * the result is that of the same sums done one by one on the host; a stump
 * with alpha = +inf (a perfect stump) decides alone.  labels [n] receive
 * C(x), scores [n] (may be NULL) the scores.  Needs vjb_enumerate_haar.
 * Errors: VJB_EINVAL (a stump outside the feature list, polarity not +-1,
 * NaN alpha), VJB_ESTATE, VJB_ENOMEM, VJB_ECUDA. */
int vjb_classify(vjb_ctx *c, const uint8_t *pixels, int32_t n, const vjb_stump *stumps, int32_t T,
                 uint8_t *labels, double *scores);

/* ---- batches: many jobs per launch ------------------------------------------------
 * A batch trains many independent jobs (each its own windows, labels and
 * number of rounds) with one launch of each round kernel for all of them,
 * replayed as one CUDA graph per round.  Each job computes exactly what it
 * computes alone in a context (same kernels per row and per block): its
 * stumps and weights are bit-identical to a plain run.
 * The batch owns an HBM arena of `table_budget_bytes` for the jobs' sorted
 * tables (2 * F * npad bytes each, see vjb_batch_table_bytes); a job whose
 * table does not fit the free arena is rejected with VJB_EFULL.  Everything
 * else of a job lives in its own context, allocated when it is added.
 * At most 256 jobs; a job's n must leave its weights within 32768 floats
 * (every n up to VJB_MAX_SAMPLES does). */
typedef struct vjb_batch vjb_batch;

typedef struct {
    int32_t jobs;               /* jobs in the batch                                  */
    int32_t warps, stages, unroll, rows_per_warp;  /* search launch shape and schedule */
    int32_t box_lines;          /* lines per TMA stage                                */
    int64_t budget_bytes;       /* the table arena                                    */
    int64_t free_bytes;         /* free arena                                         */
    int64_t largest_free_bytes; /* largest free block (the largest table that fits)   */
    double  search_bytes;       /* algorithmic bytes of one batched search: sum 2 F N */
    int64_t launches;           /* kernels the batch has launched                     */
} vjb_batch_info;

/* Create a batch on `device` (stream may be NULL) with a table arena of
 * `table_budget_bytes`.  Errors: VJB_EINVAL, VJB_ENOMEM, VJB_ECUDA. */
int vjb_batch_create(vjb_batch **out, int device, void *cuda_stream, int64_t table_budget_bytes);
void vjb_batch_destroy(vjb_batch *b);

/* Arena bytes the sorted table of an n-sample h x w job needs. */
int vjb_batch_table_bytes(int32_t n, int32_t h, int32_t w, int64_t *bytes);

/* Add a job: copies its windows and labels (host, as vjb_load_windows),
 * builds its integral images, features and sorted table (in the arena) and
 * sets the Table 2 weights.  It will be trained until it has kept `rounds`
 * stumps (or training ends).  *job_id receives its id.  Errors: VJB_EFULL
 * (arena or slots), the errors of vjb_load_windows / vjb_enumerate_haar. */
int vjb_batch_add_job(vjb_batch *b, const uint8_t *pixels, const uint8_t *labels, int32_t n,
                      int32_t h, int32_t w, int32_t rounds, int32_t *job_id);

/* Remove a job and free its table space.  Errors: VJB_EINVAL (unknown id). */
int vjb_batch_remove_job(vjb_batch *b, int32_t job_id);

/* Run up to `max_rounds` batched rounds: every job that has kept fewer
 * stumps than its `rounds` and is not done takes part in each.
 * *rounds_run (may be NULL) receives the rounds launched.  Errors:
 * VJB_EDEVICE, VJB_ECUDA. */
int vjb_batch_train(vjb_batch *b, int32_t max_rounds, int32_t *rounds_run);

/* Autotuner of the batched search: times `trial_rounds` real rounds (after
 * one untimed round) with each of a list of launch shapes (warps, stages,
 * unroll, features per warp and work item) and keeps the fastest.  The rounds
 * count toward the jobs' training, whose results do not depend on the shape;
 * it stops trying when the jobs have fewer rounds left than a trial needs.
 * *rounds_run (may be NULL) receives the rounds it ran; `trials` (may be
 * NULL) up to `max_trials` timed shapes and *n_trials (may be NULL) their
 * number. */
typedef struct {
    int32_t warps, stages, unroll, rows_per_warp;  /* the shape tried                  */
    int32_t box_lines;                             /* lines per TMA stage              */
    float   ms_per_round;                          /* its timed rounds, on the device  */
} vjb_batch_trial;
int vjb_batch_autotune(vjb_batch *b, int32_t trial_rounds, int32_t *rounds_run, vjb_batch_trial *trials,
                       int32_t max_trials, int32_t *n_trials);

/* A job's kept stumps so far and its status (VJB_OK, VJB_DONE_*, or a
 * negative code if a kernel flagged it). */
int vjb_batch_job_state(vjb_batch *b, int32_t job_id, int32_t *rounds_done, int32_t *status);

/* A job's kept stumps [first, first + count) and its current weights (host). */
int vjb_batch_get_stumps(vjb_batch *b, int32_t job_id, int32_t first, int32_t count, vjb_stump *out);
int vjb_batch_get_weights(vjb_batch *b, int32_t job_id, float *out);

/* Launch shape of the batched search (stage height box_lines: a multiple of 4
 * up to 32 lines) and its schedule (rows_per_warp):
 *  - VJB_BATCH_INTERLEAVED (the default): the plain search's row order, one
 *    job after the other: warp w of the grid's G warps takes rows w, w + G, ...
 *    so the whole GPU streams one compact window of consecutive rows; a CTA
 *    synchronises at every job;
 *  - VJB_BATCH_PARTITIONED: each CTA takes one contiguous range of all jobs'
 *    rows with the same number of table lines (recomputed each round for the
 *    jobs taking part), so it synchronises once or twice a round;
 *  - > 0: a queue of work items of that many rows per warp.
 * Results do not depend on the choice.  A field or rows_per_warp of 0 keeps
 * its value. */
#define VJB_BATCH_PARTITIONED (-1)
#define VJB_BATCH_INTERLEAVED (-2)
int vjb_batch_set_search_shape(vjb_batch *b, const vjb_search_shape *shape, int32_t rows_per_warp);
int vjb_batch_get_info(vjb_batch *b, vjb_batch_info *out);

/* CUDA-event timing of every batched round: as vjb_set_timing / vjb_get_timing
 * (enabling resets the totals; search = the batched search kernel). */
int vjb_batch_set_timing(vjb_batch *b, int32_t enable);
int vjb_batch_get_timing(vjb_batch *b, vjb_timing *out);

/* ---- serving: continuous batching of training requests ------------------------------
 * A server trains requests as they arrive, many at a time, in one batch on
 * one GPU.  A request (windows, labels, round count) waits in arrival order
 * until its sorted table fits the free part of the table budget and a job
 * slot is free; later requests may overtake one that does not fit, at most 8
 * times.  An admitted request is prepared (integral images, features, sorted
 * table) by a worker thread on a low-priority stream while the batch keeps
 * training the others on a high-priority one (the worker also frees the
 * contexts of finished requests), joins the batch at the next round and
 * leaves it when it has
 * kept `rounds` stumps (or stops early); its table space then goes to the
 * requests still waiting.  Each request's stumps and weights are those of a
 * plain run of the same job (see the batch section).
 * Times are host milliseconds since the server was created; round times
 * are CUDA-event durations of whole batched rounds. */
typedef struct vjb_server vjb_server;

#define VJB_REQ_QUEUED    0
#define VJB_REQ_PREPARING 1
#define VJB_REQ_TRAINING  2
#define VJB_REQ_DONE      3
#define VJB_REQ_FAILED    4

typedef struct {
    int64_t request_id;
    int32_t state;            /* VJB_REQ_*                                            */
    int32_t status;           /* VJB_OK, VJB_DONE_* or a negative code (failed)       */
    int32_t rounds_done;      /* stumps kept so far                                  */
    int32_t rounds_target;
    int32_t n, h, w;
    int32_t rounds_timed;     /* batched rounds it took part in                       */
    int32_t pad;
    int64_t table_bytes;      /* its share of the table budget                        */
    double  t_submit_ms, t_admit_ms, t_ready_ms, t_done_ms;  /* -1 until reached      */
    double  round_ms_sum;     /* summed duration of the rounds it took part in        */
} vjb_request_info;

typedef struct {
    int32_t queued, preparing, training, done, failed, pad;
    int64_t rounds;           /* batched rounds run                                   */
    int64_t job_rounds;       /* rounds summed over the jobs in them                  */
    int64_t budget_bytes, free_bytes;
    double  round_ms_total;   /* device time of all batched rounds                    */
    double  clock_ms;         /* time since creation                                  */
} vjb_server_summary;

/* Create a server on `device` with `table_budget_bytes` of HBM for sorted
 * tables and at most `max_jobs` (1-256) requests admitted at once. */
int vjb_server_create(vjb_server **out, int device, int64_t table_budget_bytes, int32_t max_jobs);
/* Stops the worker (requests still queued are dropped) and frees everything. */
void vjb_server_destroy(vjb_server *s);

/* Queue a request (host windows [n][h][w] and labels [n], copied).  Errors:
 * VJB_EINVAL (sizes, labels), VJB_EFULL (its table exceeds the whole budget). */
int vjb_server_submit(vjb_server *s, const uint8_t *pixels, const uint8_t *labels, int32_t n, int32_t h,
                      int32_t w, int32_t rounds, int64_t *request_id);

/* One scheduling step: admit what fits, take in prepared requests, then run
 * up to `max_rounds` batched rounds, retiring finished jobs and admitting
 * waiting requests between rounds.  When nothing trains but a request is
 * being prepared it waits for it up to 5 ms.  *rounds_run (may be NULL)
 * receives the rounds run. */
int vjb_server_step(vjb_server *s, int32_t max_rounds, int32_t *rounds_run);

/* State and times of a request. */
int vjb_server_request(vjb_server *s, int64_t request_id, vjb_request_info *out);

/* A finished request's stumps (`cap` of room; may be NULL) and final
 * weights ([n], may be NULL).  Returns its status; VJB_ESTATE while it runs. */
int vjb_server_result(vjb_server *s, int64_t request_id, vjb_stump *stumps, int32_t cap, float *weights);

/* Forget a finished request. */
int vjb_server_release(vjb_server *s, int64_t request_id);

int vjb_server_stats(vjb_server *s, vjb_server_summary *out);

/* Duration and job count of batched rounds [first, first + count). */
int vjb_server_round_times(vjb_server *s, int64_t first, int32_t count, float *ms, int32_t *jobs);

/* ---- allocation-free search ----------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory when they want a search -- a real-time
 * loop whose memory is fixed up front (a cudaMalloc can wait on the whole
 * device), or a framework whose pool owns all device memory.
 *
 * vjb_screen_noalloc runs the per-round FP32 screen (the search kernel of
 * vjb_train_round, without its compensated re-scan) over a caller-owned
 * sorted table and allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library routine.  Its scratch (one partial per CTA and a
 * counter) is a file-scope device array of 8.4 KiB that every GPU loading
 * the library holds until the process exits; at most 1024 CTAs fit it.
 *
 * Arguments (all pointers are device memory on the current device, owned by
 * the caller):
 *   rows          [nfeat][npad] uint16 sorted table, 16-byte aligned: entry =
 *                 sample index (bits 0-14) | bit 15 when the value at this
 *                 position is below the next one; positions n .. npad-1
 *                 hold n.  Entries naming a sample above n read as padding.
 *   v             [n + 1] float: +w_i for a face, -w_i for a non-face,
 *                 v[n] = 0.
 *   n, npad       samples (1 .. VJB_MAX_SAMPLES) and row length (a multiple
 *                 of 64, >= n).
 *   nfeat         features (rows), 1 .. 2^31 - 1.
 *   t_pos, t_neg  face and non-face weight totals (finite, >= 0).
 *   ctas          CTAs to launch, 0 = one per SM; at most 1024.
 *   feature_err   [nfeat] float out: each feature's least stump error.
 *   best_err      [1] float out: the smallest of them; NaN if a TMA wait
 *                 timed out.
 *   best_feature  [1] int32 out: its feature (lowest index on ties), or -1
 *                 if a TMA wait timed out (feature_err is then undefined)
 *                 or no feature has an error that is not NaN (NaN weights;
 *                 best_err is then +inf).
 *   cuda_stream   cudaStream_t to run on (NULL: the legacy default stream).
 * The call is asynchronous on the stream.  The first call on a device does
 * that device's set-up (the scratch array's device address, the kernel's
 * shared-memory limit); make that first call before any stream capture.
 * Every call shares the one scratch array, so calls that overlap on the GPU
 * (on two streams, or from two host threads) race; serialise them.
 * Errors: VJB_EINVAL (a size or pointer outside the limits above, or ctas
 * above 1024), VJB_ECUDA; vjb_last_error() gives the message. */
int vjb_screen_noalloc(const uint16_t *rows, const float *v, int32_t n, int32_t npad,
                       int64_t nfeat, double t_pos, double t_neg, int32_t ctas,
                       float *feature_err, float *best_err, int32_t *best_feature,
                       void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* VJB_H */
