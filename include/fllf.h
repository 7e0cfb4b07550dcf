/*
 * fllf.h -- C ABI of the GB300 Fourier local Laplacian filter (libfllf.so).
 *
 * The filter is Fourier LLF (Sumiya, Otsuka, Maeda, Fukushima, "Gaussian
 * Fourier Pyramid for Local Laplacian Filter", IEEE SPL, arXiv 2206.04681).
 * Local Laplacian filtering (Sec. II-C) remaps the input about every
 * pyramid coefficient's own Gaussian value g = G_l[I]_p and keeps the
 * remapped Laplacian coefficient; Fourier LLF expands the remap detail in a
 * sine series (Eqs. (9)-(11)) so that only 2K+1 pyramids are needed
 * (Eq. (14), Fig. 1).  With the remap
 *
 *     r_g(i) = i + f(i - g),  f(d) = (m - 1) d exp(-d^2 / (2 sigma_r^2)),
 *     f(d) ~= sum_{k=1..K} a_k sin(omega_k d),  omega_k = 2 pi k / T,
 *
 * every output Laplacian level below the top is
 *
 *     L_l[O] = L_l[I] + sum_k a_k [cos(omega_k G_l[I]) L_l[sin(omega_k I)]
 *                                - sin(omega_k G_l[I]) L_l[cos(omega_k I)]],
 *
 * the top level is G_top[I], and O is the collapse of Eq. (4).  Pyramids use
 * the 5-tap binomial kernel [1 4 6 4 1]/16 with reflect-101 borders at every
 * level; coarse sizes are ceil(n/2).
 *
 * Conventions for every entry point:
 *   - Every call returns an fllf_status; no C++ exception crosses the ABI.
 *     On an error, fllf_last_error() returns a thread-local description.
 *   - Images are planar float32, C x H x W, contiguous (row pitch W, plane
 *     pitch H*W).  Values are expected in [0, 1] (the period T is chosen for
 *     that range); values outside it are filtered as-is, without clamping.
 *   - Device pointers are CUDA device addresses on the plan's device; host
 *     pointers are ordinary (preferably pinned) host memory.
 *   - Stream arguments are cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Device-pointer calls only enqueue work on that
 *     stream; results are valid once the stream reaches that point.
 *   - Output buffers are written only when the call returns FLLF_OK.
 */
#ifndef FLLF_H
#define FLLF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FLLF_OK = 0,
  FLLF_EINVAL = 1,   /* invalid argument or parameter set */
  FLLF_ENOMEM = 2,   /* device or host allocation failed; nothing leaked */
  FLLF_ECUDA = 3,    /* a CUDA call failed; see fllf_last_error() */
  FLLF_EAGAIN = 4,   /* asynchronous work still pending */
  FLLF_ETIMEOUT = 5, /* a bounded wait ran out */
  FLLF_EBUSY = 6     /* no slot or memory free and the queue is full */
} fllf_status;

/* Storage type of the 2K Gaussian Fourier pyramids (Sec. III-A, Fig. 1).
 * Arithmetic is float32 in every mode; the guide pyramid G_l[I], the
 * residual collapse and the output are always float32. */
typedef enum { FLLF_FP32 = 0, FLLF_FP16 = 1, FLLF_BF16 = 2 } fllf_precision;

/* How a_k is obtained from (m, sigma_r, T, K). */
typedef enum {
  FLLF_COEFF_QUADRATURE = 0, /* (2/T) * integral over one period of f(x) sin(omega_k x) */
  FLLF_COEFF_CLOSED_FORM = 1 /* Eqs. (9)-(11): (m-1) 2 sigma_r^2 alpha_k omega_k */
} fllf_coeff_mode;

/* Which local Laplacian filter a plan computes. */
typedef enum {
  FLLF_METHOD_FOURIER = 0, /* Fourier LLF (Sec. III, Eq. (14)): 2K+1 pyramids */
  FLLF_METHOD_FAST = 1     /* fast LLF (Sec. II-D), the paper's comparison method:
                            * S samples g_j = j / (S - 1) of [0, 1], the Laplacian
                            * pyramids of the remapped images r(I, g_j) with the
                            * exact remap, linearly interpolated at each pixel
                            * between the two samples bracketing G_l[I]_p; S + 1
                            * pyramids.  The S sampled pyramids are held as
                            * ceil(S/2) complex planes (pairs of samples), so a
                            * fast plan's K is ceil(S/2); K, T and coeff_mode are
                            * not used.  Not available in batches, the server or
                            * fllf_run_adaptive. */
} fllf_method;

typedef struct {
  int H, W;          /* image size, >= 1 each */
  int C;             /* planes filtered independently (1 = gray, 3 = planar RGB), 1..64 */
  int levels;        /* pyramid levels including level 0; 1..16 (top = levels-1) */
  int K;             /* Fourier orders, 1..64 (2K+1 pyramids) */
  double m;          /* remap gain: 1 = identity, > 1 enhances, < 1 smooths */
  double sigma_r;    /* remap range scale, > 0 */
  double T;          /* Fourier period, > 0 (2 covers differences in [-1, 1]) */
  int precision;     /* fllf_precision */
  int coeff_mode;    /* fllf_coeff_mode */
  int method;        /* fllf_method (0: Fourier LLF) */
  int samples;       /* fast LLF: intensity samples S, 2..128 (unused by Fourier LLF) */
} fllf_params;

typedef struct fllf_plan fllf_plan;

/* Human-readable name of a status code (static string). */
const char *fllf_status_str(fllf_status s);

/* Detail text of the last error raised on the calling thread ("" if none). */
const char *fllf_last_error(void);

/* Checks a parameter set: FLLF_OK or FLLF_EINVAL with the reason. */
fllf_status fllf_params_validate(const fllf_params *p);

/* Fourier sine coefficients a_1..a_K of the remap detail f for this
 * parameter set, in float64 (Eqs. (9)-(11); quadrature or closed form per
 * coeff_mode).  a_out: host array of p->K doubles, written on FLLF_OK. */
fllf_status fllf_coeffs(const fllf_params *p, double *a_out);

/* Fourier period of Eq. (12): the T minimising
 *     E_K(T) = erfc(pi sigma_r (2K + 1) / T) + erfc((T - R) / sigma_r)
 * for an R-tone image (R = 1 for images in [0, 1], 256 for 8-bit ones),
 * the bound on the cosine-series error of the Gaussian w_r used by
 * Eqs. (9)-(10).  Host only (no device work).  sigma_r > 0, R > 0, finite,
 * 1 <= K <= 64, T_out non-NULL; otherwise FLLF_EINVAL.  *T_out is written
 * on FLLF_OK.  Example: sigma_r = 30, K = 10, R = 256 gives 405.5 (the
 * paper prints 405.9 for its experiments). */
fllf_status fllf_optimal_period(double sigma_r, int K, double R, double *T_out);

/* Bytes of device scratch a plan for this parameter set allocates: the
 * guide pyramid G_l (l >= 1), the Fourier pyramids Z_l (K complex planes
 * per level l >= 1, in the storage precision) and the residual pyramid
 * E_l = O_l - G_l (1 <= l <= levels-2), for all C planes.  0 if invalid. */
size_t fllf_plan_scratch_bytes(const fllf_params *p);

/* Creates a plan on CUDA device `device`: validates p, computes a_k on the
 * host in float64, uploads them as float32, and allocates the scratch.
 * On failure nothing stays allocated and *out is NULL.  The caller owns the
 * plan and frees it with fllf_plan_destroy. */
fllf_status fllf_plan_create(const fllf_params *p, int device, fllf_plan **out);

/* Frees the plan and its scratch; NULL is accepted.  The caller must make
 * sure no work of the plan is still running on any stream, and poll every
 * ticket of the plan (fllf_submit, fllf_submit_host) to completion first. */
fllf_status fllf_plan_destroy(fllf_plan *plan);

/* Copies the plan's parameters (a fast LLF plan reports K = ceil(samples/2))
 * / float64 coefficients (K doubles; FLLF_EINVAL for a fast LLF plan). */
fllf_status fllf_plan_params(const fllf_plan *plan, fllf_params *out);
fllf_status fllf_plan_coeffs(const fllf_plan *plan, double *a_out);

/* Filters one C x H x W image: d_in -> d_out, both device pointers on the
 * plan's device, non-overlapping (d_in == d_out is FLLF_EINVAL).  Enqueues
 * the kernels on `stream` and returns; the plan's scratch is in use until
 * the stream passes this work, so one plan must not run concurrently on two
 * streams. */
fllf_status fllf_run(fllf_plan *plan, const float *d_in, float *d_out, void *stream);

/* Pixel-by-pixel enhancement (Sec. III-B): filters like fllf_run, but the
 * remap gain m is a per-pixel map instead of the plan's constant (Fourier
 * LLF plans only; a fast LLF plan gets FLLF_EINVAL).  The
 * Gaussian Fourier pyramids do not depend on the remap, so only the
 * coefficients change: at level l < top the Fourier term of Eq. (14) is
 * scaled by (m_{l,p} - 1) / (m - 1), where m is the plan's gain and
 * m_{l,p} = G_l[gain]_p is the Gaussian pyramid of the map at that pixel
 * (a constant map reproduces fllf_run with that gain).
 *   d_gain: device H x W float32 map (row pitch W) of the gain m_p, shared
 *           by the C planes; read only.
 *   The plan's m must differ from 1 (FLLF_EINVAL otherwise); sigma_r, T and
 *   K stay the plan's.  The map's pyramid lives in a plan-owned device
 *   buffer allocated on the first call.  d_in, d_out and d_gain must not
 *   overlap d_out.  Stream-ordered like fllf_run. */
fllf_status fllf_run_adaptive(fllf_plan *plan, const float *d_in, const float *d_gain, float *d_out,
                              void *stream);

/* Colour by luma, the colour processing of the paper's experiments
 * (Sec. IV): LLF is applied to the Y channel of YUV and the other
 * components are kept.  YUV is BT.601 (Y = 0.299 R + 0.587 G + 0.114 B);
 * keeping U and V means every output channel is the input channel plus
 * Y' - Y, with Y' the filtered luma.
 *   plan: C == 1 (it filters the H x W luma plane), otherwise FLLF_EINVAL.
 *   d_rgb_in, d_rgb_out: device planar RGB, 3 x H x W float32, not
 *   overlapping.  Two plan-owned H x W luma buffers are allocated on the
 *   first call.  Stream-ordered like fllf_run. */
fllf_status fllf_run_luma(fllf_plan *plan, const float *d_rgb_in, float *d_rgb_out, void *stream);

/* End-to-end variant for host buffers: copies h_in to a plan-owned device
 * buffer, filters, copies the result to h_out and waits for the work.
 * Allocates the two device I/O buffers on first use (kept by the plan).
 * With C >= 2 planes the planes are pipelined: the plan's two copy streams
 * (created on first use) move plane c in and plane c-2 out while `stream`
 * filters plane c-1, each plane on a one-plane view of the plan's scratch;
 * the output is the same as fllf_run's, bit for bit.  Pinned host buffers
 * let the copies overlap. */
fllf_status fllf_run_host(fllf_plan *plan, const float *h_in, float *h_out, void *stream);

/* Asynchronous form of fllf_run: enqueues the work and records a
 * completion event; *ticket identifies it for fllf_poll.  After the run a
 * one-thread kernel copies the plan's fault word into a host-mapped word
 * (64 per plan, one per pending ticket of fllf_submit or fllf_submit_host;
 * allocated on first use), which fllf_poll reads without a device-to-host
 * copy; so each ticket reports a bounded wait that gave up in its own run or
 * an earlier one.  Tickets beyond 64 pending read the device word. */
fllf_status fllf_submit(fllf_plan *plan, const float *d_in, float *d_out, void *stream,
                        uint64_t *ticket);

/* Asynchronous end-to-end form for host buffers, for a stream of frames.
 * Enqueues three steps and returns with *ticket for fllf_poll, which
 * reports the frame done once h_out holds its result:
 *   1. the copy of h_in into one of the plan's two device staging slots
 *      (the plan's host-to-device copy stream);
 *   2. the filtering of the whole frame on `stream` (fllf_run's path, the
 *      same bits);
 *   3. the copy of the result to h_out (the device-to-host copy stream).
 * Successive submits take the slots in turn, so frame n+1's input copy and
 * frame n-1's output copy overlap frame n's filtering.  A slot is reused
 * only after its previous frame was filtered (input) and copied back
 * (output); events order this on the device, without a host wait.
 *   h_in, h_out: host, H x W x C float32 planar; h_in must stay unchanged
 *   and h_out unread until the ticket is done.  Pinned memory lets the
 *   copies run asynchronously; pageable memory works, with copies that
 *   block the caller.
 *   Allocates the two slots (4 frame buffers) and the copy streams on the
 *   first call (kept by the plan; FLLF_ENOMEM if the slots do not fit).
 *   Like fllf_run, one plan's runs share its scratch: submit them on one
 *   stream.  A kernel's bounded wait that gave up is reported by fllf_poll
 *   (FLLF_ETIMEOUT), from the frame's fault-word snapshot as for
 *   fllf_submit. */
fllf_status fllf_submit_host(fllf_plan *plan, const float *h_in, float *h_out, void *stream,
                             uint64_t *ticket);

/* Waits up to timeout_us microseconds (0 = just test, < 0 = up to
 * FLLF_POLL_MAX_US) for a submitted ticket.  FLLF_OK: done (ticket
 * consumed); FLLF_EAGAIN: still running after a zero timeout;
 * FLLF_ETIMEOUT: still running after the timeout (the ticket stays valid),
 * or the work finished but one of its kernels' bounded waits gave up
 * (ticket consumed, output undefined); FLLF_EINVAL: unknown or already
 * consumed ticket; FLLF_ECUDA: the work failed on the device. */
#define FLLF_POLL_MAX_US 60000000
fllf_status fllf_poll(uint64_t ticket, int timeout_us);

/* ---- Batched execution ------------------------------------------------------
 * A batch groups n plans (same device and storage precision; each with its
 * own size, levels, K and remap) so that one launch per stage kind and level
 * covers every image, or one persistent dataflow launch covers every stage of
 * every image (see fllf_batch_set_mode): the REDUCE and combine work items
 * of all images share the persistent grids, and small images and small
 * levels fill the GPU beside large ones.  The launch sequence is captured in
 * a CUDA graph at the first run and replayed afterwards.  The batch uses the plans' scratch:
 * a plan must not run on its own while a batch that holds it is running, and
 * the plans must outlive the batch. */
typedef struct fllf_batch fllf_batch;

/* Builds the batch's argument tables (device memory owned by the batch). */
fllf_status fllf_batch_create(fllf_plan *const *plans, int n, fllf_batch **out);

/* Frees the batch (not the plans); NULL is accepted. */
fllf_status fllf_batch_destroy(fllf_batch *batch);

/* Filters image i of the batch from d_in[i] to d_out[i] (device pointers,
 * planar C x H x W of plan i, non-overlapping) for every i, enqueued on
 * `stream`.  Host arrays d_in / d_out are read before the call returns. */
fllf_status fllf_batch_run(fllf_batch *batch, const float *const *d_in, float *const *d_out,
                           void *stream);

/* After the batch's work completed: FLLF_ETIMEOUT if a kernel's bounded wait
 * ran out (the status is then cleared), else FLLF_OK. */
fllf_status fllf_batch_check(fllf_batch *batch);

/* One-shot form of the above (the batch call of the boundary, with the plans
 * passed directly): builds a batch of the n plans, filters d_in[i] ->
 * d_out[i] for every i on `stream`, waits for the stream, reports a bounded
 * wait that gave up (FLLF_ETIMEOUT) and frees the batch.  Synchronous; the
 * batch's small argument tables are allocated and freed inside.  Keep a
 * fllf_batch for repeated runs of the same plans. */
fllf_status fllf_batch_run_plans(fllf_plan *const *plans, const float *const *d_in, float *const *d_out,
                                 int n, void *stream);

/* ---- Serving: continuous batching of filter requests ----------------------
 * A server owns one device memory pool of `hbm_budget` bytes (allocated at
 * creation) and a worker thread.  Requests (any size, levels, K, remap,
 * storage precision) wait in a FIFO queue; the worker admits them as slots
 * (at most `max_slots` requests admitted and not finished) and pool memory
 * for their pyramids free up, builds their plans inside the pool (no device
 * allocation per request), and launches each group admitted together as a
 * batched wave on one of `max_waves` streams, so requests that arrive while
 * others run are admitted and overlap them on the device.  A request's
 * result does not depend on the other requests it shares a wave with.
 * Plans stay resident: the coefficients of every parameter set seen (m,
 * sigma_r, T, K, coefficient mode) are cached on the host and in a device
 * slot; a new set's quadrature runs in fllf_server_submit on the caller's
 * thread, and admission only encodes the request's tensor maps for its pool
 * range.
 * Latency is measured from fllf_server_submit to the worker seeing the
 * request's wave complete. */
typedef struct fllf_server fllf_server;

typedef struct {
  uint64_t submitted, completed, rejected;
  double p50_ms, p99_ms, mean_ms, max_ms; /* latency of completed requests */
  double mpixel_per_s;   /* H*W of completed requests / (last completion - first submit) */
  size_t pool_bytes, pool_peak_bytes;
  int max_active;        /* peak number of admitted, unfinished requests */
  int waves;             /* waves launched */
  uint64_t plan_cache_hits;     /* submissions whose coefficient set was resident */
  uint64_t plan_cache_misses;   /* submissions that computed theirs (in fllf_server_submit) */
  uint64_t admission_quadratures; /* coefficient quadratures run at admission (always 0) */
} fllf_server_stats;

/* Creates a server on `device`.  hbm_budget: pool bytes (>= 1 MiB); max_slots:
 * 1..4096; max_queue: pending requests before FLLF_EBUSY (>= 1);
 * max_waves: concurrent waves (streams), 1..16. */
fllf_status fllf_server_create(int device, size_t hbm_budget, int max_slots, int max_queue,
                               int max_waves, fllf_server **out);

/* Stops the worker after the waves in flight finish, and frees the server.
 * Requests not yet admitted are cancelled; NULL is accepted.  No call on the
 * server may run concurrently with or after this one. */
fllf_status fllf_server_destroy(fllf_server *server);

/* Queues a request: d_in (read) and d_out (written) are caller-owned device
 * buffers (planar C x H x W float32, non-overlapping) that must stay valid
 * until fllf_server_poll returns FLLF_OK for the ticket.  FLLF_EBUSY: the
 * queue is full; FLLF_ENOMEM: the request can never fit in the pool. */
fllf_status fllf_server_submit(fllf_server *server, const fllf_params *p, const float *d_in,
                               float *d_out, uint64_t *ticket);

/* Waits up to timeout_us (0 = test only, < 0 = up to FLLF_POLL_MAX_US) for a request.
 * FLLF_OK: finished, d_out holds the result (ticket consumed);
 * FLLF_EAGAIN / FLLF_ETIMEOUT: still pending; FLLF_EINVAL: unknown ticket;
 * FLLF_ECUDA: the request's wave failed, or one of its kernels' bounded waits
 * gave up (ticket consumed, d_out undefined).  Thread-safe. */
fllf_status fllf_server_poll(fllf_server *server, uint64_t ticket, int timeout_us);

/* Statistics since creation or the last reset. */
fllf_status fllf_server_stats_get(fllf_server *server, fllf_server_stats *out);
fllf_status fllf_server_stats_reset(fllf_server *server);

/* ---- Filtering without any device allocation -------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc (code running inside a memory pool or an
 * allocator it does not own, real-time loops where an allocation could block
 * or fragment memory, plugin hosts that hand out only the image buffers).
 *
 * fllf_run_noalloc filters one C x H x W image (d_in -> d_out, device
 * pointers on the current device, non-overlapping) exactly like fllf_run
 * with a plan of the same parameters, but keeps the coefficients and the
 * guide, Fourier and residual pyramids in one fixed device array compiled
 * into the library (FLLF_NOALLOC_SCRATCH_BYTES per GPU, held by every GPU
 * that loads the library until the process exits).  It allocates no device
 * memory and enqueues on `stream`.
 *   - Returns FLLF_EINVAL, with the byte counts in fllf_last_error(), when
 *     the parameter set needs more scratch than the array holds
 *     (fllf_plan_scratch_bytes(p) + 512 bytes must fit), and for the usual
 *     invalid arguments.
 *   - All calls on one GPU share the array, which keeps the last call's
 *     contents; calls whose GPU work overlaps (two streams or threads)
 *     race on it, so serialise them.  Each call starts by clearing the
 *     array's status words; the pyramids need no clearing.
 *   - The coefficients reach the device as a by-value kernel argument, so
 *     nothing reads host memory after the call returns.
 *   - The first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress on the current device (this may load the
 *     module), so make the first call before any stream capture.  The
 *     address is kept until the process exits: do not call this across a
 *     cudaDeviceReset.
 *   - A kernel's bounded wait that gives up (about 2 s) is not reported:
 *     the call has already returned FLLF_OK and the output is incomplete.
 *     fllf_run_host or fllf_poll on a plan do report it (FLLF_ETIMEOUT). */
#define FLLF_NOALLOC_SCRATCH_BYTES (32u << 20)
fllf_status fllf_run_noalloc(const fllf_params *p, const float *d_in, float *d_out, void *stream);

/* ---- Diagnostics: per-stage device timing -------------------------------
 * Stage kinds of the path (Fig. 1 read as a pipeline): */
enum {
  FLLF_STAGE_UP0 = 0,   /* level 0 -> 1: trig of I + REDUCE of I and the 2K Fourier images */
  FLLF_STAGE_UP = 1,    /* level l -> l+1 REDUCE of G_l and Z_l (Eq. (1)) */
  FLLF_STAGE_DOWN = 2,  /* level l >= 1: Eq. (14) product-sum fused with the collapse */
  FLLF_STAGE_DOWN0 = 3, /* level 0: Eq. (14) l = 0 case + final collapse, writes O */
  FLLF_STAGE_CHAIN = 4, /* the small levels (REDUCE up, then combines down) in one launch */
  FLLF_STAGE_DOWN_S = 5, /* level l >= 2 below small_pixels: FLLF_STAGE_DOWN on 32 x 16 tiles */
  FLLF_STAGE_GRAPH = 6,  /* every stage in one persistent dataflow launch (fllf_tuning.dataflow) */
  FLLF_NSTAGE = 7
};

/* When enabled, every run of the plan records CUDA events around each
 * kernel launch on the run's stream.  Adds no synchronisation. */
fllf_status fllf_plan_enable_timing(fllf_plan *plan, int enable);

/* Times only the stage kinds whose bit is set in `mask` (bit k = stage kind
 * k; 0 disables timing), so that a measurement of one kernel adds no events
 * around the others. */
fllf_status fllf_plan_set_timing_mask(fllf_plan *plan, unsigned mask);

/* Waits for the recorded events, then writes per stage kind the summed
 * kernel time in milliseconds (ms[FLLF_NSTAGE]) and the number of launches
 * (launches[FLLF_NSTAGE]) since the last call, and clears the record. */
fllf_status fllf_plan_stage_times(fllf_plan *plan, double *ms, int *launches);

/* Host-only check of the dataflow launch's task list (no device work): builds
 * the list for n parameter sets (one batch; n == 1 is a plan's own list) with
 * the given task sizes (task_items[5] as in fllf_tuning, NULL = defaults),
 * with or without the fused level-1/level-0 combine, and from first_level up
 * (0: every stage; 2..15: the list of dataflow mode 3), then runs it in
 * order on one host worker.  FLLF_OK when every work item of every stage is in
 * exactly one task, every task comes after the tasks whose row bands it
 * reads, and every band reaches the count its readers wait for;
 * FLLF_EINVAL with the reason otherwise.  *ntasks, *nbands (may be NULL):
 * the list's size. */
fllf_status fllf_dataflow_check(const fllf_params *ps, int n, const int *task_items, int with_d10,
                                int first_level, int *ntasks, int *nbands);

/* Test hook for the bounded device waits (failure detection; the paper has
 * no counterpart).  Every wait in the kernels gives up
 * after about 2 s of SM clock, sets the plan's fault word and leaves the
 * kernel, and the host reports FLLF_ETIMEOUT.  This sets, for the plan's next
 * runs, a shorter limit (wait_cycles > 0, in SM cycles; 0 = the default) and
 * a number of arrivals that the grid barriers of the chained launch
 * (fllf_tuning.chain_pixels > 0) wait for beyond the grid (0 = none): with a
 * positive count no barrier can complete, so each one gives up after the
 * limit, with no copy in flight.  Both settings are cleared when a run
 * reports the timeout.  Synchronises the device. */
fllf_status fllf_plan_set_wait_test(fllf_plan *plan, long long wait_cycles, unsigned extra_arrivals);

/* ---- Launch tuning and the autotuner ---------------------------------------
 * The kernels' tile shapes and orders per chunk are fixed at compile time
 * (they set the TMA box geometry and the thread mappings).  What a plan can
 * tune at run time is how the path is launched:
 *   chain_pixels    levels >= 2 whose planes hold at most this many pixels
 *                   (over all C planes) run in one chained cooperative launch
 *                   with grid barriers between stages; 0 = no chained launch
 *                   (default: with programmatic dependent launch between the
 *                   per-level kernels, separate launches measured faster at
 *                   every size from 512 x 512 to 8K RGB).
 *   ctas_per_sm[k]  resident CTAs per SM of the persistent grid of stage kind
 *                   k (FLLF_STAGE_*); 0 = as many as fit (default).
 *   reduce_reverse  1 (default): the level 1 -> 2 REDUCE visits its work
 *                   items last to first, reading what the level-0 REDUCE
 *                   wrote last while it is still in L2.
 *   small_pixels    combines at levels >= 2 (outside the chained launch)
 *                   whose planes hold at most this many pixels run on
 *                   32 x 16 tiles with two pixels per thread
 *                   (FLLF_STAGE_DOWN_S) instead of 64 x 32 tiles with eight:
 *                   four times the tiles and a quarter of each thread's
 *                   serial work.  Default 2^40 (every level: the small tiles
 *                   measured as fast or faster at every size tried); 0 = never.
 *   dataflow        1: every stage of a Fourier LLF run without a gain map
 *                   in ONE persistent launch (FLLF_STAGE_GRAPH): the stages
 *                   are cut into tasks of a few tiles of one row band; a
 *                   band's tasks are pushed onto a device queue once every
 *                   row band they read is complete, and the CTAs pop ready
 *                   tasks, so the REDUCE of a level starts on the first rows
 *                   the level below has finished and no launch boundary
 *                   separates the levels.  2: the same without the fused
 *                   level-1/level-0 combine, which follows as its own
 *                   kernel.  3: the stages below dataflow_level as their own
 *                   kernels and one dataflow launch for the REDUCE from that
 *                   level to the top and the combines back down to it (the
 *                   small, latency-bound levels).  0 (default; measured
 *                   faster at 4K RGB): one launch per stage kind and level
 *                   (the settings above).
 *                   The same stage code on the same work items: the same
 *                   output, bit for bit.
 *   task_items[5]   work items per task of the dataflow launch for the
 *                   level-0 REDUCE (tiles of 32 x 14 level-1 outputs), the
 *                   REDUCE at levels >= 1 (tile-chunks; at level 1, halved
 *                   per level above), the combines at levels >= 2 (32 x 16
 *                   tiles; at level 2, halved per level above), the fused
 *                   level-1/0 combine (64 x 32 tiles) and the level-0
 *                   combine of 2-level images; 1..4096 each, 0 = the
 *                   default (4, 8, 4, 2, 4).
 *   dataflow_level  first level of the dataflow launch of mode 3: 2..15, or
 *                   0 for the default (3).
 *   reduce_bands    > 1: the level-0 REDUCE and the level 1 -> 2 REDUCE run
 *                   in this many row bands (all planes in turn), each band
 *                   of the level-1 REDUCE launched right after the level-0
 *                   band that completes its inputs, so that it reads Z_1
 *                   while it is still in L2; 0 or 1: one launch each
 *                   (default).  0..256.
 * Every setting computes the same output, bit for bit. */
typedef struct {
  long long chain_pixels;
  int ctas_per_sm[FLLF_NSTAGE];
  int reduce_reverse;
  long long small_pixels;
  int dataflow;
  int task_items[5];
  int dataflow_level;
  int reduce_bands;
} fllf_tuning;

/* Reads / replaces a plan's launch tuning.  set: chain_pixels >= 0,
 * small_pixels >= 0, ctas_per_sm 0..32, reduce_reverse 0 or 1, dataflow 0
 * to 3, task_items 0..4096, dataflow_level 0 or 2..15, reduce_bands 0..256;
 * otherwise FLLF_EINVAL.  A change of task_items
 * rebuilds the plan's task list (allocates its tables anew; synchronises the
 * device). */
fllf_status fllf_plan_get_tuning(const fllf_plan *plan, fllf_tuning *out);
fllf_status fllf_plan_set_tuning(fllf_plan *plan, const fllf_tuning *t);

/* Autotuner: times the plan on d_in -> d_out (device buffers as for
 * fllf_run; d_out is overwritten many times) with CUDA events on `stream`,
 * `reps` timed runs per candidate after one untimed run, each timed run
 * after an L2 flush (it allocates a buffer of twice the L2 size for the
 * search and frees it; FLLF_ENOMEM if that fails).  It searches by
 * coordinate descent, from the plan's current tuning: first the dataflow
 * launch against the per-stage launches; with the dataflow launch, its
 * resident CTAs per SM and the task sizes of each stage kind; otherwise the
 * chain start (0, 2^15, 2^17, 2^19, 2^21, 2^23 pixels), the small-tile
 * threshold (0 or the pixel count of a combined level >= 2), the resident
 * CTAs per SM of each stage kind (1 .. as many as fit), the REDUCE order and
 * the REDUCE row bands (1, 2, 4, 6, 8, 12, 16).  A candidate
 * replaces the setting only if it is at least 1% faster.  The plan keeps
 * the best setting; *best_ms (may be NULL) receives its time per run.
 * Synchronises the stream.  reps 1..10000. */
fllf_status fllf_plan_autotune(fllf_plan *plan, const float *d_in, float *d_out, int reps, void *stream,
                               double *best_ms);

/* Batches: resident CTAs per SM of the four batched stage kinds (level-0
 * REDUCE, REDUCE, combine at levels >= 2 on 32 x 16 tiles, and the level-0
 * stage: the fused level-1/level-0 combine, or the level-0 combine of the
 * 2-level images), 0 = as many as fit.  Changing them makes the next
 * fllf_batch_run capture its CUDA graph again.  The batch autotuner times fllf_batch_run on the given
 * buffers (as for fllf_batch_run; outputs overwritten) and keeps the best
 * caps, with the same search and 1% rule as fllf_plan_autotune. */
fllf_status fllf_batch_get_ctas(const fllf_batch *batch, int *ctas_per_sm /* [4] */);

/* Launch mode of a batch: 1: ONE persistent dataflow launch runs every stage
 * of every image (tasks of a few tiles of one row band, pushed onto a device
 * queue once the row bands they read are complete, popped by the CTAs;
 * ctas_per_sm[0] caps its grid); 2: the same without the fused
 * level-1/level-0 combine, which follows as one batched launch
 * (ctas_per_sm[3]); 0 (default; measured faster on mixed batches): one
 * launch per stage kind and level over all images.
 * task_items[5] (may be NULL): task sizes as in fllf_tuning.  Every mode
 * computes the same output, bit for bit.  Setting a mode or task sizes
 * synchronises the device and rebuilds the task list; the next run captures
 * its CUDA graph again.  The batch autotuner searches the mode, the caps of
 * the kinds the mode launches and the task sizes. */
fllf_status fllf_batch_get_mode(const fllf_batch *batch, int *mode, int *task_items);
fllf_status fllf_batch_set_mode(fllf_batch *batch, int mode, const int *task_items);
fllf_status fllf_batch_set_ctas(fllf_batch *batch, const int *ctas_per_sm /* [4] */);
fllf_status fllf_batch_autotune(fllf_batch *batch, const float *const *d_in, float *const *d_out, int reps,
                                void *stream, double *best_ms);

#ifdef __cplusplus
}
#endif

#endif /* FLLF_H */
