/*
 * iwpp.h -- C ABI of libiwpp, a GB300 (sm_103a) implementation of the
 * irregular wavefront propagation pattern (IWPP) of Teodoro, Pan, Kurc, Kong,
 * Cooper and Saltz, "Efficient Irregular Wavefront Propagation Algorithms on
 * Hybrid CPU-GPU Machines" (arXiv:1209.3314), for its two operations:
 *
 *   - grayscale morphological reconstruction by dilation (Section 2.1,
 *     Algorithms 2 and 5);
 *   - Euclidean distance transform by nearest-feature propagation
 *     (Section 2.2, Algorithms 3 and 6).
 *
 * Conventions shared by every entry point
 *   - Image buffers are DEVICE pointers owned by the caller, row-major, with
 *     a pitch counted in elements (pitch >= w).  The library never frees or
 *     retains them past the call's completion on the stream.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All work is enqueued on it.
 *   - The context owns a device workspace (tile queues, flags, spill
 *     buffers, counters) that it grows on demand; calls that share a context
 *     must be ordered on one stream (two streams need two contexts).
 *   - Synchronous entry points return after the work finished and the
 *     device status word was read back; *_async entry points only enqueue
 *     and report device-side failures at the next iwpp_sync().
 *   - Return value: IWPP_OK or a negative IWPP_E* code; iwpp_last_error()
 *     gives a one-line message.  No entry point aborts the process.
 */
#ifndef IWPP_H
#define IWPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IWPP_OK 0
#define IWPP_EINVAL (-1)    /* bad shape, dtype, pitch, connectivity or size  */
#define IWPP_ENOMEM (-2)    /* workspace would exceed the HBM budget / cudaMalloc failed */
#define IWPP_ECUDA (-3)     /* a CUDA runtime call failed                      */
#define IWPP_ETIMEOUT (-4)  /* a device-side wait gave up (bounded spin)       */
#define IWPP_EOVERFLOW (-5) /* tile queue overflowed more often than allowed   */

typedef enum { IWPP_U8 = 0, IWPP_I32 = 1 } iwpp_dtype;

/* Distance-transform polarity.  FEATURE_ZERO (default) is the paper's: the
 * distance of every pixel to the nearest background (value 0) pixel
 * (Section 2.2).  FEATURE_NONZERO measures the distance to the nearest
 * non-zero pixel instead. */
#define IWPP_EDT_FEATURE_ZERO 0
#define IWPP_EDT_FEATURE_NONZERO 1
/* Distance-transform mode (or-ed with the polarity): after the 8-neighbour
 * propagation has reached its fixpoint, a second wavefront runs the same
 * update rule with a wider window -- every offset (dy, dx) with |dy|,
 * |dx| <= k -- whose half-width k grows with the pixel's current distance
 * (Section 2.2: a sufficiently large neighbourhood makes the propagation
 * exact).  k = 1 below the distance edt_wide_step, one more for each further
 * edt_wide_step, at most 8.  This removes the departures from the exact
 * distance that the 8-neighbour rule leaves (Figure 3); the window sizes
 * come from measured departure distances (errors need a window that widens
 * with the distance), and every tested image, up to 16384^2 in both
 * polarities, comes out bit-identical to the exact transform. */
#define IWPP_EDT_EXACT_PROPAGATION 2

typedef struct iwpp_ctx iwpp_ctx;

/* A device image: data (device pointer), h rows, w columns, pitch in
 * elements between row starts, dtype. */
typedef struct {
    void *data;
    int32_t h, w;
    int64_t pitch;
    int32_t dtype; /* iwpp_dtype */
} iwpp_image;

/* Counters accumulated by a context since creation (or iwpp_stats_reset). */
typedef struct {
    uint64_t calls;            /* entry-point invocations                        */
    uint64_t tiles_processed;  /* tile visits (first visits + re-visits)         */
    uint64_t tiles_initial;    /* tiles in the initial queues                    */
    uint64_t seeds;            /* wavefront seeds found by the tile seed scans   */
    uint64_t pushes;           /* pixel-queue insertions during propagation      */
    uint64_t spills;           /* insertions that went to the global spill queue */
    uint64_t rescans;          /* tile rescans after the spill queue was full    */
    uint64_t relaunches;       /* whole-image relaunches after tile-queue overflow */
    uint64_t rounds;           /* propagation rounds summed over tile visits     */
    uint64_t wait_ns;          /* time persistent CTAs spent waiting for a tile, summed */
    uint64_t visit_ns;         /* time persistent CTAs spent visiting tiles, summed     */
    uint64_t phase_ns[4];      /* visit time by phase: staging, sweeps and seeds,
                                  queue rounds, store and border test (summed)  */
    uint64_t kernel_launches;  /* kernels this library launched                  */
    uint64_t kernel_ns;        /* device time from the first to the last persistent
                                  launch of each call, summed (only while the
                                  `timing` option is set; resolved at iwpp_sync) */
    uint64_t sweep_sets;       /* raster + anti-raster sweep sets run, summed over
                                  tile visits                                    */
    uint64_t revisits;         /* tile visits of tiles visited before in the same
                                  call (tiles_processed - revisits = first visits) */
} iwpp_stats_t;

/* Tunables; iwpp_get_options() fills the defaults: tile 0, blocks_per_sm 0,
 * sweeps 3, queue_factor 32, spill_cap 8192, max_relaunch 1, timeout_ms
 * 10000, timing 0, revisit_sweep_min 0, edt_sweeps 2, edt_revisit_sweep_min
 * 64, revisit_sweeps -1, queue_mode 0, test_empty_slot 0, gdt_sweeps 8,
 * batch_split 1, ws_sweeps 6, ws_revisit_sweep_min 0, gdt_revisit_sweep_min
 * 4, edt_wide_step 12.  The tile side is fixed at 64 pixels (the field
 * accepts 0 or 64).  Values are validated by iwpp_set_options().  New fields
 * are only ever appended. */
typedef struct {
    int32_t tile;            /* tile side in pixels: fixed at 64 (0 or 64)    */
    int32_t blocks_per_sm;   /* persistent CTAs per SM, 0 = as many as fit    */
    int32_t sweeps;          /* raster+anti-raster sweep sets per bulk visit   */
    int32_t queue_factor;    /* tile-queue slots = queue_factor * tiles (>= 1);
                                the shortest-path and watershed propagations
                                (also SKIZ) take 4 * queue_factor            */
    int32_t spill_cap;       /* global spill slots per CTA and buffer (>= 0)   */
    int32_t max_relaunch;    /* device-side relaunches after queue overflow    */
    int32_t timeout_ms;      /* bound on a device-side wait that sees no
                                progress: a tile claim gives up after this
                                long without any visit finishing or tile
                                being queued anywhere; the TMA waits and the
                                round guard of one tile visit give up this
                                long after the visit began.  A call of any
                                length that keeps making progress is never
                                cut off.                                      */
    int32_t timing;          /* 1: bracket the persistent launches with CUDA
                                events and add their duration to kernel_ns    */
    int32_t revisit_sweep_min; /* reconstruction: a later visit of a tile runs
                                the sweeps when more halo pixels than this can
                                propagate inward, else only the queue       */
    int32_t edt_sweeps;      /* distance transform: vector-propagation sweep
                                sets per bulk visit (0 = queue only)          */
    int32_t edt_revisit_sweep_min; /* distance transform: a later visit sweeps
                                when more halo pixels than this changed       */
    int32_t revisit_sweeps;  /* reconstruction: sweep sets on a later visit
                                (-1: the same as sweeps)                      */
    int32_t queue_mode;      /* intra-tile queue design, for ablations (the
                                result is the same in every mode):
                                0  warp-aggregated pushes (ballot / prefix
                                   sum, one shared atomic per warp) into the
                                   block queue in shared memory, spilling to
                                   the CTA's queue in global memory
                                1  one shared atomic per pushing thread
                                2  warp-aggregated, block queue bypassed:
                                   every item in the global queue
                                3  both                                       */
    int32_t test_empty_slot; /* tests of the timeout path only: 1 leaves one
                                slot of the initial tile queue unfilled, so
                                one claim waits until timeout_ms runs out and
                                the call returns IWPP_ETIMEOUT (no fault, no
                                hang: every device wait is bounded)           */
    int32_t gdt_sweeps;      /* shortest paths: sweep sets per bulk visit
                                (obstacles bend the paths, so more sets pay)  */
    int32_t batch_split;     /* batches of several operations: 0 one
                                persistent launch with the kernel that runs
                                them all; 1 one persistent launch per
                                operation family, back to back on the stream
                                (each with its smaller, faster kernel; the
                                default); the autotuner tries both            */
    int32_t ws_sweeps;       /* watershed plateau-distance and label
                                propagations (also the SKIZ labels): sweep
                                sets per bulk visit                           */
    int32_t ws_revisit_sweep_min; /* the same propagations: a later visit
                                runs the sweeps when more halo pixels than
                                this can propagate inward, else only the
                                queue                                         */
    int32_t gdt_revisit_sweep_min; /* the same for the shortest-path
                                propagation (also the SKIZ distances)         */
    int32_t edt_wide_step;   /* IWPP_EDT_EXACT_PROPAGATION: the window's
                                half-width grows by one per this many pixels
                                of distance (default 12; smaller is wider)    */
} iwpp_options;

/* Creates a context on `device`.  hbm_budget_bytes bounds the workspace the
 * context may hold (0 = unlimited).  *out receives the handle. */
int iwpp_ctx_create(iwpp_ctx **out, int device, size_t hbm_budget_bytes);
/* Waits for nothing; frees the workspace.  Passing NULL is a no-op. */
int iwpp_ctx_destroy(iwpp_ctx *ctx);
/* Message of the last failure on this context (never NULL). */
const char *iwpp_last_error(const iwpp_ctx *ctx);

int iwpp_get_options(const iwpp_ctx *ctx, iwpp_options *out);
int iwpp_set_options(iwpp_ctx *ctx, const iwpp_options *opt);

/*
 * Morphological reconstruction by dilation of `mask` (I) from `marker` (J),
 * Section 2.1 (definition: elementary geodesic dilations clipped by the
 * mask, repeated to stability) computed by the tile-parallel wavefront of
 * Algorithm 5.  conn = 4 or 8.  marker, mask and out share h, w and dtype
 * (IWPP_U8 or IWPP_I32); pitches may differ.  out may alias marker (in
 * place) but not mask.  A marker above the mask is first clipped to it.
 * Result is exact (bit-identical to any correct sequential algorithm).
 */
int iwpp_recon(iwpp_ctx *ctx, const iwpp_image *marker, const iwpp_image *mask,
               int conn, iwpp_image *out, void *stream);
int iwpp_recon_async(iwpp_ctx *ctx, const iwpp_image *marker, const iwpp_image *mask,
                     int conn, iwpp_image *out, void *stream);

/*
 * Distance transform by nearest-feature propagation, Section 2.2,
 * Algorithms 3 and 6, 8-connected.  binary: IWPP_U8 image (0 / non-zero).
 * Outputs (dense h*w int32, device): sqdist = squared Euclidean distance to
 * the feature assigned to the pixel, nearest = that feature's linear index
 * y*w + x.  With no feature in the image: sqdist = INT32_MAX, nearest = -1.
 * Limits: max(h, w) <= 32768.  Like the paper's method, the assignment is
 * approximate at rare pixels (Section 2.2, Figure 3): each result is a
 * fixpoint of the propagation rule (no 8-neighbour's feature is strictly
 * closer), and where several fixpoints exist the one reached may depend on
 * the processing order.
 */
int iwpp_edt(iwpp_ctx *ctx, const iwpp_image *binary, int32_t *sqdist,
             int32_t *nearest, int flags, void *stream);
int iwpp_edt_async(iwpp_ctx *ctx, const iwpp_image *binary, int32_t *sqdist,
                   int32_t *nearest, int flags, void *stream);

/*
 * Exact distance transform: sqdist = min over features f of |p - f|^2 (the
 * definition of Section 2.2, which the propagation method approximates;
 * Figure 3 shows a pixel where it departs), computed by the separable
 * method rather than by propagation.  It runs a column pass (per column,
 * the nearest feature row, in bands of 128 rows) and a row pass that builds
 * each row's lower envelope of the parabolas (x - i)^2 + dy_i^2, one CTA
 * per row, so its cost does not depend on the distances.  All comparisons
 * are exact integer arithmetic.  Same arguments, flags, limits and
 * no-feature convention as iwpp_edt; nearest may be any of several equally
 * near features.  The context workspace grows to h*w*4 bytes plus band
 * summaries.  Synchronous: returns after the work on `stream` completed.
 */
int iwpp_edt_exact(iwpp_ctx *ctx, const iwpp_image *binary, int32_t *sqdist,
                   int32_t *nearest, int flags, void *stream);

/*
 * Shortest paths on a grid with obstacles, which Section 1 names as a
 * further instance of the IWPP, by the same tile-parallel wavefront.
 * mask, seeds: IWPP_U8 images of one shape (pitches may differ); a pixel is
 * free where mask != 0 (0 = obstacle) and a source where it is free and
 * seeds != 0.  Paths move to any free 8-neighbour at cost 5 (horizontal or
 * vertical) or 7 (diagonal): this build's choice of grid metric, the 5-7
 * chamfer weights.  dist (dense h*w int32, device) receives each pixel's
 * least path cost from any source: 0 at sources, INT32_MAX at obstacles
 * and unreachable pixels.  Exact (integer costs; the least cost is unique)
 * while every least path cost stays below 2^30: always with fewer than
 * 153 M free pixels (a shortest path visits a pixel at most once, at cost
 * <= 7 per step), and on open fields far beyond (at most 7*max(h, w)
 * without obstacles).  Limits: h*w < 2^31.  Not part of mixed job batches.
 */
int iwpp_geodesic(iwpp_ctx *ctx, const iwpp_image *mask, const iwpp_image *seeds,
                  int32_t *dist, void *stream);
int iwpp_geodesic_async(iwpp_ctx *ctx, const iwpp_image *mask, const iwpp_image *seeds,
                        int32_t *dist, void *stream);

/*
 * Influence zones of labelled sources inside a mask and their skeleton
 * (SKIZ), which Section 1 names among the IWPP algorithms.  The paper gives
 * no definition; this is the geodesic SKIZ (Lantuejoul, 1980) with the
 * grid metric of iwpp_geodesic:
 *   mask     IWPP_U8 image, free where != 0;
 *   labels   IWPP_I32 image of the same shape (pitches may differ): a free
 *            pixel with a label != 0 is a source of that label.  Labels
 *            must lie in [INT32_MIN + 2, INT32_MAX - 1];
 *   zones    (dense h*w int32, device) the least label among the labels
 *            whose sources are nearest (least path cost, 8 moves at cost
 *            5 / 7 through free pixels); 0 at obstacles and unreachable
 *            pixels;
 *   skiz     (optional, may be NULL: dense h*w uint8) 1 where two or more
 *            labels are nearest (the skeleton by influence zones), else 0;
 *   dist     (optional, may be NULL: dense h*w int32) the least path cost,
 *            as iwpp_geodesic.
 * Exact and unique under iwpp_geodesic's bound on the path costs.  Steps:
 * the shortest-path propagation, then one launch that propagates the least
 * label and the least negated label along the shortest-path edges.  Outputs must not overlap the inputs.  The context
 * holds 6*h*w bytes of planes (10*h*w without dist) besides its workspace.
 * Limits: h*w < 2^31.  Synchronous.
 */
int iwpp_skiz(iwpp_ctx *ctx, const iwpp_image *mask, const iwpp_image *labels,
              int32_t *zones, uint8_t *skiz, int32_t *dist, void *stream);

/*
 * Watershed from markers, which Section 1 names among the IWPP algorithms,
 * as three wavefront propagations on the tile wavefront.  The paper gives
 * no definition; this is the image foresting transform with the
 * highest-value path cost (Falcao, Stolfi and Lotufo, 2004), plateaus
 * split by distance (Lotufo and Falcao, 2000), ties to the least label:
 *   relief   IWPP_U8 or IWPP_I32 image; markers: IWPP_I32 image of the
 *            same shape (pitches may differ), 0 = no marker, any other
 *            value but INT32_MAX a label;
 *   levels   (optional, may be NULL: dense h*w of the relief's type,
 *            device) the flooding level: the least, over the 8-connected
 *            paths from a marker pixel, of the highest relief value on the
 *            path (a marker pixel's own relief value);
 *   labels   (dense h*w int32, device) the least marker value among the
 *            marker pixels from which the pixel is reached along optimal
 *            edges: from a lower-level neighbour into a pixel with one, or
 *            within a level region from a neighbour one breadth-first step
 *            nearer to the region's entry pixels (its markers and its
 *            pixels with a lower neighbour).  A marker pixel keeps its
 *            value.  Without any marker: labels 0 and levels the type's
 *            maximum.
 * The result is unique (no dependence on the processing order).  Steps:
 * the levels by a reconstruction by dilation of the complemented images,
 * then the plateau distances and the labels by min-propagations along
 * per-pixel in-edge masks.  labels and levels must not overlap the inputs.
 * The context holds 2*h*w*size(relief) + 5*h*w bytes of planes besides
 * its workspace.  Limits: h*w < 2^30.  Synchronous.
 */
int iwpp_watershed(iwpp_ctx *ctx, const iwpp_image *relief, const iwpp_image *markers,
                   int32_t *labels, void *levels, void *stream);

/*
 * Batched entry points: n independent images in ONE persistent launch
 * (tiles of all images share one tile queue).  Arrays are host arrays of n
 * descriptors / pointers; the images themselves are on the device.
 */
int iwpp_recon_batched(iwpp_ctx *ctx, int n, const iwpp_image *markers,
                       const iwpp_image *masks, int conn, iwpp_image *outs,
                       void *stream);
int iwpp_edt_batched(iwpp_ctx *ctx, int n, const iwpp_image *bins,
                     int32_t *const *sqdists, int32_t *const *nearests, int flags,
                     void *stream);

/* One job of a mixed batch: op 0 = reconstruction (a = marker, b = mask,
 * out = result, conn), op 1 = distance transform (a = binary, sqdist,
 * nearest, flags). */
typedef struct {
    int32_t op;
    int32_t conn;
    int32_t flags;
    int32_t reserved;
    iwpp_image a, b, out;
    int32_t *sqdist, *nearest;
} iwpp_job;

#define IWPP_OP_RECON 0
#define IWPP_OP_EDT 1

/* Mixed reconstruction / distance-transform batch in one persistent launch. */
int iwpp_run_jobs(iwpp_ctx *ctx, int n, const iwpp_job *jobs, void *stream);
int iwpp_run_jobs_async(iwpp_ctx *ctx, int n, const iwpp_job *jobs, void *stream);

/*
 * Asynchronous jobs with tickets: the operations of Sections 2.1 and 2.2
 * (one iwpp_job each, device images as in iwpp_run_jobs) enqueued on the
 * context's own stream, which the first iwpp_submit creates.  That stream
 * is a blocking stream: it runs after work enqueued earlier on the legacy
 * default stream and before work enqueued there later, so inputs written
 * on the default stream are ready.  Submitted jobs run in submission order
 * and share the context's workspace: do not mix them with *_async calls of
 * the same context on other streams unless those are synchronised.
 *   iwpp_submit  validates and enqueues the job; returns at once with a
 *                ticket (> 0) in *ticket.  Argument errors are returned
 *                directly and give no ticket.
 *   iwpp_poll    returns 1 when the job has finished (its outcome, IWPP_OK
 *                or a negative IWPP_E* code, in *status; may be NULL) and
 *                retires the ticket; 0 while it is pending; IWPP_EINVAL
 *                for an unknown or retired ticket.
 *   iwpp_wait    blocks until the job has finished, stores its outcome in
 *                *status and retires the ticket; IWPP_EINVAL for an unknown
 *                or retired ticket.
 * Every submitted job is counted by iwpp_stats like any other call.  For a
 * continuous-batching request loop over host images see iwpp_server_*.
 */
int iwpp_submit(iwpp_ctx *ctx, const iwpp_job *job, uint64_t *ticket);
int iwpp_poll(iwpp_ctx *ctx, uint64_t ticket, int *status);
int iwpp_wait(iwpp_ctx *ctx, uint64_t ticket, int *status);

/*
 * Plans: a fixed batch of jobs prepared once for repeated launches -- tile
 * layout, TMA tensor maps, the device job table and the plan's own
 * workspace are set up by iwpp_plan_create (which may allocate and copy).
 * iwpp_plan_launch then only enqueues kernels (no allocation, no host
 * encoding, no copies), so it is legal inside a CUDA stream capture;
 * iwpp_plan_launch_graph captures that launch sequence into a CUDA graph
 * on its first call and replays the graph afterwards.  The images the jobs
 * name must stay valid while the plan lives; their contents may change
 * between launches.  Plan launches share the context's status block: order
 * them on one stream with the context's other calls and read failures with
 * iwpp_sync().
 *
 * iwpp_plan_autotune times `reps` launches of each candidate option set on
 * the plan's own images: first sweep sets (reconstruction 2..4, distance
 * transform 1..3), revisit thresholds, CTAs per SM (max / max-1) and one
 * launch or one launch per operation family; then, from the best of those,
 * the tile-queue capacity (queue_factor 8 / 16 / 32 slots per tile) and the
 * per-CTA spill capacity (spill_cap 1024 / 8192).  It keeps the fastest in
 * the plan, stores it in the context under a key of (kernel family, log2
 * pixels, log2 jobs, SM count) so that later plans of the same kind start
 * tuned, and copies it to *best (may be NULL).  It synchronises `stream`.
 */
typedef struct iwpp_plan iwpp_plan;
int iwpp_plan_create(iwpp_ctx *ctx, int n, const iwpp_job *jobs, iwpp_plan **out);
int iwpp_plan_launch(iwpp_plan *plan, void *stream);
int iwpp_plan_launch_graph(iwpp_plan *plan, void *stream);
int iwpp_plan_autotune(iwpp_plan *plan, void *stream, int reps, iwpp_options *best);
int iwpp_plan_destroy(iwpp_plan *plan);

/*
 * Served mode: a continuous-batching request server on one GPU.  Requests
 * name HOST images (dense, row-major; pinned memory gives overlapped
 * copies).  A worker thread admits queued requests while their device
 * memory fits `hbm_budget_bytes` next to the work in flight, runs each
 * admitted group as one persistent launch on one of `streams` streams
 * (each with its own resident context), and keeps admitting new arrivals
 * onto free streams while earlier batches run.  Results are copied back to
 * the request's host buffers; the latency reported is submit-to-completion.
 * The request images come from a memory pool of the server's own, which
 * never makes one stream wait for another's frees.
 * Admission counts, against the budget, the images of every request in
 * flight and the device memory of every stream's context (its workspace
 * grows to the largest batch it has run and stays resident).  A request
 * that cannot fit even alone completes with IWPP_ENOMEM; creation fails with
 * IWPP_ENOMEM when the contexts alone exceed the budget.  poll / wait hand a
 * result out once: the ticket is then retired and a second poll or wait on
 * it returns IWPP_EINVAL.  iwpp_server_destroy finishes every submitted
 * request first.
 */
typedef struct {
    int32_t op;             /* IWPP_OP_RECON or IWPP_OP_EDT                      */
    int32_t conn;           /* reconstruction: 4 or 8                            */
    int32_t flags;          /* distance transform: IWPP_EDT_FEATURE_*            */
    int32_t dtype;          /* reconstruction: IWPP_U8 or IWPP_I32               */
    int32_t h, w;
    const void *marker;     /* recon: marker; edt: binary image (uint8)          */
    const void *mask;       /* recon: mask                                       */
    void *out;              /* recon: result                                     */
    int32_t *sqdist;        /* edt: squared distances (h*w)                      */
    int32_t *nearest;       /* edt: nearest-feature linear indices (h*w)         */
} iwpp_request;

typedef struct {
    uint64_t submitted, completed, batches, pending;
    uint64_t bytes_in_use;       /* request images in flight + resident workspaces */
    uint64_t peak_bytes_in_use;  /* peak of bytes_in_use (admission keeps it <= budget) */
    uint64_t workspace_bytes;    /* device memory the streams' contexts hold */
    uint64_t pool_used_high;     /* high-water mark of the server's memory pool
                                    (request images) since server creation */
    uint64_t records;            /* finished results not yet handed out */
} iwpp_server_stats_t;

typedef struct iwpp_server iwpp_server;
int iwpp_server_create(iwpp_server **out, int device, size_t hbm_budget_bytes, int streams, int max_batch);
int iwpp_server_submit(iwpp_server *srv, const iwpp_request *req, uint64_t *ticket);
/* 1 when the request finished (its status in *status; the ticket is then
 * retired), 0 while pending, IWPP_EINVAL for an unknown or retired ticket. */
int iwpp_server_poll(iwpp_server *srv, uint64_t ticket, int *status);
/* Blocks until the request finished; *status is its outcome. */
int iwpp_server_wait(iwpp_server *srv, uint64_t ticket, int *status, double *latency_ms);
int iwpp_server_stats(iwpp_server *srv, iwpp_server_stats_t *out);
int iwpp_server_destroy(iwpp_server *srv);

/* Waits for `stream`, reads the device status of the async calls enqueued
 * on it since the last sync, returns IWPP_OK or the first failure. */
int iwpp_sync(iwpp_ctx *ctx, void *stream);

int iwpp_stats(iwpp_ctx *ctx, iwpp_stats_t *out);
int iwpp_stats_reset(iwpp_ctx *ctx);

/*
 * Allocation-free uint8 reconstruction.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory --
 * code running inside another allocator's accounting (a caching allocator
 * that owns the device budget) and real-time paths that forbid allocation
 * after start-up (cudaMalloc may block and synchronise the device).
 *
 * Same operation and result as iwpp_recon on IWPP_U8 images, without a
 * context: marker, mask and out are device pointers with pitches in bytes;
 * out may be marker exactly (in place, equal pitches) but must not overlap
 * the mask or partly overlap the marker; conn = 4 or 8; the work is
 * enqueued on `stream` and the call returns after it finished.  All
 * scratch (tile queue, tile states, spill queues, status block) lives in one
 * statically sized device array of IWPP_NOALLOC_SCRATCH_BYTES held by every
 * GPU that loads the library until process exit; the call itself allocates
 * nothing.  Limits and rules:
 *   - at most IWPP_NOALLOC_MAX_TILES tiles of 64x64 pixels (e.g. 16384 x
 *     16384); larger images return IWPP_EINVAL;
 *   - all calls share the array, which keeps the last call's contents (each
 *     call clears its status block and refills its queue before it runs):
 *     calls whose GPU work overlaps (different streams or threads on one
 *     device) race -- serialise them;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress);
 *   - a device-side wait gives up after 10 s without progress.
 * Returns IWPP_OK, IWPP_EINVAL, IWPP_ECUDA, IWPP_ETIMEOUT or IWPP_EOVERFLOW.
 */
#define IWPP_NOALLOC_MAX_TILES 65536
#define IWPP_NOALLOC_SCRATCH_BYTES ((size_t)12 << 20)
int iwpp_recon_u8_noalloc(const uint8_t *marker, int64_t marker_pitch, const uint8_t *mask,
                          int64_t mask_pitch, uint8_t *out, int64_t out_pitch, int h, int w,
                          int conn, void *stream);

/* Library version as major*10000 + minor*100 + patch. */
int iwpp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* IWPP_H */
