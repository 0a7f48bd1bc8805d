/*
 * ccd.h -- C ABI of the GB300 continuous-collision-detection library.
 *
 * The library computes, for two triangle meshes given at t = 0 and t = 1 with
 * linear vertex trajectories and a shared topology, the earliest time of
 * impact t* in [0, 1] (+inf when nothing collides), as defined in Section
 * "Preliminaries" and Algorithm 1 (CCD = BuildBoxes, BroadPhase, NarrowPhase)
 * of "Time of Impact Dataset for Continuous Collision Detection and a Scalable
 * Conservative Algorithm" (Belgrod et al.).
 *
 * Conventions for every entry point:
 *   - Device pointers are CUDA global-memory pointers on the context's device,
 *     owned by the caller, never freed or retained by the library.
 *   - V0, V1: FP64 vertex positions, structure of arrays [3][nV]: x[0..nV),
 *     then y, then z.  E: int32 [nE][2] vertex ids.  F: int32 [nF][3].
 *     Ids must lie in [0, nV); coordinates must be finite with magnitude
 *     below 2^100 (the single-precision boxes and the error bound assume it).
 *   - Box numbering: vertices 0..nV-1, edges nV..nV+nE-1, faces after.
 *   - Pair lists: int32 [n][2].  Vertex-face pairs are (vertex id, face id);
 *     edge-edge pairs are (lower edge id, higher edge id).
 *   - All work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream).  Calls return after enqueueing unless stated otherwise.
 *   - Return value: a CCD_* status.  On an error nothing is guaranteed about
 *     the outputs.  ccd_status_str() describes a status.
 *   - A context is not thread-safe: one host thread and one stream at a time.
 */
#ifndef GB300_CCD_H
#define GB300_CCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ccd_ctx ccd_ctx;

enum {
    CCD_OK = 0,
    CCD_EINVAL = 1,    /* bad argument: null pointer, negative size, bad option */
    CCD_ENOMEM = 2,    /* device allocation failed */
    CCD_ETRUNC = 3,    /* an output list was too small; counts hold the sizes needed */
    CCD_EQUEUE = 4,    /* the narrow-phase interval queue overflowed (work was kept
                          on the lane that owned it, results stay correct) */
    CCD_ETIMEOUT = 5,  /* a bounded device-side wait gave up; results are invalid */
    CCD_ECUDA = 6,     /* a CUDA runtime call failed */
    CCD_EDEVICE = 7    /* the device is not a compute capability 10.3 GPU */
};

/* Per-query flag bits written by ccd_narrow. */
#define CCD_FLAG_ITER_CAP 1u   /* more than max_iter intervals: the TOI is the
                                  earliest left end of the live intervals */
#define CCD_FLAG_LEVEL_CAP 2u  /* an interval could not be split further
                                  (53 levels on every axis); accepted as a hit */

/* Options fixed at context creation (ccd_default_opts fills the defaults). */
typedef struct {
    double delta;            /* codomain tolerance of the stop rule w(B) < delta
                                (Algorithm 3); default 1e-6 */
    double min_sep;          /* minimum separation, added to the error box on every
                                axis (Section "Avoiding Time of Impacts Equal to
                                Zero"); default 0 */
    int64_t max_iter;        /* per-query cap on processed intervals; default 1e6 */
    int32_t broad_fp64;      /* 0 (default): single-precision outward-rounded boxes
                                then an exact FP64 filter; 1: FP64 boxes throughout */
    int32_t sweep_kernel;    /* 0 (default): cell sweep (boxes are also binned
                                into a grid of cells on the two other axes and
                                swept per cell, each pair reported in one cell
                                only);
                                1: one warp per box, one sorted list (Algorithm 2
                                as printed); 2: tiled sweep over one sorted list
                                (a block walks the sweep ranges of 256 boxes
                                through shared memory) */
    int64_t pair_capacity;   /* initial pair-buffer capacity used by ccd_step
                                (0 = auto); grows on demand in synchronous calls */
    int64_t queue_capacity;  /* interval-queue slots, a power of two (0 = auto) */
    int32_t export_budget;   /* tail phase: every 32 x export_budget intervals a
                                warp evaluates, its busy lanes hand their
                                shallowest pending siblings to the queue
                                (0 = 16) */
    int32_t profile_stages;  /* 1: record CUDA events around the stages of each
                                call (read with ccd_stage_times); default 0 */
    int32_t no_zero_toi;     /* 1: ccd_step applies the zero-TOI rule of the appendix
                                "Zero time of impact and minimum separation": when
                                the earliest time is 0, the narrow phase runs again
                                with min_sep = 0, intervals starting at t = 0 are
                                always split, and the result is scaled by 0.8
                                (decided on the device); default 0 */
    int32_t use_graph;       /* 1: ccd_step with a device output and ccd_step_batch
                                capture their launch sequence into a CUDA graph on
                                the first call and replay it while the arguments
                                (pointers, sizes, parameters) stay the same;
                                default 0 */
    int32_t pad0;
    double strip_width;      /* cell sweep: cell width as a multiple of the mean
                                box width on each cell axis (0 = auto: 3); more
                                cells mean fewer comparisons but more copies of
                                boxes that straddle cell borders */
    int64_t memory_limit;    /* device bytes ccd_step may size its buffers for (by the
                                memory model, ccd_get_memory_model; 0 = no limit).
                                A synchronous step whose candidate pairs exceed the
                                capacity that fits runs the paper's batching
                                (Section "Batching"): the sorted boxes are swept in
                                ranges whose pairs fit, each range's narrow phase
                                carrying the earliest time over (cell sweep only, no
                                zero-TOI rule); an asynchronous step raises
                                CCD_ETRUNC instead */
} ccd_opts;

/* Work counters of the last broad/narrow/step call (see ccd_get_status). */
typedef struct {
    int64_t n_boxes;         /* boxes built */
    int32_t sweep_axis;      /* axis of largest centre variance (0 x, 1 y, 2 z) */
    int32_t pad0;
    int64_t n_superset;      /* pairs passing the single-precision box test */
    int64_t n_vf, n_ee;      /* candidate pairs after the exact test */
    int64_t n_intervals;     /* narrow-phase intervals evaluated */
    int64_t n_exported;      /* subtrees handed to the queue (other warps) */
    int64_t n_capped;        /* queries that hit max_iter */
    int64_t queue_peak;      /* largest queue occupancy seen */
    int32_t device_status;   /* CCD_* status raised by the kernels */
    int32_t pad1;
    int64_t n_launches;      /* kernels this context launched since creation */
    int64_t narrow_bulk_ns;  /* narrow kernel: start until every query was taken */
    int64_t narrow_tail_ns;  /* narrow kernel: from then until the last lane ended */
    int64_t n_donated;       /* subtrees passed between lanes of one warp, or between
                                warps of one block through shared memory */
    int64_t n_intervals_tail;  /* intervals evaluated after every query was taken */
    int64_t n_intervals_fp64;  /* intervals the single-precision filter left to FP64 */
    int64_t n_box_copies;    /* cell sweep: boxes placed in cells, counting each
                                cell a box overlaps (n_boxes for the other sweeps) */
    int64_t n_ranges;        /* ranges the last step swept under memory_limit (0: one pass) */
} ccd_stats;

/* Fill *o with the defaults. */
void ccd_default_opts(ccd_opts *o);

/* Create a context on CUDA device `device`: checks the device, keeps a copy
 * of *o (NULL = defaults) and allocates the fixed scratch (status words,
 * counters).  Size-dependent scratch grows on first use.  *out receives the
 * context; free it with ccd_destroy. */
int ccd_create(ccd_ctx **out, const ccd_opts *o, int device);

/* Release every device buffer of the context (synchronizes its device). */
int ccd_destroy(ccd_ctx *ctx);

/*
 * Broad phase (Section "Broad-Phase", Algorithm 2, with the boxes of Section
 * "Construction of the Boxes"): every vertex-face pair (v, f) with v not a
 * vertex of f, and every edge-edge pair without a shared endpoint, whose
 * boxes swept over [0, 1] overlap on all three axes (closed intervals).  The
 * set is exactly the one defined by the FP64 extents (the single-precision
 * sweep is followed by an exact FP64 test), returned in unspecified order.
 *
 * vf_out [vf_cap][2], ee_out [ee_cap][2]: device outputs.
 * n_vf, n_ee: HOST pointers, receive the total numbers of pairs found.
 * Synchronizes `stream`.  Returns CCD_ETRUNC when a total exceeds its
 * capacity (only the first `cap` pairs were written; call again with room
 * for the returned totals).
 */
int ccd_broad(ccd_ctx *ctx, const double *V0, const double *V1, int64_t nV,
              const int32_t *E, int64_t nE, const int32_t *F, int64_t nF,
              int32_t *vf_out, int64_t vf_cap, int64_t *n_vf,
              int32_t *ee_out, int64_t ee_cap, int64_t *n_ee, void *stream);

/*
 * One shard of the broad phase: the decomposition of the sweep over several
 * GPUs (the paper's multi-GPU broad phase, Section "Conclusion and Future
 * Work"), callable on one.  Every shard builds and sorts all boxes (the same
 * small work on each), then sweeps from its own contiguous part
 * [n s / n_shards, n (s + 1) / n_shards) of the n sorted cell copies,
 * reading past the part's end; each pair is reported from exactly one copy,
 * so the shards' pair sets are disjoint and their union is ccd_broad's set.
 * The earliest time of the whole step is the minimum over the shards of the
 * narrow phase (mode 1) on each shard's pairs: the only exchange a multi-GPU
 * step needs is that one minimum.  Arguments and outputs as in ccd_broad,
 * plus 0 <= shard < n_shards.  Cell sweep only (sweep_kernel 0); synchronous.
 */
int ccd_broad_shard(ccd_ctx *ctx, const double *V0, const double *V1, int64_t nV,
                    const int32_t *E, int64_t nE, const int32_t *F, int64_t nF,
                    int32_t shard, int32_t n_shards,
                    int32_t *vf_out, int64_t vf_cap, int64_t *n_vf,
                    int32_t *ee_out, int64_t ee_cap, int64_t *n_ee, void *stream);

/*
 * Narrow phase (Section "Narrow-Phase", Algorithm 3): conservative interval
 * bisection over (t, u, v) with an FP64 inclusion function and error box, for
 * the given pairs.  mode 0: each pair gets its own time of impact (toi_vf,
 * toi_ee: device double [n], +inf for no collision; flags_vf, flags_ee:
 * device uint8 [n], CCD_FLAG_* bits).  mode 1: only the earliest time over
 * all pairs is wanted (Algorithm 3 as printed: one shared t* prunes every
 * pair); the per-pair arrays may be NULL and are not meaningful.
 * toi_min: device double [1], receives the earliest time over all pairs.
 * delta, min_sep, max_iter override the context options for this call.
 * Asynchronous; device errors are reported by ccd_get_status.
 */
int ccd_narrow(ccd_ctx *ctx, const int32_t *vf, int64_t n_vf, const int32_t *ee, int64_t n_ee,
               const double *V0, const double *V1, int64_t nV,
               const int32_t *E, int64_t nE, const int32_t *F, int64_t nF,
               double delta, double min_sep, int64_t max_iter, int32_t mode,
               double *toi_vf, double *toi_ee, uint8_t *flags_vf, uint8_t *flags_ee,
               double *toi_min, void *stream);

/*
 * Whole CCD step (Algorithm 1): boxes, broad phase, earliest-TOI narrow phase,
 * using the context's own pair buffers.  toi_min may be a device pointer
 * (asynchronous; an overflow of the pair buffers is reported by
 * ccd_get_status as CCD_ETRUNC and the result must then be discarded) or a
 * host pointer (synchronous; the pair buffers are grown and the step rerun
 * when they overflow, and the device status is returned).
 */
int ccd_step(ccd_ctx *ctx, const double *V0, const double *V1, int64_t nV,
             const int32_t *E, int64_t nE, const int32_t *F, int64_t nF,
             double delta, double min_sep, int64_t max_iter, double *toi_min, void *stream);

/*
 * Narrow phase without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc where they
 * need the query (under an allocator they do not own, in hosts that forbid
 * allocation, in loops that must not allocate).  Same computation, results
 * and arguments as ccd_narrow, but no context: the scratch is one fixed array
 * in the library's device memory (about 1.4 MB per GPU, kept until the
 * process exits).  Limit: n_vf + n_ee <= 65536; larger calls return
 * CCD_EINVAL.  Its interval ring is smaller than ccd_narrow's (2^14 cells);
 * that changes only how much tail work can move between warps, not results.
 * status: device int32 [1], receives the kernels' CCD_* status.
 * The first call on a device sets it up from the current device (occupancy
 * query for the grid size); make that first call before any stream capture.
 * Every call looks up the array's device address (a host-side lookup) and
 * first resets all of the array that the kernels read (counters, status,
 * t*, interval ring), so no state of an earlier call -- finished, failed or
 * cut off -- reaches it.  Calls share the array: calls that overlap on the
 * GPU race.  Asynchronous.
 */
int ccd_narrow_noalloc(const int32_t *vf, int64_t n_vf, const int32_t *ee, int64_t n_ee,
                       const double *V0, const double *V1, int64_t nV,
                       const int32_t *E, int64_t nE, const int32_t *F, int64_t nF,
                       double delta, double min_sep, int64_t max_iter, int32_t mode,
                       double *toi_vf, double *toi_ee, uint8_t *flags_vf, uint8_t *flags_ee,
                       double *toi_min, int32_t *status, void *stream);

/*
 * Batched step: Algorithm 1 on many independent scenes (environments) of
 * uneven size in one launch sequence -- one sort, one sweep, one narrow-phase
 * launch for all of them.  The scenes are concatenated: scene s owns vertices
 * [vert_off[s], vert_off[s+1]), edges [edge_off[s], edge_off[s+1]) and faces
 * [face_off[s], face_off[s+1]) (device int64 arrays of n_scenes + 1 entries,
 * each starting at 0); E and F hold global vertex ids, and every edge or face
 * uses vertices of its own scene.  Pairs never cross scenes; each scene has
 * its own sweep axis (largest centre variance) and its own earliest time.
 * toi_out: device double [n_scenes], +inf for a scene without collision.
 * Asynchronous and allocation-free once the context's buffers have grown to
 * the sizes of a first call (it can then be captured in a CUDA graph); an
 * overflow of the pair buffers is reported by ccd_get_status (CCD_ETRUNC).
 * Each scene has its own cell layout under the cell sweep (more than
 * 65,536 scenes take the tiled sweep).  Requires the single-precision broad
 * phase, the cell or tiled sweep (sweep_kernel 0 or 2), and no zero-TOI rule.
 */
int ccd_step_batch(ccd_ctx *ctx, int32_t n_scenes, const int64_t *vert_off, const int64_t *edge_off,
                   const int64_t *face_off, const double *V0, const double *V1, int64_t nV,
                   const int32_t *E, int64_t nE, const int32_t *F, int64_t nF,
                   double delta, double min_sep, int64_t max_iter, double *toi_out, void *stream);

/* Settings chosen by ccd_autotune. */
typedef struct {
    int32_t sweep_kernel;    /* 0 cells or 2 tiled */
    int32_t export_budget;   /* tail phase: a warp hands off every 32 x this many
                                evaluations */
    double strip_width;      /* cell width in mean box widths (cell sweep) */
    int64_t queue_capacity;  /* interval-queue slots */
    double broad_ms;         /* median broad-phase time with the chosen settings */
    double narrow_ms;        /* median narrow-phase time with the chosen settings */
    double default_ms;       /* median broad + narrow time with the previous settings */
    int32_t n_trials;        /* settings timed */
    int32_t pad;
} ccd_tuning;

/*
 * Autotuner: times the broad phase with the cell sweep at cell widths of
 * 1.5-6 mean box widths and with the tiled sweep, then the narrow phase with
 * hand-off budgets of 16-256 intervals, each as the median of `reps` runs on
 * this mesh, and keeps the fastest settings in the context (later calls use
 * them; captured graphs are dropped).  The interval queue then shrinks to the
 * smallest power of two at least 16 times the peak occupancy seen (and at
 * least 1024 slots) unless that slows the narrow phase by more than 2%.
 * Synchronous; not for use under stream capture.  Requires the
 * single-precision broad phase.  On an error the previous settings stay.
 */
int ccd_autotune(ccd_ctx *ctx, const double *V0, const double *V1, int64_t nV, const int32_t *E, int64_t nE,
                 const int32_t *F, int64_t nF, int32_t reps, ccd_tuning *out, void *stream);

/* The autotuner on batched scenes (arguments as in ccd_step_batch): times
 * the batched broad phase and the per-scene narrow phase. */
int ccd_autotune_batch(ccd_ctx *ctx, int32_t n_scenes, const int64_t *vert_off, const int64_t *edge_off,
                       const int64_t *face_off, const double *V0, const double *V1, int64_t nV,
                       const int32_t *E, int64_t nE, const int32_t *F, int64_t nF, int32_t reps,
                       ccd_tuning *out, void *stream);

/*
 * Device memory model.  Section "Batching" sizes the candidate list C from
 * the free memory M as S_C = (M - S_P) / (S_Q + S_i): per pair, the query
 * data of the narrow phase plus the pair itself.  The same accounting for
 * this implementation: a step over n_boxes boxes (in n_scenes scenes) with
 * room for P candidate pairs needs
 *     bytes_fixed + n_boxes * bytes_per_box + n_scenes * bytes_per_scene
 *       + P * bytes_per_pair
 * bytes of device memory (buffers grow to these sizes and are kept).
 * o: the context's options (NULL = defaults; the interval-queue capacity
 * enters bytes_fixed).
 */
typedef struct {
    int64_t bytes_per_box;    /* boxes, sort keys, cell copies, sorted arrays */
    int64_t bytes_per_pair;   /* pair, candidate slots, narrow-phase query scratch */
    int64_t bytes_per_scene;  /* per-scene statistics and cell layout */
    int64_t bytes_fixed;      /* control block and interval queue */
} ccd_memory_model;

int ccd_get_memory_model(const ccd_opts *o, ccd_memory_model *m);

/* The largest pair capacity P that fits mem_bytes for a step over n_boxes
 * boxes in n_scenes scenes under the model above (0 when even the boxes do
 * not fit).  Use it as opts.pair_capacity for a memory budget. */
int64_t ccd_pair_capacity_for(const ccd_opts *o, int64_t mem_bytes, int64_t n_boxes, int32_t n_scenes);

/* Enqueue on `stream` a copy of the context's device status (a CCD_*
 * value raised by its kernels, e.g. CCD_ETRUNC when pairs did not fit) into
 * *status (host pinned or device memory); no synchronization. */
int ccd_status_async(ccd_ctx *ctx, int32_t *status, void *stream);

/* Synchronize the context's last stream and read its device status and
 * counters (stats may be NULL).  Returns the device status. */
int ccd_get_status(ccd_ctx *ctx, ccd_stats *stats);

/* Stages timed when opts.profile_stages is set. */
enum { CCD_STAGE_BOXES = 0, CCD_STAGE_SORT = 1, CCD_STAGE_SWEEP = 2, CCD_STAGE_NARROW = 3,
       CCD_STAGE_NARROW_KERNEL = 4, CCD_NSTAGES = 5 };

/* Milliseconds spent in each stage by the last ccd_broad / ccd_narrow /
 * ccd_step call (CUDA events on its stream; boxes = box build and axis
 * choice, sort = keys (cell sweep: copies per cell), radix sort and
 * gather, sweep = sweep with the exact filter, narrow = query records and
 * the narrow-phase kernel, narrow_kernel = the narrow-phase kernel alone,
 * inside the narrow stage); stages the call did not run read 0.
 * Synchronizes the stream.  Returns CCD_EINVAL unless profile_stages was set. */
int ccd_stage_times(ccd_ctx *ctx, double ms[CCD_NSTAGES]);

/* Self-test of the narrow phase's failure detection, with no GPU fault:
 * runs the narrow-phase kernel on no queries with one unit counted as
 * pending that no lane will ever take.  Every warp idles until its idle
 * limit (about half a second) and leaves; the last one to leave finds the
 * count above zero and raises CCD_ETIMEOUT, as it would for work lost in a
 * real call.  *status (host memory) receives the device status the kernel
 * left: CCD_ETIMEOUT when detection works.  Synchronous on `stream`; the
 * context stays usable (the next call resets its status).  Returns CCD_OK,
 * or CCD_EINVAL / CCD_ENOMEM / CCD_ECUDA if it could not run. */
int ccd_selftest_unfinished_work(ccd_ctx *ctx, int32_t *status, void *stream);

/* Self-test of the broad phase's radix sort (Section "Broad-Phase": the boxes
 * sorted by their minimum; here the cell-and-minimum keys of the cell sweep):
 * sorts n (key, value) pairs in place, stably, by the low key_bits bits of
 * the key (0: all; key_bytes 4 or 8), with the library's kernels -- one
 * counting pass and one pass per 8-bit digit.  Passes of a digit that every
 * key shares are skipped two at a time, or (skip_all != 0, as the cell sort
 * does) all of them, with the result's buffers named on the device.  keys
 * (n x key_bytes) and vals (n x uint32) are device arrays.  n_cap >= n sizes
 * the launch; with n_cap > n the count is read from device memory, as the
 * broad phase does.
 * Allocates and frees its own buffers.  *status (host) receives the device
 * status (CCD_OK, or CCD_ETIMEOUT if a cross-tile wait ran out).  Synchronous
 * on `stream`.  Returns CCD_OK, CCD_EINVAL (bad sizes, n_cap >= 2^32),
 * CCD_ENOMEM or CCD_ECUDA. */
int ccd_selftest_radix_sort(ccd_ctx *ctx, int key_bytes, int key_bits, int64_t n, int64_t n_cap, int skip_all,
                            void *keys, uint32_t *vals, int32_t *status, void *stream);

/* Human-readable text of a CCD_* status (static storage). */
const char *ccd_status_str(int status);

/*
 * Measure this device's FP64 fused-multiply-add throughput with a kernel of
 * independent DFMA chains (the narrow phase's bound).  *gflops receives
 * 2 x DFMA per second / 1e9.  Synchronous; allocates and frees its own
 * small buffer.
 */
int ccd_measure_fp64_peak(int device, double *gflops);

/*
 * Serving.  Continuous batching of steps that arrive one scene at a time
 * (Section "Batching" runs the method over many independent inputs; here
 * they arrive over time).  The server owns a pinned host arena, n_slots
 * contexts each with its own stream, and a scheduler thread.  A client asks
 * for space for one scene (ccd_server_request), writes the scene there --
 * V0 and V1 as structure of arrays [3][nV], E [nE][2] and F [nF][3] with
 * vertex ids local to the scene -- and queues it (ccd_server_submit).
 * Whenever a slot is free, the scheduler takes the queued scenes in arrival
 * order, up to max_scenes scenes and max_boxes boxes and within the slot's
 * share of memory_cap (by the memory model above), and runs them as one
 * batched step (ccd_step_batch) on the slot's stream: one copy of the
 * scenes' contiguous arena range to the device, one kernel that lays them
 * out, the step, one copy of the per-scene earliest times back.  Slots run
 * concurrently, so copies of one batch overlap the work of another.
 * ccd_server_wait returns a scene's earliest time (+inf: no collision) and
 * its latency from submission to completion.  A scene's result does not
 * depend on the other scenes of its batch.
 */
typedef struct ccd_server ccd_server;

typedef struct {
    int32_t n_slots;         /* batches in flight at once (1-16); default 2 */
    int32_t max_scenes;      /* scenes per batch (1-65536); default 256 */
    int64_t max_boxes;       /* boxes per batch; default 2^24 */
    int64_t memory_cap;      /* device bytes for all slots (admission); default 64 GiB */
    int64_t arena_bytes;     /* pinned host arena; default 1 GiB */
    double delta, min_sep;   /* as in ccd_opts */
    int64_t max_iter;
    double pairs_per_box;    /* candidate pairs per box the admission budgets for
                                (0 = 4); a batch with more pairs fails with
                                CCD_ETRUNC */
    int32_t autotune;        /* 1: each slot runs ccd_autotune_batch on its first
                                batch (cell width, hand-off budget, queue) */
    int32_t pad;
} ccd_server_opts;

typedef struct {
    int64_t n_submitted;     /* scenes submitted */
    int64_t n_done;          /* scenes completed */
    int64_t n_batches;       /* batches launched */
    int64_t max_batch_scenes;  /* largest batch */
    double sum_latency_ms;   /* sum of completed scenes' latencies */
    int64_t max_batch_bytes; /* largest device-memory need of one batch (memory
                                model) that was admitted */
    int64_t max_inflight_bytes;  /* largest sum of those needs over the batches
                                    in flight at one time (at most memory_cap) */
} ccd_server_stats;

void ccd_server_default_opts(ccd_server_opts *o);

/* Start a server on `device` (o: NULL = defaults).  Errors: CCD_EINVAL (bad
 * option), CCD_ENOMEM (arena or context allocation), CCD_EDEVICE. */
int ccd_server_create(ccd_server **out, const ccd_server_opts *o, int device);

/* Stop the scheduler after the submitted scenes complete and free
 * everything (scenes requested but never submitted are dropped). */
int ccd_server_destroy(ccd_server *srv);

/* Reserve arena space for one scene of nV vertices, nE edges, nF faces; the
 * four pointers receive where to write it (pinned host memory, valid until
 * the scene's ccd_server_wait returns).  Blocks while the arena is full.
 * Scenes are batched in the order of their requests; a requested scene holds
 * back later ones until it is submitted.  CCD_ENOMEM: the scene alone does
 * not fit the arena, max_boxes or a slot's memory share. */
int ccd_server_request(ccd_server *srv, int64_t nV, int64_t nE, int64_t nF, double **V0, double **V1,
                       int32_t **E, int32_t **F, uint64_t *ticket);

/* Queue a written scene (thread-safe). */
int ccd_server_submit(ccd_server *srv, uint64_t ticket);

/* ccd_server_request, a copy of the scene from the caller's host arrays
 * (V0, V1 as [3][nV], E [nE][2], F [nF][3], local vertex ids) into the arena,
 * and ccd_server_submit, in one call (thread-safe; blocks while the arena is
 * full).  *ticket receives the scene's ticket for ccd_server_wait. */
int ccd_server_submit_scene(ccd_server *srv, int64_t nV, int64_t nE, int64_t nF, const double *V0,
                            const double *V1, const int32_t *E, const int32_t *F, uint64_t *ticket);

/* Wait up to timeout_ms (< 0: forever) for a submitted scene; on completion
 * writes its earliest time and latency (ms from submission to completion),
 * releases the ticket and returns the batch's device status (CCD_OK, or e.g.
 * CCD_ETRUNC).  CCD_ETIMEOUT: not done yet (the ticket stays valid). */
int ccd_server_wait(ccd_server *srv, uint64_t ticket, double timeout_ms, double *toi, double *latency_ms);

/* Counters; returns the first launch error seen (CCD_OK if none). */
int ccd_server_get_stats(ccd_server *srv, ccd_server_stats *st);

#ifdef __cplusplus
}
#endif

#endif /* GB300_CCD_H */
