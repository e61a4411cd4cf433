/*
 * vcm.h -- C ABI of libvcm, a GB300 (sm_103a) engine for visibility color maps.
 *
 * A visibility color map (VCM, Def. 1 of Section II-A of "Scalable
 * Visibility Color Map Construction in Spatial Databases") gives every point
 * of a discretised space a color in [0,1] that grows with how much of a
 * target T is visible from that point.  Visibility is the target's perceived
 * size: the visual angle (Eq. 1, Section II-B.1), shrunk by oblique viewing
 * (Section II-B.1, "Angle") and by obstacles that cut the line of sight
 * (point-to-point visibility, Def. 2 of Section II-B.2).
 *
 * This library computes the target-centric VCM on a dense viewpoint grid:
 *   - the target is an axis-aligned rectangle (3D) or segment (2D) split into
 *     patches_u x patches_w equal patches represented by their centres (each
 *     cell is represented by its centre, end of Section III-A);
 *   - viewpoints are the centres of the cells of an nx x ny grid on each of
 *     n_layers heights;
 *   - the segment from viewpoint q to patch centre p is blocked iff it meets
 *     an obstacle box; touching a box counts as meeting it (the shadow of an
 *     obstacle contains the points whose segment to T "intersects or
 *     touches" it, Def. 4 of Section III-B);
 *   - v(q) = sum over unblocked patches with cos(theta) > 0 of
 *     A cos(theta) / d^2 in 3D (solid angle of the visible part) or
 *     len cos(theta) / d in 2D (visible subtended angle; for an unobstructed
 *     target seen head-on this is Eq. 1);
 *   - color = 0 if v == 0, else 1 + min(L-2, floor((L-1) v / v_ref)), with
 *     v_ref the largest v of the request unless the caller gives one; level 0
 *     is the color of obstructed points (Section III-C).
 *
 * COORDINATES.  All lengths are metres, float32, and must lie on the lattice
 * of 2^-10 m with magnitude <= 16384 m (VCM_COORD_LIMIT_M); derived patch
 * centres and viewpoints are rounded to that lattice (halves away from zero).
 * Off-lattice, NaN or infinite inputs are rejected with VCM_E_ARG.  On this
 * lattice the occlusion bits are exact: they equal the real-number answer.
 *
 * CONVENTIONS.  Every call returns a vcm_status and never throws or aborts.
 * Host inputs are copied before the call returns; the caller keeps them.
 * Buffers returned in vcm_result belong to the context until
 * vcm_result_release.  Viewpoint order in outputs is ((layer*ny)+iy)*nx+ix.
 * Occlusion bits (VCM_EMIT_BITS) are ceil(P/32) uint32 words per viewpoint,
 * bit j of the viewpoint's bit string set iff patch j = iw*patches_u + iu is
 * blocked.  vcm_last_error returns a message for the calling thread's last
 * failed call.  A context may be used from several threads; calls that
 * change the scene (load, build) must not overlap running requests.
 */
#ifndef VCM_H
#define VCM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vcm_ctx vcm_ctx;

typedef enum {
    VCM_OK = 0,
    VCM_PENDING = 1,       /* vcm_poll: not finished yet */
    VCM_E_ARG = -1,        /* invalid argument, off-lattice or non-finite input */
    VCM_E_IO = -2,         /* scene file missing or malformed */
    VCM_E_NOMEM = -3,      /* device memory or the context's budget exhausted */
    VCM_E_CUDA = -4,       /* CUDA runtime error (message in vcm_last_error) */
    VCM_E_TIMEOUT = -5,    /* vcm_poll wait elapsed, or a device-side bounded wait gave up */
    VCM_E_CANCELLED = -6,  /* request cancelled before it ran */
    VCM_E_STATE = -7       /* call out of order (e.g. submit before build) */
} vcm_status;

/* Axis codes for target orientation. */
enum { VCM_AXIS_PX = 0, VCM_AXIS_NX = 1, VCM_AXIS_PY = 2, VCM_AXIS_NY = 3,
       VCM_AXIS_PZ = 4, VCM_AXIS_NZ = 5 };

/* Request flags.
 * VCM_EMIT_BITS: also produce the per-patch occlusion bits.
 * VCM_STRICT:    a viewpoint keeps the whole target's measure only if no
 *                patch is blocked, and gets 0 otherwise: the visible region
 *                holds the points from which the target is completely
 *                visible (Def. 3; end of Section III-B).
 * VCM_VIEWER:    viewer-centric VCM (Section IV-B): `center` is the viewer,
 *                `width` the size S of an object placed at every grid cell
 *                facing the viewer; a cell's value is the object's visual
 *                angle 2 atan(S / 2D) (2D, Eq. 1) or the solid angle of an
 *                S x S square, 4 asin(S^2 / (S^2 + 4 D^2)) (3D), with D the
 *                distance to the viewer, or 0 if the segment from the cell to
 *                the viewer meets a box (or D = 0).  Axes, height and patch
 *                counts are ignored; bits (one per cell) mark blocked cells.
 * VCM_TWO_SIDED: the target counts from both of its faces: a patch's term
 *                uses |n.(q - p)| instead of requiring n.(q - p) > 0, so
 *                viewpoints behind the target are measured too (viewpoints
 *                in its plane still get 0).  Not with VCM_VIEWER.
 * VCM_CACHE_BITS: (vcm_submit) keep the request's occlusion bits in the
 *                context, so that a later request for the same target,
 *                patch counts and viewpoint grid (scene unchanged) that
 *                differs only in field of view, gaze, sides, strictness,
 *                color levels or v_ref is served from them by recolouring,
 *                with no occlusion test (Section IV-C: when the gaze turns,
 *                the work done for every direction is reused).  The bits
 *                count against the budget; the least recently used are
 *                dropped when admission needs the memory, and all when the
 *                scene changes.  Ignored by the direct calls; not with
 *                VCM_VIEWER. */
enum { VCM_EMIT_BITS = 1u, VCM_STRICT = 2u, VCM_VIEWER = 4u, VCM_TWO_SIDED = 8u, VCM_CACHE_BITS = 16u };

#define VCM_UNITS_PER_M 1024
#define VCM_COORD_LIMIT_M 16384.0f
#define VCM_MAX_PATCHES_SIDE 4096u
#define VCM_MAX_PATCHES 65536u
#define VCM_MAX_LAYERS 4096u
#define VCM_MAX_GRID_SIDE 65536u

/* One VCM query (Def. 1: target-centric VCM of target T over a grid).
 * 3D: T is the rectangle centred at `center`, spanning `width` along axis_u
 * and `height` along axis_w, facing `normal` (three distinct axes).
 * 2D: T is the segment centred at (center[0], center[1]) spanning `width`
 * along axis_u (x or y), facing `normal` (the other of x, y); height,
 * axis_w, patches_w, n_layers and layer_z are ignored.
 * Patch (iu, iw) has centre center + ((iu+1/2)/patches_u - 1/2) width e_u
 * + ((iw+1/2)/patches_w - 1/2) height e_w, e_u and e_w the signed unit
 * vectors of axis_u and axis_w.
 * Viewpoint (ix, iy, layer) is (grid_origin + (i+1/2) grid_step, layer_z[layer]). */
typedef struct {
    int32_t dims;            /* 2 or 3 */
    float center[3];
    int32_t axis_u, axis_w, normal;
    float width, height;
    uint32_t patches_u, patches_w;
    float grid_origin[2], grid_step[2];
    uint32_t grid_nx, grid_ny;
    uint32_t n_layers;
    const float *layer_z;    /* host pointer, n_layers heights; copied */
    uint32_t color_levels;   /* L, 2..256 */
    float v_ref;             /* > 0: normalise by this; <= 0: by the largest v */
    uint32_t flags;          /* VCM_EMIT_BITS | VCM_STRICT | VCM_VIEWER | VCM_TWO_SIDED | VCM_CACHE_BITS */
    /* Field of view of the target (Section III-B: the visible region starts
     * as the part of space inside the FOV, 120 degrees by default in
     * Table II; Section IV-C turns the gaze).  fov_deg in (0, 360): patch p
     * counts for viewpoint q only if q lies in p's cone of half-angle
     * fov_deg / 2 around the axis `gaze` (world x, y, z; all 0 = the
     * target's facing normal; z ignored in 2D), i.e. with r = q - p and
     * a = g / |g|:  a.r >= cos(fov_deg / 2) |r|  (|a.r| with VCM_TWO_SIDED).
     * 0 or >= 360: no cone.  The kernels evaluate the inequality in float32
     * with one rounding per operation, in this order (world x, y, z):
     *   c = (float) cos(fov_deg * pi / 360)        (in double, then rounded)
     *   a = (float) (g / |g|) per component         (in double, then rounded)
     *   d = (a.x r.x + a.y r.y) + a.z r.z, |d| with VCM_TWO_SIDED
     *   inside iff d >= c * sqrt((r.x r.x + r.y r.y) + r.z r.z)
     * which errs in the margin a.r - c |r| by at most about 10.5 u |r|
     * (u = 2^-24), so it can differ from the exact decision only for pairs
     * within 1e-6 |r| of the cone's edge.  In strict mode a viewpoint still
     * gets 0 if any patch is blocked, and otherwise the sum over the patches
     * inside the cone.  Not with VCM_VIEWER. */
    float fov_deg;
    float gaze[3];
} vcm_request;

/* Values of vcm_stats.error: a device-side failure; a request whose error
 * is nonzero has an incomplete result.
 * VCM_DEVERR_BOUNDS:     a bounds check of a checked build (libvcm_checked,
 *                        compiled with VCM_CHECKED) failed; the access was
 *                        skipped instead of made.
 * VCM_DEVERR_SPILL_WAIT: a block of a launch that shares the GPU with other
 *                        launches gave up its bounded wait for a spill region
 *                        (a buffer for candidate lists longer than shared
 *                        memory holds) and cut such a list short.  vcm_poll
 *                        reports it as VCM_E_TIMEOUT.
 * The direct calls (vcm_compute, vcm_compute_batch, vcm_compute_static,
 * vcm_recolor) return once their work is enqueued: the caller finds a
 * failure in the error word of d_stats after the stream has run.  Their
 * launches own their spill regions, so only VCM_DEVERR_BOUNDS can occur
 * there. */
enum { VCM_DEVERR_NONE = 0, VCM_DEVERR_BOUNDS = 1, VCM_DEVERR_SPILL_WAIT = 2 };

/* Per-request counters written by the device. */
typedef struct {
    float v_ref;                       /* the v_ref used for colors */
    uint32_t vmax_bits;                /* largest v (float bits), accumulated on device */
    uint32_t edge_cells;               /* viewpoints within 1e-5 (relative) of a color bin edge */
    uint32_t error;                    /* VCM_DEVERR_*: nonzero if a device-side check failed */
    unsigned long long slab_tests;     /* lane-level slab tests executed in the row sweep */
    unsigned long long rechecked;      /* segment-box pairs re-decided by the exact float64 predicate */
    unsigned long long segments;       /* viewpoint-patch pairs decided (= viewpoints x patches) */
    unsigned long long boxes_listed;   /* sum over tiles of culled candidate-list lengths */
    unsigned long long corner_tests;   /* segment-box tests of the one-box-blocks-all check */
    unsigned long long shortcut_viewpoints;  /* viewpoints decided by that check */
    unsigned long long shared_viewpoints;    /* open viewpoints handed from their tile to the chunk pass */
} vcm_stats;

/* Results of a submitted request; all pointers owned by the context. */
typedef struct {
    const float *v;            /* host: visibility per viewpoint */
    const uint8_t *color;      /* host: color level per viewpoint */
    const uint32_t *bits;      /* host: occlusion bits (VCM_EMIT_BITS) or NULL */
    const float *d_v;          /* device copies of the same */
    const uint8_t *d_color;
    const uint32_t *d_bits;
    uint64_t n_viewpoints;
    uint32_t words_per_viewpoint;
    vcm_stats stats;
    double latency_ms;         /* submit -> completion observed by the context */
    double queue_ms;           /* submit -> its launch began (admission and queueing) */
    double device_ms;          /* device time of the launch that ran it: its whole group, from its
                                  descriptor upload to its results copied to host memory, with any
                                  wait for the kernels of the launch before it */
    uint32_t group_size;       /* requests in that launch */
    uint32_t launch_form;      /* VCM_FORM_* of that launch */
    double launch_ms;          /* host time the scheduler spent enqueuing that launch */
    double chain_ms;           /* of device_ms, the wait for the kernels of the launch before it
                                  (0 when that launch had finished) */
} vcm_result;

/* How the scheduler launched a group (vcm_result.launch_form).
 * VCM_FORM_PERSISTENT: a persistent grid with the chunk pass (every launch
 *   but those below).
 * VCM_FORM_ONE_TILE:   one block per tile, whose blocks claim spill regions
 *   with a bounded wait (VCM_INJECT_SPILL_BUSY).
 * VCM_FORM_RECOLOR:    recoloured from occlusion bits cached by an earlier
 *   request (VCM_CACHE_BITS); stats.slab_tests and corner_tests are 0. */
enum { VCM_FORM_PERSISTENT = 0, VCM_FORM_ONE_TILE = 1, VCM_FORM_RECOLOR = 2 };

/* Autotuned launch shape for one class of request (see vcm_autotune). */
typedef struct {
    uint32_t tile_x, tile_y;   /* viewpoints per tile (a tile is one block's work item) */
    uint32_t patch_k;          /* patch rows per lane held in registers per pass (0 = auto; at most 8) */
    uint32_t box_cap;          /* candidate boxes staged in shared memory per tile */
} vcm_tune;

/* ---- context --------------------------------------------------------- */

/* Create a context on CUDA device `device`.  mem_budget_bytes bounds the
 * device memory of the asynchronous path (0 = 64 GiB): the result buffers
 * of admitted requests, the occlusion bits kept for recolouring
 * (VCM_CACHE_BITS), and the scratch of the scheduler's execution slots.
 * A slot's scratch is a descriptor buffer, a spill list of n_boxes ints per
 * block that can be resident (about 365 MB per slot for 100,000 boxes on
 * 152 SMs) and a 74 MB work buffer through which the blocks of a launch
 * share the open viewpoints of expensive tiles; it is allocated when the
 * slot first runs a launch that needs it and kept.  The direct path
 * (vcm_compute, vcm_compute_batch, vcm_recolor) has scratch of its own,
 * which the budget does not count. */
vcm_status vcm_ctx_create(int device, size_t mem_budget_bytes, vcm_ctx **out);

/* Wait for all work of the context, then free everything it owns. */
void vcm_ctx_destroy(vcm_ctx *ctx);

/* Message for the calling thread's last failed call ("" if none).  Valid
 * until the next call on the same thread. */
const char *vcm_last_error(vcm_ctx *ctx);

/* ---- scene ------------------------------------------------------------ */

/* Obstacles (the set O of Def. 1) as axis-aligned boxes, given by corners.
 * lo/hi: host arrays of n_boxes x dims floats (dims = 2: rectangles in the
 * plane; 3: boxes), lo <= hi componentwise, on the lattice.  Replaces any
 * previous scene; the index must then be rebuilt with vcm_build. */
vcm_status vcm_scene_load_mem(vcm_ctx *ctx, const float *lo, const float *hi,
                              uint32_t n_boxes, int32_t dims);

/* Same, from a file: "VCMS" magic, uint32 version = 1, int32 dims, uint32 n,
 * then n*dims float32 lo and n*dims float32 hi (little endian). */
vcm_status vcm_scene_load(vcm_ctx *ctx, const char *path);

/* Write the current scene in the format read by vcm_scene_load. */
vcm_status vcm_scene_save(vcm_ctx *ctx, const char *path);

/* Build the device uniform-grid index over the box footprints (cell edge
 * grid_cell_m metres, > 0; 0 picks one from the scene's density).  Boxes
 * are bucketed by centre and each bucket keeps the bounds of its boxes.
 * The scene is immutable afterwards until the next load.  Synchronous. */
vcm_status vcm_build(vcm_ctx *ctx, float grid_cell_m);

/* ---- direct device path ---------------------------------------------- */

/* Enqueue one request on `stream` (a cudaStream_t; NULL = legacy default)
 * writing into caller-owned device buffers: d_v (n_viewpoints floats),
 * d_color (n_viewpoints bytes, or NULL to skip colors), d_bits
 * (n_viewpoints * ceil(P/32) words, required iff VCM_EMIT_BITS) and d_stats
 * (one vcm_stats).  Returns once the work is enqueued.  Calls on one
 * context share its scratch and must not overlap on the device; issue them
 * on one stream.  The first call for a larger shape may allocate scratch
 * (and synchronises the device once). */
vcm_status vcm_compute(vcm_ctx *ctx, const vcm_request *req, float *d_v, uint8_t *d_color,
                       uint32_t *d_bits, vcm_stats *d_stats, void *stream);

/* ---- asynchronous requests (continuous batching) --------------------- */

/* Queue a request.  Non-blocking: a scheduler thread admits queued requests
 * as execution slots and budgeted memory free up, and runs each admitted
 * group as one batched persistent launch while another group is still on
 * the device: its upload and counters go at once, its kernels follow the
 * other's back to back, and the results of one are copied while the next
 * computes.
 * A launch whose parameters equal those of the slot's previous launch of
 * the same form is replayed from a CUDA graph captured then; others are
 * launched directly.  VCM_E_NOMEM if the request's results together with
 * one slot's scratch exceed the budget. */
vcm_status vcm_submit(vcm_ctx *ctx, const vcm_request *req, uint64_t *ticket);

/* Queue several requests that must run together in one batched launch. */
vcm_status vcm_submit_batch(vcm_ctx *ctx, const vcm_request *reqs, uint32_t n, uint64_t *tickets);

/* VCM_OK when finished, VCM_PENDING if still queued or running after
 * waiting up to wait_ms (-1 = forever), or the request's error: VCM_E_NOMEM
 * (its buffers could not be allocated with nothing else in flight),
 * VCM_E_CUDA (a launch or copy failed, or a device-side bounds check),
 * VCM_E_TIMEOUT (a bounded device-side wait gave up, VCM_DEVERR_SPILL_WAIT),
 * VCM_E_CANCELLED. */
vcm_status vcm_poll(vcm_ctx *ctx, uint64_t ticket, int32_t wait_ms);

/* Results of a finished request (host copies and device buffers). */
vcm_status vcm_result_get(vcm_ctx *ctx, uint64_t ticket, vcm_result *out);

/* Free a finished or cancelled request's buffers and forget the ticket. */
vcm_status vcm_result_release(vcm_ctx *ctx, uint64_t ticket);

/* Cancel a request that has not been admitted yet (VCM_E_STATE if it has). */
vcm_status vcm_cancel(vcm_ctx *ctx, uint64_t ticket);

/* Scheduler limits: number of execution slots (1..16; 2 by default), i.e.
 * the launches in flight at once, each on a stream of its own, and the
 * largest number of requests merged into one launch (64 by default).  Each
 * slot holds scratch (see vcm_ctx_create). */
vcm_status vcm_set_slots(vcm_ctx *ctx, uint32_t slots, uint32_t max_batch);

/* Device memory of the asynchronous path, in bytes. */
typedef struct {
    uint64_t budget;             /* the context's budget */
    uint64_t results;            /* result buffers of admitted requests not yet released */
    uint64_t slot_scratch;       /* scratch the scheduler's slots hold now */
    uint64_t slot_scratch_need;  /* scratch one slot needs for the current scene (counted
                                    against the budget before a slot first runs) */
    uint64_t cached_bits;        /* occlusion bits kept for recolouring (VCM_CACHE_BITS) */
    uint32_t cache_entries;
} vcm_memory;
vcm_status vcm_get_memory(vcm_ctx *ctx, vcm_memory *out);

/* Drop the occlusion bits kept for recolouring (VCM_CACHE_BITS) that no
 * running request uses. */
vcm_status vcm_cache_clear(vcm_ctx *ctx);

/* Per-request metric lines and latency percentiles of the asynchronous
 * path (a serving aid; the paper reports only total times and error
 * percentages).  With a path, every request whose scheduler launch
 * completes appends one JSON object, on a line of its own, to that file:
 * ticket, status (0 or the request's vcm_status), latency_ms, queue_ms,
 * launch_ms, device_ms, chain_ms, group_size, launch_form, viewpoints,
 * patches, segments, and the counters of vcm_stats (slab_tests,
 * corner_tests, rechecked, edge_cells, shortcut_viewpoints,
 * shared_viewpoints, v_ref).  The scheduler's waiter threads write the
 * lines after each launch, outside the context lock, and flush the file.
 * The file is opened for appending; NULL closes it.  VCM_E_ARG if it cannot
 * be opened. */
vcm_status vcm_set_request_log(vcm_ctx *ctx, const char *path);

/* Latency (submit to completion) percentiles, nearest rank, over the last
 * 4,096 requests the scheduler completed without error, and how many it has
 * completed since the context was created.  p50 and p99 are 0 before the
 * first. */
vcm_status vcm_latency_summary(vcm_ctx *ctx, double *p50_ms, double *p99_ms, uint64_t *completed);

/* Host-side fault injection, for testing how failures surface (nothing
 * here faults or stalls the GPU).
 * VCM_INJECT_SPILL_BUSY: the next `count` launches of the scheduler run one
 *   block per tile with every spill region already marked held and a claim
 *   limit of 8 rounds (microseconds), so a tile whose candidate list is
 *   longer than shared memory holds gives up its bounded wait: its request
 *   finishes with VCM_E_TIMEOUT.
 * VCM_INJECT_ALLOC_FAIL: the next `count` device allocations of request
 *   buffers by the scheduler fail as if the device had no memory left.
 * VCM_INJECT_NONE with count 0 clears both. */
enum { VCM_INJECT_NONE = 0, VCM_INJECT_SPILL_BUSY = 1, VCM_INJECT_ALLOC_FAIL = 2 };
vcm_status vcm_inject(vcm_ctx *ctx, uint32_t kind, uint32_t count);

/* ---- batching and tuning --------------------------------------------- */

/* Run n requests as one persistent launch on `stream`, into caller-owned
 * device buffers (arrays of n pointers, same meaning as vcm_compute). */
vcm_status vcm_compute_batch(vcm_ctx *ctx, const vcm_request *reqs, uint32_t n, float *const *d_v,
                             uint8_t *const *d_color, uint32_t *const *d_bits, vcm_stats *d_stats,
                             void *stream);

/* Time candidate launch shapes on the given sample requests and keep the
 * fastest per request class (patch count bucket); later launches use it.
 * Writes the chosen shape for each sample to out (may be NULL).  Viewer-
 * centric requests (VCM_VIEWER) keep a fixed shape of 32 x 16 cells. */
vcm_status vcm_autotune(vcm_ctx *ctx, const vcm_request *samples, uint32_t n, vcm_tune *out);

/* Force a launch shape for all later launches (tile_x = 0 restores tuning). */
vcm_status vcm_set_tune(vcm_ctx *ctx, const vcm_tune *tune);

/* Launch shape the context would use for this request launched alone
 * (a launch with fewer tiles than four waves of resident blocks has its
 * tiles shrunk, 16 x 16 -> 16 x 8 -> 8 x 8 -> 8 x 4, unless a shape is
 * forced with vcm_set_tune). */
vcm_status vcm_get_tune(vcm_ctx *ctx, const vcm_request *req, vcm_tune *out);

/* ---- without device allocation ----------------------------------------- */

#define VCM_STATIC_MAX_BOXES 4096u
#define VCM_STATIC_MAX_COORDS 65536u   /* patches_u + patches_w + grid_nx + grid_ny + n_layers */
#define VCM_STATIC_SCRATCH_BYTES (8u << 20)

/* One request computed without allocating any device memory, for callers
 * that must not call cudaMalloc: code running under an allocator that owns
 * all device memory (a framework's caching pool, a fixed memory budget), or
 * a plug-in that may not change the process's device footprint while it
 * runs.  The paper has no counterpart; this is an interface convenience.
 *
 * Inputs: the obstacle boxes as host arrays lo/hi of n_boxes x dims floats
 * (same rules as vcm_scene_load_mem) and the request.  Outputs: caller-owned
 * device buffers with the meaning of vcm_compute (d_v, d_color or NULL,
 * d_bits iff VCM_EMIT_BITS, d_stats).  No context is needed.  The index,
 * descriptors and counters live in one file-scope device array of
 * VCM_STATIC_SCRATCH_BYTES, which every GPU that loads libvcm holds until
 * the process exits.  Requests beyond VCM_STATIC_MAX_BOXES boxes or
 * VCM_STATIC_MAX_COORDS coordinates are rejected with VCM_E_ARG.
 *
 * The work is enqueued on `stream` (a cudaStream_t, NULL = legacy default)
 * of the current device; host inputs are consumed before the call returns.
 * The first call on a device looks up the array's device address and
 * uploads constant tables; make that first call before any stream capture.
 * Every call on a device reuses that device's array and leaves the last
 * call's contents in it (each call clears what must start at zero).  Calls
 * whose work overlaps on the same GPU, e.g. on two streams, race on the
 * array: serialise them, for instance by issuing them on one stream. */
vcm_status vcm_compute_static(const float *lo, const float *hi, uint32_t n_boxes, int32_t dims,
                              const vcm_request *req, float *d_v, uint8_t *d_color, uint32_t *d_bits,
                              vcm_stats *d_stats, void *stream);

/* ---- incremental gaze change ------------------------------------------ */

/* Recolour a target-centric request from occlusion bits made earlier, with
 * no occlusion test (Section IV-C: when the gaze turns, only the field of
 * view changes, so the work done once for every direction is reused).  A
 * request's occlusion bits do not depend on its field of view, gaze, sides
 * or strictness.  So one vcm_compute with VCM_EMIT_BITS serves every later
 * gaze: `req` must describe the same target, patch counts and viewpoint
 * grid as that computation, while its fov_deg, gaze, VCM_TWO_SIDED,
 * VCM_STRICT, color_levels and v_ref may differ (VCM_EMIT_BITS is ignored;
 * VCM_VIEWER is rejected with VCM_E_ARG).  The result equals what
 * vcm_compute would give for `req`.
 *
 * d_bits: device, n_viewpoints x ceil(P/32) words as VCM_EMIT_BITS wrote
 * them (read only).  d_v (n_viewpoints floats), d_color (n_viewpoints bytes,
 * or NULL) and d_stats (one vcm_stats; slab_tests and corner_tests stay 0):
 * caller-owned device outputs.  At most 2^31 - 1 viewpoints.  Enqueued on
 * `stream` (a cudaStream_t, NULL = legacy default); needs no scene.  The
 * context keeps n_viewpoints ints of device scratch (grown on demand).  The caller keeps d_bits unchanged
 * until the work has run.  The call uses the context's descriptor buffer
 * and so is serialised with vcm_compute on the same context. */
vcm_status vcm_recolor(vcm_ctx *ctx, const vcm_request *req, const uint32_t *d_bits, float *d_v,
                       uint8_t *d_color, vcm_stats *d_stats, void *stream);

/* ---- profiling --------------------------------------------------------- */

/* Record two caller-created CUDA events (cudaEvent_t) on the launch stream
 * immediately before and after the tile kernel (both of its passes) of every
 * later direct-path launch (vcm_compute, vcm_compute_batch) and the recolour
 * kernel of every later vcm_recolor; NULL, NULL stops.  The events must
 * outlive their use. */
vcm_status vcm_set_timing_events(vcm_ctx *ctx, void *before_tiles, void *after_tiles);

#ifdef __cplusplus
}
#endif
#endif /* VCM_H */
