/*
 * dqj.h -- C ABI of libdqj, a GB300 (sm_103a) renderer for isosurfaces of 3-D
 * slices of dual-quaternion Julia sets (Kenwright, "Dual-Quaternion Julia
 * Fractals").
 *
 * Method (paper references by section / equation):
 *   - zeta_{n+1} = zeta_n^2 + c in 8-component dual-quaternion algebra
 *     (Method, "Dual-Quaternion Julia Sets", Eq. dqjulia2; products from the
 *     appendix, "Dual-Quaternion Operations");
 *   - a sample escapes at the first n with modulus > R^2, and counts as inside
 *     when it has not escaped after max_iter steps (Method, "Practical
 *     Considerations");
 *   - the 8-D space is cut by a 3-D slice, five coordinates held fixed
 *     (Method, "Dimension Reduction");
 *   - each pixel's ray is marched through a bounding box, the first inside
 *     sample refined by bisection, or sphere-traced by the distance estimate of
 *     Eq. distfract2 (Method, "Ray-Marching"); a normal comes from central
 *     differences of neighbouring samples (Method, "Lighting/Illumination")
 *     and is shaded with the ambient and diffuse terms of Eq. phong, and its
 *     specular term when k_specular > 0.
 *
 * All functions return a dqj_status; no C++ exception crosses this boundary.
 * On a non-OK status, dqj_last_error() returns a message for the calling thread.
 * Functions are thread-safe unless stated otherwise.
 */
#ifndef DQJ_H
#define DQJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DQJ_ABI_VERSION 1

typedef struct dqj_ctx dqj_ctx;
typedef uint64_t dqj_ticket;

typedef enum {
    DQJ_OK = 0,
    DQJ_ERR_INVALID = 1,   /* bad argument or parameter block                      */
    DQJ_ERR_NOMEM = 2,     /* device or host allocation failed                     */
    DQJ_ERR_BUSY = 3,      /* serving queue full (max_pending reached)             */
    DQJ_ERR_TIMEOUT = 4,   /* a bounded wait ran out                               */
    DQJ_ERR_CUDA = 5,      /* a CUDA runtime call failed; message has the detail   */
    DQJ_ERR_NOT_FOUND = 6, /* unknown or already consumed ticket                   */
    DQJ_ERR_CANCELLED = 7  /* request cancelled by dqj_destroy                     */
} dqj_status;

/* dqj_params.precision */
enum {
    DQJ_FP32 = 0,         /* FP32 throughout                                         */
    DQJ_FP32_RECHECK = 1, /* FP32, samples within recheck_margin of R^2 re-evaluated
                             in FP64 on the GPU; a pixel whose FP64 decision differs
                             is re-rendered in FP64                                  */
    DQJ_FP64 = 2          /* FP64 throughout                                         */
};

/* dqj_params.square_mode (Method, "Dual-Quaternion Julia Sets") */
enum {
    DQJ_SQUARE_ALGEBRAIC = 0,          /* zeta^2 = q_r^2 + (q_r q_d + q_d q_r) eps   */
    DQJ_SQUARE_PAPER_COMPONENTWISE = 1 /* zeta^2 = q_r^2 + q_d^2 eps, as printed     */
};

/* dqj_params.traversal (Method, "Ray-Marching").  MARCH: march_steps + 1
 * equally spaced samples over the box, the first inside one refined by
 * bisect_steps halvings.  DE: the paper's own traversal, sphere tracing by the
 * distance estimate of Eq. distfract2, d = 0.5 |zeta_n| / |zeta'_n| ln |zeta_n|
 * at the escape step n, with |zeta'_{n+1}| = 2 |zeta_n| |zeta'_n| (Eq. distfract)
 * and |zeta| = sqrt(modulus): from the entry into the box (and the bounding
 * sphere of radius de_bound_radius, when positive) a ray samples, hits at an
 * inside sample or one whose estimate is below de_epsilon, otherwise advances
 * by de_step_scale times the estimate, and misses when it leaves the volume
 * or after de_max_steps samples.  A hit's depth is its sample's t and n* its
 * escape count (max_iter when inside); a miss reports the largest escape
 * count over its samples.  DE supports every precision.  Its FP32 +
 * FP64-recheck mode re-traces every hit pixel in FP64 (the FP32 trace's ray
 * parameter accumulates the rounding of each estimate) and rechecks in FP64 the
 * samples of the other pixels whose escape test came within the margin of R^2
 * or whose estimate lies near de_epsilon, re-tracing in FP64 the pixels whose
 * decisions could differ. */
#define DQJ_TRAVERSAL_MARCH 0
#define DQJ_TRAVERSAL_DE 1

/* dqj_params.modulus_mode (Introduction; appendix, magnitude) */
enum {
    DQJ_MODULUS_EUCLID8 = 0, /* |q_r|^2 + |q_d|^2                                   */
    DQJ_MODULUS_DUALNUM = 1  /* |q_r|^2, the dual-number modulus of zeta zeta*      */
};

/* dqj_config.device value for a CPU-only context whose serving entry points run
 * against a mock device (for testing admission, budgets and timeouts without a
 * GPU); it cannot render.  The mock reads DQJ_MOCK_DELAY_US (run time of a
 * request, default 1000) and DQJ_MOCK_FAIL ("nomem": every admission fails,
 * "hang": no request ever completes, "throw_start" / "throw_admit": a host
 * allocation fails while serving starts / while a batch is admitted) from the
 * environment when serving starts.  It loads a tile cache written for device
 * "unknown" with 0 SMs (dqj_tile_shape then reports its entries). */
#define DQJ_DEVICE_MOCK (-1)

/* Per-context configuration for dqj_create. */
typedef struct {
    int32_t device;            /* CUDA device ordinal, or DQJ_DEVICE_MOCK               */
    uint64_t mem_budget_bytes; /* serving: device bytes admitted requests may occupy
                                  (outputs the library allocates + scratch); 0 = 16 GiB */
    int32_t max_pending;       /* serving: host queue bound; 0 = 4096                   */
    const char *autotune_cache;/* path of the tile-shape cache (JSON) or NULL: the
                                  env var DQJ_AUTOTUNE_CACHE, else built-in defaults    */
} dqj_config;

/*
 * One render request.  Every length is in scene units, angles in degrees.
 * Dual quaternions are 8 doubles (q_r | q_d), scalar first in each half
 * (appendix, quaternion definition).
 */
typedef struct {
    double c[8];                /* Julia constant (Eq. dqjulia2)                      */
    double slice_origin[8];     /* 8-D point the 3-D slice passes through             */
    double slice_basis[3][8];   /* orthonormal 3-frame: scene x,y,z -> R^8
                                   ("Dimension Reduction"); orthonormal to 1e-9       */
    double eye[3], target[3], up[3];
    double fov_y_deg;           /* vertical field of view, 0 < fov < 180              */
    int32_t width, height;      /* 1..16384 each                                      */
    int32_t max_iter;           /* 1..1024 ("Practical Considerations")               */
    double escape_radius;       /* R > 0; escape when modulus > R^2 (strict)          */
    int32_t march_steps;        /* N in 1..65535: samples t_in + k (t_out-t_in)/N,
                                   k = 0..N, over the ray's part inside the box       */
    int32_t bisect_steps;       /* B in 0..30 halvings of the first crossing          */
    double normal_h;            /* central-difference step h > 0                      */
    double box_min[3], box_max[3]; /* march volume, box_min < box_max                 */
    double light_dir[3];        /* direction to the light (normalised internally)     */
    double k_ambient, k_diffuse;/* Eq. phong coefficients                             */
    double albedo[3];           /* per-channel factor in [0, 1]                       */
    int32_t precision;          /* DQJ_FP32 | DQJ_FP32_RECHECK | DQJ_FP64             */
    double recheck_margin;      /* DQJ_FP32_RECHECK: |modulus - R^2| <= margin * R^2
                                   marks a sample for FP64 re-evaluation; 0..0.5      */
    int32_t square_mode;        /* DQJ_SQUARE_*                                       */
    int32_t modulus_mode;       /* DQJ_MODULUS_*                                      */
    double k_specular;          /* Eq. phong specular coefficient k_s >= 0 (0: off)   */
    double shininess;           /* Eq. phong specular exponent s, 0..10000            */
    int32_t traversal;          /* DQJ_TRAVERSAL_MARCH | DQJ_TRAVERSAL_DE             */
    int32_t de_max_steps;       /* DE: samples per ray at most, 1..1000000            */
    double de_epsilon;          /* DE: a sample whose estimate is below this is a hit */
    double de_step_scale;       /* DE: step = scale * estimate, (0, 1]                */
    double de_bound_radius;     /* DE: bounding sphere about the origin, 0 = box only */
} dqj_params;

/*
 * Output planes, row-major with a row pitch in pixels (>= width).  Pixel (x, y)
 * lives at element y * pitch_px + x; normal holds 3 floats and rgba 4 bytes per
 * pixel at 3x / 4x that element offset.  For dqj_render / dqj_submit these are
 * DEVICE pointers owned by the caller, valid until the render completes; for
 * dqj_render_host they are HOST pointers.  Any plane may be NULL (not written).
 *
 *   iter   hit: escape count of the final outside bisection end (max_iter when
 *          the first march sample is inside); miss: largest escape count over
 *          the march samples (0 when the ray misses the box)
 *   depth  ray parameter of the hit (midpoint of the final bracket), +inf on miss
 *          (DQJ_TRAVERSAL_DE: the hit sample's t and escape count, see
 *          dqj_params.traversal)
 *   normal unit normal (+gradient of the modulus field), (0,0,0) on miss
 *   rgba   shaded colour, alpha 255 on hit; (0,0,0,0) on miss
 *   stats  optional DEVICE (render) / HOST (render_host) array of DQJ_NSTATS
 *          int64 counters, overwritten with this render's counts
 */
typedef struct {
    int32_t *iter;
    float *depth;
    float *normal;
    uint8_t *rgba;
    int64_t pitch_px;
    int64_t *stats;
} dqj_outputs;

/* Indices into dqj_outputs.stats. */
enum {
    DQJ_STAT_CLASS_ITERS = 0,  /* DQ iterations of march + bisection (or DE) samples  */
    DQJ_STAT_NORMAL_ITERS = 1, /* DQ iterations of the six normal evaluations         */
    DQJ_STAT_SAMPLES = 2,      /* classified samples (march + bisection, or DE)       */
    DQJ_STAT_HITS = 3,         /* hit pixels                                          */
    DQJ_STAT_RECHECKS = 4,     /* samples re-evaluated in FP64                        */
    DQJ_STAT_FIXUPS = 5,       /* pixels re-rendered in FP64 after a disagreement     */
    DQJ_STAT_FIXUP_ITERS = 6,  /* DQ iterations spent by those re-renders             */
    DQJ_STAT_OVERFLOW = 7,     /* recheck-queue overflows (pixel re-rendered instead) */
    DQJ_STAT_MARCH_ITERS = 8,  /* part of CLASS_ITERS spent by march samples          */
    DQJ_STAT_RESERVED = 9,
    DQJ_NSTATS = 10
};

/* Fill *p with the defaults of the single-frame scene: c = (-0.2, 0.6, 0.2, 0.2 |
 * 0.1, 0, 0, 0.05), real-quaternion coordinates 0..2 free, 256x256, max_iter 12,
 * R = 4, N = 256, B = 8, h = 1e-4, box [-2,2]^3, eye (0,0,3.5) looking at the
 * origin, up +y, fov 45, light (1,1,1), k_a 0.15, k_d 0.85, white albedo,
 * DQJ_FP32, margin 1e-3, algebraic square, EUCLID8 modulus, no specular term
 * (k_s 0, s 32), DQJ_TRAVERSAL_MARCH (DE fields: 512 steps, epsilon 1e-3,
 * scale 1, no bounding sphere). */
dqj_status dqj_default_params(dqj_params *p);

/* Check a parameter block on the host (no device needed).  DQJ_ERR_INVALID
 * with a message naming the first offending field. */
dqj_status dqj_validate_params(const dqj_params *p);

/* Create a context on cfg->device (NULL cfg: device 0, defaults).  The context
 * owns its scratch memory, streams and the serving thread. */
dqj_status dqj_create(const dqj_config *cfg, dqj_ctx **out);

/* Enqueue one frame on cuda_stream (a cudaStream_t; NULL = legacy default) and
 * return without waiting.  Outputs are caller-owned device memory.  Renders on one
 * context are ordered with each other across streams (they share scratch).
 * Stream capture (CUDA graphs): a render may be captured once the context has
 * rendered a frame at least as large (with the same precision class), since a
 * captured render neither allocates nor synchronizes (DQJ_ERR_INVALID
 * otherwise).  Renders captured together are ordered with each other; the
 * caller orders the capture after the context's earlier work (e.g. by
 * synchronizing first), replays of graphs holding renders of one context
 * must not overlap each other or other renders on it, and such graphs are
 * destroyed before the context (they use its events and scratch memory). */
dqj_status dqj_render(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *out, void *cuda_stream);

/* Frame split (several GPUs, one process each): render only the tiles t of
 * the frame with t mod parts == part, writing their pixels' outputs and
 * leaving every other pixel of the planes untouched.  Tile t covers the pixels
 * with (y / th) * ceil(width / tw) + x / tw == t, where (tw, th) is
 * dqj_tile_shape's tile for the march and 8 x 4 for DQJ_TRAVERSAL_DE.  The
 * parts' planes put together (each pixel from the part that owns its tile)
 * equal dqj_render's exactly: every pixel's arithmetic is its own.  part = 0,
 * parts = 1 is dqj_render.  DQJ_ERR_INVALID unless 0 <= part < parts <= 65536.
 * Stats count the part's own work.  An interface of this library (the frame
 * split across GPUs); the paper has no counterpart. */
dqj_status dqj_render_tiles(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *out, void *cuda_stream,
                            int32_t part, int32_t parts);

/* Enqueue n frames on cuda_stream, p[i] into the device outputs out[i] (the
 * output sets must not overlap), and return without waiting.  The frames
 * alternate between two context-owned scratch sets and two context-owned
 * streams forked from and joined back into cuda_stream; each frame's march
 * starts after the previous frame's march, so a frame's bisection and FP64
 * recheck passes run beside the next frame's march.  Results and stats equal
 * n calls of dqj_render.  Every frame is validated before any work starts
 * (DQJ_ERR_INVALID); n = 0 does nothing, n = 1 is dqj_render.  Ordered with
 * the context's other renders like dqj_render.  Not under stream capture
 * (DQJ_ERR_INVALID; capture dqj_render calls instead).  Holds a second
 * scratch set as large as the largest frame needs.  An interface of this
 * library (throughput of a batch of frames); the paper has no counterpart. */
dqj_status dqj_render_batch(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *out, int32_t n,
                            void *cuda_stream);

/* Render one frame into HOST buffers: the library renders into context-owned
 * device planes, copies the requested planes to the host and waits.  Blocking. */
dqj_status dqj_render_host(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *host_out);

/* Render n frames into HOST buffers, p[i] into host_out[i], and wait.  The
 * context keeps two device plane sets, so the copy back of frame i overlaps
 * the render of frame i + 1 (use page-locked host buffers for the overlap);
 * the renders themselves are pipelined as in dqj_render_batch.
 * Every frame is validated before any work starts (DQJ_ERR_INVALID); results
 * equal n calls of dqj_render_host.  n = 0 does nothing.  Blocking.  An
 * interface of this library (throughput for host-resident outputs); the paper
 * has no counterpart. */
dqj_status dqj_render_host_batch(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *host_out, int32_t n);

/* Serving: queue a request and return a ticket at once.  Outputs are
 * caller-owned device memory that must stay valid until dqj_poll reports done
 * and must have no pending work on any stream at submit: the library writes
 * them from its own streams, unordered with the caller's.
 * Requests are admitted to the GPU while their footprint fits the context's
 * memory budget; admitted requests run together in one persistent launch.
 * DQJ_ERR_BUSY when max_pending requests are queued and not yet admitted. */
dqj_status dqj_submit(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *out, dqj_ticket *ticket);

/* Serving counters since the context started serving, DQJ_NSERVE_STATS int64
 * values (all 0 before the first dqj_submit):
 *   [0] persistent launches      [1] launches stopped to recycle control blocks
 *   [2] requests run in the persistent launch   [3] requests run as plain frames
 *   [4] admission batches        [5] host nanoseconds spent admitting batches
 *   [6] requests completed       [7] scheduler loop iterations
 *   [8] most requests admitted and unfinished at the same time
 *   [9] requests of the persistent launch whose device execution (first work
 *       item claimed to completion, by the device clock) overlapped that of
 *       another request among the 256 that finished before it
 * An interface of this library (observability); the paper has no counterpart. */
#define DQJ_NSERVE_STATS 10
dqj_status dqj_serve_stats(dqj_ctx *ctx, int64_t *out);

/* Order in which queued requests are admitted and the persistent launch
 * serves the admitted ones (requests that run as plain frames keep their
 * admission position):
 *   DQJ_SERVE_FIFO      arrival order (the default);
 *   DQJ_SERVE_SHORTEST  earliest estimated finish: each request's key is its
 *                       arrival time at dqj_submit plus an estimate of its own
 *                       march time (width x height x (march_steps + 1) samples
 *                       at 2^-9 ns each).  Small requests overtake a large one
 *                       that arrived less than their difference in cost
 *                       earlier, in the host queue (admission waits for the
 *                       memory budget and a device slot in key order) and on
 *                       the device; no request is overtaken by one that
 *                       arrives after its own estimated finish, so none starves.
 * A request takes the policy in force when it is submitted; results are
 * unchanged (every request equals its dqj_render alone).  DQJ_ERR_INVALID for
 * an unknown policy.
 * An interface of this library (serving latency); the paper has no counterpart. */
#define DQJ_SERVE_FIFO 0
#define DQJ_SERVE_SHORTEST 1
dqj_status dqj_serve_policy(dqj_ctx *ctx, int32_t policy);

/* Non-blocking completion check.  *done = 1 and *result = the request's status
 * once finished; the ticket is then consumed (a second poll: DQJ_ERR_NOT_FOUND). */
dqj_status dqj_poll(dqj_ctx *ctx, dqj_ticket ticket, int *done, dqj_status *result);

/* Cancel queued requests (their tickets finish with DQJ_ERR_CANCELLED), wait for
 * admitted ones for at most DQJ_DESTROY_TIMEOUT_MS (environment, default 10000)
 * and free everything.  DQJ_ERR_TIMEOUT when admitted requests were still
 * running; their device memory is then left allocated rather than freed under a
 * kernel that may still use it. */
dqj_status dqj_destroy(dqj_ctx *ctx);

/* Autotuning of the march tile shape (an interface of this library; the paper
 * has no counterpart).  For each of the first max_classes frame-size classes
 * (<= 256^2, <= 512^2, <= 1024^2, larger; 0 = all four) and each iteration bucket
 * (max_iter <= 12, <= 20, <= 28, larger) renders a probe frame with every
 * candidate shape of the paired FP32 march (8x8, 16x4, 4x16, 32x2, 64x1 rays),
 * keeps the fastest (CUDA events, best of three) for later renders and served
 * requests on this context, and writes the table to the cache file (the
 * dqj_config path, else DQJ_AUTOTUNE_CACHE, else none).  dqj_create loads a
 * cache written on the same device model.  Blocking; allocates ~50 MB of
 * temporary planes. */
dqj_status dqj_autotune(dqj_ctx *ctx, int32_t max_classes);

/* The march kernel variant (0 one ray per lane, 1 two rays per lane) and tile
 * shape this context would use for p. */
dqj_status dqj_tile_shape(dqj_ctx *ctx, const dqj_params *p, int32_t *variant, int32_t *tile_w, int32_t *tile_h);

/* Profiling: with ring_frames > 0 (at most 4096), every later render on this
 * context records CUDA events on its own stream before its first pass and after
 * each pass, into a ring that keeps the last ring_frames renders; 0 turns this
 * off.  dqj_pass_ms waits for the `frames` most recent recorded renders (oldest
 * first, frames <= ring_frames) and writes 4 floats per render: elapsed ms of
 * the march, of bisection + normal + shading, of the FP64 recheck and of the
 * FP64 re-render (0 for passes that did not run).  DQJ_ERR_NOT_FOUND when fewer
 * renders were recorded. */
dqj_status dqj_set_profiling(dqj_ctx *ctx, int32_t ring_frames);
dqj_status dqj_pass_ms(dqj_ctx *ctx, int32_t frames, float *ms);

/*
 * dqj_voxelize -- voxel occupancy grid (Fig. voxels: the paper's voxel
 * prototype, which the paper compares with the ray-traced image).
 *
 * Classifies the centre of every cell of a grid_n^3 grid over the march box
 * [box_min, box_max] like a ray sample: cell (i, j, k) has centre
 * box_min + (idx + 1/2) (box_max - box_min) / grid_n per axis, is mapped into
 * the slice (slice_origin, slice_basis) and iterated (c, max_iter,
 * escape_radius, square_mode, modulus_mode, precision; recheck_margin for
 * DQJ_FP32_RECHECK).  The camera, image size, march, normal and shading fields
 * of p are validated but unused.
 *
 * Outputs (caller-owned device memory, linear index (k grid_n + j) grid_n + i,
 * x fastest; either may be NULL but not both):
 *   occupancy  uint8[grid_n^3]: 1 when the centre stays bounded for max_iter
 *              steps (inside), else 0;
 *   counts     uint16[grid_n^3], 2-byte aligned: escape count 1..max_iter, 0 inside;
 *   stats      int64[DQJ_NSTATS] or NULL: [CLASS_ITERS] DQ iterations of the
 *              classification, [SAMPLES] cells, [HITS] inside cells of the
 *              final grid, [RECHECKS] cells re-classified in FP64, [FIXUPS]
 *              cells the FP64 pass changed, [FIXUP_ITERS] its iterations,
 *              [OVERFLOW] recheck-queue overflows (the whole grid is then
 *              re-classified in FP64).
 * Stream-ordered on cuda_stream like dqj_render, and ordered with the
 * context's renders.  Errors: DQJ_ERR_INVALID for a bad p, grid_n outside
 * 1..DQJ_VOXEL_MAX_GRID, misaligned or both-NULL outputs, or a mock context.
 */
#define DQJ_VOXEL_MAX_GRID 1024
dqj_status dqj_voxelize(dqj_ctx *ctx, const dqj_params *p, int32_t grid_n, uint8_t *occupancy, uint16_t *counts,
                        int64_t *stats, void *cuda_stream);

/*
 * dqj_render_voxels -- image of a voxel grid from the scene camera (Fig. voxels
 * sets the ray-traced image beside renders of 50^3 and 100^3 voxel grids; the
 * paper drew its cubes with a geometry shader, here each camera ray walks the
 * grid).
 *
 * The grid is drawn as the union of its occupied cells, cell (i, j, k) being the
 * closed cube box_min + [idx, idx + 1] (box_max - box_min) / grid_n per axis.
 * Each pixel's camera ray (eye, target, up, fov_y_deg, width, height: the
 * camera of dqj_render) shows the first occupied cube it crosses, found by
 * walking the ray through the grid cell by cell in FP64.  Outputs, as for
 * dqj_render (caller-owned device planes, any may be NULL, pitch_px >= width,
 * 4-byte aligned):
 *   iter    cells the ray crossed up to and including the hit cube; on a miss
 *           all cells it crossed (0 when it misses the box);
 *   depth   ray parameter at which the ray enters the hit cube (the box entry
 *           when the first cell is occupied); +inf on a miss;
 *   normal  outward normal of the face entered, -sign(d_a) e_a (-d when the eye
 *           is inside the hit cube); (0,0,0) on a miss;
 *   rgba    the ambient, diffuse and (k_specular > 0) specular terms of Eq. phong
 *           with that normal; (0,0,0,0) on a miss.
 * occupancy is grid_n^3 bytes of device memory, nonzero = occupied, linear index
 * (k grid_n + j) grid_n + i as written by dqj_voxelize.  The Julia, march and
 * precision fields of p are validated but unused.  Stream-ordered on
 * cuda_stream; uses no context memory.  A choice between two cell faces that
 * lie within rounding of each other may go either way.  Errors: DQJ_ERR_INVALID
 * for a bad p or outputs, grid_n outside 1..DQJ_VOXEL_MAX_GRID, NULL occupancy
 * or a mock context; DQJ_ERR_CUDA for a failed launch.
 */
dqj_status dqj_render_voxels(dqj_ctx *ctx, const dqj_params *p, int32_t grid_n, const uint8_t *occupancy,
                             const dqj_outputs *out, void *cuda_stream);

/* Largest width * height dqj_render_noalloc accepts (e.g. 512 x 512). */
#define DQJ_NOALLOC_MAX_PIXELS 262144u

/*
 * dqj_render_noalloc -- the plain render (either traversal) without any device
 * allocation.  (An interface of this library; the paper has no counterpart.)
 *
 * For callers that must not allocate device memory.  Examples: a host
 * application that reserves all device memory for its own pool before loading
 * this library, or a frame loop that must not block on the allocator.
 * It needs no context: its scratch (the counter block and hit list of the march
 * and bisection passes) is a fixed array inside the library, about 4 MiB, which
 * every device that loads the library holds until the process exits.
 *
 * p, out and cuda_stream as for dqj_render: out holds caller-owned DEVICE planes
 * (and an optional device stats array).  Runs on the current device; the first
 * call on each device looks up the array's device address with
 * cudaGetSymbolAddress.  Under lazy module loading (the CUDA default) that
 * first call is also when the array is placed on the device, so make it before
 * reserving the device's memory for your own pool, and before any stream
 * capture.  The address is kept for the life of the process: cudaDeviceReset
 * after the first call is not supported.  The march kernel and tile shape are
 * dqj_render's defaults (no autotuned shapes: there is no context).
 * Stream-ordered: enqueues and returns.  Allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  Errors: DQJ_ERR_INVALID when
 * width * height > DQJ_NOALLOC_MAX_PIXELS or precision is DQJ_FP32_RECHECK
 * (only DQJ_FP32 and DQJ_FP64 are supported), plus dqj_render's checks.
 * Every call shares the one array and clears its counters at the start; calls
 * that overlap on the GPU (different streams or threads) race on it, so order
 * them on one stream.
 */
dqj_status dqj_render_noalloc(const dqj_params *p, const dqj_outputs *out, void *cuda_stream);

/* Message for the last non-OK status on this thread ("" if none). */
const char *dqj_last_error(void);

/* Measurement: FMA throughput of this GPU with independent dependency chains
 * (the roofline denominator of the renderer).  variant 0 = scalar fma.rn.f32,
 * 1 = paired fma.rn.f32x2, 2 / 3 = as 0 / 1 with two integer operations per
 * eight FMAs, 4 = fma.rn.f64; only FMAs count as flops.  Runs `launches` timed
 * launches on device `device`; *flops_per_s gets the best.  An interface of
 * this library; the paper has no counterpart. */
dqj_status dqj_fma_peak(int32_t device, int32_t variant, int32_t launches, double *flops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* DQJ_H */
