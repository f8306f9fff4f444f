/*
 * rf.h -- C ABI of the GB300 (sm_103a) Radiant Foam renderer.
 *
 * Differentiable ray tracing through a 3D Voronoi foam (Govindarajan et al.,
 * "Radiant Foam: Real-Time Differentiable Ray Tracing", arXiv 2502.01157).
 * The scene is a set of sites p_i (Sec. 3.2, Eq. 5); each Voronoi cell carries
 * a density sigma_i and spherical-harmonic colour coefficients (Sec. 3.4).
 * Rays walk cell to cell (Alg. 1) and composite Eq. (3)-(4).
 *
 * Conventions for every call:
 *   - Pointers documented "device" are CUDA device pointers owned by the
 *     caller; the library never frees them.  "host" pointers are read during
 *     the call only.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t, NULL = the
 *     legacy default stream); outputs are valid once the stream reaches that
 *     point.  Calls return after enqueueing.
 *   - Every call returns an rf_status; on failure rf_last_error() gives a
 *     message (thread-local, valid until the next call on the same thread).
 *     Invalid arguments are rejected before anything is enqueued.
 *   - Per-ray anomalies (the step cap was reached) are reported in the
 *     optional per-ray status output, not as a call failure.
 *   - Calls that use one rf_scene must be ordered on one stream: the scene
 *     owns a small device workspace (start cells per camera) that renders
 *     reuse.
 */
#ifndef RF_H
#define RF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
#define RF_API extern "C" __attribute__((visibility("default")))
#else
#define RF_API __attribute__((visibility("default")))
#endif

#define RF_VERSION 1
#define RF_MAX_SH_DEGREE 3

typedef enum rf_status {
    RF_OK = 0,
    RF_ERR_INVALID_ARG = 1,  /* a pointer, size, dtype or camera is invalid */
    RF_ERR_CUDA = 2,         /* a CUDA runtime call failed (message has the reason) */
    RF_ERR_OOM = 3,          /* device allocation failed */
    RF_ERR_BUSY = 4,         /* serving: request not admitted (memory or slots) */
    RF_ERR_NOT_READY = 5,    /* serving: request still in flight */
    RF_ERR_TIMEOUT = 6,      /* a bounded wait ran out */
    RF_ERR_BAD_SCENE = 7,    /* adjacency / positions failed validation */
    RF_ERR_NOT_FOUND = 8     /* serving: unknown request id */
} rf_status;

/* Storage type of the per-cell attributes (density, SH coefficients).
 * Geometry, plane intersections and compositing are always FP32. */
typedef enum rf_dtype { RF_F32 = 0, RF_BF16 = 1, RF_F16 = 2 } rf_dtype;

/* Per-ray status codes (optional output). */
enum { RF_RAY_OK = 0, RF_RAY_MAX_STEPS = 1 };

/*
 * Scene description (Sec. 3.2: "a learnable point cloud" of Voronoi sites
 * whose Delaunay adjacency N(i) is maintained alongside; Sec. 3.4: per-cell
 * density and degree <= 3 SH colour).
 *
 *   pos       device float [n_sites][3]   site positions p_i.
 *   adj_off   device int32 [n_sites+1]    CSR offsets, adj_off[0] = 0,
 *                                          adj_off[n_sites] = n_edges.
 *   adj_idx   device int32 [n_edges]      neighbour ids N(i) of each site, in
 *                                          the order exits are tie-broken
 *                                          (first wins).  Must be symmetric,
 *                                          in range, without self loops or
 *                                          duplicate positions.  A superset of
 *                                          the Delaunay neighbours renders the
 *                                          same image; a missing neighbour
 *                                          does not.
 *   density   device [n_sites] of attr_dtype          sigma_i >= 0 (after
 *                                                     the activation).
 *   sh        device [n_sites][(deg+1)^2][3] of attr_dtype  coefficients,
 *             real orthonormal SH index l*l+l+m, RGB innermost; the colour is
 *             max(0, sum_k sh[i][k][c] Y_k(d) + 0.5).
 *             density and sh are BORROWED: the scene keeps the pointers; the
 *             caller keeps them alive and may rewrite their contents between
 *             renders (see rf_scene_set_attributes to swap them).
 *             Both must be 16-byte aligned.
 *   aabb_min/max  scene box; every ray is clipped to it.  If min > max on
 *             any axis the box of the sites is computed on the device.
 */
typedef struct rf_scene_desc {
    int64_t n_sites;
    int64_t n_edges;
    const float *pos;
    const int32_t *adj_off;
    const int32_t *adj_idx;
    const void *density;
    const void *sh;
    int32_t sh_degree;
    int32_t attr_dtype;
    float aabb_min[3];
    float aabb_max[3];
} rf_scene_desc;

/*
 * Camera (the ray origins o and unit directions d of Alg. 1; the camera
 * models and the rolling shutter are the non-linear cameras of the paper's
 * ray-based effects figure, Fig. 2).
 *   c2w      row-major 3x4 [R | t]: camera-frame point x -> R x + t; the
 *            camera frame is OpenCV (+x right, +y down, +z forward); t is the
 *            centre.
 *   fx, fy, cx, cy  intrinsics in pixels; pixel (u,v) casts the ray through
 *            its centre: x = (u+.5-cx)/fx, y = (v+.5-cy)/fy and
 *            RF_CAM_PINHOLE:  d = normalise(R (x, y, 1));
 *            RF_CAM_FISHEYE:  equidistant, th = sqrt(x^2+y^2) is the angle to
 *                             the optical axis, d = R (x sin(th)/th,
 *                             y sin(th)/th, cos(th)).
 *   width, height   image size; ray index = v * width + u.
 *   t_near, t_far   compositing interval along d, intersected with the scene
 *            box (t_far <= 0: no limit).
 *   model    RF_CAM_PINHOLE or RF_CAM_FISHEYE.
 *   shutter  rolling shutter: displacement of the centre over the frame;
 *            row v's rays start at t + ((v+.5)/height - .5) * shutter
 *            (all zero: global shutter, every ray starts at t).
 */
enum { RF_CAM_PINHOLE = 0, RF_CAM_FISHEYE = 1 };

typedef struct rf_camera {
    float c2w[12];
    float fx, fy, cx, cy;
    int32_t width, height;
    float t_near, t_far;
    int32_t model;
    float shutter[3];
} rf_camera;

/*
 *   eps        transmittance threshold: a ray continues while T > eps
 *              (Alg. 1).  Default when opts == NULL: 1e-4.
 *   max_steps  cap on cell steps per ray (<= 0: 65536); a capped ray gets
 *              RF_RAY_MAX_STEPS.
 *   flags      0, or RF_RENDER_SHARED_CELLS for the backward: the crossing
 *              terms of a cell are summed over the lanes of a warp that
 *              share it before their atomic, in warp iterations whose rays
 *              are in at most 2 distinct cells.  Faster where many rays
 *              cross the same cells (large empty cells, cameras far from the
 *              foam: a 1M-site Gaussian-mixture frame's backward 1.93 ->
 *              1.19 ms on a GB300), slower on dense uniform foams (~4 rays
 *              per cell: 3M uniform sites 9.15 -> 10.1 ms).  Same results
 *              up to the order of the floating-point atomics.  Other bits:
 *              RF_ERR_INVALID_ARG.
 *   max_bounces, sphere, sphere_ior  optional analytic sphere met in the
 *              same walk (reflection / refraction of Fig. 2): centre
 *              sphere[0..2], radius sphere[3] > 0; sphere_ior = 0 for a
 *              perfect mirror, > 0 for clear glass of that refractive index
 *              (Snell refraction, total internal reflection).  In each cell
 *              a hit before the exit face ends the segment there; the ray
 *              bends at the hit point and walks on from the same cell with
 *              t0 = 0, clipped to the scene box only.  A ray meets the
 *              sphere at most max_bounces times, then passes through it.
 *              max_bounces = 0: no sphere.  Depth is the path length along
 *              the bent ray.  The sphere is fixed: it receives no gradient
 *              and passes none to the sites.
 */
#define RF_RENDER_SHARED_CELLS 1u

typedef struct rf_render_opts {
    float eps;
    int32_t max_steps;
    uint32_t flags;
    int32_t reserved;
    int32_t max_bounces;
    float sphere[4];
    float sphere_ior;
} rf_render_opts;

typedef struct rf_scene rf_scene;

RF_API int32_t rf_version(void);
RF_API const char *rf_last_error(void);

/*
 * Packs the foam for traversal: per site a 16-byte record (position, first
 * neighbour) and per directed edge (i, j) a 16-byte face record holding the
 * bisector normal scaled by 2/|p_j - p_i|^2 and j, so each face test of
 * Alg. 1 is one coalesced 16-byte load.  Validates the adjacency on the
 * device (range, self loops, symmetry, zero-length edges) and returns
 * RF_ERR_BAD_SCENE if it fails.  Allocates the packed copy (16 B per edge
 * plus 20 B per site) with cudaMalloc; synchronises `stream` once.
 */
RF_API rf_status rf_scene_create(const rf_scene_desc *desc, void *stream, rf_scene **out);

/* Swaps the borrowed attribute pointers / dtype (same n_sites, sh_degree). */
RF_API rf_status rf_scene_set_attributes(rf_scene *scene, const void *density, const void *sh,
                                         int32_t attr_dtype);

/* Re-packs after the sites moved (same adjacency); pos: device [n_sites][3]. */
RF_API rf_status rf_scene_update_positions(rf_scene *scene, const float *pos, void *stream);

/* Scene facts: counts, the box used (6 floats, may be NULL) and device bytes owned. */
RF_API rf_status rf_scene_info(const rf_scene *scene, int64_t *n_sites, int64_t *n_edges,
                               float *aabb6, size_t *device_bytes);

/* Frees the packed copy; waits for the device. */
RF_API rf_status rf_scene_destroy(rf_scene *scene);

/*
 * Forward render of n_cams cameras in one launch (Alg. 1 per ray, Eq. 3-4).
 * Outputs are concatenated camera after camera (ray r of camera c at
 * sum_{c'<c} W_c' H_c' + r):
 *   rgb    device float [R][3]   composited colour (black background).
 *   trans  device float [R]      final transmittance T.
 *   depth  device float [R]      sum_n T_n alpha_n (a_n + b_n)/2 over the
 *                                composited part [a_n, b_n] of each segment.
 *   steps  device int32 [R] or NULL   cells visited.
 *   ray_status device uint8 [R] or NULL   RF_RAY_*.
 * cams is a host array.  A ray that misses the scene box gives rgb 0, T 1,
 * depth 0, steps 0.
 */
RF_API rf_status rf_render_fwd(rf_scene *scene, const rf_camera *cams, int32_t n_cams,
                               const rf_render_opts *opts, float *rgb, float *trans,
                               float *depth, int32_t *steps, uint8_t *ray_status, void *stream);

/*
 * Backward of rf_render_fwd: each ray is walked again with bit-identical
 * arithmetic (no per-segment storage) and the gradient of
 *   L = sum d_rgb . rgb + sum d_trans * trans + sum d_depth * depth
 * is ACCUMULATED (+=) into
 *   g_density device float [n_sites]
 *   g_sh      device float [n_sites][(deg+1)^2][3]
 *   g_pos     device float [n_sites][3]   (through the segment widths only,
 *                                          Sec. 3.1)
 * rgb / trans / depth are the forward outputs of the same call arguments
 * (depth may be NULL when d_depth is NULL); d_trans / d_depth may be NULL
 * (zero).  Any gradient output may be NULL to skip it.
 */
RF_API rf_status rf_render_bwd(rf_scene *scene, const rf_camera *cams, int32_t n_cams,
                               const rf_render_opts *opts, const float *rgb,
                               const float *trans, const float *depth, const float *d_rgb,
                               const float *d_trans, const float *d_depth, float *g_density,
                               float *g_sh, float *g_pos, void *stream);

/*
 * Extended forward / backward with the quantile loss of Eq. (6) (Sec. 3.3):
 *   L_q = E_{u1,u2 ~ U[0,1]} |W^-1(u1) - W^-1(u2)|,
 * W^-1 the quantile function of the ray's weight distribution T(t) sigma(t)
 * normalised over the composited interval, i.e. 2 int F(1 - F) dt with
 * F = (1 - T(t)) / (1 - T_final); 0 for a ray with no weight.  It is
 * accumulated in the same walk as the colour (closed form per segment).
 *
 *   outputs of rf_render_fwd_ex (device, rays of all cameras concatenated):
 *     rgb, trans, depth  required, as rf_render_fwd
 *     steps, ray_status  optional
 *     quantile           optional float [R]
 *     quantile_aux       float [R][5], required with quantile: per-ray sums the
 *                        backward of the quantile loss reads
 *     walk_record        optional device buffer, 16-byte aligned, of
 *                        walk_record_bytes >=
 *                        rf_walk_record_bytes(cams, n_cams, walk_record_steps):
 *                        the forward stores there, for the first
 *                        walk_record_steps steps of every ray, the segment it
 *                        composited (Eq. 3-4): the neighbour it left the cell
 *                        for, the exit parameter, the cell's density and its
 *                        colour before the clamp (24 bytes per step).  Given
 *                        to rf_render_bwd_ex with the same cameras, options
 *                        and scene, it lets the backward rebuild those steps
 *                        instead of reading the faces and attributes again;
 *                        the gradients are the same up to the order of the
 *                        floating-point atomics.  A record of another scene
 *                        gives wrong gradients; a neighbour id outside the
 *                        scene ends that ray's backward walk (no access out of
 *                        bounds).
 */
typedef struct rf_fwd_outputs {
    float *rgb;
    float *trans;
    float *depth;
    int32_t *steps;
    uint8_t *ray_status;
    float *quantile;
    float *quantile_aux;
    uint8_t *walk_record;
    size_t walk_record_bytes;
    int32_t walk_record_steps;
} rf_fwd_outputs;

/*   inputs of rf_render_bwd_ex (device):
 *     rgb, trans, depth      forward outputs (depth may be NULL without d_depth)
 *     quantile_aux           forward output, required with d_quantile
 *     d_rgb                  required; d_trans, d_depth, d_quantile optional
 *     walk_record            optional: the forward's walk record (same
 *                            walk_record_bytes and walk_record_steps)
 *   gradients (device, FP32, accumulated +=, each may be NULL):
 *     density [N], sh [N][(deg+1)^2][3], pos [N][3]
 *   With density or pos requested, the first backward on a scene allocates a
 *   16-byte-per-site workspace owned by the scene (counted in rf_scene_info's
 *   device_bytes; RF_ERR_OOM if it cannot), and every backward zeroes it on
 *   the stream, sums the site terms into it and adds it to pos and density
 *   after the walk. */
typedef struct rf_bwd_inputs {
    const float *rgb;
    const float *trans;
    const float *depth;
    const float *quantile_aux;
    const float *d_rgb;
    const float *d_trans;
    const float *d_depth;
    const float *d_quantile;
    const uint8_t *walk_record;
    size_t walk_record_bytes;
    int32_t walk_record_steps;
} rf_bwd_inputs;

/* Bytes of a walk record of `steps` steps per ray for these cameras: 24
 * bytes per step for every ray slot of the 16x8 tiles (rays are grouped by
 * warps of 32); 0 for bad arguments. */
RF_API size_t rf_walk_record_bytes(const rf_camera *cams, int32_t n_cams, int32_t steps);

typedef struct rf_grads {
    float *density;
    float *sh;
    float *pos;
} rf_grads;

RF_API rf_status rf_render_fwd_ex(rf_scene *scene, const rf_camera *cams, int32_t n_cams,
                                  const rf_render_opts *opts, const rf_fwd_outputs *out,
                                  void *stream);
RF_API rf_status rf_render_bwd_ex(rf_scene *scene, const rf_camera *cams, int32_t n_cams,
                                  const rf_render_opts *opts, const rf_bwd_inputs *in,
                                  const rf_grads *grads, void *stream);

/*
 * Debug / parity: the cells each ray of one camera visits, in order.
 *   cells   device int32 [R][max_per_ray]  (-1 after the last cell)
 *   counts  device int32 [R]                total cells visited (may exceed
 *                                           max_per_ray)
 */
RF_API rf_status rf_trace_cells(rf_scene *scene, const rf_camera *cam,
                                const rf_render_opts *opts, int32_t max_per_ray,
                                int32_t *cells, int32_t *counts, void *stream);

/*
 * Serving: continuous batching of render requests over a resident scene
 * (the paper's renderer, Sec. 3.4, turned into a request loop).
 *
 *   mem_budget_bytes  device memory reserved for in-flight outputs: 20 B per
 *                     ray (rgb, T, depth); the same number of rays x 12 B of
 *                     pinned host memory receives the images.  A request is
 *                     admitted only if its rays fit in the free part.
 *   max_inflight      admitted requests not yet collected.
 *   n_streams         batches that may run on the device at the same time.
 *   max_batch         cameras (any resolutions) per launch, 1..16.
 *   eps, max_steps    as in rf_render_opts.
 *
 * A scheduler thread launches waiting admitted requests, up to max_batch at a
 * time, on any free stream; requests that arrive while others run start as
 * soon as a stream frees up.  Images are bit-identical to rf_render_fwd of
 * the same camera (rays are independent).  The server borrows the scene,
 * which must outlive it.  All calls are thread-safe.
 */
typedef struct rf_serve_config {
    size_t mem_budget_bytes;
    int32_t max_inflight;
    int32_t n_streams;
    int32_t max_batch;
    float eps;
    int32_t max_steps;
} rf_serve_config;

typedef struct rf_serve_metrics {
    int64_t completed;     /* requests rendered (since creation or the last reset) */
    int64_t rejected;      /* submits refused (RF_ERR_BUSY or too large) */
    int64_t rays_done;
    int64_t batches;       /* launches */
    double p50_ms, p99_ms, mean_ms, max_ms;  /* latency: submit -> image in host memory */
    double mrays_s;        /* rays_done / (last completion - first submit) */
    double mean_batch;     /* requests per launch */
    int32_t max_busy_streams;
    int32_t inflight;
} rf_serve_metrics;

typedef struct rf_server rf_server;

RF_API rf_status rf_serve_create(rf_scene *scene, const rf_serve_config *cfg, rf_server **out);
/* Admits one request (cam: host) or returns RF_ERR_BUSY (no memory / slot);
 * RF_ERR_INVALID_ARG if it can never fit. */
RF_API rf_status rf_serve_submit(rf_server *srv, const rf_camera *cam, uint64_t *req_id);
/* *done = 1 once rendered; then the image (rgb, [H*W][3] floats) is copied to
 * host_rgb (may be NULL), the latency reported and the request released. */
RF_API rf_status rf_serve_poll(rf_server *srv, uint64_t req_id, float *host_rgb, int32_t *done,
                               double *latency_ms);
/* As rf_serve_poll but waits up to timeout_ms (RF_ERR_TIMEOUT after). */
RF_API rf_status rf_serve_wait(rf_server *srv, uint64_t req_id, int32_t timeout_ms, float *host_rgb,
                               double *latency_ms);
RF_API rf_status rf_serve_stats(rf_server *srv, rf_serve_metrics *out);
RF_API rf_status rf_serve_reset_stats(rf_server *srv);
/* Stops the scheduler, waits for launched work, frees the pools. */
RF_API rf_status rf_serve_destroy(rf_server *srv);

/*
 * Forward render that allocates no device memory (no counterpart in the
 * paper; an interface of this library).  It is for callers that cannot call
 * cudaMalloc -- code running under another runtime or engine that owns the
 * device allocator and forbids allocations from outside, or a latency-bound
 * render loop where an allocation would stall -- and so cannot create an
 * rf_scene, whose packed copy and workspace are allocated.
 *
 * Inputs are the caller's own device arrays, as in rf_scene_desc (pos
 * [n_sites][3], adj_off [n_sites+1], adj_idx [n_edges], density, sh), plus
 * the scene box aabb6 (HOST, min xyz then max xyz, min <= max required);
 * outputs rgb [R][3], trans [R], depth [R] as in rf_render_fwd, with the same
 * values (the face records are formed on the fly with the packer's FP32
 * operations).  The adjacency is not validated; out-of-range offsets or ids
 * end the affected ray instead of being read.
 *
 * Its only scratch, one 64-bit start-cell key per camera, lives in a fixed
 * device array inside the library (64 entries, 512 bytes, held on every
 * device that loads the library until the process exits).  Hence:
 *   - at most 64 cameras per call; more returns RF_ERR_INVALID_ARG;
 *   - every call shares that array: calls that overlap on the GPU (on
 *     different streams, or from different threads) race and must not be
 *     issued concurrently; calls ordered on one stream are safe;
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress), so make that first call before any stream
 *     capture.
 * Pinhole and fisheye cameras are supported; a rolling shutter (nonzero
 * camera shutter) or a sphere (opts->max_bounces > 0) returns
 * RF_ERR_INVALID_ARG: their per-ray start cells and bounces need the packed
 * scene.
 */
RF_API rf_status rf_render_fwd_noalloc(int64_t n_sites, int64_t n_edges, const float *pos,
                                       const int32_t *adj_off, const int32_t *adj_idx,
                                       const void *density, const void *sh, int32_t sh_degree,
                                       int32_t attr_dtype, const float *aabb6,
                                       const rf_camera *cams, int32_t n_cams,
                                       const rf_render_opts *opts, float *rgb, float *trans,
                                       float *depth, void *stream);

/*
 * Densification and pruning statistics (Sec. 3.3 "Densification",
 * "Pruning").
 *
 * rf_densify_scores: score[i] = |g_pos[i]| * r_i with r_i half the mean
 *   distance from site i to its Delaunay neighbours (the approximate cell
 *   radius: the faces lie halfway to the neighbours).  g_pos: device float
 *   [N][3] (e.g. the accumulated position gradient); score: device float [N].
 * rf_prune_mask: mask[i] = 1 iff density[i] < threshold and density[j] <
 *   threshold for every neighbour j (a low-density cell that does not bound a
 *   denser one).  mask: device uint8 [N]; reads the scene's current
 *   attributes.
 * rf_sample_multinomial: m draws of indices in [0, n) with probability
 *   weights[k] / sum (negative weights count as 0), as in the paper's
 *   multinomial choice of densification candidates.  u: device float [m],
 *   uniform numbers in [0, 1) supplied by the caller; a draw takes the first
 *   k whose inclusive FP64 prefix sum exceeds u * total.  workspace: device,
 *   8-byte aligned, at least rf_multinomial_workspace_bytes(n) bytes (the
 *   prefix sums); n <= 16,777,216.  out: device int32 [m].
 */
RF_API rf_status rf_densify_scores(rf_scene *scene, const float *g_pos, float *score, void *stream);
RF_API rf_status rf_prune_mask(rf_scene *scene, float threshold, uint8_t *mask, void *stream);
RF_API size_t rf_multinomial_workspace_bytes(int64_t n);
RF_API rf_status rf_sample_multinomial(const float *weights, int64_t n, const float *u, int64_t m,
                                       void *workspace, size_t workspace_bytes, int32_t *out,
                                       void *stream);

/*
 * GPU Voronoi adjacency: the neighbour lists N(i) the walk traverses (the
 * Delaunay graph of the sites), built from the positions alone and rebuilt
 * whenever they move (the paper keeps this adjacency through training and
 * updates it after position steps: the "Voronoi optimization" paragraph of
 * Sec. 4, with the tracing of Sec. 3.2).
 *
 * j is a neighbour of i iff their Voronoi cells share a face of positive area
 * inside the domain box (the part of the bisector plane of p_i and p_j that
 * is no farther from them than from any other site).  Each cell is built on
 * the GPU as the domain box cut by the bisector half-spaces of nearby sites;
 * every inside/outside decision is the FP64 one.  The lists are symmetric,
 * sorted by neighbour id, without self loops: ready for rf_scene_desc.
 *
 * rf_adjacency_build: pos device float [n_sites][3] (1 <= n_sites <= 10^8);
 *   domain6 HOST float[6] (min xyz, max xyz) holding every site, or NULL for
 *   the sites' bounding box grown by 5% of its extent (at least 1e-3) on
 *   every side.  Faces that
 *   lie entirely outside the domain are not produced, so the domain should
 *   hold the cameras as well as the sites.  incremental = 1 seeds each cell
 *   with its previous neighbours (the sites moved a little since the last
 *   build of the same n_sites); the result is the same as a full build.  The
 *   call waits for the GPU three times (sites' box, edge count, completion).
 *   Errors: RF_ERR_INVALID_ARG (bad sizes, non-finite positions, a site
 *   outside domain6), RF_ERR_OOM, RF_ERR_BAD_SCENE (too many one-sided edges:
 *   heavily degenerate sites).
 * rf_adjacency_result: device pointers to the CSR (adj_off [n_sites + 1],
 *   adj_idx [n_edges]) owned by the handle and valid until its next build or
 *   destroy, and statistics (host).
 */
typedef struct rf_adjacency rf_adjacency;
typedef struct rf_adjacency_stats {
    int64_t n_sites, n_edges;
    int64_t edges_before_symmetry;  /* directed edges the cells produced */
    int64_t asym_added;             /* reverse edges added for symmetry */
    int64_t wide_sites;             /* cells rebuilt with room for up to 186 faces */
    int64_t failed_sites;           /* cells that could not be built (empty rows) */
    int64_t fp64_tests;             /* vertex tests decided in FP64 */
    int32_t max_degree;
    int32_t reserved;
    float domain[6];
} rf_adjacency_stats;
RF_API rf_status rf_adjacency_create(rf_adjacency **out);
RF_API rf_status rf_adjacency_build(rf_adjacency *adj, int64_t n_sites, const float *pos,
                                    const float *domain6, int32_t incremental, void *stream);
RF_API rf_status rf_adjacency_result(rf_adjacency *adj, const int32_t **adj_off,
                                     const int32_t **adj_idx, rf_adjacency_stats *stats);
/* Copies the CSR into caller device arrays (adj_off [n_sites + 1], adj_idx
 * [n_edges]), asynchronously on stream. */
RF_API rf_status rf_adjacency_copy(rf_adjacency *adj, int32_t *adj_off, int32_t *adj_idx, void *stream);
RF_API rf_status rf_adjacency_destroy(rf_adjacency *adj);

/*
 * MSE loss helper for a training step (device, n = 3 * rays):
 *   d_rgb[k] = 2 * scale * (rgb[k] - target[k]);  *loss += scale * sum_k (rgb[k]-target[k])^2
 * loss is a device float accumulated with atomics (zero it first).
 */
RF_API rf_status rf_mse_grad(const float *rgb, const float *target, int64_t n, float scale,
                             float *d_rgb, float *loss, void *stream);

#endif /* RF_H */
