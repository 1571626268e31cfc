/*
 * st.h -- C ABI of the synchronized blobtree tracer (sm_103a).
 *
 * The library renders the first ray / iso-surface crossing f(r(t)) = 0 of a
 * blobtree implicit surface for every pixel (Zanni 2023, Sec. 2.2).  It follows the paper's
 * two-step tile pipeline:
 *   1. st_build_tiles: a low-resolution A-buffer holding, for every screen
 *      tile, the primitives whose volume of interest is hit by at least one
 *      of the tile's pixel rays, with conservative entry / exit depths,
 *      sorted by entry depth (the per-tile structure of Sec. 3 and Sec. 6).
 *   2. st_trace: synchronized sphere tracing of each tile's subfrustums over
 *      a blobtree pruned to the subfrustum's active primitives by the sparse
 *      bottom-up traversal (Sec. 7, Sec. 8 Algorithm 2 and 3, Sec. 9).
 *
 * Conventions for every entry point:
 *   - Return value: ST_OK (0) or a negative ST_ERR_* code; st_last_error()
 *     returns a thread-local message for the last failure.  No C++ exception
 *     crosses this boundary.
 *   - Calls taking a cudaStream_t (passed as void*; NULL = legacy default
 *     stream) enqueue their device work on that stream.  st_scene_create and
 *     st_build_tiles also synchronise that stream once (host preparation /
 *     sizing of the A-buffer); st_trace and st_render_batch do not.
 *   - "device pointer" = memory on the current CUDA device, owned by the
 *     caller unless stated; "host pointer" = ordinary host memory.
 *   - All floating point data is IEEE binary32 unless stated.
 */
#ifndef ST_H
#define ST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define ST_OK 0
#define ST_ERR_INVALID (-1)   /* malformed argument, tree or sizes          */
#define ST_ERR_CAPACITY (-2)  /* a fixed-size buffer is too small           */
#define ST_ERR_CUDA (-3)      /* a CUDA runtime call failed                 */
#define ST_ERR_TIMEOUT (-4)   /* a bounded device-side wait expired         */
#define ST_ERR_NOMEM (-5)     /* device allocation failed                   */

/* ---- node kinds (scene description) ------------------------------------ */
/* Primitives (leaves); rotation and translation only (Sec. 4). */
#define ST_PRIM_SPHERE 0   /* rec[0:3] centre, rec[3] radius                */
#define ST_PRIM_RBOX 1     /* rec[0:3] centre, rec[3:12] world->local rotation
                              M row-major (local = M (x - centre)),
                              rec[12:15] half extents, rec[15] rounding      */
#define ST_PRIM_CAPSULE 2  /* rec[0:3] end a, rec[3:6] end b, rec[6] radius */
/* Further families of Sec. 10's primitive list (kind numbers equal their
 * node codes in a pruned view): */
#define ST_PRIM_TORUS 12   /* rec[0:3] centre, rec[3:6] axis (any length > 0),
                              rec[6] major radius R >= 0, rec[7] minor
                              radius r > 0; exact distance               */
#define ST_PRIM_SCONE 13   /* sphere-cone, the convex hull of two balls:
                              rec[0:3] centre a, rec[3:6] centre b, rec[6]
                              radius r_a, rec[7] radius r_b (>= 0, not both
                              0, |b - a| > |r_a - r_b|); exact distance   */
#define ST_PRIM_ELLIPSOID 14 /* rec[0:3] centre, rec[3:12] world->local
                              rotation M as ST_PRIM_RBOX, rec[12:15] radii
                              > 0; field min(r) (|M (x - c) / r| - 1), a
                              Lipschitz-1 bound of the distance           */
#define ST_PRIM_RTRI 15    /* rounded triangle: rec[0:3], rec[3:6], rec[6:9]
                              vertices a, b, c (not collinear), rec[9]
                              rounding r > 0; field = exact distance to the
                              triangle minus r.  Its volume of interest is
                              the sphere-triangle of Sec. 6.1 (points within
                              r + d of the triangle)                      */
#define ST_PRIM_QUADRIC 11 /* bounded quadric: the solid {q <= 0} inside an
                              oriented box.  rec[0:3] centre, rec[3:7]
                              rotation quaternion (w, x, y, z; any length >
                              0; local = R^T (x - centre) for the rotation R
                              it represents), rec[7:10] box half extents >
                              0, rec[10:15] alpha, beta, gamma, delta,
                              kappa of q(u) = alpha u0^2 + beta u1^2 +
                              gamma u2^2 + delta u2 + kappa in local
                              coordinates u (not all of alpha..delta zero).
                              Field max(q(clamp(u)) / G, box distance) with
                              G = |(2|alpha| e0, 2|beta| e1, 2|gamma| e2 +
                              |delta|)| >= |grad q| on the box: Lipschitz 1,
                              exact zero set.  Volume of interest: the
                              oriented box of half extents e + d.
                              (Kind 11 maps to view code 16; the other
                              primitive kinds equal their view codes.)    */
/* Operators (binary): compact smooth operators G_op of Sec. 5 (Eq.
 * "smooth_comp" with the smooth polynomial operators of Eq. 4-7 and the
 * transition b_r), rec[0] = blend range k > 0, rec[1] = operator range bound
 * d_o with 6 d_o > k; and sharp CSG operators of Eq. 1-3 (no parameters). */
#define ST_OP_UNION 16
#define ST_OP_INTER 17
#define ST_OP_DIFF 18
#define ST_OP_SHARP_UNION 19
#define ST_OP_SHARP_INTER 20
#define ST_OP_SHARP_DIFF 21

#define ST_REC_FLOATS 16   /* floats per node record in a description     */
#define ST_MAX_NODES 8388606 /* 23-bit ancestor pointers (Sec. 4)          */
#define ST_MAX_STACK 32    /* evaluation stack entries (Sec. 10 uses 22)   */

/* Blobtree description: a binary tree in any node numbering.  The library
 * linearises it in post-order (Sec. 4).  All pointers are host pointers,
 * read during the call only. */
typedef struct {
    int32_t n_nodes;        /* 2 N - 1 for N primitives                    */
    int32_t root;           /* index of the root node                      */
    const int32_t *kind;    /* [n_nodes] ST_PRIM_* or ST_OP_*              */
    const int32_t *left;    /* [n_nodes] left child, -1 for primitives     */
    const int32_t *right;   /* [n_nodes] right child, -1 for primitives    */
    const float *params;    /* [n_nodes][ST_REC_FLOATS] node records       */
    float voi_pad;          /* absolute slack added to every volume of
                               interest extent to absorb FP32 rounding in
                               the culling tests (scene units); <= 0 means
                               the default 1e-5                           */
} st_scene_desc;

/* Pinhole camera.  Basis (computed in double, then rounded to float):
 *   F = normalize(target - eye), R = normalize(F x up), U = R x F,
 *   dot(a, a) = (a.x a.x + a.y a.y) + a.z a.z, normalize = a / sqrt(dot),
 *   th = tan(vfov_deg * pi / 360), R' = (R * th) * (width / height),
 *   U' = U * th.
 * Ray of pixel (i, j), i = column, j = row from the top, FP32 without FMA:
 *   u = (float)(2i+1) / (float)width - 1,  v = 1 - (float)(2j+1) / (float)height,
 *   d = (F + u R') + v U'  per component;  points o + t d, o = eye.
 * t is the planar view depth (d . F = 1). */
typedef struct {
    float eye[3], target[3], up[3];
    float vfov_deg;
    int32_t width, height;
} st_camera;

/* A-buffer: CSR over tiles in row-major tile order (tile (tx, ty) has index
 * ty * tiles_x + tx).  Entries of tile t are [offsets[t], offsets[t+1]),
 * sorted by (z_in ascending, prim ascending).  z values are planar depths t
 * clipped to t >= 0.  prim is the post-order address of the primitive node.
 * All arrays are device pointers owned by the scene object; they stay valid
 * until the next st_build_tiles on the same scene or st_scene_destroy. */
typedef struct {
    int32_t tile;           /* tile edge in pixels                         */
    int32_t tiles_x, tiles_y;
    const uint32_t *offsets;  /* [tiles_x * tiles_y + 1]                   */
    const float *z_in;        /* [n_entries]                               */
    const float *z_out;       /* [n_entries]                               */
    const uint32_t *prim;     /* [n_entries]                               */
    uint64_t n_entries;
    uint32_t max_overlap;     /* longest tile list                         */
} st_tiles;

/* Tracing options.  Zero-initialised fields take the defaults in brackets. */
#define ST_STEP_PLAIN 0        /* z += f / (L |d|)                          */
#define ST_STEP_LEARNED 1      /* relaxed step with omega proposed per step by
                                  the MLP of st_mlp_* (BF16 tensor cores),
                                  verified like ST_STEP_OVERRELAX        */
#define ST_STEP_OVERRELAX 2    /* z += omega f / (L |d|), verified: a step whose
                                  landing sphere does not overlap the previous
                                  one is rejected, the ray returns to the
                                  previous point, takes the plain step and
                                  relaxes again once it has crossed the stored
                                  landing sphere (Sec. 10)                 */
#define ST_STEP_CROSSING 3     /* the ray processing of Sec. 10 as stated:
                                  ST_STEP_OVERRELAX's verified relaxed steps,
                                  every step at least min_step long, a hit at
                                  the first sample with f <= 0 (eps unused),
                                  no step cap (max_steps unused).  A relaxed
                                  step that lands inside the solid is
                                  rejected and plain steps bracket the
                                  crossing                                 */
typedef struct {
    float eps;              /* hit when f <= eps [1e-4]                    */
    float lipschitz;        /* L of the step f / L [1.45, Sec. 10]         */
    int32_t max_steps;      /* per-ray field evaluation cap [256]          */
    int32_t step_mode;      /* ST_STEP_* [plain]                            */
    float depth_slab_frac;  /* subfrustum depth limit d as a fraction of the
                               scene diameter measured at st_scene_create
                               (edits keep it) [0.05 = 1:20, Sec. 8]       */
    int32_t max_new_per_turn; /* new primitives fetched per subfrustum, at
                                 most 1024; a tile takes at least an eighth
                                 of its list per turn [32; Sec. 8 uses 6] */
    int32_t newton_iters;   /* Newton refinements of a hit, each ray
                               stopping at its own convergence [2]      */
    float newton_clamp;     /* Newton step bound, distance units [64 eps]  */
    const void *mlp;        /* ST_STEP_LEARNED: device pointer (16-byte
                               aligned) to MLP weights packed by st_mlp_pack */
    uint32_t *tile_stats;   /* optional device uint32[n_tiles][24] per-tile
                               diagnostics: [0] total, [1] segmentation +
                               view build, [2] marching, [3] hit refinement
                               SM clock cycles / 16 (first warp); [4]
                               subfrustums; [5] tracing steps; [6] longest
                               view; [7] A-buffer list length; [12]
                               refinement cycles / 16 summed over warps;
                               [13] sum of view lengths, [14] sum of
                               operator levels; [8] discard, [9] fetch,
                               [10] view build, [11] parameter cache fill
                               cycles / 16 (first warp); [15] marching
                               cycles / 16 summed over warps; [16]
                               lockstep iterations and [17] live rays
                               summed over them (lane use), [18] rays
                               evaluated by the warp-wide tail mode, [19]
                               hit refinement passes and [20] live lanes
                               summed over them, all summed over warps;
                               [21] CTA-split passes (see
                               cta_eval_min_view) and [22] live rays
                               summed over them; [23] 0; a tile split across CTAs
                               reports its first part only (NULL = off) */
    float omega;            /* relaxation factor of ST_STEP_OVERRELAX and
                               ST_STEP_CROSSING [1.7, Sec. 10]             */
    float min_step;         /* ST_STEP_CROSSING: shortest step, distance
                               units [1/32000 of the largest extent of the
                               primitives' bounding box measured at
                               st_scene_create, Sec. 10]                   */
    int32_t split_kcycles;  /* a tile still tracing this many thousand SM
                               cycles after its CTA started it hands parts
                               of its pending rays to other CTAs at its next
                               subfrustum boundary (the output does not
                               change); 0 = default [2000], < 0 = never   */
    int32_t heavy_split_len; /* > 0: a tile whose A-buffer list holds at
                               least this many entries is split across CTAs
                               before its first subfrustum (about one part
                               per 512 list entries, at most 8; each part
                               builds the tile's views itself), and CTAs
                               take open parts before whole tiles (the
                               output does not change); <= 0 = never
                               [never: the repeated view builds cost more
                               than the balance gains on the clustered
                               workloads]                                 */
    int32_t heavy_split_rank; /* > 0: the tiles of the heavy_split_rank
                               longest lists (each at least 1024 entries
                               and four times the mean list) split as
                               heavy_split_len describes; the threshold is
                               taken on the device from the launch's own
                               lists; 0 = default [see st_trace_opts
                               defaults below], < 0 = never; a positive
                               heavy_split_len takes precedence           */
    uint32_t wait_spin_limit; /* bound on the polls of a warp waiting for
                               the other warps of its tile and of a CTA
                               waiting for parts of split tiles; a warp
                               wait that runs out sets error bit 3 and the
                               kernel carries on without the waiting warp
                               (results of that call are undefined) [0 =
                               built-in bounds, 2^22 and 2^21 polls]      */
    int32_t check_status;   /* 1: st_trace and st_trace_noalloc synchronise
                               `stream` after the launch and return
                               ST_ERR_TIMEOUT when a bounded device wait
                               ran out, ST_ERR_CAPACITY or ST_ERR_INVALID
                               for the other device error bits [0: the
                               call stays asynchronous; the bits are in
                               counters[7] when counters are given]      */
    int32_t cta_eval_min_view; /* launches whose views live in global
                               memory (tile lists over 1024 entries): a
                               subfrustum whose pruned view has at least
                               this many nodes is, once at most 64 of its
                               rays are unfinished, stepped by one warp
                               while all four warps of the CTA evaluate a
                               quarter of the view each (Algorithm 3 cut
                               at subtree boundaries; the same values bit
                               for bit); 0 = default [1024 for st_trace
                               launches bound by their heaviest tiles
                               (those with the large parameter cache);
                               no split otherwise, nor for batches],
                               < 0 = never; st_trace_noalloc never
                               splits                                   */
    int32_t full_views;     /* 1: evaluate each subfrustum's pruned view
                               as Algorithm 1 builds it (Sec. 8-9); 0
                               [default]: without the subtrees whose
                               values its usage rewrite discards (the
                               operand an operator rewritten to "left",
                               "right" or "+inf" drops: 50-70 % of the
                               nodes on the synthetic scenes), by
                               building the view again from the
                               primitives whose values reach the root.
                               Every value computed, hence every output
                               byte, is the same; only counters [8], [9]
                               differ                                   */
} st_trace_opts;

/* Optional per-call counters (device pointer to ST_NUM_COUNTERS uint64,
 * accumulated with atomics; the caller zeroes them):
 *   [0] tracing steps (field evaluations on live rays)
 *   [1] useful primitive evaluations (pruned-view primitives x live steps)
 *   [2] useful operator evaluations
 *   [3] algorithmic FP32 flops of those evaluations (fixed per-node counts)
 *   [4] subfrustums processed (each part of a tile split across CTAs
 *       counts those it marches)
 *   [5] rejected learned steps
 *   [6] finalisation field evaluations (Newton + normal)
 *   [7] device error flags (bit 0: view capacity, bit 1: stack overflow,
 *       bit 2: a tile list longer than the launch's capacity, bit 3: a
 *       bounded wait between the warps of a tile expired)
 *   [8] view nodes evaluated on live steps (the views actually evaluated:
 *       without discarded subtrees unless full_views)
 *   [9] FP32 flops of those evaluations (fixed per-node counts, + the step) */
#define ST_NUM_COUNTERS 10

/* ---- scenes --------------------------------------------------------------
 * st_scene_create: host preparation of a tree structure (the preparation
 * step of Sec. 10 / Sec. 11): post-order linearisation, isLeft, ignoreMod, fast
 * ancestor pointers (Sec. 7.2, cut at intersections and at right-operand ->
 * difference edges, Sec. 9), ranges of interest propagated from the root
 * (Sec. 5), then upload of the node arrays to the current device.  Fails with
 * ST_ERR_INVALID on a malformed tree (cycle, bad child, kind out of range,
 * k <= 0 or 6 d_o <= k), more than ST_MAX_NODES nodes or a tree whose
 * post-order evaluation needs more than ST_MAX_STACK stack entries.  *out
 * receives an opaque handle owned by the library. */
typedef struct st_scene st_scene;
int st_scene_create(const st_scene_desc *desc, st_scene **out, void *stream);

/* Update the parameter records of n primitives (no preparation re-run, the
 * tree structure is unchanged; Sec. 1 "no preprocessing when primitive
 * parameters are updated").  ids: host int32[n] description node indices of
 * primitives; params: host float[n][ST_REC_FLOATS].  The copy is staged and
 * enqueued on `stream`. */
int st_scene_update_prims(st_scene *scene, const int32_t *ids, const float *params, int n,
                          void *stream);

/* Post-order address of every description node: host int32[n_nodes] out. */
int st_scene_addresses(const st_scene *scene, int32_t *po_of_desc);

/* Facts of the preparation, host double[4] out: [0] scene diameter (the
 * diagonal of the axis-aligned box of all primitive bounds, measured at
 * st_scene_create; it scales the subfrustum depth slab), [1] the largest
 * edge of that box, [2] primitives, [3] post-order evaluation stack depth. */
int st_scene_info(const st_scene *scene, double *out);

void st_scene_destroy(st_scene *scene);

/* ---- per-frame calls -------------------------------------------------------
 * st_build_tiles: fills the tile A-buffer of `scene` seen by `cam` (Sec. 6):
 * volumes of interest are recomputed from the current primitive parameters
 * (sphere -> sphere r + d, rounded box -> oriented box b + r_round + d,
 * capsule -> capsule r + d, plus voi_pad); every (primitive, tile) pair whose
 * conservative screen bound covers the tile is tested with one ray per pixel
 * centre of the tile (FP32, fixed operation order documented in the kernel
 * source, identical on every call); the entry is kept iff at least one ray
 * hits, with z_in = min over hitting rays of max(t0, 0) and z_out = max of
 * t1.  Buffers grow on demand (the call synchronises `stream` once to size
 * them).  tile must be 8, 16 or 32. */
int st_build_tiles(st_scene *scene, const st_camera *cam, int tile, st_tiles *out, void *stream);

/* st_trace: synchronized sphere tracing of every tile (Algorithm 2) over the
 * A-buffer built for the same scene and camera.  Outputs are caller-owned
 * device buffers of width * height pixels, row-major from the top row:
 *   depth  float[H*W]   Euclidean eye distance of the hit, +inf on a miss
 *   normal float[H*W*3] unit normal (field gradient) at the hit, 0 on a miss
 *   evals  uint32[H*W]  tracing field evaluations of the ray
 *   flags  uint8[H*W]   bit 0 hit, bit 1 step cap reached (reported as miss)
 * counters: optional device uint64[ST_NUM_COUNTERS] (may be NULL). */
int st_trace(st_scene *scene, const st_camera *cam, const st_tiles *tiles,
             const st_trace_opts *opts, float *depth, float *normal, uint32_t *evals,
             uint8_t *flags, uint64_t *counters, void *stream);

/* Copy an A-buffer out (cudaMemcpyDefault: each destination may be host or
 * device memory; offsets gets tiles_x * tiles_y + 1 words, the others
 * n_entries each; NULL destinations are skipped).  Enqueued on `stream`,
 * then the stream is synchronised. */
int st_tiles_copy(const st_tiles *tiles, uint32_t *offsets, float *z_in, float *z_out, uint32_t *prim,
                  void *stream);

/* ---- batched rendering of many scenes ------------------------------------------
 * Not a paper step: the paper renders one scene per frame.  A batch renders
 * n scenes (each with its own camera, resolution and output buffers) with
 * the same per-scene results as st_build_tiles + st_trace: culling, sorting
 * and tracing of all scenes run as batched launches over a concatenated
 * primitive / tile space, and tracing is ONE persistent launch whose CTAs
 * pull (scene, tile) items from a single queue.  The launch sequence is
 * captured once in a CUDA graph and replayed by every st_batch_render.
 *
 * Per-scene tile size (8, 16 or 32), new primitives per subfrustum and the
 * subfrustum depth slab come from an autotuner (st_autotune) whose results
 * are kept in a JSON cache file keyed by st_tune_key; other trace options
 * (eps, Lipschitz bound, step cap and mode, MLP) are the caller's opts for
 * every scene.  Outputs per scene are identical, bit for bit, to
 * st_build_tiles(tile) + st_trace with those parameters.
 *
 * st_tune: one tuned configuration; ms = measured tiles + trace time of the
 * scene it was tuned on (informative).
 * st_tune_key: "m<mode>_n<round(log2 n_prims)>_<W>x<H>" into key[0..cap).
 * st_tune_load / st_tune_store: look up / insert-or-replace one entry of
 * the cache file (host only; store rewrites the whole file).  load returns
 * ST_ERR_INVALID when the file or key is absent or malformed.
 * st_autotune: times every candidate (tile 8/16/32 x max_new 16/32/64 x
 * depth slab 0.05/0.15 of the scene diameter) on `scene` seen by `cam`
 * with `opts` (1 untimed + 2 timed runs each, CUDA events on `stream`),
 * writes the fastest to *out and, when cache_path is not NULL, stores it.
 * Synchronises `stream`.
 *
 * st_batch_create: plans a batch.  scenes/cams: host arrays of n; depth,
 * normal, evals, flags: host arrays of n device pointers (per scene layout as
 * st_trace).  autotune_cache: JSON cache path, or NULL for tile 16 and the
 * opts' subfrustum parameters; a scene whose key is missing from an existing
 * cache path is tuned (st_autotune) and stored.  The plan runs the culling
 * once to size its buffers (entries x 1.5, longest list x 1.25), then
 * captures the graph.  Synchronises `stream`.  Scenes must outlive the
 * batch; their primitive parameters may change between renders
 * (st_scene_update_prims), their tree may not.
 * st_batch_render: replays the graph on the plan's stream, then synchronises
 * it and checks the batch status word; when an edit made the lists outgrow
 * the planned buffers it re-plans, re-captures and renders again (at most
 * twice), else returns ST_ERR_CAPACITY.  counters: optional host
 * uint64[ST_NUM_COUNTERS] receiving the counters of the render.
 * st_batch_tiles: the tile size chosen for scene i (0 when out of range).
 * st_batch_graph_kernels: kernel launches one render replays.
 * st_render_batch: create + render + destroy in one call. */
typedef struct {
    int32_t tile;
    int32_t max_new_per_turn;
    float depth_slab_frac;
    float ms;
} st_tune;
typedef struct st_batch st_batch;
int st_tune_key(int n_prims, int width, int height, int step_mode, char *key, int cap);
int st_tune_load(const char *path, const char *key, st_tune *out);
int st_tune_store(const char *path, const char *key, const st_tune *t);
int st_autotune(st_scene *scene, const st_camera *cam, const st_trace_opts *opts, const char *cache_path,
                st_tune *out, void *stream);
int st_batch_create(st_scene *const *scenes, const st_camera *cams, int n, const st_trace_opts *opts,
                    float *const *depth, float *const *normal, uint32_t *const *evals,
                    uint8_t *const *flags, const char *autotune_cache, st_batch **out, void *stream);
int st_batch_render(st_batch *batch, uint64_t *counters);
int st_batch_tiles(const st_batch *batch, int i);
int st_batch_graph_kernels(const st_batch *batch);
void st_batch_destroy(st_batch *batch);
int st_render_batch(st_scene *const *scenes, const st_camera *cams, int n, const st_trace_opts *opts,
                    float *const *depth, float *const *normal, uint32_t *const *evals,
                    uint8_t *const *flags, const char *autotune_cache, void *stream);

/* ---- learned relaxation factor (MLP 6 -> 32 -> 32 -> 1) ---------------------------
 * Not part of the paper: a small network proposes the relaxation factor
 * omega in (1, 2) of each sphere-tracing step (ST_STEP_LEARNED) from the
 * local ray state; every proposal goes through the rejection test of
 * ST_STEP_OVERRELAX, so the plain step stays the fallback.
 * Features of a step (fixed scaling): 8 f / L; 8 f_prev / L (f when none);
 * 8 x previous step length (0 when none); steps / 64;
 * log2(1 + primitives in the pruned view) / 8; log2(1 + tile list length) / 8.
 * Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), o = w3 . h2 + b3,
 * omega = 1 + sigmoid(o).  FP32 parameter vector (st_mlp_param_count() =
 * 1313 floats): W1[32][6], b1[32], W2[32][32], b2[32], w3[32], b3.
 *
 * st_trace_record: plain synchronized tracing (as st_trace) that also writes
 * one training record per plain step of the rays whose pixel index is a
 * multiple of ray_stride: 8 floats = the 6 features of the step, the label
 * 0.97 x 2 / (1 + k) clamped to [1, 2] with k = 1 - f_next / f (the largest
 * factor whose relaxed step passes the overlap test when the field drops
 * linearly), and 0.  records: device float[rec_cap][8]; rec_count: device
 * uint32 zeroed by the caller, returns the number of records produced (it
 * may exceed rec_cap; only rec_cap are stored).
 *
 * st_mlp_grad: adds to grad (device float[1313]) the gradient, and to
 * loss_sum (device float[1]) the value, of sum_i w_i (omega_i - y_i)^2 over
 * records i (x: device float[n][6], y: device float[n]), w_i = 4 when
 * omega_i > y_i else 1.  FP32.
 * st_mlp_grad_bf16: the same sums with the products on BF16 tensor cores
 * (FP32 accumulation; params stay FP32): inputs, weights and post-ReLU
 * activations rounded to BF16 as in the tracer's inference, and the
 * backpropagated signals rounded to BF16 where they enter a product (the
 * layer-2 signal dout x w3 before it meets W2 and h1, the layer-1 signal
 * before it meets x); bias gradients sum the signals before that rounding.
 * st_mlp_adam: one Adam step on params with grad x grad_scale (bias
 * corrected for step >= 1); m, v: device float[1313] moments.
 * st_mlp_pack: host float[1313] -> host buffer of st_mlp_pack_size() bytes
 * (BF16 weights, FP32 biases) for opts.mlp / st_mlp_infer.
 * st_mlp_infer: omega for n feature rows with the tracer's BF16 tensor-core
 * inference (packed: device, 16-byte aligned). */
int st_trace_record(st_scene *scene, const st_camera *cam, const st_tiles *tiles,
                    const st_trace_opts *opts, float *depth, float *normal, uint32_t *evals,
                    uint8_t *flags, float *records, uint32_t rec_cap, uint32_t *rec_count,
                    int ray_stride, void *stream);
size_t st_mlp_pack_size(void);
int st_mlp_param_count(void);
int st_mlp_pack(const float *params, void *packed);
int st_mlp_grad(const float *params, const float *x, const float *y, int n, float *grad,
                float *loss_sum, void *stream);
int st_mlp_grad_bf16(const float *params, const float *x, const float *y, int n, float *grad,
                     float *loss_sum, void *stream);
int st_mlp_adam(float *params, const float *grad, float *m, float *v, int step, float lr,
                float beta1, float beta2, float eps, float grad_scale, void *stream);
int st_mlp_infer(const void *packed, const float *x, int n, float *omega, void *stream);

/* ---- tracing without device allocation ----------------------------------------
 * st_trace_noalloc: same arguments, outputs and results as st_trace, but the
 * call itself allocates no device memory (no cudaMalloc or cudaFree and no
 * allocating library routine).  It is meant for callers that cannot allocate
 * at draw time: render loops that run under a fixed memory budget or must
 * not stall on an allocation (cudaMalloc can synchronise the device), and
 * hosts whose device memory is owned by another allocator.  The paper has no
 * counterpart to this call.  Every step mode of st_trace (ST_STEP_LEARNED
 * reads the caller's packed weights, opts.mlp), and the same launch:
 * parameter cache size, longest-list-first tile order, tiles split across
 * CTAs, opts.check_status.
 *
 * Its scratch memory (the work-queue counter, the status word, the job
 * record, the tile order, for long tile lists the per-CTA work areas, then
 * as many split records as fit) is one fixed 32 MiB device array defined in
 * the library; every device that loads the library holds it until the
 * process exits (st_trace_noalloc_scratch_bytes() returns the size).  A
 * launch whose tile order or work areas would not fit returns
 * ST_ERR_CAPACITY with the needed size in st_last_error(), before anything
 * is enqueued; st_trace has no such limit.
 * st_trace_noalloc_last_layout(out[3]) reports the last call's layout:
 * out[0] 1 when its per-CTA work areas were carved from the array (lists
 * too long for shared memory), out[1] bytes of the array in use, out[2]
 * split records.
 *
 * The first call on a device resolves the array's device address (with that
 * device current); make that first call before any stream capture.  Every
 * call reuses the same array, which keeps the previous call's contents: the
 * call clears what must start at zero, but two calls whose work overlaps on
 * the GPU (different streams, or without ordering between them) race on the
 * array and give undefined results. */
int st_trace_noalloc(st_scene *scene, const st_camera *cam, const st_tiles *tiles,
                     const st_trace_opts *opts, float *depth, float *normal, uint32_t *evals,
                     uint8_t *flags, uint64_t *counters, void *stream);
size_t st_trace_noalloc_scratch_bytes(void);
int st_trace_noalloc_last_layout(uint64_t *out);

/* ---- the non-synchronized variants of Table 1 ---------------------------------
 * The paper measures its pipeline against per-pixel processing over a
 * full-resolution A-buffer ("dexel" buffer) in which every field evaluation
 * runs the sparse bottom-up traversal of Algorithm 1 on the ray's own active
 * primitives, with parent pointers (Sec. 7.1, "ParentPtr/Full") or fast
 * ancestor pointers (Sec. 7.2, "FastPtr/Full").  These calls provide them
 * for comparison; st_build_tiles + st_trace is the method.
 *
 * st_build_dexels: one list per pixel of every primitive whose volume of
 * interest the pixel's centre ray hits (FP32 tests of the tile culling), with
 * entry and exit depths, sorted by (z_in, post-order address).  `tiles` must
 * come from st_build_tiles for the same scene, camera and primitive
 * parameters (their lists hold every primitive hit by a ray of the tile).
 * *out: tile = 1, tiles_x = width, tiles_y = height, CSR over pixels
 * (row-major), library-owned device buffers valid until the next call on the
 * scene; max_overlap = longest pixel list.  Synchronises `stream` once (to
 * size the buffers).
 *
 * st_trace_dexels: per-pixel sphere tracing (one thread per ray): the ray's
 * own list is cut into subintervals by the rule st_trace applies per tile
 * (Sec. 8: discard, fetch up to max_new_per_turn with no empty space and
 * within the depth slab), a step never passes a subinterval's end, and each
 * step evaluates f_A by Algorithm 1 with field values, with
 * traversal ST_TRAVERSE_PARENT or ST_TRAVERSE_FAST.  Step ST_STEP_PLAIN only
 * (eps, L, max_steps, Newton refinement and normals as st_trace).  Outputs as
 * st_trace.  Counters: [0] tracing steps, [1] primitive evaluations, [2]
 * operators reached by the traversals' climbs, [3] operators evaluated, [4]
 * active-set changes, [7] error bits (1 malformed traversal, 2 stack).
 * Library-owned scratch of max_overlap x 8 bytes per thread of a persistent
 * grid.
 *
 * st_eval_sparse: f_A at points (device float[npts][3] -> f device
 * float[npts]) by the same traversal over the active primitives `act`
 * (device, ascending post-order addresses); equal bit for bit to
 * st_eval_pruned over the pruned view of the same set.  status: device
 * uint32, error bits OR-ed in (zero it first). */
#define ST_TRAVERSE_PARENT 0
#define ST_TRAVERSE_FAST 1
int st_build_dexels(st_scene *scene, const st_camera *cam, const st_tiles *tiles, st_tiles *out, void *stream);
int st_trace_dexels(st_scene *scene, const st_camera *cam, const st_tiles *dexels, const st_trace_opts *opts,
                    int traversal, float *depth, float *normal, uint32_t *evals, uint8_t *flags,
                    uint64_t *counters, void *stream);
int st_eval_sparse(const st_scene *scene, const uint32_t *act, int n, const float *pts, int npts, int traversal,
                   float *f, uint32_t *status, void *stream);

/* ---- inspection of the hot-path steps ----------------------------------------
 * st_pruned_view: the pruned tree view of an active set, built on the device
 * by the same code st_trace uses: the warp-parallel form of Algorithm 1 (the
 * operators of the view are the lowest common ancestors of consecutive
 * active primitives; the usage rewrite of Sec. 9 through each node's nearest
 * blocking ancestor).
 * st_pruned_view_alg1: the same view by Algorithm 1 as stated (one thread,
 * fast ancestor pointers, clamping, popRequiredA / popRequiredB and the
 * usage rewrite); same arguments and outputs.
 * st_pruned_view_live: the view st_trace evaluates by default (full_views =
 * 0): st_pruned_view's view without the subtrees that its usage rewrite
 * discards (the operators rewritten to "left operand", "right operand" or
 * "+inf" and the operands they drop), i.e. the pruned view of the active
 * primitives whose values reach the root; same arguments; info[0] is the
 * length of that view, info[3] still the number of active primitives.  When
 * the root is unused, or the view has more than 65,535 nodes or more than 64
 * operator levels, the view is st_pruned_view's.
 *   act        device uint32[n], post-order addresses of active primitives,
 *              strictly ascending, 1 <= n <= number of primitives
 *   view       device uint32[2n-1] out: bits 27..31 node code (0 sphere,
 *              1 rounded box, 2 capsule, 3/4/5 compact union / intersection /
 *              difference, 6/7/8 sharp ones, 9 +inf, 10 right operand, 11 left
 *              operand, 12 torus, 13 sphere-cone, 14 ellipsoid, 15 rounded
 *              triangle, 16 bounded quadric), bit 26 set (record in the
 *              scene's global array), bits 0..25 record word offset
 *   view_addr  device uint32[2n-1] out (optional): post-order address per entry
 *   info       device int32[4] out: view length, root usage bit, error (0 ok),
 *              number of primitives
 * Uses a library-owned scratch stack; calls on one scene must be stream ordered.
 *
 * st_eval_pruned: f_A (Sec. 3) at points by Algorithm 3 over a view from
 * st_pruned_view, with the FP32 evaluator of st_trace (approximate square root
 * and reciprocal).  pts device float[npts][3]; f device float[npts] (+inf when
 * the root is unused); grad optional device float[npts][3] forward-mode
 * gradient (then the IEEE square root is used). */
int st_pruned_view(const st_scene *scene, const uint32_t *act, int n, uint32_t *view, uint32_t *view_addr,
                   int32_t *info, void *stream);
int st_pruned_view_alg1(const st_scene *scene, const uint32_t *act, int n, uint32_t *view, uint32_t *view_addr,
                        int32_t *info, void *stream);
int st_pruned_view_live(const st_scene *scene, const uint32_t *act, int n, uint32_t *view, uint32_t *view_addr,
                        int32_t *info, void *stream);
int st_eval_pruned(const st_scene *scene, const uint32_t *view, const int32_t *info, const float *pts,
                   int npts, float *f, float *grad, void *stream);

/* st_eval_pruned_levels: f_A (Sec. 3) at points over the pruned view of an
 * active set, evaluated as st_trace's tail mode does for the last rays of a
 * subfrustum: the view is built as by st_pruned_view, its operators are
 * grouped by height in the view (operands always sit lower), and one warp
 * evaluates a point: the primitives in parallel, then the operators level by
 * level, one per lane (the same node values as Algorithm 3 over the view, in
 * another order).
 *   act, n     as st_pruned_view;   view  device uint32[2n-1] out
 *   info       device int32[4] out: view length, root usage bit, error (0 ok),
 *              operator levels (0: the view has no level schedule -- a single
 *              primitive, more than 64 levels or an unused root -- and f is NaN)
 *   pts        device float[npts][3];   f  device float[npts] out
 * Uses the library-owned scratch of st_pruned_view (stream ordered on one
 * scene).  ST_ERR_INVALID on bad arguments. */
int st_eval_pruned_levels(const st_scene *scene, const uint32_t *act, int n, uint32_t *view, int32_t *info,
                          const float *pts, int npts, float *f, void *stream);

/* ---- host-only preparation (no GPU needed) ----------------------------------
 * The preparation step of st_scene_create on its own, for inspection: every
 * output is a host array indexed by post-order address (n_nodes entries):
 *   po_of_desc  post-order address of each description node (desc-indexed)
 *   blob        packed node word: bit 31 isPrimitive, bits 26..30 kind,
 *               bits 24..25 ignoreMod, bit 23 isLeft, bits 0..22 fast
 *               ancestor address (0x7FFFFF for the root)   (Sec. 4 layout)
 *   parent      parent address, -1 for the root
 *   roi         upper bound d_n of the node's range of interest (Sec. 5)
 * Returns the post-order evaluation stack depth (>= 1), or a negative code. */
int st_prep_tree(const st_scene_desc *desc, int32_t *po_of_desc, uint32_t *blob,
                 int32_t *parent, float *roi);

/* Number of kernels this library has launched in this process so far. */
uint64_t st_kernel_launches(void);

/* Number of device allocations (cudaMalloc) this library has made in this
 * process so far: scene arrays, tile and work buffers growing on demand,
 * batch buffers.  st_trace_noalloc never adds to it. */
uint64_t st_device_allocations(void);

const char *st_last_error(void);
const char *st_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ST_H */
