/*
 * v3dg.h -- C ABI of the GB300 (sm_103a) implementation of V3DG's online per-frame path:
 * footprint-based LOD-cut selection over instanced cluster hierarchies (Sec. 3.3-3.4) followed by
 * tile-based splatting of only the selected Gaussians (Sec. 2.1, Sec. 5.1).
 *
 * Conventions shared by every call:
 *  - Every call returns a v3dg_status.  No exception or longjmp crosses this boundary.  On an
 *    error the context keeps its previous state and v3dg_last_error() holds a one-line reason.
 *  - "host" pointers are read during the call only; the library copies what it keeps.
 *    "device" pointers must be CUDA device (or managed) memory of the context's device and stay
 *    owned by the caller.
 *  - All work is enqueued on the context's stream (v3dg_set_stream; default: the legacy stream).
 *    Device memory the library needs comes from the allocator given to v3dg_create (e.g. a
 *    PyTorch caching allocator) or, when none is given, from cudaMalloc.
 *  - One context per host thread; a context is not thread-safe, except v3dg_submit and v3dg_poll,
 *    which any thread may call while a server runs.
 *  - There is no CPU fallback: without a usable CUDA device v3dg_create returns V3DG_ECUDA.
 */
#ifndef V3DG_H
#define V3DG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct v3dg_ctx v3dg_ctx;

typedef enum {
  V3DG_OK = 0,
  V3DG_EINVAL = 1,     /* bad argument or malformed input; nothing changed */
  V3DG_ENOMEM = 2,     /* allocator returned NULL; nothing changed */
  V3DG_ECUDA = 3,      /* a CUDA call failed; the message names it */
  V3DG_EBUSY = 4,      /* the requested result is not ready */
  V3DG_ETIMEOUT = 5,   /* a bounded device-side wait gave up; the frame's outputs are invalid */
  V3DG_EOVERFLOW = 6,  /* a device capacity was exceeded and could not be grown */
  V3DG_ENOTFOUND = 7   /* unknown asset id or no frame selected yet */
} v3dg_status;

/* Device-memory provider.  alloc returns device memory of at least `bytes` bytes aligned to 256
 * bytes, or NULL; free releases a pointer alloc returned.  `user` is passed through. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* user;
} v3dg_allocator;

/* Pinhole camera V with image size w x h (Sec. 3.4 selects with "the camera view V and image
 * resolution w x h").  OpenCV axes: x right, y down, z forward.  world_to_cam is the row-major
 * 3x4 [R | t] mapping world points to camera space.  Intrinsics are in pixels; pixel (px, py)
 * samples the point (px + 0.5, py + 0.5).  near_z <= 0 selects the default 0.01. */
typedef struct {
  double world_to_cam[12];
  float fx, fy, cx, cy;
  int32_t width, height;
  float near_z;
} v3dg_camera;

/* One asset's bundle (Sec. 3.1-3.2, Algorithm 1): Gaussians plus the cluster tree.
 *  - Gaussians, SoA, host pointers, n_gauss entries each: means (3n), log_scales (3n),
 *    quats (4n; w, x, y, z; need not be unit length), opacity (n; activated, in (0, 1]),
 *    sh (n * (sh_degree + 1)^2 * 3; per Gaussian coefficient-major then RGB).
 *  - Clusters (tree nodes), n_nodes entries each: node_first / node_count give the node's
 *    Gaussians [first, first + count) with 1 <= count <= 64; node_level is 0 for the finest
 *    clusters; node_parent is -1 for the root and otherwise a node one level up.
 *  - own_sphere (4 * n_nodes; cx, cy, cz, r): the bounding sphere of the cluster group the node
 *    belongs to (Sec. 3.3, Fig. 4).  The parent sphere (c_p, r_p) of Sec. 3.4 is the parent's
 *    own sphere, so the library derives it; a leaf has F_c := 0 and the root F_p := +inf.
 *  - gaussians_per_group: the nominal Gaussians per cluster group, used to turn a per-Gaussian
 *    pixel tolerance into the area tolerance (tau_F = n * tau_px^2).
 * Validation (V3DG_EINVAL): counts in range, ranges inside [0, n_gauss), parents one level up
 * and acyclic, exactly one root, finite spheres with r >= 0, sh_degree <= 3. */
typedef struct {
  uint32_t n_gauss, n_nodes, sh_degree;
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity;
  const float* sh;
  const uint32_t* node_first;
  const uint32_t* node_count;
  const uint8_t* node_level;
  const int32_t* node_parent;
  const float* own_sphere;
  uint32_t gaussians_per_group;
} v3dg_hierarchy_desc;

/* Counters of the last frame (filled by v3dg_frame_stats, which synchronises the stream). */
typedef struct {
  uint64_t cut_nodes;       /* |{(i, n) : F_c <= tau < F_p}| over all instances (Sec. 3.4) */
  uint64_t cut_gaussians;   /* Gaussians in those clusters */
  uint64_t render_nodes;    /* cut clusters left after the conservative visibility cull */
  uint64_t visible;         /* Gaussians that survive the projection culls */
  uint64_t pairs;           /* (tile, Gaussian) pairs sorted and blended */
  uint32_t overflow;        /* nonzero if a capacity was exceeded in the last frame, or in any
                               frame rendered since the previous v3dg_frame_stats call */
  uint32_t timeout;         /* likewise for a bounded device wait that gave up */
  uint64_t blend_evals;     /* (pixel, Gaussian) pairs the blend evaluated inside the Gaussian's
                               pixel box (only with V3DG_OPT_COUNT_WORK, else 0) */
  uint64_t blend_contribs;  /* of those, the ones with alpha >= 1/255 that were blended */
  uint64_t conic_fp64;      /* Gaussians whose 2D covariance had det < 1e-12 (eps2d = 0, Sec. 5.1, lets
                               it approach 0) and was formed and inverted in FP64 */
  uint64_t render_clusters; /* distinct (asset, cluster) among the render list's entries, counted
                               when the projection takes them grouped by cluster (see
                               V3DG_OPT_PROJECT_ORDER) and the loaded assets hold at most 2^24
                               nodes in all; else 0 */
} v3dg_stats;

/* Options for v3dg_set_option. */
enum {
  V3DG_OPT_SYNC_CHECK = 1,  /* 1 (default): v3dg_render waits for the frame and re-runs it with
                               larger buffers on overflow; 0: fully asynchronous, the caller
                               checks v3dg_frame_stats */
  V3DG_OPT_STAGE_TIMING = 2, /* 1: record CUDA events around every stage (see v3dg_stage_times) */
  V3DG_OPT_CAP_NODES = 3,    /* current render-list capacity in clusters (>= 64); grows on demand */
  V3DG_OPT_CAP_PAIRS = 4,    /* current (tile, Gaussian) pair capacity (>= 4096); grows on demand */
  V3DG_OPT_COUNT_WORK = 5,   /* 1: the blend also counts its evaluations (v3dg_stats.blend_*) */
  V3DG_OPT_SPLIT_PAIRS = 6,  /* tiles with at least this many pairs are blended as four 8x8
                                quadrants by separate blocks (default 2^32 - 1: no split; the
                                image does not depend on it) */
  V3DG_OPT_ATTR_FP16 = 7,    /* 1: assets loaded from now on keep opacity and SH in float16 (rounded
                                to nearest even); means, scales and rotations stay float32 and all
                                arithmetic stays float32 */
  V3DG_OPT_SELECT_TOPDOWN = 8, /* 1: v3dg_select walks each instance's tree from its roots, level by
                                level, testing only nodes whose parent's footprint exceeds tau_F and
                                skipping subtrees that the visibility cull rejects as a whole; the
                                cut is the same as the flat test of every node (F grows from a node
                                to its parent, Sec. 3.4), in the same order.  0: the flat test of
                                every (instance, node).  2 (default): top-down when that would be
                                more than 8M tests, else flat. */
  V3DG_OPT_BLEND_BATCH = 9,    /* records the blend stages per batch in shared memory: 128, 256
                                or 512 (default); the image does not depend on it */
  V3DG_OPT_BLEND_MODE = 11,    /* blend kernel variant, the same image bit for bit: 0 (default)
                                two phases per batch, a record-parallel alpha test into per-pixel
                                masks, then pixel-parallel compositing; 1: each batch staged into
                                shared memory by bulk copies (cp.async.bulk, one per 48-byte record,
                                completing on an mbarrier with a bounded wait), then composited by
                                warps that each own two pixel rows and walk only the records whose
                                box spans them.  Variant 1 always blends whole tiles
                                (V3DG_OPT_SPLIT_PAIRS is ignored). */
  V3DG_OPT_SERVE_MERGE = 12,   /* server (read at v3dg_server_start): a slot that takes a request
                                also takes up to this many - 1 queued requests with the same image
                                size, intrinsics and near plane whose memory estimates fit the
                                budget, and renders them as the views of one frame (each view its
                                own scene, camera and tolerance; every stage one launch for all);
                                each image is the one its request gives alone, bit for bit.  Only
                                while at least as many requests wait as there are slots.  1..64,
                                default 1 (one request per frame). */
  V3DG_OPT_PROJECT_ORDER = 13, /* order in which the projection takes the render list; no result
                                depends on it: 0 list order; 1 grouped by cluster (a radix sort of
                                the entries' cluster ids), so that the instances drawing one cluster
                                read its attributes one after the other and share one HBM read
                                through L2; 2 (default): grouped when the instances outnumber the
                                assets they draw at least twice over. */
  V3DG_OPT_GRAPHS = 10         /* 1: v3dg_select only stages the camera and instances, and
                                v3dg_render runs the selection and the whole render as one CUDA
                                graph, captured the first time a configuration (instance and view
                                count, image size and intrinsics, buffer capacities, options,
                                output pointers) is seen and replayed after that.  Same images;
                                the frame counters are valid after v3dg_render.  Not used while
                                V3DG_OPT_STAGE_TIMING is on.  Default 0. */
};

/* Create a context on CUDA device `device`.  `alloc` may be NULL (cudaMalloc/cudaFree). */
v3dg_status v3dg_create(int device, const v3dg_allocator* alloc, v3dg_ctx** out);
/* Release every device buffer of the context (after synchronising its stream). */
void v3dg_destroy(v3dg_ctx* ctx);
/* Last error text of the context (never NULL; "" after success). */
const char* v3dg_last_error(const v3dg_ctx* ctx);
/* Stream (a cudaStream_t of the context's device) on which all later work is enqueued. */
v3dg_status v3dg_set_stream(v3dg_ctx* ctx, void* cuda_stream);
v3dg_status v3dg_set_option(v3dg_ctx* ctx, int option, int64_t value);

/* Upload one asset's bundle (the bundles that the online stage reads, Sec. 3, Fig. 2).  The
 * Gaussians are repacked on the device into 64-slot cluster blocks, attribute-major.  On success
 * *asset_id receives the asset's index (0, 1, ... in load order). */
v3dg_status v3dg_load_hierarchy(v3dg_ctx* ctx, const v3dg_hierarchy_desc* desc, uint32_t* asset_id);

/* Set the composed scene (Sec. 4.2, App. B.2): n instances, instance i places asset asset_id[i]
 * with rotation rot[9i..9i+8] (row-major, proper), translation trans[3i..3i+2] and uniform scale
 * scale[i] > 0: x_world = scale R x_asset + t.  Host pointers, FP64.  Instances may change every
 * frame (rigid dynamic scenes, App. B.3). */
v3dg_status v3dg_set_instances(v3dg_ctx* ctx, uint32_t n, const uint32_t* asset_id,
                               const double* rot, const double* trans, const double* scale);

/* Select the cut for one camera (Sec. 3.4): for every instance i and cluster n, with footprints
 * F = pi r'^2 fx fy / z^2 of the own and parent spheres (Sec. 3.3, Fig. 4; r' = s_i r, +inf when
 * |z| <= r'), keep (i, n) iff F_c <= tau_F < F_p, with tau_F = float32(gaussians_per_group *
 * tau_px^2).  Clusters whose Gaussians provably cannot reach a pixel are dropped afterwards (this
 * changes no pixel).  Enqueued only; counters are available through v3dg_frame_stats.
 * V3DG_EINVAL for an image of more than 2^20 16x16 tiles (above 16384 x 16384 pixels). */
v3dg_status v3dg_select(v3dg_ctx* ctx, const v3dg_camera* cam, float tau_px);

/* v3dg_select for n_views cameras at once (a batch of frames of the same instances): every stage
 * of the following v3dg_render covers all views in one launch -- selection over (view, instance,
 * cluster), one depth sort of every view's Gaussians, pairs keyed by (view, tile) -- and it writes
 * n_views images one after the other (view v at offset v * height * width).  Each image is the one
 * v3dg_select with that camera alone gives, bit for bit.  The cameras must share image size,
 * intrinsics and near plane (V3DG_EINVAL otherwise); the views' tiles together are at most 2^20.
 * The parity read-backs then report instance v * n_instances + i for instance i in view v, and
 * v3dg_get_tile_ranges the (view, tile) ranges.  The paper renders one view at a time (Sec. 5). */
v3dg_status v3dg_select_views(v3dg_ctx* ctx, const v3dg_camera* cams, uint32_t n_views, float tau_px);

/* Splat the selected Gaussians (Sec. 2.1; Sec. 5.1: no 2D dilation): projection to 2D means and
 * conics, binning to 16x16 tiles, (tile, depth) sort with ties broken by Gaussian id, and per
 * pixel front-to-back blending C = sum_i c_i a_i prod_{j<i}(1 - a_j) with
 * a = min(0.999, o exp(-q/2)), a < 1/255 skipped, stopping before T < 1e-4; background 0.
 * rgb_out: device, height * width * 3 float32 (row-major, RGB interleaved); T_out: device,
 * height * width float32 final transmittance, or NULL.  Requires a prior v3dg_select
 * (V3DG_ENOTFOUND otherwise). */
v3dg_status v3dg_render(v3dg_ctx* ctx, float* rgb_out, float* T_out);

/* Autotuner of the blend's kernel variant, batch size and work split.  Re-runs the blend stage of
 * the last rendered frame (its sorted pairs and records are still on the device) with every
 * combination of variant (V3DG_OPT_BLEND_MODE 0, 1), records per batch (128, 256, 512) and, for
 * variant 0, long-tile split threshold (4096, 16384, 65536 pairs, or none), times each with CUDA
 * events (best of 3 after one warm-up run) and keeps the fastest as V3DG_OPT_BLEND_MODE,
 * V3DG_OPT_BLEND_BATCH and V3DG_OPT_SPLIT_PAIRS for the frames that follow.  None changes the
 * image.  Synchronous; the caller's image is not touched.  V3DG_ENOTFOUND without a rendered
 * frame, V3DG_EOVERFLOW if that frame was not valid.  mode, batch, split_pairs, best_ms: the choice
 * and its time, each may be NULL.  The paper has no counterpart (its rasterizer is fixed). */
v3dg_status v3dg_autotune_blend(v3dg_ctx* ctx, uint32_t* mode, uint32_t* batch, uint32_t* split_pairs, float* best_ms);

/* v3dg_render into HOST buffers (same layouts): the image is produced on the device and copied
 * back before the call returns. */
v3dg_status v3dg_render_host(v3dg_ctx* ctx, float* rgb_host, float* T_host);

/* Synchronise the stream and report the last frame's counters. */
v3dg_status v3dg_frame_stats(v3dg_ctx* ctx, v3dg_stats* out);

/* Parity read-back (synchronising, host outputs).
 * v3dg_get_cut: the cut of the last v3dg_select before the visibility cull, as (instance, node)
 *   pairs in ascending (instance, node) order; 2 * cap uint32 slots; *n receives the size.
 * v3dg_get_projected: every visible Gaussian of the last render in global-id order; per entry
 *   inst, local (asset-local Gaussian index), u (2), conic (3; q = A dx^2 + 2B dx dy + C dy^2),
 *   opacity, rgb (3), depth_key (bits of the float32 view depth), rect (4; tx0, tx1, ty0, ty1).
 *   Any output pointer may be NULL.
 * v3dg_get_pairs: the sorted (tile, Gaussian) pairs of the last render, as tile id, depth key,
 *   instance and asset-local index.
 * v3dg_get_tile_ranges: for each tile t, [range[2t], range[2t+1]) indexes the sorted pairs. */
v3dg_status v3dg_get_cut(v3dg_ctx* ctx, uint32_t* inst_node, uint64_t cap, uint64_t* n);
v3dg_status v3dg_get_projected(v3dg_ctx* ctx, uint64_t cap, uint64_t* n, uint32_t* inst,
                               uint32_t* local, float* u, float* conic, float* opacity,
                               float* rgb, uint32_t* depth_key, int32_t* rect);
v3dg_status v3dg_get_pairs(v3dg_ctx* ctx, uint64_t cap, uint64_t* n, uint32_t* tile,
                           uint32_t* depth_key, uint32_t* inst, uint32_t* local);
v3dg_status v3dg_get_tile_ranges(v3dg_ctx* ctx, uint32_t* range, uint64_t cap, uint64_t* n_tiles);

/* Per-stage device times (ms) of the last frame when V3DG_OPT_STAGE_TIMING is on, in the order
 * select, project, depth-sort, bin, tile-sort, ranges, blend; also the number of kernels the
 * library has launched since the context was created (*launches may be NULL). */
v3dg_status v3dg_stage_times(v3dg_ctx* ctx, float* ms, int n, uint64_t* launches);

/* Stable LSD radix sort of n (key, value) uint32 pairs on key bits [begin_bit, end_bit), in
 * place, on the context's stream (the sort of the splatting stage, exposed on its own).  keys
 * and vals are device pointers; scratch memory comes from the context's allocator. */
v3dg_status v3dg_sort_pairs(v3dg_ctx* ctx, uint32_t* keys, uint32_t* vals, uint64_t n,
                            int begin_bit, int end_bit);

/* Diagnostic of the bounded device-side waits (the paper has no counterpart).  Every chained scan
 * of the path (selection compaction, pair expansion, radix-sort passes) finds its offsets with a
 * decoupled look-back that polls earlier tiles' status words at most a fixed number of times and
 * then gives up, flags the frame (V3DG_ETIMEOUT) and returns, so that a wait can never hang the
 * GPU.  This call runs both look-back variants (the sort's, one thread with several words per
 * round, and the warp-wide one) as tile 1 of a two-tile chain, with at most spin_limit polls
 * (1 .. 2^20).  predecessor_publishes != 0: tile 0 publishes its prefix first; the call returns
 * V3DG_OK and *prefix (may be NULL) receives the prefix found (1000).  0: tile 0 never publishes;
 * the waits give up after spin_limit polls, the kernel returns, and the call reports
 * V3DG_ETIMEOUT.  Synchronous on the context's stream; the context stays usable either way. */
v3dg_status v3dg_check_wait(v3dg_ctx* ctx, uint32_t spin_limit, int predecessor_publishes, uint32_t* prefix);

/* Release the frame buffers of the context (render list, sort keys and values, records, pairs,
 * images of v3dg_render_host, ...), which grow with the largest frame rendered and are otherwise
 * kept for the next frames; they grow again on demand, and the next v3dg_render needs a new
 * v3dg_select.  Device memory goes back to the context's allocator (or to cudaFree).  *released
 * (may be NULL): the bytes released.  V3DG_EBUSY while a server runs.  The paper has no
 * counterpart. */
v3dg_status v3dg_release_buffers(v3dg_ctx* ctx, uint64_t* released);

/* Largest n that v3dg_sort_pairs_noalloc accepts (its fixed scratch holds this many pairs). */
#define V3DG_SORT_NOALLOC_MAX_PAIRS (1u << 20)

/* The same stable radix sort as v3dg_sort_pairs, for callers that cannot allocate device memory
 * (the paper has no counterpart: this serves hosts that own every device allocation themselves,
 * such as an engine that reserves its pools at start-up, or a real-time loop where cudaMalloc /
 * cudaFree would stall a frame).  It allocates nothing and needs no context: its scratch is one
 * fixed device array of the library, sized for V3DG_SORT_NOALLOC_MAX_PAIRS pairs (about 8.5 MB),
 * held by every GPU that loads the library until the process exits.
 *  - keys, vals: device pointers of the calling thread's current device, n uint32 each, sorted in
 *    place on key bits [begin_bit, end_bit); cuda_stream: a stream of that device (NULL: legacy).
 *  - n > V3DG_SORT_NOALLOC_MAX_PAIRS returns V3DG_EOVERFLOW and does nothing; bad pointers or
 *    bit ranges return V3DG_EINVAL; a bounded device wait that gave up returns V3DG_ETIMEOUT.
 *  - Synchronises cuda_stream before returning.  The first call on a device looks up the scratch
 *    array's address and keeps it; make that first call before any stream capture.  The kept
 *    address does not survive cudaDeviceReset: after a device reset the entry point must not be
 *    used again in the same process.  All calls share the one array: calls whose work overlaps on
 *    the GPU race with each other. */
v3dg_status v3dg_sort_pairs_noalloc(uint32_t* keys, uint32_t* vals, uint64_t n, int begin_bit, int end_bit,
                                    void* cuda_stream);

/* ---------------------------------------------------------------- serving
 * Many independent frames (each its own scene, camera and tolerance) rendered concurrently for
 * interactive or batch clients.  The paper measures one viewer at a time (Sec. 5); serving
 * repeats its per-frame path (select, Sec. 3.4, then splat, Sec. 2.1) once per request.
 *
 * v3dg_server_start starts `slots` workers (1..64) on the context's device.  Each worker owns its
 * own streams and frame buffers (from the server's stream-ordered memory pool: the context's
 * allocator is only ever called from the thread that owns the context) and shares the loaded
 * assets (load them all first).  Requests wait in arrival order; a free worker takes the next one
 * at once when none is in flight, and beside others while two or more requests wait and the
 * device-memory estimates of the requests in flight plus its own fit `hbm_budget` bytes (0: 3/4 of
 * the device memory free at start), so frames overlap on the GPU when requests pile up (a frame
 * started beside others would otherwise only take turns with them kernel by kernel: every stage
 * runs on a persistent grid).  A request's estimate (also used to size its frame buffers before its
 * first frame) grows with its instances, the square root of 1 / tau_px and, for its pairs, of its
 * pixel count (about 9 MB per instance of a 1M-leaf crowd at 1920x1080, tau 1).  A request
 * estimated above half its slot's share of the budget is heavy: it saturates the GPU on its own,
 * so at most one heavy request is in flight (light ones still overlap it).  A
 * request that starts while no other one is in flight, or whose estimate is at most a quarter of
 * every running one's, runs on a high-priority stream, the others on low-priority streams, so a
 * frame alone keeps its solo latency and later ones fill idle SMs.
 * Each frame is checked and re-run with larger buffers on overflow, as v3dg_render does with
 * V3DG_OPT_SYNC_CHECK.  Device memory: the slots allocate from one stream-ordered pool of the
 * server; a slot that holds more frame buffers than half its share of the budget releases them
 * to the pool after its request; a request that runs out of device memory beside others is
 * rendered again once no other request is on the GPU (new requests wait meanwhile), and fails
 * with V3DG_ENOMEM only alone.  While a server runs,
 * v3dg_set_option and v3dg_load_hierarchy return V3DG_EBUSY.  Status EBUSY if a server already
 * runs, ENOTFOUND if no asset is loaded. */
v3dg_status v3dg_server_start(v3dg_ctx* ctx, int slots, uint64_t hbm_budget);

/* Finish every queued request, then stop the workers and free their buffers (results not yet
 * polled are dropped).  v3dg_destroy does this too. */
v3dg_status v3dg_server_stop(v3dg_ctx* ctx);

/* One frame request.  Instance arrays are host pointers as in v3dg_set_instances and camera /
 * tau_px are as in v3dg_select; all are copied by v3dg_submit.  rgb_out (h*w*3 float32) and t_out
 * (h*w float32, or NULL) are host memory when out_on_device == 0 (pinned memory copies faster),
 * else device memory; they are written before the request completes and must stay valid until
 * v3dg_poll reports it. */
typedef struct {
  uint32_t n_instances;
  int32_t out_on_device;
  const uint32_t* asset_id;
  const double* rot;
  const double* trans;
  const double* scale;
  v3dg_camera camera;
  float tau_px;
  float* rgb_out;
  float* t_out;
} v3dg_request;

/* Completion record.  Times are milliseconds on the server's steady clock since it started. */
typedef struct {
  v3dg_status status;    /* the frame's own status (V3DG_OK, V3DG_ETIMEOUT, V3DG_ECUDA, ...) */
  uint32_t batch_views;  /* requests rendered together in this request's frame (V3DG_OPT_SERVE_MERGE) */
  double submit_ms, start_ms, done_ms;
  uint64_t visible;      /* visible Gaussians of the frame (of all its views when batch_views > 1) */
  uint64_t pairs;        /* (tile, Gaussian) pairs of the frame (likewise) */
} v3dg_result;

/* Queue a request; *ticket receives its id (1, 2, ...).  Validation errors are returned here
 * (EINVAL; ENOTFOUND for an unknown asset id or when no server runs; EBUSY while it stops) and
 * nothing is queued then.  v3dg_submit and v3dg_poll may be called from any thread and leave
 * v3dg_last_error unchanged; they must not overlap v3dg_server_stop or v3dg_destroy. */
v3dg_status v3dg_submit(v3dg_ctx* ctx, const v3dg_request* req, uint64_t* ticket);

/* Wait up to timeout_us microseconds for request `ticket`.  V3DG_OK: *out holds its completion
 * record and the ticket is forgotten; V3DG_EBUSY: not done yet (poll again); V3DG_ENOTFOUND: a
 * ticket that was never issued or was already reported. */
v3dg_status v3dg_poll(v3dg_ctx* ctx, uint64_t ticket, uint32_t timeout_us, v3dg_result* out);

#ifdef __cplusplus
}
#endif
#endif /* V3DG_H */
