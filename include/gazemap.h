/*
 * gazemap.h -- C ABI of libgazemap, a GB300 (sm_103a) implementation of surface-based
 * fixation density maps (Javerliat & Lavoue, "GPU accelerated surface-based gaze mapping
 * for XR experiences").
 *
 * The method (Section 3): sample mesh surfaces at a chosen density (samples per m^2); for
 * every sample x fixation pair, keep the pair when the sample lies inside the gaze cone cut
 * at 4 sigma and is visible from the eye, and add the duration-weighted angular Gaussian of
 * Section 3.2.1 to the sample; finally divide every value by the maximum (Section 3.2.3).
 *
 * Conventions for every call:
 *  - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream). All device work
 *    is enqueued on it; calls return once the work is enqueued unless stated otherwise.
 *  - Pointers marked "host or device" are classified with cudaPointerGetAttributes; host
 *    memory is copied to the device inside the call (synchronously for pageable memory).
 *    Input buffers are borrowed for the duration of the call only.
 *  - Handles (gm_ctx, gm_scene, gm_samples, gm_map, gm_field) own their device memory and are
 *    released by the matching gm_*_free / gm_destroy. A handle must outlive every handle built
 *    from it (samples need their scene; maps need their samples).
 *  - Errors: every call returns a gm_status; gm_last_error() returns a thread-local message
 *    for the last failing call on this thread. Kernel-side faults detected by the library
 *    (a BVH deeper than the traversal stack) are reported by the next gm_sync / info call.
 *  - Nothing here falls back to the CPU: without a usable sm_103a device, gm_create fails.
 */
#ifndef GAZEMAP_H
#define GAZEMAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gm_ctx gm_ctx;
typedef struct gm_scene gm_scene;
typedef struct gm_samples gm_samples;
typedef struct gm_map gm_map;
typedef struct gm_field gm_field;
typedef struct gm_batch gm_batch;
typedef void* gm_stream; /* cudaStream_t */

typedef enum {
    GM_OK = 0,
    GM_ERR_INVALID_ARG = 1,  /* bad pointer, size, NaN/Inf input, theta <= 0, ... */
    GM_ERR_CUDA = 2,         /* a CUDA runtime call failed (message has the CUDA error) */
    GM_ERR_OOM = 3,          /* device allocation failed */
    GM_ERR_TIMEOUT = 4,      /* a bounded device wait ran out */
    GM_ERR_UNSUPPORTED = 5,  /* no sm_103a device, or a size beyond a documented limit */
    GM_ERR_INTERNAL = 6,     /* a device-side consistency check failed */
    GM_WARN_EMPTY = 100      /* success, but a map's maximum is 0 (all values 0) */
} gm_status;

/* One mesh of the scene. Section 3.3.4: the sampling density may differ per mesh. */
typedef struct {
    const float* vertices;     /* n_verts x 3 FP32, mesh-local (host or device) */
    const uint32_t* indices;   /* n_tris x 3 vertex indices (host or device) */
    uint32_t n_verts;
    uint32_t n_tris;
    double transform[16];      /* row-major 4x4 local -> world (metres), applied in FP64 */
    uint32_t object_id;        /* reported per sample (Section 3.3.3 export format) */
} gm_mesh_desc;

/* Fixations, structure of arrays (host or device). */
typedef struct {
    const float* eye_xyz;      /* n x 3, world-space eye position */
    const float* gaze_xyz;     /* n x 3, gaze direction (any non-zero length) */
    const float* duration_s;   /* n, fixation duration t in seconds (weights g, Section 3.2.1) */
    const double* timestamp_s; /* n, fixation start time (windowing, Section 3.3.4) */
    uint32_t n;
} gm_fixations;

/* Generation parameters (Section 3.3.4 lists theta, per-mesh density and the time interval). */
typedef struct {
    float theta_rad;      /* angular deviation theta = one standard deviation (> 0) */
    float cutoff_sigmas;  /* cone cut-off in sigmas; 4 in the paper (Fig. 4, Section 3.3.2) */
    float eps_rel;        /* occlusion segment stops (1 - eps_rel) of the way to the sample */
    double t_begin;       /* fixations with t_begin <= timestamp < t_end are used */
    double t_end;
    double window_s;      /* > 0: one map per window of this length from t_begin; else one map */
    int32_t normalize;    /* non-zero: divide each map by its maximum in place (Section 3.2.3) */
    int32_t flags;        /* GM_F_* below */
    uint64_t debug_pair_cap; /* > 0 with GM_F_DEBUG_PAIRS: record up to this many in-cone pairs */
} gm_params;

enum {
    GM_F_TIMING = 1,        /* record CUDA events around each stage (gm_map_stats.*_ms) */
    GM_F_DEBUG_PAIRS = 2,   /* record in-cone pairs (sample, fixation, visible, weight) */
    GM_F_NO_REORDER = 4,    /* process samples in stored order (no spatial work order) */
    GM_F_NO_COMPACT = 8,    /* trace each lane's in-cone rays in place (no per-warp ray queue; 4
                               samples per thread unless GM_F_SPT1) */
    GM_F_WIDE_BVH = 16,     /* traverse the 4-wide collapse of the tree instead of the binary tree */
    GM_F_REGCAP64 = 32,     /* cap the accumulation kernel at 64 registers (4 blocks per SM; the
                               one-sample ray-queue kernel, the default, always fits 64) */
    GM_F_TILE_CONSECUTIVE = 64, /* multi-sample warp tiles of consecutive samples (else runs of 32 spread
                               over 8 tiles' span); a one-sample tile is one run of 32 either way */
    GM_F_STATIC_TILES = 128, /* one warp tile per warp of a full grid (else warps pull tiles from a counter) */
    GM_F_NO_TILE_CULL = 256, /* test every sample against every fixation (no warp-tile sphere test) */
    GM_F_BLOCK128 = 512,    /* blocks of 128 threads instead of 256 for the ray-queue binary-tree
                               kernel (one sample per thread: 8 per SM; with GM_F_SPT4: 7 per SM at
                               72 registers, 8 with GM_F_REGCAP64); with the eye grid: 6 per SM */
    GM_F_EYE_GRID = 1024,   /* occlusion through per-fixation eye grids instead of the BVH (ray-queue
                               kernel only: with NO_COMPACT, WIDE_BVH or REGCAP64 the BVH is kept) */
    GM_F_GRID64 = 2048,     /* with GM_F_EYE_GRID: 64 x 64 cells per fixation instead of 128 x 128 */
    GM_F_SPT1 = 4096,       /* warp tiles of 32 samples (1 per thread); the default of the ray-queue
                               binary-tree kernel (the eye grid's default is 4 per thread); with
                               GM_F_NO_COMPACT: one-sample tiles traced in place */
    GM_F_SPT2 = 8192,       /* warp tiles of 64 samples (2 per thread): ray-queue binary tree and eye grid */
    GM_F_BLOCK512 = 16384,  /* blocks of 512 threads: eye grid (1 or 2 samples per thread) and the
                               one-sample ray-queue binary-tree kernel */
    GM_F_FIX_L1 = 32768,    /* ray-queue binary-tree kernel: read the fixations one by one through L1
                               (warp-wide broadcasts) instead of staging them 32 at a time in each
                               warp's shared memory */
    GM_F_SPT4 = 65536       /* warp tiles of 128 samples (4 per thread): the ray-queue binary-tree kernel
                               (the in-place and 4-wide kernels always take 4) */
};

typedef struct {
    uint64_t pairs;           /* nominal sample x fixation pairs (valid fixations only) */
    uint64_t in_cone;         /* pairs inside the cut-off cone = occlusion rays traced */
    uint64_t visible;         /* in-cone pairs whose ray reached the sample */
    uint32_t n_windows;
    uint32_t n_fixations_used;
    float prep_ms;            /* fixation prep + window sort (GM_F_TIMING) */
    float accumulate_ms;      /* cone + occlusion + Gaussian + store + max kernel */
    float normalize_ms;
    uint32_t launches;        /* kernels this call launched */
    uint64_t nodes_visited;   /* BVH nodes fetched by all occlusion rays (eye grid: cell entries read) */
    uint64_t tris_tested;     /* ray/triangle tests performed by all occlusion rays */
    uint64_t pairs_tested;    /* sample x fixation cone tests evaluated (pairs of warp tiles whose bounding
                                 sphere the cone misses are skipped without a per-sample test) */
    float grid_ms;            /* eye-grid frames, counts and (first chunk's) cell lists (GM_F_TIMING) */
    uint32_t grid_chunks;     /* fixation chunks the eye grid was built in (0: BVH occlusion, the default) */
    uint32_t grid_launches;   /* accumulation launches over runs of fixations (eye grid) */
} gm_map_stats;

/* ---- context ------------------------------------------------------------------------ */

/* Bind `device` (must be compute capability 10.3) and create a context. */
gm_status gm_create(int device, gm_ctx** out);
void gm_destroy(gm_ctx* ctx);
const char* gm_last_error(void);
/* Wait for `stream`, then report any device-side fault recorded by library kernels. */
gm_status gm_sync(gm_ctx* ctx, gm_stream stream);
/* Failure-detection check of the bounded device waits (not in the paper): one block waits, with
 * the wait the tensor-core field kernels use, on an mbarrier that nothing completes, gives up
 * after `iterations` polls (1 .. 2^16) and records the timeout; the next gm_sync returns
 * GM_ERR_TIMEOUT and clears it, and the context stays usable. Nothing hangs or faults. */
gm_status gm_debug_wait_timeout(gm_ctx* ctx, uint32_t iterations, gm_stream stream);
/* Number of kernels this context has launched so far (every library launch site counts). */
gm_status gm_ctx_launches(const gm_ctx* ctx, uint64_t* kernel_launches);

/* ---- scene (meshes -> world triangles -> BVH) ----------------------------------------- */

/* Transform every mesh to world space (FP64, rounded to FP32), then build a BVH over all
 * triangles: Morton codes of centroids, LSD radix sort, then PLOC clustering (default) or
 * Karras' HPG 2012 hierarchy, bottom-up boxes, internal nodes stored depth-first. The BVH
 * replaces the per-view z-buffer of Section 3.2.2 as the occlusion structure. Meshes are
 * concatenated in order; global triangle ids follow that order. Synchronises `stream` (to
 * check the tree depth; the clustering reads its cluster count back once per round). */
gm_status gm_build_scene(gm_ctx* ctx, const gm_mesh_desc* meshes, uint32_t n_meshes,
                         gm_stream stream, gm_scene** out);
/* Builders of the hierarchy (same node layout and traversal either way):
 *  GM_BUILD_LBVH: Karras' linear BVH from the Morton order (HPG 2012), fastest to build;
 *  GM_BUILD_PLOC: parallel locally-ordered clustering (Meister & Bittner, TVCG 2018) from the same
 *                 Morton order, merging mutual nearest neighbours by union-box surface area
 *                 within +-ploc_radius positions (8 by default); a tighter tree for a few more
 *                 milliseconds of build (the default used by gm_build_scene). */
enum { GM_BUILD_LBVH = 0, GM_BUILD_PLOC = 1, GM_BUILD_DEFAULT = GM_BUILD_PLOC };
typedef struct {
    int32_t builder;
    int32_t dynamic;   /* nonzero: keep the mesh-local triangles (48 B per triangle) so that
                          gm_scene_pose can move the meshes later */
    int32_t ploc_radius; /* GM_BUILD_PLOC: neighbours searched on each side, 4, 8, 16, 32 or 64 (0: 8) */
} gm_build_opts;
gm_status gm_build_scene_opts(gm_ctx* ctx, const gm_mesh_desc* meshes, uint32_t n_meshes,
                              const gm_build_opts* opts, gm_stream stream, gm_scene** out);
gm_status gm_scene_info(const gm_scene* scene, uint32_t* n_tris, uint32_t* bvh_depth);
/* Dynamic scenes. The surface-bound map ties densities to objects, not to world space (Section 2
 * contrasts this with volumetric maps, which leave fixations behind when an object moves), so a
 * mesh that moves carries its samples with it. gm_scene_pose gives every mesh a new row-major
 * 4 x 4 transform (`transforms`: n_meshes x 16 FP64, host memory): the world triangles are
 * recomputed from the kept mesh-local ones exactly as at build time (a pose equal to the build's
 * transforms reproduces them bit for bit), the BVH boxes are refit bottom-up over the unchanged
 * hierarchy (same depth, looser boxes as meshes move apart), the export's local frames follow,
 * and the 4-wide collapse is dropped. Requires a scene built with gm_build_opts.dynamic;
 * GM_ERR_INVALID_ARG otherwise or on a non-finite transform. Synchronises `stream` once. Sample
 * sets of the scene keep stale positions until gm_samples_follow. */
gm_status gm_scene_pose(gm_scene* scene, const double* transforms, gm_stream stream);
/* Copy the world triangles (n_tris x 9 FP32, v0 v1 v2) to `dst` (host or device). */
gm_status gm_scene_triangles(const gm_scene* scene, float* dst, gm_stream stream);
void gm_scene_free(gm_scene* scene);

/* ---- samples (Section 3.1) ----------------------------------------------------------- */

/* Area-weighted surface sampling. Triangle i of mesh m gets count_i samples with
 * |count_i - k_m A_i| < 1 (A_i its FP64 world area): counts are differences of the rounded
 * running total of k_m A_i in 32.32 fixed point. Global sample j (mesh order, triangle order,
 * then j) is placed from Philox4x32-10(key = seed, counter = (j lo, j hi, session, 0)) words
 * w0, w1: u = ((w >> 9) + 1/2) 2^-23, barycentrics (1 - sqrt u1, sqrt u1 (1 - u2), sqrt u1 u2).
 * density_per_mesh: n_meshes samples-per-m^2 values (host memory). Synchronises `stream`
 * once (to read the sample count). Fails with GM_ERR_UNSUPPORTED beyond 2^31 - 1 samples. */
gm_status gm_sample_surface(gm_scene* scene, const double* density_per_mesh, uint64_t seed,
                            uint32_t session, gm_stream stream, gm_samples** out);
/* The paper's own sampler (Section 3.1): triangle i gets the integer resolution r_i of the adaptive
 * rule (D = 1 + 8 k_m A_i; r = 1 if D < 25, else rint((-3 + sqrt(D)) / 2)) and the
 * (r+1)(r+2)/2 samples of its barycentric grid (Eq. 1), indexed in O(1) (Eq. 2): local sample idx
 * sits at row = max m with m(m+1)/2 <= idx, col = idx - row(row+1)/2, with weights
 * (col/r, 1 - row/r, (row - col)/r) on (v0, v1, v2) (Eq. 3; its printed third weight does not
 * sum to one, 1 - w1 - w2 is used). Samples on shared edges and vertices are repeated per
 * triangle, as in the paper. Same layout and calls as gm_sample_surface (bary2 = (w2, w3)).
 * Synchronises `stream` once. Resolutions of 65535 or more return GM_ERR_UNSUPPORTED. */
gm_status gm_sample_surface_grid(gm_scene* scene, const double* density_per_mesh, gm_stream stream,
                                 gm_samples** out);
/* Explicit query points (n x 3 FP32 world positions, each on triangle tri[i], which is
 * excluded from its occlusion test), host or device. Used for GM_Q_PLAIN queries. */
gm_status gm_samples_from_points(gm_scene* scene, const float* xyz, const uint32_t* tri,
                                 uint64_t n, gm_stream stream, gm_samples** out);
gm_status gm_samples_info(const gm_samples* s, uint64_t* n_samples);
/* Copy the per-triangle start offsets (n_tris + 1 int64) to `dst` (host or device). */
gm_status gm_samples_offsets(const gm_samples* s, int64_t* dst, gm_stream stream);
/* Copy sample data in stored order; any destination may be NULL (host or device):
 * xyz n x 3 FP32, tri n global triangle ids, bary2 n x 2 FP32 (b1, b2; b0 = 1 - b1 - b2),
 * obj n object ids (Section 3.3.3 export fields). */
gm_status gm_samples_copy(const gm_samples* s, float* xyz, uint32_t* tri, float* bary2,
                          uint32_t* obj, gm_stream stream);
/* Samples [begin, end) of `src` in its stored order, as a sample set of their own (positions and
 * barycentrics copied, a spatial work order of their own): the slice one GPU takes when the path
 * is sharded by samples (each sample's value depends on no other sample, so the slices' maps are
 * the whole map's values, bit for bit). The slice is a set of fixed points: it has no per-triangle
 * offsets and does not follow re-posed meshes. */
gm_status gm_samples_slice(const gm_samples* src, uint64_t begin, uint64_t end, gm_stream stream, gm_samples** out);
void gm_samples_free(gm_samples* s);
/* Re-place a Philox or grid sample set on its scene's current pose: same triangle, same
 * barycentrics (same counts per triangle: the densities of the first pose stand), positions from
 * the posed vertices by the sampler's own arithmetic. GM_ERR_INVALID_ARG for explicit points. */
gm_status gm_samples_follow(gm_samples* s, gm_stream stream);

/* The export record of Section 3.3.3, one entry per sample in stored order; any destination may
 * be NULL, each host or device: value (FP32, the map's window `window`, normalised iff the map
 * was), object id, triangle id (global), barycentrics (w0, w1, w2) FP32 x 3, mesh-local position
 * FP32 x 3 (the world position mapped back by the inverse of the mesh transform, FP64),
 * world position FP32 x 3. */
typedef struct {
    float* value;
    uint32_t* object_id;
    uint32_t* triangle;
    float* bary3;
    float* local_xyz;
    float* world_xyz;
} gm_export_dst;
gm_status gm_samples_export(const gm_samples* s, const gm_map* map, uint32_t window, const gm_export_dst* dst,
                            gm_stream stream);

/* Allocation-free per-triangle sample offsets. The paper has no counterpart: this is a service
 * for callers that cannot allocate device memory when they need the offsets -- an engine
 * plugin whose host application owns all device memory through its own allocator, or a
 * real-time (per-frame) thread on which cudaMalloc may stall or fail. It computes exactly the
 * offsets gm_sample_surface computes (FP64 area, rint(k A 2^32), int64 prefix, rounded starts;
 * bit-identical) and calls no allocator.
 *   tri_xyz:         n_tris x 9 FP32 world vertices (v0 v1 v2), device memory
 *   density_per_tri: n_tris FP64 samples per m^2, device memory
 *   offsets:         n_tris + 1 int64 output, device memory (also used as the prefix buffer)
 * Scratch: the per-block partial sums live in a file-scope __device__ array of 65 536 int64
 * (512 KiB) that every GPU loading this library holds until the process exits, so n_tris is
 * limited to 65 536 * 2 048 = 134 217 728; larger inputs return GM_ERR_UNSUPPORTED without
 * launching anything. Every call shares that array and it keeps the last call's contents;
 * nothing in it needs to start at zero (each call writes every partial it reads), but calls
 * that overlap on the GPU (different streams, or other threads) race on it and must be
 * serialised by the caller. The first call with each gm_ctx looks up the array's device address
 * (cudaGetSymbolAddress, with the context's device current); make that first call before any
 * stream capture. Densities that are negative, NaN or give a triangle 2^31 or more samples set that
 * triangle's count to 0 and are reported by the next gm_sync (GM_ERR_INTERNAL). A scene whose
 * expected total (the FP64 sum of k A over its triangles) exceeds 2^31 - 16 samples would wrap
 * the int64 prefix: then every offset is written as 0 and the next gm_sync returns
 * GM_ERR_UNSUPPORTED. The scratch address is looked up per gm_ctx: after a cudaDeviceReset,
 * create a new context (the old one's device memory is gone anyway) and it looks it up again. */
gm_status gm_tri_offsets_noalloc(gm_ctx* ctx, const float* tri_xyz, const double* density_per_tri,
                                 uint32_t n_tris, int64_t* offsets, gm_stream stream);

/* ---- accumulation (Section 3.2) -------------------------------------------------------- */

/* For every sample s and every fixation f whose timestamp lies in [t_begin, t_end):
 *   p = s - e_f, r^ = r_f/|r_f|, d1 = p.r^, d2 = |p x r^|, sigma = tan(theta);
 *   the pair counts when d1 > 0, d2/d1 <= cutoff * sigma (the 4 sigma cone), and the segment
 *   from e_f to e_f + (1 - eps_rel) p meets no triangle but the sample's own;
 *   then value[window(f)][s] += t_f / (sigma sqrt(2 pi)) exp(-(d2/d1)^2 / (2 sigma^2)).
 * Sums are compensated (Kahan) FP32 in fixation order. The maximum of each window's map is
 * kept; with params->normalize the map is divided by it in place (max 0 => map stays 0 and
 * the call returns GM_WARN_EMPTY at gm_map_info).
 * Occlusion: by default every segment walks the scene's BVH. With GM_F_EYE_GRID each fixation
 * gets an eye grid instead -- the triangles that can meet its cone, binned by their image in the
 * gaze frame into 128 x 128 cells (GM_F_GRID64: 64 x 64) and sorted by depth -- and a segment
 * tests the triangles of its own cell. Both give the same maps (the same triangle test over every
 * triangle it can report).
 * The eye grid's memory is taken on the stream for the call: at most a third of the free device
 * memory for the cell lists of one chunk of fixations (more fixations run in several chunks) and
 * 1 GiB of offset tables; the environment variable GM_EYEGRID_CHUNK_ENTRIES, read at each call,
 * lowers the per-chunk entry budget (a chunk always takes at least one fixation). Within a chunk
 * the accumulation can run once per run of fixations whose lists hold at most GM_EYEGRID_L2_ENTRIES
 * entries (of 8 bytes; default: one launch per chunk), carrying the sums over. The call reads the per-fixation list sizes back once (it
 * synchronises the stream). */
gm_status gm_accumulate_fixations(gm_scene* scene, gm_samples* samples, const gm_fixations* fix,
                                  const gm_params* params, gm_stream stream, gm_map** out);
/* The same accumulation for a scene whose meshes move from window to window (params->window_s > 0
 * gives the windows; one window otherwise). `window_transforms` holds n_windows x n_meshes x 16
 * FP64 row-major transforms in host memory. For each window k in order: gm_scene_pose with the
 * window's transforms, gm_samples_follow on `samples`, then the fixations of window k only
 * (window k = floor((t - t_begin) / window_s), as above) are accumulated into window k of one
 * map; every window is normalised at the end when params->normalize. The scene and the samples
 * are left in the last window's pose. GM_F_TIMING is ignored (no stage times). Requires a scene
 * built with gm_build_opts.dynamic and a Philox or grid sample set. */
gm_status gm_accumulate_dynamic(gm_scene* scene, gm_samples* samples, const gm_fixations* fix,
                                const gm_params* params, const double* window_transforms, gm_stream stream,
                                gm_map** out);
/* ---- the paper's z-buffer occlusion path (Sections 3.2.2, 3.3.2, Appendix A) -------------
 * The same accumulation with the paper's visibility test in place of the exact ray: for every
 * fixation a camera at the eye (forward and up hints per fixation: the head pose; NULL forward =
 * the gaze, NULL up = +y), the crop window of the cutoff cone on the near plane, a z-buffer of
 * res x res pixels over that window holding the linear view depth w of the nearest surface at
 * each pixel centre (geometry clipped to near <= w <= far, triangles two-sided), and a pair
 * counts as visible when the sample lies in the crop frustum (the NDC filter of Section 3.3.2)
 * and |w_sample - w_zbuffer| <= eps (Section 3.2.2). The crop window is the exact bounding box of
 * the cone's section (Appendix A centres its box on the gaze point E, which is not the centre of
 * an oblique conic section, so the printed box can cut the cone). The cone test, the Gaussian,
 * windows, compensated sums and normalisation are those of gm_accumulate_fixations. Fixations
 * whose cone reaches behind their camera have no crop window and are skipped (counted). With
 * `compare` the exact ray test also runs on every in-cone pair and the disagreements are counted
 * (gm_zbuffer_stats). Z-buffers are built for chunks of fixations of at most `zbuffer_bytes`
 * (0: 2 GiB). Synchronises `stream` a few times per chunk. */
typedef struct {
    uint32_t res;            /* z-buffer pixels per side (a generation parameter, Section 3.3.4) */
    float near_m, far_m;     /* clip planes, metres, 0 < near < far */
    float eps_m;             /* the +-eps of the depth comparison, metres */
    uint32_t compare;        /* nonzero: count disagreements with the exact ray test */
    uint64_t zbuffer_bytes;  /* device memory for one chunk of z-buffers (0: 2 GiB) */
} gm_zbuffer_params;
gm_status gm_accumulate_zbuffer(gm_scene* scene, gm_samples* samples, const gm_fixations* fix,
                                const float* cam_forward, const float* cam_up, const gm_params* params,
                                const gm_zbuffer_params* zb, gm_stream stream, gm_map** out);
/* Statistics of a z-buffer map: fixations skipped (no crop window), in-cone pairs the z-buffer
 * calls visible but the ray test hides, pairs it hides but the ray test sees (both 0 unless
 * `compare`), and (fixation, triangle) pairs sent to the rasteriser. */
gm_status gm_zbuffer_stats(const gm_map* map, uint64_t* skipped_fixations, uint64_t* flips_to_visible,
                           uint64_t* flips_to_hidden, uint64_t* raster_pairs);
/* The z-buffers themselves, for n fixations in input order (no windows, no accumulation):
 * zbuf (host or device) receives n x res x res FP32 depths (row = pixel y from the window's
 * bottom, +inf where no surface), crop (host, may be NULL) n x 4 FP64 (l, r, b, t on the near
 * plane; NaN for a fixation without a crop window). Synchronises `stream`. */
gm_status gm_zbuffer_render(gm_scene* scene, const float* eye, const float* gaze, const float* cam_forward,
                            const float* cam_up, uint32_t n, float theta_rad, float cutoff_sigmas,
                            const gm_zbuffer_params* zb, float* zbuf, double* crop, gm_stream stream);

/* Number of windows, samples and statistics; waits for the map's work to finish. */
gm_status gm_map_info(gm_map* map, uint32_t* n_windows, uint64_t* n_samples, gm_map_stats* stats);
/* Copy window `window` (n_samples FP32 values in stored sample order) to `dst` (host or
 * device), and its maximum to *max_out (may be NULL). Values are normalised iff the map was
 * accumulated with params->normalize. */
gm_status gm_map_copy(const gm_map* map, uint32_t window, float* dst, float* max_out, gm_stream stream);
/* The maximum of every window (n_windows floats, host or device): the map's own raw maxima, or
 * those it was normalised by. */
gm_status gm_map_max(const gm_map* map, float* out, gm_stream stream);
/* Divide every window of a raw map (accumulated with params.normalize = 0) by `maxima` (n_windows
 * floats >= 0, host or device; NULL: the map's own maxima) and keep those as the map's maxima;
 * windows whose maximum is 0 stay 0. Section 3.2.3's normalisation when the maximum comes from
 * elsewhere: the ranks of a sample-sharded run normalise their slices by the maximum over all
 * ranks. Call it once per map. */
gm_status gm_map_normalize(gm_map* map, const float* maxima, gm_stream stream);
/* Device pointer to the map values (n_windows x n_samples FP32, window-major), owned by map. */
const float* gm_map_device_values(const gm_map* map);
/* Recorded in-cone pairs (GM_F_DEBUG_PAIRS), in no particular order: sample index (stored
 * order), fixation index (input order), visible flag, weight g. Host arrays of `cap`
 * entries; *n returns how many pairs were found (may exceed cap). */
gm_status gm_map_debug_pairs(const gm_map* map, uint32_t* sample, uint32_t* fix, uint8_t* visible,
                             float* g, uint64_t cap, uint64_t* n);
void gm_map_free(gm_map* map);

/* ---- batched sessions (a persistent, graph-captured launch; not in the paper) ------------ */

/* One independent problem: its scene, its samples (built on that scene) and its fixations
 * (host or device, copied into the plan at creation). */
typedef struct {
    gm_scene* scene;
    gm_samples* samples;
    gm_fixations fix;
} gm_session_desc;

/* Plan many sessions of uneven size as one call: all sessions' fixations are staged once; a
 * work list of warp tiles (32 x 4 consecutive work-order samples of one session) is ordered by
 * decreasing cost; the fixation prep, a persistent accumulation kernel that pulls work items
 * from a device counter, and the per-session normalisation are captured into one CUDA graph.
 * Every session gets its own map (windows as in gm_accumulate_fixations). The variant flags in
 * params (GM_F_NO_COMPACT, GM_F_WIDE_BVH, GM_F_REGCAP64) pick the kernel; gm_batch_autotune picks
 * them by measurement. The plan borrows the scenes and samples: free it before them. Scalar
 * parameters are shared by all sessions. Synchronises `stream` once. */
gm_status gm_batch_create(gm_ctx* ctx, const gm_session_desc* sessions, uint32_t n_sessions,
                          const gm_params* params, gm_stream stream, gm_batch** out);
/* Replay the plan on `stream` (one graph launch; nothing is allocated or copied). */
gm_status gm_batch_run(gm_batch* batch, gm_stream stream);
/* Session i's map, owned by the plan and valid until gm_batch_free (refreshed by every run). */
gm_status gm_batch_map(gm_batch* batch, uint32_t session, gm_map** map);
/* Plan facts; *last_ms is the device time of the last completed run (0 if none). */
gm_status gm_batch_info(gm_batch* batch, uint32_t* n_sessions, uint64_t* n_work_items, uint64_t* pairs,
                        float* last_ms, int32_t* variant_flags);
/* The plan groups its sessions into three size buckets (fewer than 2^14, fewer than 2^17, more
 * triangles); each bucket's work items run in their own persistent launch of the graph, with
 * their own variant. gm_batch_autotune times every accumulation variant on every bucket's own
 * launch (events recorded in the graph), keeps each bucket's fastest (re-capturing the graph) and
 * returns the flags of the bucket with the most work and the time of a replay with the chosen
 * variants. Cached per bucket and size; see gm_autotune_accumulate. */
gm_status gm_batch_autotune(gm_batch* batch, gm_stream stream, int32_t* best_flags, float* best_ms);
/* Per bucket (3): its variant flags, sessions, work items and the device time of its launch in
 * the last completed replay (0 if none). Any output may be NULL. */
gm_status gm_batch_buckets(gm_batch* batch, uint32_t* n_buckets, int32_t* flags, uint32_t* sessions,
                           uint32_t* work_items, float* last_ms);
void gm_batch_free(gm_batch* batch);
/* One-shot form: plan, run once, hand every session's map to the caller (free each with
 * gm_map_free). */
gm_status gm_accumulate_batch(gm_ctx* ctx, const gm_session_desc* sessions, uint32_t n_sessions,
                              const gm_params* params, gm_stream stream, gm_map** out_per_session);
/* Pick the fastest accumulation variant for one problem. Candidates: with the BVH, ray
 * queue on/off, binary or 4-wide tree, 80- or 64-register cap, spread or consecutive warp tiles,
 * persistent or static scheduling (32), and blocks of 128 instead of 256 threads for the
 * ray-queue binary-tree kernels (8 more); with the eye grid (GM_F_EYE_GRID), 128 or 64 cells a side times the
 * warp-tile and block shape (4, 2 or 1 samples per thread; 256, 128 or 512 threads) times spread
 * or consecutive tiles (28). Each is timed (fixation prep + eye grid + accumulation, best of two)
 * on a prefix of the fixations (a sixteenth, at least 256); the two fastest are timed again on
 * all of them and the faster is kept. *best_flags gets the GM_F_* variant bits to OR into
 * params->flags. Results are
 * cached per size bucket (log2 of samples, fixations and triangles) for the process and, when the
 * environment variable GM_TUNE_CACHE names a file, in that JSON file across processes. */
gm_status gm_autotune_accumulate(gm_scene* scene, gm_samples* samples, const gm_fixations* fix,
                                 const gm_params* params, gm_stream stream, int32_t* best_flags, float* best_ms);

/* ---- neural density field (a learned stand-in for the map; not in the paper) ------------- */

/* Parameters of the field, FP32, packed in this order: W1 (64 x 64, row = output unit), b1, W2,
 * b2, W3, b3, W4, b4 (hidden layers), w5 (64), b5 (output). */
#define GM_FIELD_N_PARAMS 16705

typedef struct {
    uint32_t steps;   /* Adam steps */
    uint32_t batch;   /* points per step, drawn by Philox4x32-10(key = seed, counter = (step, i)) mod n */
    float lr;         /* learning rate at step 0, cosine-decayed ... */
    float lr_min;     /* ... to this at the last step */
    uint64_t seed;
} gm_field_cfg;

/* The field f(x) = softplus(w5 . h4 + b5), h_l = bf16(relu(h_{l-1} bf16(W_l)^T + b_l)),
 * h0 = bf16(features), features = [x~, sin(2^k pi x~), cos(2^k pi x~), k = 0..9, 0] of
 * x~ = (x - centre) / (half the largest side of the box [box_lo, box_hi]). Hidden-layer products
 * run on the tensor cores (BF16 in, FP32 accumulate). init_params: GM_FIELD_N_PARAMS FP32
 * values (host or device), copied. Adam moments start at zero. */
gm_status gm_field_create(gm_ctx* ctx, const float* box_lo, const float* box_hi, const float* init_params,
                          gm_stream stream, gm_field** out);
/* Train on a map: inputs are the samples' positions, targets the map values of `window` (use a
 * map accumulated with normalize set, so targets lie in [0, 1]); mean squared error, Adam
 * (beta 0.9, 0.999, eps 1e-8, bias-corrected). *final_loss (may be NULL) gets the last batch's
 * mean squared error. Synchronises `stream` once at the end. */
gm_status gm_field_train(gm_field* field, const gm_samples* samples, const gm_map* map, uint32_t window,
                         const gm_field_cfg* cfg, gm_stream stream, float* final_loss);
/* One Adam step on the points xyz[batch_idx[i]] (n x 3 FP32) with targets target[batch_idx[i]];
 * all device memory; batch_idx NULL draws the batch with Philox as gm_field_train does. */
gm_status gm_field_step(gm_field* field, const float* xyz, const float* target, uint64_t n,
                        const uint32_t* batch_idx, uint32_t batch, float lr, gm_stream stream);
/* Loss (mean squared error) and its gradient (GM_FIELD_N_PARAMS FP32, host or device) on one
 * batch without updating the parameters; inputs in device memory. */
gm_status gm_field_loss_grad(gm_field* field, const float* xyz, const float* target, uint64_t n,
                             const uint32_t* batch_idx, uint32_t batch, float* grad_out, float* loss_out,
                             gm_stream stream);
/* Evaluate the field at n points (n x 3 FP32, host or device) into out (host or device). The
 * default kernel runs the four hidden layers on the 5th-generation tensor cores: 128-point tiles,
 * tcgen05.mma (bf16 x bf16, FP32 accumulator in tensor memory), point tiles brought in by bulk
 * asynchronous copies; the other computes them with warp-level mma.sync. Both round every
 * activation to bf16 and accumulate in FP32; they may differ in the last bits of a sum. A device
 * wait that does not complete is reported by the next gm_sync. */
enum { GM_FIELD_QUERY_TCGEN05 = 0, GM_FIELD_QUERY_MMA_SYNC = 1 };
gm_status gm_field_query(const gm_field* field, const float* xyz, uint64_t n, float* out, gm_stream stream);
gm_status gm_field_query_kernel(gm_field* field, int32_t kernel);
/* The kernel that computes training gradients (gm_field_train, gm_field_step, gm_field_loss_grad).
 * GM_FIELD_QUERY_TCGEN05 (default): one persistent block per SM over 128-point tiles; every
 * hidden-layer product of the forward and backward passes, the weight gradients dZ^T H and the
 * bias gradients runs as tcgen05.mma with FP32 accumulators in tensor memory, the gradients stay
 * there across a block's tiles, and the blocks' partial sums are added in a fixed order, so the
 * gradient of a batch does not depend on scheduling. GM_FIELD_QUERY_MMA_SYNC: warp-level mma.sync,
 * one block per 128 points, gradients summed with atomics. Same definition and rounding; sums
 * may differ in their last bits. */
gm_status gm_field_train_kernel(gm_field* field, int32_t kernel);
/* Copy the FP32 master parameters (GM_FIELD_N_PARAMS) to out (host or device). */
gm_status gm_field_params(const gm_field* field, float* out, gm_stream stream);
/* Checkpoint and resume of training (the field is not in the paper): the FP32 parameters, the two
 * Adam moment vectors (GM_FIELD_N_PARAMS floats each, the layout of gm_field_params) and the number
 * of Adam steps taken, which sets both the bias corrections and the batch draws of the next
 * gm_field_train. Buffers host or device; get: any pointer may be NULL (that part is skipped);
 * set: all three are required, the bf16 weight copies are refreshed from theta. A field restored
 * from a checkpoint and trained on continues exactly as the original would. */
gm_status gm_field_get_state(const gm_field* field, float* theta, float* m, float* v, uint32_t* steps,
                             gm_stream stream);
gm_status gm_field_set_state(gm_field* field, const float* theta, const float* m, const float* v, uint32_t steps,
                             gm_stream stream);
gm_status gm_field_info(const gm_field* field, uint32_t* n_params, uint32_t* steps_taken, float* last_loss,
                        float* train_ms);
void gm_field_free(gm_field* field);

/* ---- queries -------------------------------------------------------------------------- */

typedef enum {
    GM_Q_SAMPLE = 0,  /* gather: out[i] = map value of sample idx[i] (window `window`) */
    GM_Q_PLAIN = 1,   /* evaluate the plain accumulation at explicit points (see below) */
    GM_Q_FIELD = 2    /* evaluate a trained neural density field at explicit points */
} gm_query_mode;

/* GM_Q_SAMPLE: `map` and `sample_idx` (n indices, host or device) are used.
 * GM_Q_PLAIN: unused here; build points with gm_samples_from_points and accumulate them.
 * GM_Q_FIELD: `field` and `xyz` (n x 3 FP32 world points, host or device) are used.
 * out: n FP32 values (host or device). */
gm_status gm_query_density(const gm_map* map, const gm_field* field, gm_query_mode mode,
                           uint32_t window, const uint32_t* sample_idx, const float* xyz,
                           uint64_t n, float* out, gm_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* GAZEMAP_H */
