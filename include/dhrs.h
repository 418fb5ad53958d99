/*
 * dhrs.h -- C ABI of libdhrs: the server-side hot path of DHR+S (distributed
 * hybrid rendering with soft shadows and ambient occlusion) on one NVIDIA
 * B300 (sm_103a).
 *
 * Per frame the server receives a camera (Section 4.1: the client sends its
 * camera data), traces per-pixel visibility -- one cone-jittered shadow ray
 * per light (Section 3.1, Fig. 1) and N cosine-weighted ambient-occlusion
 * rays of length r (Section 3.2, Eqs. 1-3) -- from a G-buffer produced by
 * primary rays (standing in for the client rasteriser of Section 1), and
 * reconstructs the noisy result with the modified SVGF of Section 3.3.
 * Outputs per pixel: a visibility bitmask with one bit per light (Fig. 1)
 * and the 8-bit count N_unoccluded (Section 3.2), or their filtered form.
 *
 * Conventions
 *  - Every call returns dhr_status; nothing throws across the ABI.  On
 *    failure dhr_last_error() returns a thread-local message.
 *  - "device" pointers are CUDA global-memory pointers of the current
 *    device; "host" pointers are CPU memory.  Per-frame inputs and outputs
 *    are owned by the caller; scenes, SVGF history and sessions are owned by
 *    the library and freed by their destroy call.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Kernels
 *    are enqueued asynchronously on it; a launch error is reported by the
 *    call that enqueued it, an execution error by the next synchronising
 *    call (DHR_ERR_CUDA).
 *  - Images are row-major, row 0 at the top, W*H pixels.  A pixel is
 *    background when its primary ray misses: depth +inf, mesh id
 *    DHR_BACKGROUND.
 */
#ifndef DHRS_H
#define DHRS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DHR_OK = 0,
    DHR_ERR_INVALID = 1,    /* bad argument (size, range, null pointer)      */
    DHR_ERR_OOM = 2,        /* device or host allocation failed             */
    DHR_ERR_CUDA = 3,       /* a CUDA runtime call or kernel failed         */
    DHR_ERR_TIMEOUT = 4,    /* a bounded wait gave up                       */
    DHR_ERR_ADMISSION = 5,  /* serving: session refused (memory budget)     */
    DHR_ERR_STATE = 6       /* call not valid in the object's current state */
} dhr_status;

typedef enum { DHR_FP32 = 0, DHR_FP16 = 1 } dhr_precision;

#define DHR_MAX_LIGHTS 8
#define DHR_BACKGROUND 0xFFFFFFFFu

/* Pinhole camera with an orthonormal basis.  The ray of pixel (x, y) has
 * direction forward + sx right + sy up with
 *   sx = (2 (x + 0.5) / W - 1) tan_half_fov_y W / H,
 *   sy = (1 - 2 (y + 0.5) / H) tan_half_fov_y. */
typedef struct {
    float pos[3];
    float forward[3];
    float right[3];
    float up[3];
    float tan_half_fov_y;
    int32_t width;
    int32_t height;
} dhr_camera;

/* BVH builders.  Both start from 63-bit Morton codes of the triangle
 * centroids sorted on the device.  PLOC (parallel locally-ordered
 * clustering) merges mutual nearest neighbours by surface area and gives
 * a tree close to a sweep-SAH build; LBVH (Karras 2012) splits on the Morton
 * bits and builds faster. */
#define DHR_BUILD_PLOC 0u
#define DHR_BUILD_LBVH 1u

/* Triangle soup, host memory; read during dhr_create_scene only. */
typedef struct {
    const float* vertices;     /* [n_vertices][3] */
    const uint32_t* indices;   /* [n_triangles][3], each < n_vertices */
    const uint32_t* mesh_ids;  /* [n_triangles]; NULL = all 0 */
    uint32_t n_vertices;
    uint32_t n_triangles;
    uint32_t builder;          /* DHR_BUILD_PLOC (0, default) or DHR_BUILD_LBVH */
} dhr_scene_desc;

typedef struct dhr_scene dhr_scene;

typedef struct {
    uint32_t n_triangles;
    uint32_t n_nodes;          /* internal BVH nodes */
    uint32_t height;           /* longest root-to-leaf path (edges) */
    uint64_t device_bytes;     /* scene + BVH memory held on the device */
    float build_ms;            /* device time of the LBVH build */
} dhr_scene_info;

/* Visibility tracing parameters (Sections 3.1, 3.2). */
typedef struct {
    uint32_t n_lights;                      /* 1..DHR_MAX_LIGHTS directional lights */
    float light_dir[DHR_MAX_LIGHTS][3];     /* direction toward light k, any nonzero finite
                                               length: the library normalises it in double
                                               and rounds once to binary32 */
    float cone_half_angle[DHR_MAX_LIGHTS];  /* radians in [0, pi/2); 0 = hard shadow */
    float ao_radius;                        /* r > 0: a hit at t < r occludes */
    uint32_t ao_spp;                        /* N in 1..255 (8-bit count, Section 3.2) */
    uint32_t frame;                         /* hash input: frame index */
    uint32_t seed;                          /* hash input: xored into the frame */
    uint32_t primary;                       /* how the primary G-buffer is found (both give
                                               identical outputs): DHR_PRIMARY_RASTER
                                               (0, default) or DHR_PRIMARY_TRAVERSE */
} dhr_trace_params;

/* Primary visibility (Section 1 and Section 3.3: the client rasterises the
 * G-buffer).  TRAVERSE: one closest-hit ray per pixel through the BVH.
 * RASTER: every triangle is binned into the 8 x 4-pixel tiles its clipped
 * screen bounds overlap and tested against those pixels' centre rays with
 * the same watertight test, each pixel keeping the nearest hit (ties: the
 * smaller original triangle index) -- the closest hit of the pixel-centre
 * ray by construction; tiles with long lists are traversed.  Each tile's
 * list is kept in the tile's own G-buffer depth storage and the list of
 * screen-filling triangles in the mesh-id buffer, until the trace overwrites
 * them, so it needs no memory of its own (images under 1024 pixels are
 * traversed).  dhr_trace_visibility(_selective), dhr_trace_timed,
 * dhr_trace_stats and sessions honour RASTER; the server always traverses. */
#define DHR_PRIMARY_RASTER 0u
#define DHR_PRIMARY_TRAVERSE 1u

/* G-buffer (caller-owned device memory, W*H pixels).
 *  FP32: depth_normal = float4 per pixel (linear view depth, unit normal x,
 *        y, z facing the camera);
 *  FP16 (the 16-bit storage form): depth_normal = 8 bytes per pixel:
 *        binary32 linear depth, then the normal as two octahedral
 *        coordinates in 16-bit signed-normalised fixed point (q / 32767;
 *        depth stays binary32: the depth edge-stopping weight of Section 3.3
 *        compares depth differences below 16-bit resolution).
 *  mesh_id = uint32 per pixel (DHR_BACKGROUND on a miss).
 *  Both pointers must be 16-byte aligned. */
typedef struct {
    dhr_precision precision;
    int32_t width;
    int32_t height;
    void* depth_normal;
    uint32_t* mesh_id;
} dhr_gbuffer;

/* Modified SVGF parameters (Section 3.3). */
typedef struct {
    float alpha;          /* temporal blend (0, 1]; effective max(alpha, 1/n) */
    float sigma_z;        /* depth edge stopping */
    float sigma_n;        /* normal edge stopping exponent (>= 0) */
    float sigma_l;        /* luminance edge stopping */
    float eps_z;          /* > 0: keeps the depth weight's denominator away from 0 */
    float eps_l;          /* > 0: same for the luminance weight */
    uint32_t ao_spp;      /* N used to turn the AO count into [0, 1] */
    uint32_t levels;      /* a-trous iterations, 0..8 (step 2^i) */
    uint32_t fixed_alpha; /* 1: effective alpha = alpha once history exists */
    uint32_t wl_in_atrous;/* 1: luminance term in the a-trous weights */
    uint32_t shadow_light;/* which light's visibility bit (0..DHR_MAX_LIGHTS-1) is the
                             shadow channel filtered from a u8 bitmask; one SVGF state
                             per light gives every light's filtered shadow.  Unused by
                             the differentiable form (real-valued planes). */
    uint32_t kernel_width;/* a-trous footprint: 5 (or 0) = 5x5 B3-spline taps
                             (1/16, 1/4, 3/8, 1/4, 1/16) per axis; 3 = 3x3 taps (1/4, 1/2,
                             1/4) per axis, the smaller kernel of the lightweight denoiser
                             Section 3.3 proposes (with levels = 1).  The differentiable
                             form takes 5 only. */
} dhr_svgf_params;

typedef struct dhr_svgf_state dhr_svgf_state;

/* Device views of an SVGF state's buffers (owned by the state). */
typedef struct {
    void* illum;        /* float4 [W*H] temporal colour AO, shadow, variance AO, shadow (variance -1 on background) */
    void* moments;      /* current moments.  FP32: float4 [W*H] mu1 AO, mu1 shadow, mu2 AO, mu2 shadow.
                           FP16: 12-byte records [W*H]: mu1 AO, mu1 shadow as 16-bit
                           unsigned-normalised values (q / 65535), then the variances
                           mu2 - mu1^2 of AO and shadow as binary32 */
    void* color_hist;   /* float2 [W*H] colour history for the next frame (binary32 in both forms) */
    uint8_t* histlen;   /* [W*H] history length n (current) */
} dhr_svgf_buffers;

typedef struct dhr_session dhr_session;

/* ---------------------------------------------------------------------- */
/* Errors                                                                  */
/* ---------------------------------------------------------------------- */
/* Message of the last failing call on this thread ("" if none). */
const char* dhr_last_error(void);

/* ---------------------------------------------------------------------- */
/* Scene and BVH (Section 3.2: scene objects grouped hierarchically into   */
/* bounding volumes).  Builds an LBVH over 63-bit Morton codes of the      */
/* triangle centroids on the device.                                        */
/* ---------------------------------------------------------------------- */
/* Copies the soup to the device, builds the BVH on `stream`, synchronises.
 * It also builds the start cells of bounded rays: loose grids over the
 * scene box, 128 cells along its longest axis at the finest level and
 * sqrt(2) times wider cells at each coarser one.  Each cell holds up to four
 * BVH nodes under which lies every triangle that overlaps the cell.  An AO
 * ray (length r) and a shadow ray (clipped to the scene box) start their
 * traversal at those nodes of the finest cell that holds their segment's
 * box (16 bytes per cell, in the scene's device memory).
 * Errors: DHR_ERR_INVALID (null desc, index out of range, more than 2^31
 * triangles), DHR_ERR_OOM, DHR_ERR_CUDA. */
dhr_status dhr_create_scene(const dhr_scene_desc* desc, void* stream, dhr_scene** out);
void dhr_destroy_scene(dhr_scene* scene);
dhr_status dhr_scene_get_info(const dhr_scene* scene, dhr_scene_info* out);

/* ---------------------------------------------------------------------- */
/* Visibility tracing                                                      */
/* ---------------------------------------------------------------------- */
/* Primary G-buffer + shadow bitmask + AO count for every pixel of `cam`.
 *  gbuf_out: caller device buffers sized cam->width x cam->height (its
 *            width/height must match the camera; FP32 or FP16).
 *  shadow_mask_out (device, W*H bytes): bit k = light k unoccluded;
 *            0 where the jittered direction points below the surface;
 *            all light bits set on background.
 *  ao_count_out (device, W*H bytes): N_unoccluded in 0..ao_spp (Eq. 3);
 *            ao_spp on background.
 * Errors: DHR_ERR_INVALID (sizes, ao_spp outside 1..255, n_lights outside
 * 1..8, cone angle outside [0, pi/2), zero or non-finite light direction,
 * ao_radius <= 0, null pointers), DHR_ERR_CUDA. */
dhr_status dhr_trace_visibility(const dhr_scene* scene, const dhr_camera* cam,
                                const dhr_trace_params* params, dhr_gbuffer* gbuf_out,
                                uint8_t* shadow_mask_out, uint8_t* ao_count_out, void* stream);

/* Generic ray casting through the scene's BVH (device arrays of n rays).
 *  origins, dirs: float [n][3]; tmin, tmax: float [n]; a hit needs
 *  tmin < t < tmax.  any_hit = 1: occlusion query (t_out = some hit
 *  distance).  t_out: float [n] (+inf on miss); tri_out: int32 [n]
 *  (scene triangle index or -1). */
dhr_status dhr_cast_rays(const dhr_scene* scene, const float* origins, const float* dirs,
                         const float* tmin, const float* tmax, int32_t any_hit, int64_t n,
                         float* t_out, int32_t* tri_out, void* stream);

/* Converts a G-buffer between the FP32 and FP16 storage forms (device to
 * device, same size; mesh ids are copied).  Errors: DHR_ERR_INVALID for
 * size mismatch or equal precisions. */
dhr_status dhr_gbuffer_convert(const dhr_gbuffer* src, dhr_gbuffer* dst, void* stream);

/* Traversal work counters of one dhr_trace_visibility frame (runs a
 * counting variant of the trace kernel into scratch buffers it allocates;
 * synchronises `stream`).  counters (host, 9 values): rays traced
 * {primary, shadow, AO}, internal BVH nodes visited {primary, shadow, AO},
 * triangles tested {primary, shadow, AO}.  With params->primary =
 * DHR_PRIMARY_RASTER the primary figures are the rasterised ones: each
 * tile-list entry a pixel tests counts as a triangle test, and only the
 * traversed tiles visit nodes.  Errors as dhr_trace_visibility. */
dhr_status dhr_trace_stats(const dhr_scene* scene, const dhr_camera* cam,
                           const dhr_trace_params* params, uint64_t* counters, void* stream);

/* ---------------------------------------------------------------------- */
/* Selective shadow rays (Section 5: a shadow map marks the pixels whose    */
/* shadow it cannot decide -- potential penumbra, widened by the light's    */
/* angular size times the distance to the occluder -- and only those are   */
/* ray traced; the rest take the map's verdict, after Lauterbach and        */
/* Manocha).                                                                */
/* ---------------------------------------------------------------------- */
typedef struct dhr_shadow_map dhr_shadow_map;

typedef struct {
    int32_t resolution;      /* R texels per side (power of two) */
    int32_t levels;          /* log2(R) + 1: level 0 the depths, level l the
                                minimum over 2^l x 2^l texels */
    float light_dir[3];      /* unit L, toward the light */
    float axis_u[3], axis_v[3]; /* map plane axes (L, axis_u, axis_v orthonormal) */
    float u0, v0, texel;     /* texel (i, j) centre: u0 + (i + 1/2) texel along
                                axis_u, v0 + (j + 1/2) texel along axis_v */
    float plane;             /* depth of a point x is plane - L . x */
    float depth_min;         /* smallest depth in the map (+inf when empty) */
    const float* depth;      /* device, owned by the map: level 0 as [R][R]
                                (row j, column i), then levels 1.. each
                                [R >> l][R >> l], level l starting at element
                                4 (R^2 - (R >> l)^2) / 3; +inf where the texel
                                ray meets no surface */
    uint64_t bytes;          /* device bytes held */
    float build_ms;          /* device time of the build */
} dhr_shadow_map_info;

/* Renders the shadow map of one directional light over the whole scene:
 * the R x R texels cover the scene's bounds projected along the light,
 * each holding the depth of the closest surface met by a ray cast from the
 * light plane along -L through its centre (closest hit through the BVH),
 * plus the min pyramid.  light_dir: host float[3], any nonzero length
 * (normalised here).  resolution: power of two in 16..8192 (4/3 R^2 floats
 * of device memory).  Synchronises `stream`.  The map belongs to `scene` and
 * stays valid while the scene lives.  Errors: DHR_ERR_INVALID (null
 * pointer, bad resolution, zero or non-finite direction), DHR_ERR_OOM,
 * DHR_ERR_CUDA. */
dhr_status dhr_shadow_map_create(const dhr_scene* scene, const float* light_dir, int32_t resolution,
                                 void* stream, dhr_shadow_map** out);
void dhr_shadow_map_destroy(dhr_shadow_map* map);
dhr_status dhr_shadow_map_get_info(const dhr_shadow_map* map, dhr_shadow_map_info* out);

/* dhr_trace_visibility with the ray mask: for light k with maps[k] set,
 * each receiver is classified against the map --
 *   lit   (no texel of its penumbra footprint lies more than one texel
 *          size above its tangent plane): bit k = 1, no ray;
 *   umbra (every footprint texel does, or the light's cone lies wholly
 *          below the surface): bit k = 0, no ray;
 *   else  (mixed footprint, grazing cone, footprint radius + 1 > 4 texels):
 *          the cone-jittered ray of dhr_trace_visibility, same bit.
 * The footprint radius is (receiver depth - nearest possible occluder
 * depth) tan(cone half angle) / texel, the occluder bounded through the min
 * pyramid.  maps: n_lights entries (NULL entries, or maps == NULL: that
 * light is traced everywhere); each must belong to `scene` and to the
 * light direction params->light_dir[k].  ray_mask_out (device, W*H bytes,
 * may be NULL): bit k = light k's ray was called for (0 on background).
 * G-buffer and AO outputs are those of dhr_trace_visibility.  The map's
 * verdict is an approximation (it sees the scene through texel centres
 * only); a called ray is the exact method's ray.  Errors: as
 * dhr_trace_visibility, and DHR_ERR_INVALID for a map of another scene or
 * light direction. */
dhr_status dhr_trace_visibility_selective(const dhr_scene* scene, const dhr_camera* cam,
                                          const dhr_trace_params* params, const dhr_shadow_map* const* maps,
                                          dhr_gbuffer* gbuf_out, uint8_t* shadow_mask_out,
                                          uint8_t* ao_count_out, uint8_t* ray_mask_out, void* stream);

/* dhr_trace_visibility (same arguments, outputs and errors) timed on the
 * device: ms (host, 2 values) receives the time of the primary-visibility
 * pre-pass (the rasteriser's kernels; about 0 when traversed) and of the
 * trace kernel.  Synchronises `stream`. */
dhr_status dhr_trace_timed(const dhr_scene* scene, const dhr_camera* cam, const dhr_trace_params* params,
                           dhr_gbuffer* gbuf_out, uint8_t* shadow_mask_out, uint8_t* ao_count_out,
                           float* ms, void* stream);

/* Measurement helper (not a step of the method): the L2 read bandwidth, in
 * GB/s, of a kernel that reads a zero-filled buffer of `bytes` (a multiple
 * of 16 in [1 MiB, 96 MiB], so that it stays in the 126 MB L2) `passes`
 * times with L2-only loads, the best of five timed launches after one warm
 * pass.  The traversal's node and triangle fetches are held against it.
 * Allocates and frees its buffer; synchronises `stream`.  Errors:
 * DHR_ERR_INVALID (sizes), DHR_ERR_OOM, DHR_ERR_CUDA. */
dhr_status dhr_l2_read_bandwidth(int64_t bytes, int32_t passes, float* gbs, void* stream);

/* Sampling check entry: for each of n (px, py) and the given frame, seed
 * and sample index, the accepted disk point and the binary32 AO direction
 * about normals[i] (ray type 1) and the shadow direction about `light`
 * with cone half angle `cone_half_angle` (ray type 0) -- the same device
 * functions the trace kernel uses.  All arrays are device memory:
 * px, py uint32 [n]; normals float [n][3]; light float [3];
 * disk_* float [n][2]; dir_* float [n][3]. */
dhr_status dhr_sample_directions(const uint32_t* px, const uint32_t* py, int64_t n,
                                 uint32_t frame, uint32_t seed, uint32_t sample,
                                 const float* normals, const float* light, float cone_half_angle,
                                 float* disk_ao, float* dir_ao, float* disk_sh, float* dir_sh,
                                 void* stream);

/* ---------------------------------------------------------------------- */
/* Modified SVGF (Section 3.3)                                             */
/* ---------------------------------------------------------------------- */
/* History (colour, moments, history length) for one W x H stream of frames. */
dhr_status dhr_svgf_create(int32_t width, int32_t height, dhr_precision precision,
                           dhr_svgf_state** out);
void dhr_svgf_destroy(dhr_svgf_state* state);
dhr_status dhr_svgf_get_buffers(dhr_svgf_state* state, dhr_svgf_buffers* out);

/* One frame: temporal reprojection + accumulation + variance, then
 * `levels` edge-stopping a-trous iterations.
 *  cur, prev: G-buffers of this and the previous frame (prev = NULL: no
 *  history, e.g. the first frame or a reset); both in the state's
 *  precision and size.  cam, cam_prev: their cameras (cam_prev unused when
 *  prev is NULL).  shadow_mask, ao_count: device bytes [W*H] (bit 0 of the
 *  mask is filtered).  ao_out, shadow_out: device float [W*H] (filtered
 *  AO in [0, 1] and filtered light-0 visibility; 1 on background).
 * Errors: DHR_ERR_INVALID (sizes, precision mismatch, levels > 8,
 * ao_spp outside 1..255, null pointers), DHR_ERR_CUDA. */
dhr_status dhr_svgf_reconstruct(dhr_svgf_state* state, const dhr_gbuffer* cur,
                                const dhr_gbuffer* prev, const dhr_camera* cam,
                                const dhr_camera* cam_prev, const uint8_t* shadow_mask,
                                const uint8_t* ao_count, const dhr_svgf_params* params,
                                float* ao_out, float* shadow_out, void* stream);

/* ---------------------------------------------------------------------- */
/* Debug build (libdhrs_debug.so, compiled with DHR_DEBUG)                 */
/* ---------------------------------------------------------------------- */
/* In the debug build every gather index of the a-trous taps and variance
 * Gaussian, the depth slope, the reprojection taps, the short-history
 * estimate, BVH node and triangle fetches, the rasterised tile lists and
 * the adjoint's gathers and scatters is checked against its buffer; an
 * index outside the buffer is recorded and replaced by 0 (the kernel runs
 * on, nothing is read or written outside a buffer).
 * dhr_debug_status waits for the device (cudaDeviceSynchronize), returns
 * the first recorded event since the last call (0: none) and clears the
 * record: bit 63 set, bits 40..47 the site (1 a-trous tap, 2 a-trous
 * variance, 3 depth slope, 4 reprojection, 5 short-history estimate, 6 BVH
 * node, 7 triangle, 8 tile list, 10 adjoint, 11 self test, 12 start cell
 * of an AO ray), bits 0..39 the offending index.  debug_build: 1 in the
 * debug build (first_error is always 0 in the release build).  Errors: DHR_ERR_INVALID (null),
 * DHR_ERR_CUDA. */
dhr_status dhr_debug_status(uint64_t* first_error, int32_t* debug_build);
/* Debug build only: one checked read at index 5 of a one-element buffer on
 * `stream` (synchronised), which the check records (site 11) and redirects.
 * Errors: DHR_ERR_STATE in the release build, DHR_ERR_CUDA. */
dhr_status dhr_debug_selftest(void* stream);

/* ---------------------------------------------------------------------- */
/* Differentiable form of the modified SVGF (no counterpart in the paper,  */
/* which only runs the filter forward; this is its adjoint, Section 3.3)   */
/* ---------------------------------------------------------------------- */
typedef struct dhr_svgf_tape dhr_svgf_tape;

/* Schedules of the a-trous level records (dhr_svgf_tape_set_schedule).
 * RECOMPUTE (the default): the records of two frames are kept (frame f in
 * slot f mod 2); the forward leaves the last two frames' there and the
 * backward recomputes each earlier frame's L levels from that frame's
 * stored temporal output while the adjoint of the frame after it runs (L
 * more a-trous launches per earlier frame).  The tape owns two streams for
 * this: the passes run on one of the device's highest priority, the
 * recomputation on one of its lowest, so that recompute blocks take the SM
 * slots the passes leave free; the call orders both after `stream` on
 * entry and `stream` after both on return.
 * STORE: the forward keeps the records of every frame and the backward
 * recomputes nothing.  The a-trous levels are deterministic, so the
 * recomputed records equal the stored ones bit for bit. */
#define DHR_TAPE_RECOMPUTE 0
#define DHR_TAPE_STORE 1

/* Recording space for F frames of W x H (FP32): per frame the temporal
 * output, moments and history lengths (33 B/px), plus work buffers
 * (184 B/px).  The first forward with L >= 1 levels (or more levels than
 * before, or after a schedule change) adds the level records: the inputs of
 * levels 1..L-1, the weight sums of every level and the last level's
 * output, 24 L + 16 B/px for each of two frames (RECOMPUTE; one if F = 1)
 * or of the F frames (STORE), kept with the tape until it is destroyed.
 * Errors: DHR_ERR_INVALID (size outside 1..2^27 pixels, frames outside
 * 1..1024), DHR_ERR_OOM. */
dhr_status dhr_svgf_tape_create(int32_t width, int32_t height, int32_t frames, dhr_svgf_tape** out);
void dhr_svgf_tape_destroy(dhr_svgf_tape* tape);
/* Selects the record schedule (DHR_TAPE_RECOMPUTE or DHR_TAPE_STORE).  A
 * change discards the last forward's records (the next backward needs a new
 * forward).  Errors: DHR_ERR_INVALID (null tape, unknown schedule). */
dhr_status dhr_svgf_tape_set_schedule(dhr_svgf_tape* tape, int32_t schedule);
/* Bytes of level records a forward with `levels` levels holds under the
 * tape's current schedule (0 for levels == 0).  Errors: DHR_ERR_INVALID
 * (null pointer, levels outside 0..8). */
dhr_status dhr_svgf_tape_level_bytes(const dhr_svgf_tape* tape, int32_t levels, int64_t* bytes);

/* Forward over F consecutive frames starting without history, recording
 * into `tape`.  gbufs, cams: host arrays of F FP32 G-buffer descriptors and
 * cameras (the G-buffers are device memory and must stay unchanged until
 * the backward call).  sig (device, float [F][2][H][W]): noisy AO and
 * shadow signals in [0, 1] (planes).  out (device, float [F][2][H][W]):
 * filtered AO and shadow.  Keeps every frame's temporal output and the
 * level records its schedule asks for.  Errors: DHR_ERR_INVALID
 * (mismatched G-buffers or cameras, a 3x3 kernel, FP16 G-buffers, levels
 * above 8), DHR_ERR_OOM (level records). */
dhr_status dhr_svgf_seq_forward(dhr_svgf_tape* tape, const dhr_gbuffer* gbufs, const dhr_camera* cams,
                                const float* sig, const dhr_svgf_params* params, float* out,
                                void* stream);

/* Backward of the last dhr_svgf_seq_forward on `tape` (same arguments):
 * g_out (device, [F][2][H][W]) = dL/d out.  Writes g_sig (device,
 * [F][2][H][W]) = dL/d sig and g_sigma (device, float [3]) = dL/d
 * (sigma_z, sigma_n, sigma_l).  It reads the forward's records (temporal
 * outputs, and level records, recomputed from the temporal outputs under
 * DHR_TAPE_RECOMPUTE), so gbufs, cams, sig and params must be the
 * forward's; it may run more than once after one forward.  The
 * history scatter and the short-history variance estimate accumulate with
 * atomics (summation order may vary); dL/d sigma is summed per pixel in
 * binary32 over levels and frames, then over pixels in double in a fixed
 * order.  Errors: DHR_ERR_STATE without a preceding forward or with
 * another level count than the forward's. */
dhr_status dhr_svgf_seq_backward(dhr_svgf_tape* tape, const dhr_gbuffer* gbufs, const dhr_camera* cams,
                                 const float* sig, const dhr_svgf_params* params, const float* g_out,
                                 float* g_sig, float* g_sigma, void* stream);

/* Allocation-free variant of the a-trous part of dhr_svgf_reconstruct.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they filter (a frame loop that must
 * not wait on an allocator, a process whose device memory was budgeted up
 * front, a host whose allocator belongs to another framework).  It runs
 * params->levels (1..8) edge-stopping a-trous iterations over `illum` and
 * writes the last one's colours; it calls no allocator.
 *  gbuf: device G-buffer, FP32 or FP16, at most 1,048,576 pixels
 *        (W*H larger is rejected with DHR_ERR_INVALID); background pixels
 *        have depth +inf.
 *  illum (device, float4 per pixel, 16-byte aligned; DHR_ERR_INVALID
 *        otherwise): colour AO, colour shadow, variance AO, variance shadow,
 *        variance -1 on background pixels -- the layout of
 *        dhr_svgf_buffers.illum.
 *  ao_out, shadow_out: device float [W*H].
 * Scratch: two 16 MiB images in a fixed device array that every device
 * which loads the library holds until the process exits.  Its device
 * address is looked up on the first call on each device, so make that
 * first call before capturing the stream into a CUDA graph.  The address
 * stays valid while the device's context lives: after cudaDeviceReset on
 * that device, do not call this entry point again in the process.  Every call
 * uses the same array and each level overwrites every pixel it reads next,
 * so nothing has to start at zero; two calls whose kernels overlap on the
 * GPU (different streams, or different host threads) race on the array and
 * must be serialised by the caller. */
dhr_status dhr_svgf_atrous_noalloc(const dhr_gbuffer* gbuf, const float* illum,
                                   const dhr_svgf_params* params, float* ao_out,
                                   float* shadow_out, void* stream);

/* ---------------------------------------------------------------------- */
/* Lossless packing of the raw trace outputs for transport (the paper       */
/* streams compressed frames to its clients, Sections 4.3.2 and 5)          */
/* ---------------------------------------------------------------------- */
/* The bitmask (one bit per light) and the AO count are split into bit
 * planes (the n_lights bits, then ceil(log2(ao_spp + 1)) bits of the count),
 * each plane into 32x8-pixel tiles; a tile whose pixels inside the image are
 * all 0 or all 1 costs 2 bits, any other tile 2 bits + 256 bits.  Stream of
 * 32-bit little-endian words:
 *   [0] 0x56524844, [1] W, [2] H, [3] n_lights | ao_bits << 8,
 *   [4] M = number of mixed (plane, tile) pairs,
 *   ceil(P*T/16) words of 2-bit classes (pair k = plane*T + tile at bits
 *   2(k%16).. of word k/16; 0 all zero, 1 all one, 2 mixed), then 8 words per
 *   mixed pair in increasing k (word r = tile row r, bit i = pixel x0 + i;
 *   0 outside the image).  T = ceil(W/32) * ceil(H/8) tiles, row-major.
 * Size in bytes: 4 * (5 + ceil(P*T/16) + 8*M), known on the host after
 * reading word 4.  The library allocates nothing here. */

/* Largest stream for these parameters (bytes; 0 for invalid ones). */
uint64_t dhr_visibility_pack_bound(int32_t width, int32_t height, uint32_t n_lights, uint32_t ao_spp);

/* Device scratch the packer needs (bytes; 0 for invalid parameters). */
uint64_t dhr_visibility_pack_work(int32_t width, int32_t height, uint32_t n_lights, uint32_t ao_spp);

/* Packs shadow_mask, ao_count (device u8 [H][W], as written by
 * dhr_trace_visibility with these n_lights / ao_spp) into out (device,
 * dhr_visibility_pack_bound bytes), using work (device, 256-byte aligned,
 * dhr_visibility_pack_work bytes).  Asynchronous on `stream`.
 * DHR_ERR_INVALID for bad sizes or parameters, null or misaligned buffers. */
dhr_status dhr_visibility_pack(const uint8_t* shadow_mask, const uint8_t* ao_count, int32_t width,
                               int32_t height, uint32_t n_lights, uint32_t ao_spp, void* work,
                               uint32_t* out, void* stream);

/* ---------------------------------------------------------------------- */
/* Session: trace + SVGF per frame with library-owned G-buffer ping-pong   */
/* ---------------------------------------------------------------------- */
dhr_status dhr_session_create(const dhr_scene* scene, int32_t width, int32_t height,
                              dhr_precision precision, const dhr_trace_params* trace,
                              const dhr_svgf_params* svgf, dhr_session** out);
void dhr_session_destroy(dhr_session* session);

/* Trace + reconstruct one frame seen by `cam` (frame index `frame` feeds
 * the hash).  ao_out, shadow_out: device float [W*H] or NULL (results stay
 * in the session).  Asynchronous: the trace runs on a stream of the
 * session and may overlap the filtering of the previous frame; the filter
 * starts after the work queued on `stream` before this call, and `stream`
 * waits for it, so the results are complete in `stream` order.  The session
 * keeps three G-buffer / raw-output slots in rotation (and one pair of
 * internal output planes). */
dhr_status dhr_step_frame(dhr_session* session, const dhr_camera* cam, uint32_t frame,
                          float* ao_out, float* shadow_out, void* stream);

/* Same, writing the filtered AO and shadow into HOST memory (pinned memory
 * gives the fastest copy); returns after the results are in host memory. */
dhr_status dhr_step_frame_host(dhr_session* session, const dhr_camera* cam, uint32_t frame,
                               float* ao_host, float* shadow_host, void* stream);

/* Streaming host output.  Enqueues the frame (trace + reconstruct on
 * `stream`, into one of two session-owned device output buffers) and the
 * copy of its filtered AO and shadow into ao_host / shadow_host (float
 * [W*H] each) on the session's own copy stream, then returns without
 * waiting: the copy of frame N runs while frame N + 1 is traced.  The host
 * buffers must be pinned (page-locked; pageable memory makes the copy
 * synchronous) and must stay untouched until dhr_session_wait has returned
 * for the frame's ticket.  *out_ticket receives an increasing id (1, 2, ...).
 * A frame's device output buffer is reused two frames later; the library
 * orders that reuse after the earlier copy on the device.  Errors as
 * dhr_step_frame; DHR_ERR_CUDA if an enqueue fails. */
dhr_status dhr_step_frame_host_async(dhr_session* session, const dhr_camera* cam, uint32_t frame,
                                     float* ao_host, float* shadow_host, void* stream,
                                     uint64_t* out_ticket);

/* Blocks until the host copy of `ticket` has completed.  Waiting for any of
 * the last four tickets waits for that copy alone (so a caller can keep
 * several frames in flight); an older ticket may also wait for later
 * copies.  ticket 0 or a ticket not issued yet: DHR_ERR_INVALID. */
dhr_status dhr_session_wait(dhr_session* session, uint64_t ticket);

/* Device views of the session's current G-buffer and raw trace outputs. */
dhr_status dhr_session_get_frame(dhr_session* session, dhr_gbuffer* gbuf,
                                 uint8_t** shadow_mask, uint8_t** ao_count);

/* Drops the SVGF history: the next frame starts without history. */
dhr_status dhr_session_reset(dhr_session* session);

/* Checkpoint / resume of a session's history (the state a next frame
 * reads: the current G-buffer and mesh ids, the SVGF colour history, the
 * moments and history lengths written last, the previous camera).  The
 * checkpoint is a host byte image: a header (format tag, version, size,
 * precision, camera) then those buffers, (20 + 25) B/px in FP32 and
 * (12 + 21) B/px in the 16-bit form, plus the header.
 * dhr_session_checkpoint_bytes: its size (0 for a null session).
 * dhr_session_export: copies it into dst (host memory, `size` bytes at
 * least) after the session's last frame, using `stream`; returns when the
 * copy is complete.  dhr_session_import: restores a checkpoint into a
 * session of the same size and precision (waiting for the session's own
 * work first); the next dhr_step_frame then continues exactly as the
 * exported session would have, given the same parameters and cameras.
 * Errors: DHR_ERR_INVALID (null pointer, buffer too small, not a checkpoint
 * of this format, another size or precision), DHR_ERR_CUDA. */
uint64_t dhr_session_checkpoint_bytes(const dhr_session* session);
dhr_status dhr_session_export(dhr_session* session, void* dst, uint64_t size, void* stream);
dhr_status dhr_session_import(dhr_session* session, const void* src, uint64_t size, void* stream);

/* ---------------------------------------------------------------------- */
/* Serving: many thin-client sessions with continuous batching             */
/* (Section 1 and Section 4.1 describe one remote server per client and    */
/* delayed camera data; this serves many sessions from one GPU)            */
/* ---------------------------------------------------------------------- */
typedef struct dhr_server dhr_server;

typedef struct {
    uint64_t request_id;
    int32_t session;
    uint32_t frame;
    uint64_t t_arrival_ns;   /* as given to dhr_server_submit (dhr_server_now_ns clock) */
    uint64_t t_start_ns;     /* host time its batch was launched */
    uint64_t t_done_ns;      /* device completion of its batch, on the same clock */
    uint32_t batch_size;     /* requests in that batch */
    uint32_t dropped;        /* 1: replaced by a newer request of its session; never ran */
} dhr_completion;

typedef struct {
    uint64_t budget_bytes;
    uint64_t used_bytes;
    int32_t open_sessions;
    uint64_t batches;
    uint64_t frames;
    uint64_t dropped;
} dhr_server_stats;

/* Delay reprojection (Section 4.1: camera data reaches the server late;
 * Fig. 5): warps filtered AO/shadow computed for the pose cam_source (with
 * its FP32 G-buffer `source`) to the pose cam_target (with its FP32
 * G-buffer `target`).  Each target pixel takes the value of the nearest
 * valid source pixel -- the temporal step's history-tap rule (mesh id,
 * depth within 1 % + 2 depth slopes, normal cos >= 0.9), nearest = largest
 * bilinear weight among the valid taps -- else 1.  All pointers device,
 * float [H][W]. */
dhr_status dhr_delay_warp(const dhr_gbuffer* target, const dhr_camera* cam_target,
                          const dhr_gbuffer* source, const dhr_camera* cam_source,
                          const float* src_ao, const float* src_shadow, float* out_ao,
                          float* out_shadow, void* stream);

/* Monotonic host clock (ns) used for request arrival and completion times. */
uint64_t dhr_server_now_ns(void);

/* Device bytes one session of width x height holds (admission cost). */
uint64_t dhr_server_session_bytes(int32_t width, int32_t height);

/* Server over a scene with a device-memory budget for sessions; all
 * sessions share the trace and SVGF parameters (FP32 storage).  Captures
 * one CUDA graph per batch slot (2 slots, 2 streams). */
dhr_status dhr_server_create(const dhr_scene* scene, uint64_t budget_bytes,
                             const dhr_trace_params* trace, const dhr_svgf_params* svgf,
                             dhr_server** out);
void dhr_server_destroy(dhr_server* server);

/* Admits a session if its buffers fit the remaining budget (and fewer than
 * 1024 sessions are open), else DHR_ERR_ADMISSION (retry after other
 * sessions close). */
dhr_status dhr_server_open(dhr_server* server, int32_t width, int32_t height, int32_t* session_out);

/* Closes a session; its memory returns to the budget once its frame in
 * flight (if any) completes; a queued request is reported as dropped. */
dhr_status dhr_server_close(dhr_server* server, int32_t session);

/* Queues a frame request: trace + filter the pose `cam`; if cam_target is
 * not NULL, warp the result to that pose (delay reprojection: each target
 * pixel takes the nearest valid pixel of the traced pose by the history
 * validity rule, else 1).  A newer request replaces a queued one of the
 * same session (reported as dropped).  Host memory only; no GPU work. */
dhr_status dhr_server_submit(dhr_server* server, int32_t session, const dhr_camera* cam,
                             const dhr_camera* cam_target, uint32_t frame, uint64_t t_arrival_ns,
                             uint64_t request_id);

/* Caps the pixels of one batch: a batch takes sessions in request order
 * until the next would push it past max_pixels (it always takes at least
 * one).  Smaller batches finish sooner, so a request waits less behind the
 * batch in flight.  Default 2^21 pixels (about one 1920x1080 frame);
 * 0 = no cap (all ready sessions, up to 64).
 * Errors: DHR_ERR_INVALID for a null server. */
dhr_status dhr_server_set_max_batch_pixels(dhr_server* server, uint64_t max_pixels);

/* Sessions of at least min_pixels pixels rasterise their primary visibility
 * (when the server's trace params ask for DHR_PRIMARY_RASTER, the default);
 * smaller ones trace primary rays.  Both give the same G-buffer bit for bit:
 * the choice is speed only (the binning pass costs about the same at every
 * resolution; at and above 640 x 360 it is faster than primary rays).
 * Default 131,072 pixels; 0 = every session, UINT64_MAX = none.  Takes effect for batches formed afterwards (a running device loop
 * keeps the value it started with).  Errors: DHR_ERR_INVALID for a null
 * server. */
dhr_status dhr_server_set_raster_min_pixels(dhr_server* server, uint64_t min_pixels);

/* Collects finished batches, then launches one batch if a slot is free:
 * at most one queued request per session without a frame in flight.
 * *launched = number of requests launched (0 if none).  Non-blocking. */
dhr_status dhr_server_pump(dhr_server* server, int32_t* launched);

/* Returns up to `max` completed or dropped requests.  wait = 1 blocks until
 * a batch completes when nothing is ready. */
dhr_status dhr_server_poll(dhr_server* server, dhr_completion* out, int32_t max, int32_t* n_out,
                           int32_t wait);

/* Device-resident request loop.  Instead of the host forming batches
 * (dhr_server_pump), one graph launch keeps running on the device: a
 * scheduling kernel reads each session's newest request from a mailbox in
 * mapped host memory, takes one per session -- oldest arrival first, at most
 * 64 and the batch pixel cap -- builds the batch table in device memory and
 * runs the batch's stages (trace, temporal, a-trous, target G-buffer, delay
 * warp), then writes completion records (device timestamps) to a ring in
 * mapped memory; a WHILE conditional node repeats this with no host step
 * between batches.  Two such loops run side by side on two streams over the
 * same mailboxes (a session is claimed by one of them at a time, so its
 * frames stay in order), so that one batch's tail overlaps another's head.  While it runs, dhr_server_submit writes the mailbox (a
 * newer request replaces one the loop has not taken: latest wins),
 * dhr_server_poll and dhr_server_pump collect its records, and closed
 * sessions are freed once no batch can still use them.  The loop ends when
 * dhr_server_loop_stop asks it to, when no request has arrived for idle_ms
 * (1..600000), or after max_run_ms (1..3600000); each scheduling pass waits
 * for requests at most 50 us (%globaltimer), so every device-side wait is
 * bounded.  After the loop ends by a limit, dhr_server_poll(wait = 1) with
 * nothing to report and dhr_server_loop_stop return DHR_ERR_TIMEOUT.
 * Session histories carry over between the two modes.  At most 1024
 * sessions per server.  The library makes no device-wide synchronisation
 * while the loop runs (session memory is allocated and freed stream
 * ordered); a device-wide synchronisation elsewhere in the process
 * (cudaDeviceSynchronize, cudaFree, cudaFreeHost, destroying another scene
 * or server, or a framework call that makes one) waits until the loop ends,
 * which the idle limit bounds.
 * Errors: DHR_ERR_INVALID (limits out of range, loop already running),
 * DHR_ERR_CUDA. */
dhr_status dhr_server_loop_start(dhr_server* server, uint32_t idle_ms, uint32_t max_run_ms);

/* Asks the loop to end and waits for it (bounded by its limits), collects its
 * last records, hands requests it did not take back to the host's queue.
 * DHR_OK if it ended on this request (or was not running), DHR_ERR_TIMEOUT
 * if it had already ended at its idle or run-time limit. */
dhr_status dhr_server_loop_stop(dhr_server* server);

/* *running = 1 while the loop runs; *batches (may be NULL) = scheduling
 * passes done so far. */
dhr_status dhr_server_loop_status(dhr_server* server, int32_t* running, uint64_t* batches);

/* Device pointers (float [H][W]) of the session's last completed output. */
dhr_status dhr_server_output(dhr_server* server, int32_t session, float** ao, float** shadow);

/* Copies the session's last completed output into host memory (float
 * [H][W] each) on a stream of the server's own and waits for that stream
 * only, so it may be called while the device loop runs. */
dhr_status dhr_server_read_output(dhr_server* server, int32_t session, float* ao_host, float* shadow_host);

dhr_status dhr_server_get_stats(dhr_server* server, dhr_server_stats* out);

#ifdef __cplusplus
}
#endif

#endif /* DHRS_H */
