/*
 * ddgi.h -- C ABI of the GB300 probe-based irradiance field library.
 *
 * The library maintains the data structure of Majercik, Marrs, Spjut and
 * McGuire, "Scaling Probe-Based Real-Time Dynamic Global Illumination for
 * Production" (JCGT 2021): a 3D grid of probes storing octahedral irradiance
 * and distance / squared-distance moments, which answers queries of the
 * form irradiance(location, orientation) (Sec. 1) and is refreshed every
 * frame by tracing rays from the probes (Sec. 2.3).
 *
 * Conventions shared by every call
 *   - Every call returns a ddgi_status; DDGI_OK is 0.  On failure,
 *     ddgi_last_error() returns a message for the calling thread, and no
 *     output buffer has been written unless stated.
 *   - Pointers named *_dev are CUDA device pointers owned by the caller,
 *     contiguous and 16-byte aligned (the base of any cudaMalloc or torch
 *     allocation is); a misaligned one gives DDGI_ERR_INVALID_ARG before any
 *     work is enqueued.  Pointers without the suffix are host pointers; the
 *     library copies what it needs before returning.
 *   - Device work is enqueued asynchronously on the stream passed as
 *     ddgi_stream (a cudaStream_t; NULL is the legacy default stream).  No
 *     call synchronises the device unless its comment says so.
 *   - The library owns scenes and volumes (opaque handles).  A handle may be
 *     used from one host thread at a time; different handles may be used
 *     from several host threads at once, on one device or several (the
 *     library's own once-per-device kernel setup is guarded).
 *   - Vectors are float32 [n][3] arrays unless stated.  Triangles are wound
 *     counter-clockwise seen from their front side.
 *   - Stored irradiance is the cosine-weighted mean radiance M; queries
 *     return irradiance E = pi * M.
 *   - Consecutive kernels of an update and a query are programmatic
 *     dependent launches (each may be scheduled before its predecessor on
 *     the stream has finished, and waits for it on the device).  With
 *     DDGI_NO_PDL=1 in the environment (read at each launch) they are
 *     ordinary launches; the results are the same bit for bit.
 */
#ifndef DDGI_H
#define DDGI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ddgi_scene_s*   ddgi_scene;
typedef struct ddgi_volume_s*  ddgi_volume;
typedef struct ddgi_cascade_s* ddgi_cascade;
typedef void*                 ddgi_stream;   /* cudaStream_t */

typedef enum {
    DDGI_OK = 0,
    DDGI_ERR_INVALID_ARG = 1,   /* bad pointer, size, alignment or descriptor */
    DDGI_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    DDGI_ERR_OOM = 3,           /* device allocation failed */
    DDGI_ERR_TIMEOUT = 4,       /* a bounded device wait gave up */
    DDGI_ERR_NUMERIC = 5,       /* a kernel flagged a non-finite value */
    DDGI_ERR_UNSUPPORTED = 6    /* option not built in */
} ddgi_status;

/* Probe states (Sec. 6, Fig. "probestates"); dynamic-object states are not used. */
enum {
    DDGI_STATE_UNINIT = 0,          /* not yet classified */
    DDGI_STATE_OFF = 1,             /* inside static geometry: never traced (Sec. 6.1) */
    DDGI_STATE_SLEEPING = 2,        /* no surface within probe spacing (Sec. 6.2) */
    DDGI_STATE_NEWLY_VIGILANT = 3,  /* just classified; first update uses hysteresis 0 */
    DDGI_STATE_VIGILANT = 4,        /* traced and updated every frame */
    DDGI_STATE_NEWLY_AWAKE = 5,     /* sleeping probe woken by a dynamic object (Sec. 6.3);
                                       first update uses hysteresis 0 */
    DDGI_STATE_AWAKE = 6            /* traced and updated while a dynamic object is near */
};

/* Atlas storage formats (precision variants; the paper does not fix one). */
enum {
    DDGI_IRR_FP32 = 0,      /* rgb float32 + one unused float (0), 16 B / texel */
    DDGI_IRR_FP16 = 1,      /* rgb float16 + pad, 8 B / texel */
    DDGI_IRR_RGB9E5 = 2,    /* shared-exponent 9:9:9:5, 4 B / texel */
    DDGI_DIST_FP32 = 0,     /* (mean, mean square) float32, 8 B / texel */
    DDGI_DIST_FP16 = 1      /* (mean, mean square) float16, 4 B / texel */
};

/* Blend arithmetic (precision variants of the Eq. 1 contraction). */
enum {
    DDGI_BLEND_FP32 = 0,    /* SIMT float32 */
    DDGI_BLEND_TF32 = 1,    /* tensor cores, TF32 operands, FP32 accumulate */
    DDGI_BLEND_BF16 = 2,    /* tensor cores, BF16 operands, FP32 accumulate */
    DDGI_BLEND_TF32X3 = 3   /* tensor cores, FP32-accurate: weights and values split into TF32
                               high and low parts, hi.hi + hi.lo + lo.hi accumulated in FP32 */
};

const char* ddgi_last_error(void);
int32_t     ddgi_version(void);

/* Bytes per texel of an atlas storage format: which 0 irradiance
 * (DDGI_IRR_*), 1 distance (DDGI_DIST_*).  Returns 0 for an unknown
 * combination.  Host only; needs no device.  Atlas sizes are
 * probes x (n + 2)^2 texels of this size. */
int32_t     ddgi_texel_bytes(int32_t which, int32_t format);

/* ------------------------------------------------------------------ */
/* Scenes                                                              */
/* ------------------------------------------------------------------ */

/* Register a triangle scene and build its bounding volume hierarchy on the
 * host (binned SAH), then upload it.  The probe rays of Sec. 2.3 and the
 * shadow rays of hit shading are traced against it.
 *   verts            [n_verts][3] float, host
 *   tris             [n_tris][3] int32 vertex indices, host, CCW = front
 *   tri_object       [n_tris] int32 object index in [0, n_objects)
 *   object_albedo    [n_objects][3] float diffuse albedo
 *   object_flags     [n_objects] int32; bit 0: object casts shadows
 *   tri_emitter      [n_tris] int32 emitter index in [0, n_emitters) or -1
 *   emitter_radiance [n_emitters][3] float emitted radiance (front side only)
 * n_tris is at most DDGI_MAX_TRIS.  Synchronises the device once (upload).
 * Errors: INVALID_ARG on a bad count or an index out of range (nothing
 * allocated), OOM, CUDA. */
#define DDGI_MAX_TRIS ((int64_t)1 << 27)
ddgi_status ddgi_scene_create(const float* verts, int64_t n_verts,
                              const int32_t* tris, int64_t n_tris,
                              const int32_t* tri_object, int32_t n_objects,
                              const float* object_albedo, const int32_t* object_flags,
                              const int32_t* tri_emitter, int32_t n_emitters,
                              const float* emitter_radiance, ddgi_scene* out);
void ddgi_scene_destroy(ddgi_scene scene);

/* Size of the uploaded hierarchy: node count, leaf count, triangle count. */
ddgi_status ddgi_scene_info(ddgi_scene scene, int64_t* n_nodes, int64_t* n_leaves, int64_t* n_tris);

/* Host-only check of the bounding volume hierarchy that ddgi_scene_create
 * would build for these triangles (no counterpart in the paper; a
 * diagnostic that needs no GPU).  Builds the binary SAH tree and its 4-wide
 * collapse on the host and walks the 4-wide form, writing
 *   stats[0] binary nodes, [1] 4-wide nodes, [2] leaves, [3] binary depth,
 *   [4] 4-wide depth, [5] deepest stack a walk that pushes every child
 *   needs, [6] empty child slots, [7] violations: a reference out of range,
 *   a child box not inside its parent's, a triangle outside its leaf's box,
 *   or a triangle reached other than exactly once, [8] triangles.
 * verts [n_verts][3] float, tris [n_tris][3] int32 (host).  Errors:
 * INVALID_ARG as in ddgi_scene_create. */
ddgi_status ddgi_bvh_check(const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris,
                           int64_t stats[9]);

/* Closest hit of n arbitrary rays, t in (0, inf) (the traversal used by the
 * probe update, Sec. 2.3).  orig_dev, dir_dev: [n][3] float.  Outputs:
 * t_dev [n] float (+inf on a miss), tri_dev [n] int32 original triangle
 * index or -1, backface_dev [n] int32 (1 when dir . (e1 x e2) > 0) -- may be
 * NULL.  Equal distances resolve to the lower triangle index. */
ddgi_status ddgi_trace(ddgi_scene scene, const float* orig_dev, const float* dir_dev, int64_t n,
                       float* t_dev, int32_t* tri_dev, int32_t* backface_dev, ddgi_stream stream);

/* Pinhole-camera G-buffer of the scene (input generation for queries; the
 * paper rasterises it, Sec. 7.4).  Pixel (x, y), row-major, looks along
 * normalize(fwd + sx*tan(vfov/2)*aspect*right + sy*tan(vfov/2)*up) with
 * sx = (x+0.5)/w*2-1, sy = 1-(y+0.5)/h*2.  Outputs pos_dev, nrm_dev
 * [h*w][3]: first-hit position and unit geometric normal; misses give
 * zero position and zero normal. */
ddgi_status ddgi_raycast_gbuffer(ddgi_scene scene, const float cam_pos[3], const float cam_fwd[3],
                                 const float cam_up[3], float vfov_deg, int32_t width, int32_t height,
                                 float* pos_dev, float* nrm_dev, ddgi_stream stream);

/* ------------------------------------------------------------------ */
/* Lights                                                              */
/* ------------------------------------------------------------------ */

/* One directional light and a linear sky L(w) = sky_a + sky_b (w . sky_up)
 * seen by rays that miss the scene. */
typedef struct {
    float sun_dir[3];           /* unit direction the light travels */
    float sun_irradiance[3];    /* irradiance on a surface facing the sun */
    float sky_a[3];
    float sky_b[3];
    float sky_up[3];
} ddgi_lights;

/* ------------------------------------------------------------------ */
/* Volumes                                                             */
/* ------------------------------------------------------------------ */

/* Probe volume descriptor (Sec. 2.1 grid; Sec. 2.3 / 4 parameters). */
typedef struct {
    float   origin[3];          /* position of probe (0,0,0) */
    float   spacing[3];         /* probe spacing per axis (> 0) */
    int32_t counts[3];          /* probes per axis (>= 2) */
    int32_t rays_per_probe;     /* R, 1..1024 */
    int32_t irr_n;              /* interior irradiance texels per side (6 -> 8x8 tiles) */
    int32_t dist_n;             /* interior distance texels per side (14 -> 16x16 tiles) */
    float   hysteresis_irr;     /* alpha of Eq. 1 for irradiance */
    float   hysteresis_vis;     /* alpha for distance moments */
    float   gamma;              /* perceptual exponent of Sec. 4.2 (5; 1 = off) */
    float   self_shadow_bias;   /* B of the self-shadow bias equation, Sec. 4.1 */
    float   dist_cos_power;     /* exponent of the power-cosine distance weight */
    float   t_max;              /* distance clamp for misses and far hits; <0: 2*|spacing| */
    float   thr_low;            /* per-texel change thresholds of Sec. 4.3 (0.25) */
    float   thr_high;           /* (0.8) */
    float   thr_step;           /* hysteresis reduction on a large change (0.15) */
    int32_t state_machine;      /* 1: classify probes (Sec. 6.3); 0: all probes vigilant */
    int32_t irr_format;         /* DDGI_IRR_* */
    int32_t dist_format;        /* DDGI_DIST_* */
    int32_t tracking;           /* cascades: 1 = camera-tracking window (Sec. 7.2) */
    uint64_t seed;              /* seed of the per-frame random rotation */
    int32_t optimizer_iters;    /* probe position optimizer (Sec. 5): iterations run for
                                   uninitialised probes before classification, 0..16
                                   (0: off; the paper uses 5); single volumes only */
    float   offset_limit;       /* largest probe offset per axis, fraction of the spacing,
                                   [0, 0.5) (the paper leaves it open; 0.45) */
    int32_t converge_batches;   /* optional converge pass (Sec. 6.3): 0 = off; else 1..64
                                   batches of R rays traced for Newly Vigilant / Newly
                                   Awake probes, which take the encoded weighted
                                   average over all of them (hysteresis 0) and become
                                   Vigilant / Awake before the frame's update; batch b
                                   uses the rotation of (seed + 0xD1B54A32D192ED03 (b+1),
                                   frame); single volumes only */
} ddgi_volume_desc;

/* Allocate a volume: zeroed atlases (Tab. "algtable": uniform
 * initialisation to 0), all probes UNINIT (VIGILANT when state_machine is
 * 0), plus the per-frame ray buffer [P*R] of 16-byte records.  Synchronises
 * the device once.  Errors: INVALID_ARG (a field out of range, or P*R of
 * 2^31 or more: the ray lists index rays with 32-bit ints), OOM. */
ddgi_status ddgi_volume_create(const ddgi_volume_desc* desc, ddgi_volume* out);
void ddgi_volume_destroy(ddgi_volume volume);

typedef struct {
    int64_t n_probes;
    int64_t irr_tile_texels;        /* (irr_n+2)^2 */
    int64_t dist_tile_texels;       /* (dist_n+2)^2 */
    int64_t irr_bytes;              /* atlas sizes in bytes */
    int64_t dist_bytes;
    int64_t irr_texel_bytes;
    int64_t dist_texel_bytes;
    float   t_max;                  /* resolved distance clamp */
} ddgi_volume_info;
ddgi_status ddgi_volume_get_info(ddgi_volume volume, ddgi_volume_info* info);

/* Per-call update parameters. */
typedef struct {
    int64_t frame;              /* selects the random rotation of the ray pattern */
    float   irr_hyst_scale;     /* scene-event scale on hysteresis_irr (Sec. 4.3), 1 = none */
    float   vis_hyst_scale;     /* scene-event scale on hysteresis_vis */
    int32_t blend_precision;    /* DDGI_BLEND_* */
    int32_t reserved;
} ddgi_update_params;

/* One probe update frame (Sec. 2.3, Sec. 6.3 listing):
 *   1. rays w_i = R_t * sf(i, R) for i < R, R_t a uniformly random rotation
 *      drawn from (seed, frame), shared by every probe;
 *   2. probes in UNINIT are classified by a distance-only trace: OFF when
 *      more than 25% of rays hit back faces, NEWLY_VIGILANT when a front
 *      face is closer than the minimum spacing, else SLEEPING;
 *   3. rays of NEWLY_VIGILANT and VIGILANT probes are traced and shaded
 *      (sun with shadow ray, emitters, previous-frame probes; back faces
 *      give radiance 0 and 20% depth, Sec. 4.1);
 *   4. texels blend the normalised cosine / power-cosine averages with
 *      gamma encoding and per-texel hysteresis (Eq. 1, Sec. 4.2, 4.3),
 *      NEWLY_VIGILANT probes with hysteresis 0; borders are copied
 *      (Sec. 7.1); NEWLY_VIGILANT becomes VIGILANT.
 * Errors: INVALID_ARG (nothing enqueued), CUDA. */
ddgi_status ddgi_update(ddgi_volume volume, ddgi_scene scene, const ddgi_lights* lights,
                        const ddgi_update_params* params, ddgi_stream stream);

/* ddgi_update restricted to probes [probe_begin, probe_end) (a shard): only
 * those probes are classified, traced, blended and advanced; hit shading still
 * samples every probe of the volume's current atlas.  Running the shards of a
 * frame on copies of the same state and exchanging the updated ranges gives
 * the same atlas as one ddgi_update.  Errors: INVALID_ARG on a bad range. */
/* Dynamic objects (Sec. 6.3): boxes_host [n][6] float (lo x, y, z, hi x,
 * y, z), at most DDGI_MAX_DYNAMIC_BOXES; n = 0 clears them.  From the next
 * update on, each update extends every box on each side by one probe
 * spacing plus the largest self-shadow bias offset (0.75 D B), wakes the
 * Sleeping probes inside an extended box (Newly Awake: traced and blended
 * with hysteresis 0, then Awake) and puts Awake probes inside none back to
 * Sleeping.  Needs the state machine; single volumes only (not cascades).
 * Copies the boxes to the device synchronously.  Errors: INVALID_ARG. */
#define DDGI_MAX_DYNAMIC_BOXES 1024
ddgi_status ddgi_set_dynamic_boxes(ddgi_volume volume, const float* boxes_host, int32_t n);

ddgi_status ddgi_update_range(ddgi_volume volume, ddgi_scene scene, const ddgi_lights* lights,
                              const ddgi_update_params* params, int64_t probe_begin, int64_t probe_end,
                              ddgi_stream stream);

/* Irradiance query (Sec. 2.2) at n points: self-shadow bias
 * (n*0.2 + w_o*0.8)*(0.75*D)*B with w_o towards camera_pos and D the minimum
 * spacing (Sec. 4.1), then the 8-probe cage with trilinear, backface and
 * Chebyshev visibility weights, gamma decode (Sec. 4.2).
 *   pos_dev, nrm_dev [n][3] float (unit normals; a zero normal yields 0)
 *   out_dev [n][3] float irradiance E.
 * Errors: INVALID_ARG, CUDA. */
ddgi_status ddgi_query(ddgi_volume volume, const float* pos_dev, const float* nrm_dev, int64_t n,
                       const float camera_pos[3], float* out_dev, ddgi_stream stream);

/* One frame from host memory: ddgi_update (Sec. 2.3) then ddgi_query
 * (Sec. 2.2) of n points whose G-buffer lives on the host.
 *   pos_host, nrm_host [n][3] float, host; out_host [n][3] float, host.
 * The input copy runs on an internal stream while the probe update runs on
 * `stream`.  When out_host is page-locked and mapped for the device (as
 * cudaHostAlloc memory is under unified addressing) the query writes it
 * directly; otherwise the query runs in chunks whose result copies overlap
 * the next chunk's query.  Asynchronous like the other calls: out_host holds
 * the irradiance once `stream` has completed the work enqueued here; the
 * host arrays must stay valid and unchanged until then.  Page-locked host
 * memory keeps the copies asynchronous; pageable memory works but
 * serialises them.  The volume owns the device staging buffers (three of
 * n*12 bytes); a call with a larger n than any before synchronises
 * `stream` and reallocates them.  Errors: those of ddgi_update and
 * ddgi_query, INVALID_ARG on a NULL host array with n > 0. */
ddgi_status ddgi_frame_host(ddgi_volume volume, ddgi_scene scene, const ddgi_lights* lights,
                            const ddgi_update_params* params, const float* pos_host, const float* nrm_host,
                            int64_t n, const float camera_pos[3], float* out_host, ddgi_stream stream);

/* Second-order glossy lookup (Sec. 4.4): the probes reused as prefiltered
 * radiance at reflection-ray hits.  pos_dev, nrm_dev: [n][3] float hit
 * points and unit normals; dir_dev: [n][3] float unit directions the hits
 * were reached along (the reflection rays).  out_dev [n][3] float gets M,
 * the cosine-weighted mean radiance read in the mirror direction
 * r = d - 2 (d.n) n, in radiance units (ddgi_query returns pi M); the
 * self-shadow bias uses n and -d.  A zero normal gives 0.  Errors as
 * ddgi_query. */
ddgi_status ddgi_query_glossy(ddgi_volume volume, const float* pos_dev, const float* nrm_dev,
                              const float* dir_dev, int64_t n, float* out_dev, ddgi_stream stream);

/* Copy out device state (asynchronous, device to device).
 *   which 0: irradiance atlas, [P][(irr_n+2)^2] texels in irr_format
 *   which 1: distance atlas,   [P][(dist_n+2)^2] texels in dist_format
 *   which 2: probe states,     [P] uint8
 *   which 3: probe offsets,    [P][4] float (x, y, z, 0) from the grid point
 *            (Sec. 5; zero unless the position optimizer is on)
 * bytes must equal the buffer's size.  ddgi_set_buffer copies the other way
 * (restoring a checkpoint or a shard exchanged between devices). */
ddgi_status ddgi_get_buffer(ddgi_volume volume, int32_t which, void* dst_dev, size_t bytes,
                            ddgi_stream stream);
ddgi_status ddgi_set_buffer(ddgi_volume volume, int32_t which, const void* src_dev, size_t bytes,
                            ddgi_stream stream);

/* Save and restore a volume's state (no counterpart in the paper, which
 * keeps probes for the lifetime of a level; a checkpoint of the Sec. 6 states
 * and the Sec. 2.1 atlases): a versioned host blob holding a header (magic
 * "DDGIVOL1", format version 1, the volume's descriptor, the section sizes,
 * the update count, an FNV-1a checksum of the payload), then the states
 * [P] uint8, the irradiance and distance atlases and the probe offsets
 * [P][4] float exactly as stored on the device.
 * ddgi_volume_save: host_buf NULL writes the size needed to *bytes and does
 * nothing else; otherwise *bytes is the buffer's capacity (INVALID_ARG, with
 * *bytes set to the size needed, if it is too small) and becomes the bytes
 * written.  Synchronises the stream.
 * ddgi_volume_load: the blob must come from a volume whose probe counts,
 * origin, spacing, tile sizes, storage formats and gamma equal this one's
 * (the fields that fix what the stored bytes mean; hysteresis, seed, rays and
 * the other update parameters may differ) and pass its checksum; otherwise
 * INVALID_ARG (UNSUPPORTED for another format version) and the volume is
 * unchanged.  Synchronises the stream; the next update rebuilds its probe
 * lists from the loaded states.  An update after a load continues exactly
 * as it would have on the saved volume. */
ddgi_status ddgi_volume_save(ddgi_volume volume, void* host_buf, size_t* bytes, ddgi_stream stream);
ddgi_status ddgi_volume_load(ddgi_volume volume, const void* host_buf, size_t bytes, ddgi_stream stream);

/* Ray records of the last update: records_dev [P*R][4] float (r, g, b, d)
 * in active-list order, probe_ids_dev [P] int32 (the active list), and the
 * active count written to *n_active (host; synchronises the stream). */
ddgi_status ddgi_get_ray_records(ddgi_volume volume, float* records_dev, int32_t* probe_ids_dev,
                                 int64_t* n_active, ddgi_stream stream);

/* Kernel timing: when enabled, ddgi_update records CUDA events around its
 * kernels on the update stream; ddgi_read_timings returns the summed
 * milliseconds per stage since the last read (synchronises the stream):
 * ms[0] classify, ms[1] lists, ms[2] trace+shade (the three passes below
 * with their launch gaps), ms[3] blend+border+states, ms[4] frame setup,
 * ms[5] primary pass, ms[6] shadow pass, ms[7] shading pass; counts[k]
 * launches per stage. */
ddgi_status ddgi_enable_timing(ddgi_volume volume, int32_t enable);
ddgi_status ddgi_read_timings(ddgi_volume volume, float ms[8], int32_t counts[8]);

/* Work counters of the last update's trace (measurement only; the update
 * itself runs uninstrumented).  Re-traces the last update's rays of its
 * active probes with counting builds of the primary and shadow passes
 * (hit records go to a temporary buffer the call allocates and frees) and
 * writes, summed over rays: stats[0] primary rays, [1] primary 4-wide node
 * visits (four child-box tests each), [2] primary triangle tests, [3] shadow
 * rays, [4] shadow node visits, [5] shadow triangle tests, [6] front hits
 * (each shaded with one probe query).  The visiting order follows the warp
 * schedule, so repeated calls can differ slightly.  Synchronises the stream.
 * Errors: INVALID_ARG (no update yet), OOM, CUDA. */
ddgi_status ddgi_trace_stats(ddgi_volume volume, ddgi_scene scene, const ddgi_lights* lights,
                             uint64_t stats[7], ddgi_stream stream);

/* Device status word: non-finite texel detected, or a bounded wait that
 * gave up.  Reads and clears it (synchronises the stream). */
ddgi_status ddgi_poll_status(ddgi_volume volume, ddgi_stream stream);

/* ------------------------------------------------------------------ */
/* Cascades of volumes with tracking windows                           */
/* ------------------------------------------------------------------ */

/* Nested volumes at different spacings (Sec. 7.3), densest first, each
 * optionally a camera-tracking window (desc.tracking = 1, Sec. 7.2): when the
 * camera is more than one spacing from a window's centre along an axis, the
 * plane behind it leapfrogs to the front (a circular buffer of planes) and is
 * reset to zero texels and UNINIT.  Volumes must share rays_per_probe, tile
 * sizes, formats, gamma, hysteresis and thresholds; they share one ray
 * pattern per frame (the first descriptor's seed).  n in [1, 8].
 * Synchronises the device once.  Errors: INVALID_ARG, OOM. */
ddgi_status ddgi_cascade_create(const ddgi_volume_desc* descs, int32_t n, ddgi_cascade* out);
void ddgi_cascade_destroy(ddgi_cascade cascade);

typedef struct {
    int64_t frame;
    float   camera_pos[3];      /* moves tracking windows; centres their fall-off boxes */
    float   irr_hyst_scale;
    float   vis_hyst_scale;
    int32_t blend_precision;    /* DDGI_BLEND_* */
    int32_t use_graph;          /* 1: replay the frame's launches as a CUDA graph */
} ddgi_cascade_params;

/* One update frame of every volume in one batched launch sequence: the
 * windows scroll, leapfrogged planes reset, then classification, trace and
 * shade, blend and state advance run over all volumes' probes together; hit
 * shading samples the whole cascade of the previous frame (Sec. 7.3
 * weights).  Per-frame parameters go through device memory, so with
 * use_graph the sequence is captured once (per precision, lights,
 * hysteresis scales and tuning) and replayed.  Blocks the host only while an
 * earlier frame still reads the pinned parameter slot this frame reuses
 * (two slots).  Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
ddgi_status ddgi_cascade_update(ddgi_cascade cascade, ddgi_scene scene, const ddgi_lights* lights,
                                const ddgi_cascade_params* params, ddgi_stream stream);

/* Cascade query (Sec. 2.2 per volume, Sec. 7.3 blending): volumes densest
 * first, weight = product over axes of a linear fall-off over the last cell
 * of the volume's box (for tracking windows a box tightened by one cell and
 * centred on the last update's camera), accumulated until the weights reach
 * 1, normalised by the weights taken.  Same buffers as ddgi_query. */
ddgi_status ddgi_cascade_query(ddgi_cascade cascade, const float* pos_dev, const float* nrm_dev, int64_t n,
                               const float camera_pos[3], float* out_dev, ddgi_stream stream);

/* Buffers of volume `vol` as in ddgi_get_buffer, and its current window:
 * origin (world position of logical probe (0,0,0)) and the circular shift
 * (logical (i,j,k) is stored at (i+shift) mod count). */
ddgi_status ddgi_cascade_get_buffer(ddgi_cascade cascade, int32_t vol, int32_t which, void* dst_dev,
                                    size_t bytes, ddgi_stream stream);
ddgi_status ddgi_cascade_get_window(ddgi_cascade cascade, int32_t vol, double origin[3], int32_t shift[3]);

/* Ray records of the last cascade update (Sec. 2.3 per-ray radiance and
 * distance, every volume's active probes in one list): records_dev
 * [total_probes * R][4] float (r, g, b, d) in active-list order,
 * entries_dev [total_probes] int32 with entry = (volume index << 24) | the
 * probe's stored index in that volume, and the active count written to
 * *n_active (host; synchronises the stream).  INVALID_ARG before the first
 * update or on a NULL argument. */
ddgi_status ddgi_cascade_get_ray_records(ddgi_cascade cascade, float* records_dev, int32_t* entries_dev,
                                         int64_t* n_active, ddgi_stream stream);

/* Launch shapes: trace kernels' blocks per SM (1..32) and the SIMT blend's
 * probes per CTA (4, 8 or 16).  ddgi_cascade_autotune times the update under
 * each candidate and keeps the fastest, caching the choice in a JSON file at
 * cache_path (keyed by GPU name and workload); *from_cache = 1 when the cache
 * answered.  Timing advances the volumes by the frames it runs. */
ddgi_status ddgi_cascade_set_tuning(ddgi_cascade cascade, int32_t trace_blocks_per_sm,
                                    int32_t blend_probes_per_cta);
ddgi_status ddgi_cascade_get_tuning(ddgi_cascade cascade, int32_t* trace_blocks_per_sm,
                                    int32_t* blend_probes_per_cta);
ddgi_status ddgi_cascade_autotune(ddgi_cascade cascade, ddgi_scene scene, const ddgi_lights* lights,
                                  const ddgi_cascade_params* params, const char* cache_path,
                                  int32_t* from_cache, ddgi_stream stream);
ddgi_status ddgi_cascade_poll_status(ddgi_cascade cascade, ddgi_stream stream);

/* ------------------------------------------------------------------ */
/* Differentiation                                                     */
/* ------------------------------------------------------------------ */

/* Replace the scene's materials from device arrays: albedo [n_objects][3],
 * emitter radiance [n_emitters][3] (either may be NULL to keep it). */
ddgi_status ddgi_scene_set_materials(ddgi_scene scene, const float* albedo_dev, const float* emit_dev,
                                     ddgi_stream stream);

/* Differentiable forward: resets the volume to a zero atlas with every probe
 * VIGILANT, runs n_frames (1..8) updates from first_frame (hysteresis 0,
 * so frame f holds direct light plus f bounces through the probes), keeps
 * the atlas after each frame, then queries E at the points (as ddgi_query).
 * The volume needs hysteresis 0, the state machine off and FP32 atlases
 * (UNSUPPORTED otherwise). */
ddgi_status ddgi_diff_forward(ddgi_volume volume, ddgi_scene scene, const ddgi_lights* lights, int64_t first_frame,
                              int32_t n_frames, const float* pos_dev, const float* nrm_dev, int64_t n,
                              const float camera_pos[3], float* out_dev, ddgi_stream stream);

/* Reverse pass of the last ddgi_diff_forward: given dE_dev [n][3] = dLoss/dE,
 * writes dLoss/d(albedo) [n_objects][3] and dLoss/d(emitter radiance)
 * [n_emitters][3].  The query's weights, hits and distances are constants of
 * the fixed geometry; rays are traced again rather than stored; texel
 * gradients flow back through the gamma encoding, the normalised cosine
 * blend, the border copy and each frame's hit shading into the previous
 * frame's atlas. */
ddgi_status ddgi_diff_backward(ddgi_volume volume, ddgi_scene scene, const ddgi_lights* lights,
                               int64_t first_frame, int32_t n_frames, const float* pos_dev, const float* nrm_dev,
                               int64_t n, const float camera_pos[3], const float* dE_dev, float* d_albedo_dev,
                               float* d_emit_dev, ddgi_stream stream);

/* FP64 instantiation of the differentiable forward and of its reverse pass
 * (the computation of ddgi_diff_forward / ddgi_diff_backward: Sec. 2.3 hit
 * shading, Eq. 1 blend with the gamma encoding of Sec. 4.2, the Sec. 7.1
 * border copy and the Sec. 2.2 query), with every quantity that depends on
 * the parameters in double precision and the parameters given as double
 * device arrays: albedo_dev [n_objects][3], emit_dev [n_emitters][3]
 * (NULL when the scene has no emitter); out_dev [n][3] double gets E.  Hits
 * and shadow rays keep the FP32 traversal: geometry is a constant of the
 * parameters, so central differences of this forward check the reverse
 * pass's arithmetic in FP64.  The reverse pass (after a forward with the
 * same frames) takes dE_dev [n][3] double and writes d_albedo_dev
 * [n_objects][3] and d_emit_dev [n_emitters][3] double (overwritten).
 * Needs the volume of ddgi_diff_forward (hysteresis 0, state machine off,
 * FP32 atlases) without the position optimizer.  The volume keeps the
 * double atlases of every frame (allocated by the first call).  Meant for
 * checking gradients on small volumes; the FP32 calls are the fast path.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
ddgi_status ddgi_diff_forward_f64(ddgi_volume volume, ddgi_scene scene, const ddgi_lights* lights,
                                  int64_t first_frame, int32_t n_frames, const double* albedo_dev,
                                  const double* emit_dev, const float* pos_dev, const float* nrm_dev, int64_t n,
                                  const float camera_pos[3], double* out_dev, ddgi_stream stream);
ddgi_status ddgi_diff_backward_f64(ddgi_volume volume, ddgi_scene scene, const ddgi_lights* lights,
                                   int64_t first_frame, int32_t n_frames, const double* albedo_dev,
                                   const float* pos_dev, const float* nrm_dev, int64_t n, const float camera_pos[3],
                                   const double* dE_dev, double* d_albedo_dev, double* d_emit_dev,
                                   ddgi_stream stream);

/* Texel half of the adjoint (the query of Sec. 2.2 with the gamma decode of
 * Sec. 4.2, differentiated): given dE_dev [n][3] = dLoss/dE at the n points
 * of a ddgi_query with the same pos_dev, nrm_dev and camera_pos on the
 * volume's current atlases, writes g_irr_dev [P][(irr_n+2)^2][3] float =
 * dLoss/d(stored irradiance texel value), bordered tiles in the atlas's
 * texel order, for every texel (overwritten; zero where no point reads it).
 * The values are the gamma-encoded ones the atlas stores, decoded from its
 * storage format.  E depends on irradiance texels only through the bilinear
 * samples and the decode; its trilinear, backface and Chebyshev weights do
 * not involve them, so this is the exact gradient (distance texels are not
 * differentiated).  fold_borders != 0 adds each border texel's gradient to
 * the interior texel it copies (Sec. 7.1 border copy) and leaves the border
 * entries zero: the gradient with respect to the interior texels as free
 * parameters.  Float atomics: the summation order, and so the last bits,
 * can differ between calls.  Errors: INVALID_ARG, CUDA. */
ddgi_status ddgi_query_backward(ddgi_volume volume, const float* pos_dev, const float* nrm_dev, int64_t n,
                                const float camera_pos[3], const float* dE_dev, int32_t fold_borders,
                                float* g_irr_dev, ddgi_stream stream);

/* ------------------------------------------------------------------ */
/* Allocation-free update                                              */
/* ------------------------------------------------------------------ */

/* The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory while they run, such as a renderer that plans
 * all of its GPU memory at start-up and forbids cudaMalloc in its frame loop
 * (an allocation can synchronise the device and breaks the memory plan), or a
 * plug-in whose host application owns every device buffer.
 *
 * One update frame, the same steps and results as ddgi_update, for a volume
 * whose state the caller owns: states_dev [P] uint8, irr_dev and dist_dev the
 * atlases in the layout and formats of `desc` (what ddgi_get_buffer returns
 * for a volume made from the same descriptor; start from zeroed atlases and
 * states UNINIT, or VIGILANT with the state machine off).  The call allocates
 * nothing: its scratch (ray pattern, weight tables, probe lists, counters,
 * ray records) lives in fixed arrays of the library, about 17 MiB that every
 * GPU loading the library holds until the process exits.
 *
 * Limits (INVALID_ARG beyond them): at most 32768 probes, 512 rays per
 * probe and 1048576 probes x rays; irr_n <= 8, dist_n <= 16; FP32 blend only
 * (UNSUPPORTED otherwise).
 *
 * The first call on a device loads the library's module there, which is when
 * the driver sets the arrays up, and looks up their device addresses with
 * that device current.  Make that first call as a warm-up, before the
 * region in which the caller may not allocate begins and before any stream
 * capture; later calls allocate nothing.
 * Every call shares the arrays and overwrites the previous call's contents
 * (the counters it needs zeroed are cleared by each call), so calls whose
 * work overlaps on the GPU, on any streams, race: serialise them.
 * Device-side errors (a non-finite texel) are not returned by the call; they
 * accumulate in a status word read by ddgi_update_noalloc_poll_status. */
ddgi_status ddgi_update_noalloc(ddgi_scene scene, const ddgi_volume_desc* desc,
                                const ddgi_lights* lights, const ddgi_update_params* params,
                                uint8_t* states_dev, void* irr_dev, void* dist_dev,
                                ddgi_stream stream);

/* Status of the ddgi_update_noalloc calls on the current device since the
 * last poll (no counterpart in the paper): reads and clears the device status
 * word those calls share, synchronising `stream`.  NUMERIC when a blend wrote
 * a non-finite texel, TIMEOUT when a bounded device wait gave up, OK
 * otherwise (also before any call on this device).  Allocates nothing. */
ddgi_status ddgi_update_noalloc_poll_status(ddgi_stream stream);

/* Measurement helper (no counterpart in the paper): the denominator of the
 * ray traversal's cache roofline.  Enqueues on `stream` one kernel that reads
 * the `bytes` at buf_dev `passes` times with 16-byte loads that skip L1, so
 * each load is an L2 request; with bytes well below the L2 capacity and one
 * untimed call first, the data comes from L2, and bytes * passes divided by
 * the call's event-timed duration is the device's L2 read rate.
 * buf_dev: caller-owned device buffer, 16-byte aligned, bytes a positive
 * multiple of 16 (its contents are only read).  sink_dev: one caller-owned
 * device uint32, 4-byte aligned, that the kernel may increment (it keeps the
 * loads from being optimised away).  passes >= 1.  INVALID_ARG for a NULL,
 * misaligned or zero-sized argument; CUDA when the launch fails.  Allocates
 * nothing. */
ddgi_status ddgi_measure_l2_read(const void* buf_dev, size_t bytes, int32_t passes, uint32_t* sink_dev,
                                 ddgi_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* DDGI_H */
