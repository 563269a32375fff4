/*
 * FP64 CPU oracle for the probe-based irradiance field with visibility
 * (Majercik, Marrs, Spjut, McGuire, "Scaling Probe-Based Real-Time Dynamic
 * Global Illumination for Production", JCGT 2021).
 *
 * TEST INFRASTRUCTURE ONLY.  Tests, the smoke check and the benchmark's CPU
 * baseline call this library; the product path never does.  It shares no
 * code, header or table with the CUDA library.
 *
 * Everything is plain double precision, brute force and in the paper's
 * order: closest hits test every triangle, texel values are direct sums
 * over rays, the query loops over the 8 cage probes.
 */
#ifndef DDGI_ORACLE_H
#define DDGI_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    const double*  verts;           /* [n_verts][3] */
    int64_t        n_verts;
    const int32_t* tris;            /* [n_tris][3], counter-clockwise = front */
    int64_t        n_tris;
    const int32_t* tri_object;      /* [n_tris] */
    const double*  object_albedo;   /* [n_objects][3] */
    const int32_t* object_flags;    /* [n_objects], bit0 = casts shadow */
    const int32_t* tri_emitter;     /* [n_tris], -1 = none */
    const double*  emitter_radiance;/* [n_emitters][3] */
} or_scene;

typedef struct {
    double sun_dir[3];          /* unit direction the light travels */
    double sun_irradiance[3];
    double sky_a[3];
    double sky_b[3];
    double sky_up[3];
} or_lights;

typedef struct {
    double  origin[3];
    double  spacing[3];
    int64_t counts[3];
    int64_t rays;
    int64_t irr_n;              /* interior texels per side, irradiance */
    int64_t dist_n;             /* interior texels per side, distance */
    double  hyst_irr;
    double  hyst_vis;
    double  gamma;
    double  bias_B;
    double  cos_power;
    double  t_max;
    double  thr_low;            /* 0.25 */
    double  thr_high;           /* 0.8  */
    double  thr_step;           /* 0.15 */
    int64_t state_machine;      /* 0: every probe always active */
    uint64_t seed;
    int64_t shift[3];           /* tracking window: logical (i,j,k) stored at (i+shift) mod count */
    double  blend_lo[3];        /* cascade fall-off box (outermost planes, or camera-centred) */
    double  blend_hi[3];
    double* offsets;            /* [P][3] probe offsets from the grid (Sec. 5), or NULL */
    int64_t opt_iters;          /* position-optimizer iterations for uninitialised probes (0: off) */
    double  offset_limit;       /* largest offset per axis, as a fraction of the spacing */
    const double* dyn_boxes;    /* [n_dyn][6] dynamic-object boxes (lo xyz, hi xyz), Sec. 6.3 */
    int64_t n_dyn;
    int64_t converge_batches;   /* optional converge pass for new probes (Sec. 6.3), 0 = off */
} or_volume;

enum { OR_UNINIT = 0, OR_OFF = 1, OR_SLEEPING = 2, OR_NEWLY_VIGILANT = 3, OR_VIGILANT = 4,
       OR_NEWLY_AWAKE = 5, OR_AWAKE = 6 };

/* --- frame rays --- */
uint64_t or_splitmix64_next(uint64_t* state);
void or_rotation(uint64_t seed, int64_t frame, double R[9]);
void or_sf_dir(int64_t i, int64_t n, double out[3]);
void or_frame_dirs(uint64_t seed, int64_t frame, int64_t n, double* dirs);

/* --- octahedral map and tiles --- */
void or_oct_encode(const double v[3], double u[2]);
void or_oct_decode(const double u[2], double v[3]);
void or_texel_dir(int64_t i, int64_t j, int64_t n, double v[3]);
void or_border_copy(double* tile, int64_t n, int64_t C);
void or_sample_bilinear(const double* tile, int64_t n, int64_t C, const double v[3], double* out);

/* --- tracing --- */
int or_closest_hit(const or_scene* s, const double o[3], const double d[3],
                   double* t, int64_t* tri, int* backface);
void or_trace_batch(const or_scene* s, int64_t n, const double* o, const double* d,
                    double* t, int64_t* tri, int32_t* backface);
int or_any_hit_shadow(const or_scene* s, const double o[3], const double d[3]);

/* --- probes --- */
int64_t or_probe_phys(const or_volume* v, int64_t i, int64_t j, int64_t k);
void or_probe_pos_logical(const or_volume* v, int64_t i, int64_t j, int64_t k, double x[3]);
void or_optimize(const or_scene* s, const or_volume* v, int64_t frame, int64_t n, const int64_t* phys_ids);
void or_wake(const or_volume* v, int64_t n, const int64_t* phys_ids, uint8_t* states);
void or_classify(const or_scene* s, const or_volume* v, int64_t frame,
                 int64_t n, const int64_t* phys_ids, uint8_t* states,
                 int32_t* backface_count, double* dmin_front);
void or_update(const or_scene* s, const or_lights* L, const or_volume* v, int64_t frame,
               double irr_scale, double vis_scale,
               uint8_t* states, double* irr, double* dist,
               int64_t n_subset, const int64_t* subset, double* rays_out);
void or_query(const or_volume* v, const uint8_t* states, const double* irr, const double* dist,
              int64_t n, const double* pos, const double* nrm, const double camera[3],
              double* out_E, double* weights_out);
void or_query_glossy(const or_volume* v, const uint8_t* states, const double* irr, const double* dist,
                     int64_t n, const double* pos, const double* nrm, const double* dirs, double* out_M);
void or_query_cascade(int64_t n_vol, const or_volume* vols, const uint8_t* const* states,
                      const double* const* irr, const double* const* dist,
                      int64_t n, const double* pos, const double* nrm, const double camera[3],
                      double* out_E, double* vol_weights_out);

int64_t or_tracking_scroll(or_volume* v, const double camera[3], uint8_t* states, double* irr, double* dist);
void or_update_cascade(const or_scene* s, const or_lights* L, int64_t n_vol, const or_volume* vols,
                       int64_t frame, double irr_scale, double vis_scale,
                       uint8_t* const* states, double* const* irr, double* const* dist,
                       const int64_t* n_subset, const int64_t* const* subsets, double* const* rays_out);

void or_query_texel_grad(const or_volume* v, const uint8_t* states, const double* irr, const double* dist,
                         int64_t n, const double* pos, const double* nrm, const double camera[3],
                         const double* dE, int fold, double* g_irr);
void or_diff(const or_scene* s, const or_lights* L, const or_volume* v, int64_t first_frame, int64_t n_frames,
             int64_t n, const double* pos, const double* nrm, const double camera[3], const double* dE,
             double* E_out, double* d_emit, double* d_albedo, int64_t n_emitters, int64_t n_objects);

#ifdef __cplusplus
}
#endif
#endif
