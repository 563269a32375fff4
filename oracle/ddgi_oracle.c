/*
 * FP64 CPU oracle for the probe-based irradiance field with visibility
 * (Majercik et al., "Scaling Probe-Based Real-Time Dynamic Global
 * Illumination for Production", JCGT 2021).
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code
 * with the CUDA library.  Plain double precision, brute force, in the order
 * the paper states the method:
 *
 *   frame rays       Sec. 2.3 (spherical Fibonacci, random rotation per frame)
 *   classification   Sec. 6.3 and its state listing (Off / Newly Vigilant / Sleeping)
 *   trace + shade    Sec. 2.3 (deferred shading of ray hits, previous-frame
 *                    probes for multi-bounce), Sec. 4.1 (backface rule)
 *   blend            Sec. 2.3, Eq. 1 (cosine-weighted average, hysteresis),
 *                    Sec. 4.2 (gamma encoding), Sec. 4.3 (per-texel thresholds)
 *   border copy      Sec. 7.1, Fig. "probediagram" (a)
 *   query            Sec. 2.2 (8-probe cage), Sec. 4.1 (self-shadow bias Eq.),
 *                    Sec. 4.2 (gamma decode), Sec. 7.3 (volume blending)
 *
 * Readings where the paper is silent:
 *   - Eq. 1 is read as a normalised average (the text calls it an average).
 *   - stored irradiance is the cosine-weighted mean radiance M; queries
 *     return E = pi * M, hit shading uses rho * M.
 *   - spherical Fibonacci points follow Keinert et al. 2015; the per-frame
 *     rotation is Shoemake's uniform quaternion from three SplitMix64 draws.
 *   - octahedral map of Cigolle et al. 2014; bilinear filtering in software.
 *   - per-texel change = max over channels of |new - old| in the encoded domain.
 *   - backface query weight ((1 + n.w)/2)^2 + 0.2, Chebyshev one-sided bound,
 *     final weight floor 1e-6 * w_trilinear * w_backface.
 *   - gamma decode normalises by the weight sum before squaring.
 *
 * Parity is pinned for every function here by the CPU tests (closed forms,
 * exact-arithmetic brute force, invariants); see tests/test_oracle_*.py.
 */
#include "ddgi_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }
static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1]*b[2] - a[2]*b[1];
    c[1] = a[2]*b[0] - a[0]*b[2];
    c[2] = a[0]*b[1] - a[1]*b[0];
}
static void sub3(const double a[3], const double b[3], double c[3]) { c[0]=a[0]-b[0]; c[1]=a[1]-b[1]; c[2]=a[2]-b[2]; }
static double len3(const double a[3]) { return sqrt(dot3(a, a)); }
static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }
static double signnz(double x) { return x >= 0.0 ? 1.0 : -1.0; }

/* ------------------------------------------------------------------ */
/* Frame rays (Sec. 2.3): spherical Fibonacci under a random rotation  */
/* ------------------------------------------------------------------ */
static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* SplitMix64 (Steele, Lea, Flood 2014): state += golden gamma, output mix64(state). */
uint64_t or_splitmix64_next(uint64_t* state) {
    *state += 0x9E3779B97F4A7C15ULL;
    return mix64(*state);
}

/* Uniform random rotation for (seed, frame): Shoemake's quaternion method
 * ("Uniform random rotations", Graphics Gems III) from three 53-bit uniforms. */
void or_rotation(uint64_t seed, int64_t frame, double R[9]) {
    uint64_t st = mix64(seed ^ mix64((uint64_t)frame + 0x9E3779B97F4A7C15ULL));
    double u[3];
    for (int k = 0; k < 3; ++k)
        u[k] = (double)(or_splitmix64_next(&st) >> 11) * (1.0 / 9007199254740992.0);
    double r1 = sqrt(1.0 - u[0]), r2 = sqrt(u[0]);
    double t1 = 2.0 * M_PI * u[1], t2 = 2.0 * M_PI * u[2];
    double x = r1 * sin(t1), y = r1 * cos(t1), z = r2 * sin(t2), w = r2 * cos(t2);
    R[0] = 1 - 2*(y*y + z*z); R[1] = 2*(x*y - z*w);     R[2] = 2*(x*z + y*w);
    R[3] = 2*(x*y + z*w);     R[4] = 1 - 2*(x*x + z*z); R[5] = 2*(y*z - x*w);
    R[6] = 2*(x*z - y*w);     R[7] = 2*(y*z + x*w);     R[8] = 1 - 2*(x*x + y*y);
}

/* Spherical Fibonacci point i of n (Keinert et al. 2015):
 * z = 1 - (2i+1)/n, azimuth = 2 pi frac(i / golden ratio). */
void or_sf_dir(int64_t i, int64_t n, double out[3]) {
    const double inv_phi = 0.61803398874989484820;  /* 1/golden = golden - 1 */
    double a = (double)i * inv_phi;
    double phi = 2.0 * M_PI * (a - floor(a));
    double z = 1.0 - (2.0 * (double)i + 1.0) / (double)n;
    double r = sqrt(fmax(0.0, 1.0 - z * z));
    out[0] = cos(phi) * r;
    out[1] = sin(phi) * r;
    out[2] = z;
}

void or_frame_dirs(uint64_t seed, int64_t frame, int64_t n, double* dirs) {
    double R[9];
    or_rotation(seed, frame, R);
    for (int64_t i = 0; i < n; ++i) {
        double s[3];
        or_sf_dir(i, n, s);
        for (int a = 0; a < 3; ++a)
            dirs[3*i + a] = R[3*a+0]*s[0] + R[3*a+1]*s[1] + R[3*a+2]*s[2];
    }
}

/* ------------------------------------------------------------------ */
/* Octahedral map (Cigolle et al. 2014, cited in Sec. 3)               */
/* ------------------------------------------------------------------ */
void or_oct_encode(const double v[3], double u[2]) {
    double l1 = fabs(v[0]) + fabs(v[1]) + fabs(v[2]);
    double px = v[0] / l1, py = v[1] / l1;
    if (v[2] < 0.0) {
        double qx = (1.0 - fabs(py)) * signnz(px);
        double qy = (1.0 - fabs(px)) * signnz(py);
        px = qx; py = qy;
    }
    u[0] = px; u[1] = py;
}

void or_oct_decode(const double u[2], double v[3]) {
    double x = u[0], y = u[1], z = 1.0 - fabs(u[0]) - fabs(u[1]);
    if (z < 0.0) {
        double nx = (1.0 - fabs(u[1])) * signnz(u[0]);
        double ny = (1.0 - fabs(u[0])) * signnz(u[1]);
        x = nx; y = ny;
    }
    double l = sqrt(x*x + y*y + z*z);
    v[0] = x / l; v[1] = y / l; v[2] = z / l;
}

/* Direction of interior texel (i = column, j = row) of an n x n probe. */
void or_texel_dir(int64_t i, int64_t j, int64_t n, double v[3]) {
    double u[2] = { 2.0 * ((double)i + 0.5) / (double)n - 1.0,
                    2.0 * ((double)j + 0.5) / (double)n - 1.0 };
    or_oct_decode(u, v);
}

/* Bordered tile: (n+2) x (n+2) texels, row-major by row y, C channels;
 * interior texel (i, j) sits at column i+1, row j+1. */
#define TILE(t, N, C, x, y) ((t) + ((int64_t)(y) * (N) + (x)) * (C))

/* Border copy (Sec. 7.1, Fig. probediagram a): each border texel takes the
 * interior texel that is its neighbour across the octahedral seam, i.e. the
 * edge row/column mirrored, and each corner the diagonally opposite corner. */
void or_border_copy(double* tile, int64_t n, int64_t C) {
    int64_t N = n + 2;
    for (int64_t k = 1; k <= n; ++k) {
        for (int64_t c = 0; c < C; ++c) {
            TILE(tile, N, C, 0,     k)[c] = TILE(tile, N, C, 1, n + 1 - k)[c];   /* left   */
            TILE(tile, N, C, n + 1, k)[c] = TILE(tile, N, C, n, n + 1 - k)[c];   /* right  */
            TILE(tile, N, C, k, 0    )[c] = TILE(tile, N, C, n + 1 - k, 1)[c];   /* top    */
            TILE(tile, N, C, k, n + 1)[c] = TILE(tile, N, C, n + 1 - k, n)[c];   /* bottom */
        }
    }
    for (int64_t c = 0; c < C; ++c) {
        TILE(tile, N, C, 0,     0    )[c] = TILE(tile, N, C, n, n)[c];
        TILE(tile, N, C, n + 1, 0    )[c] = TILE(tile, N, C, 1, n)[c];
        TILE(tile, N, C, 0,     n + 1)[c] = TILE(tile, N, C, n, 1)[c];
        TILE(tile, N, C, n + 1, n + 1)[c] = TILE(tile, N, C, 1, 1)[c];
    }
}

/* Bilinear sample of a bordered tile in direction v: the octahedral
 * coordinate maps [-1,1] onto the interior span [1, n+1] in texel units. */
void or_sample_bilinear(const double* tile, int64_t n, int64_t C, const double v[3], double* out) {
    int64_t N = n + 2;
    double u[2];
    or_oct_encode(v, u);
    double sx = 1.0 + (u[0] + 1.0) * 0.5 * (double)n - 0.5;
    double sy = 1.0 + (u[1] + 1.0) * 0.5 * (double)n - 0.5;
    double fx = floor(sx), fy = floor(sy);
    int64_t x0 = (int64_t)fx, y0 = (int64_t)fy;
    if (x0 > N - 2) x0 = N - 2;
    if (y0 > N - 2) y0 = N - 2;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    double tx = sx - (double)x0, ty = sy - (double)y0;
    for (int64_t c = 0; c < C; ++c) {
        out[c] = (1 - tx) * (1 - ty) * TILE(tile, N, C, x0,     y0    )[c]
               +      tx  * (1 - ty) * TILE(tile, N, C, x0 + 1, y0    )[c]
               + (1 - tx) *      ty  * TILE(tile, N, C, x0,     y0 + 1)[c]
               +      tx  *      ty  * TILE(tile, N, C, x0 + 1, y0 + 1)[c];
    }
}

/* ------------------------------------------------------------------ */
/* Tracing: brute force over every triangle (Moller & Trumbore 1997)   */
/* ------------------------------------------------------------------ */
static int tri_intersect(const or_scene* s, int64_t k, const double o[3], const double d[3],
                         double* t_out, int* backface) {
    const double* v0 = s->verts + 3 * (int64_t)s->tris[3*k + 0];
    const double* v1 = s->verts + 3 * (int64_t)s->tris[3*k + 1];
    const double* v2 = s->verts + 3 * (int64_t)s->tris[3*k + 2];
    double e1[3], e2[3], p[3], q[3], sv[3];
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(d, e2, p);
    double det = dot3(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    sub3(o, v0, sv);
    double u = dot3(sv, p) * inv;
    if (u < 0.0 || u > 1.0) return 0;
    cross3(sv, e1, q);
    double v = dot3(d, q) * inv;
    if (v < 0.0 || u + v > 1.0) return 0;
    double t = dot3(e2, q) * inv;
    if (!(t > 0.0)) return 0;
    double ng[3];
    cross3(e1, e2, ng);
    *t_out = t;
    *backface = dot3(d, ng) > 0.0;
    return 1;
}

/* Closest hit over t in (0, inf); equal t keeps the lower triangle index. */
int or_closest_hit(const or_scene* s, const double o[3], const double d[3],
                   double* t, int64_t* tri, int* backface) {
    double best = INFINITY;
    int64_t bi = -1;
    int bb = 0;
    for (int64_t k = 0; k < s->n_tris; ++k) {
        double tk;
        int bk;
        if (tri_intersect(s, k, o, d, &tk, &bk) && tk < best) {
            best = tk; bi = k; bb = bk;
        }
    }
    *t = best; *tri = bi; *backface = bb;
    return bi >= 0;
}

void or_trace_batch(const or_scene* s, int64_t n, const double* o, const double* d,
                    double* t, int64_t* tri, int32_t* backface) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < n; ++r) {
        int bf;
        if (!or_closest_hit(s, o + 3*r, d + 3*r, t + r, tri + r, &bf)) bf = 0;
        backface[r] = bf;
    }
}

/* Any hit, t in (0, inf), among triangles of shadow-casting objects. */
int or_any_hit_shadow(const or_scene* s, const double o[3], const double d[3]) {
    for (int64_t k = 0; k < s->n_tris; ++k) {
        if (!(s->object_flags[s->tri_object[k]] & 1)) continue;
        double tk;
        int bk;
        if (tri_intersect(s, k, o, d, &tk, &bk)) return 1;
    }
    return 0;
}

static void tri_unit_normal(const or_scene* s, int64_t k, double n[3]) {
    const double* v0 = s->verts + 3 * (int64_t)s->tris[3*k + 0];
    const double* v1 = s->verts + 3 * (int64_t)s->tris[3*k + 1];
    const double* v2 = s->verts + 3 * (int64_t)s->tris[3*k + 2];
    double e1[3], e2[3];
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(e1, e2, n);
    double l = len3(n);
    n[0] /= l; n[1] /= l; n[2] /= l;
}

/* ------------------------------------------------------------------ */
/* Probe grid (Sec. 2.1) and tracking-window indexing (Sec. 7.2)        */
/* ------------------------------------------------------------------ */
static int64_t pmod(int64_t a, int64_t m) { int64_t r = a % m; return r < 0 ? r + m : r; }

int64_t or_probe_phys(const or_volume* v, int64_t i, int64_t j, int64_t k) {
    int64_t a = pmod(i + v->shift[0], v->counts[0]);
    int64_t b = pmod(j + v->shift[1], v->counts[1]);
    int64_t c = pmod(k + v->shift[2], v->counts[2]);
    return a + v->counts[0] * (b + v->counts[1] * c);
}

static void probe_logical(const or_volume* v, int64_t phys, int64_t ijk[3]) {
    int64_t a = phys % v->counts[0];
    int64_t b = (phys / v->counts[0]) % v->counts[1];
    int64_t c = phys / (v->counts[0] * v->counts[1]);
    ijk[0] = pmod(a - v->shift[0], v->counts[0]);
    ijk[1] = pmod(b - v->shift[1], v->counts[1]);
    ijk[2] = pmod(c - v->shift[2], v->counts[2]);
}

void or_probe_pos_logical(const or_volume* v, int64_t i, int64_t j, int64_t k, double x[3]) {
    x[0] = v->origin[0] + (double)i * v->spacing[0];
    x[1] = v->origin[1] + (double)j * v->spacing[1];
    x[2] = v->origin[2] + (double)k * v->spacing[2];
}

/* World position of a probe: its grid point plus its offset (Sec. 5). */
static void probe_pos_phys(const or_volume* v, int64_t phys, double x[3]) {
    int64_t ijk[3];
    probe_logical(v, phys, ijk);
    or_probe_pos_logical(v, ijk[0], ijk[1], ijk[2], x);
    if (v->offsets)
        for (int a = 0; a < 3; ++a) x[a] += v->offsets[3 * phys + a];
}

static double min_spacing(const or_volume* v) {
    return fmin(v->spacing[0], fmin(v->spacing[1], v->spacing[2]));
}

/* traced and updated: vigilant probes, and sleeping probes woken by a dynamic object */
static int is_active(uint8_t s) {
    return s == OR_NEWLY_VIGILANT || s == OR_VIGILANT || s == OR_NEWLY_AWAKE || s == OR_AWAKE;
}
static int is_newly(uint8_t s) { return s == OR_NEWLY_VIGILANT || s == OR_NEWLY_AWAKE; }
static uint8_t advanced(uint8_t s) {
    return s == OR_NEWLY_VIGILANT ? OR_VIGILANT : (s == OR_NEWLY_AWAKE ? OR_AWAKE : s);
}

static int64_t irr_tile_size(const or_volume* v) { return (v->irr_n + 2) * (v->irr_n + 2) * 3; }
static int64_t dist_tile_size(const or_volume* v) { return (v->dist_n + 2) * (v->dist_n + 2) * 2; }

/* ------------------------------------------------------------------ */
/* Probe position optimizer (Sec. 5 and its listing)                   */
/* ------------------------------------------------------------------ */
/* Iteration k traces the R rays of frame (frame + k) from each probe's
 * current position, then moves its offset:
 *   more than 25% backfaces: along the vector to the closest backface
 *     (t * w) by the largest scale that keeps every component of the offset
 *     within +-limit (less 1 mm); only if that scale exceeds 1, i.e. the move
 *     goes through the backface;
 *   otherwise, unless the farthest front face lies within 60 degrees of the
 *     closest one (one visible surface): min(0.2, t) along the direction of
 *     the farthest front face, each component clamped to +-limit.
 * Closest picks the smallest t (ties: smaller ray index), farthest the
 * largest t (ties: larger ray index); misses are neither. */
void or_optimize(const or_scene* s, const or_volume* v, int64_t frame, int64_t n, const int64_t* phys_ids) {
    int64_t R = v->rays;
    if (!v->offsets || v->opt_iters <= 0 || n <= 0) return;
    double* dirs = (double*)malloc(sizeof(double) * 3 * (size_t)R);
    double lim[3];
    for (int a = 0; a < 3; ++a) lim[a] = v->offset_limit * v->spacing[a];
    for (int64_t k = 0; k < v->opt_iters; ++k) {
        or_frame_dirs(v->seed, frame + k, R, dirs);
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t q = 0; q < n; ++q) {
            int64_t p = phys_ids[q];
            double x[3];
            probe_pos_phys(v, p, x);
            int64_t bf = 0, ib = -1, icf = -1, iff = -1;
            double tb = INFINITY, tcf = INFINITY, tff = -INFINITY;
            for (int64_t i = 0; i < R; ++i) {
                double t;
                int64_t tri;
                int back;
                if (!or_closest_hit(s, x, dirs + 3*i, &t, &tri, &back)) continue;
                if (back) {
                    bf++;
                    if (t < tb) { tb = t; ib = i; }
                } else {
                    if (t < tcf) { tcf = t; icf = i; }
                    if (t >= tff) { tff = t; iff = i; }
                }
            }
            double* cur = v->offsets + 3 * p;
            if (4 * bf > R) {
                double vec[3], comb[3];
                for (int a = 0; a < 3; ++a) {
                    vec[a] = tb * dirs[3*ib + a];
                    double pos = (lim[a] - cur[a]) / vec[a];
                    double neg = (-lim[a] - cur[a]) / vec[a];
                    comb[a] = fmax(pos, neg);
                }
                double scale = fmin(fmin(comb[0], comb[1]), comb[2]) - 1e-3;
                if (scale > 1.0)
                    for (int a = 0; a < 3; ++a) cur[a] += vec[a] * scale;
            } else if (iff >= 0 && icf >= 0 && !(dot3(dirs + 3*iff, dirs + 3*icf) > 0.5)) {
                double step = fmin(0.2, tff);
                for (int a = 0; a < 3; ++a) cur[a] = clampd(cur[a] + step * dirs[3*iff + a], -lim[a], lim[a]);
            }
        }
    }
    free(dirs);
}

/* ------------------------------------------------------------------ */
/* Dynamic objects (Sec. 6.3, second step of the initialisation listing) */
/* ------------------------------------------------------------------ */
/* Each dynamic object's box is extended on every side by one grid cell
 * plus the largest self-shadow bias offset (0.75 D B); a SLEEPING probe
 * inside an extended box becomes NEWLY_AWAKE, an AWAKE probe inside none
 * goes back to SLEEPING.  Other states are untouched. */
void or_wake(const or_volume* v, int64_t n, const int64_t* phys_ids, uint8_t* states) {
    double ext[3];
    double bias = 0.75 * min_spacing(v) * v->bias_B;
    for (int a = 0; a < 3; ++a) ext[a] = v->spacing[a] + bias;
    for (int64_t q = 0; q < n; ++q) {
        int64_t p = phys_ids[q];
        uint8_t s = states[p];
        if (s != OR_SLEEPING && s != OR_AWAKE) continue;
        double x[3];
        probe_pos_phys(v, p, x);
        int inside = 0;
        for (int64_t b = 0; b < v->n_dyn && !inside; ++b) {
            const double* bx = v->dyn_boxes + 6 * b;
            inside = 1;
            for (int a = 0; a < 3; ++a)
                if (x[a] < bx[a] - ext[a] || x[a] > bx[3 + a] + ext[a]) inside = 0;
        }
        if (s == OR_SLEEPING && inside) states[p] = OR_NEWLY_AWAKE;
        else if (s == OR_AWAKE && !inside) states[p] = OR_SLEEPING;
    }
}

/* ------------------------------------------------------------------ */
/* Classification (Sec. 6.3 and its state listing)                     */
/* ------------------------------------------------------------------ */
void or_classify(const or_scene* s, const or_volume* v, int64_t frame,
                 int64_t n, const int64_t* phys_ids, uint8_t* states,
                 int32_t* backface_count, double* dmin_front) {
    int64_t R = v->rays;
    double* dirs = (double*)malloc(sizeof(double) * 3 * (size_t)R);
    or_frame_dirs(v->seed, frame, R, dirs);
    double D = min_spacing(v);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < n; ++q) {
        int64_t p = phys_ids[q];
        double x[3];
        probe_pos_phys(v, p, x);
        int64_t bf = 0;
        double dmin = INFINITY;
        for (int64_t i = 0; i < R; ++i) {
            double t;
            int64_t tri;
            int back;
            if (or_closest_hit(s, x, dirs + 3*i, &t, &tri, &back)) {
                if (back) bf++;
                else if (t < dmin) dmin = t;
            }
        }
        uint8_t st;
        if (4 * bf > R) st = OR_OFF;                 /* more than 25% backfaces: in a wall */
        else if (dmin < D) st = OR_NEWLY_VIGILANT;   /* a surface within probe spacing */
        else st = OR_SLEEPING;
        states[p] = st;
        if (backface_count) backface_count[q] = (int32_t)bf;
        if (dmin_front) dmin_front[q] = dmin;
    }
    free(dirs);
}

/* ------------------------------------------------------------------ */
/* Query (Sec. 2.2, self-shadow bias Eq. of Sec. 4.1, decode Sec. 4.2)  */
/* Returns the cosine-weighted mean radiance M (E = pi * M).           */
/* ------------------------------------------------------------------ */
/* `look` is the direction the irradiance tiles are read in: the normal n for
 * the irradiance query, the mirror direction for a second-order glossy
 * lookup (Sec. 4.4); bias and backface weights always use n. */
static void query_M_look(const or_volume* v, const uint8_t* st, const double* irr, const double* dist,
                         const double x[3], const double n[3], const double wo[3], const double look[3],
                         double M[3], double* wout) {
    double D = min_spacing(v);
    double xb[3];
    for (int a = 0; a < 3; ++a)
        xb[a] = x[a] + (0.2 * n[a] + 0.8 * wo[a]) * (0.75 * D) * v->bias_B;
    int64_t base[3];
    double fr[3];
    for (int a = 0; a < 3; ++a) {
        double g = (xb[a] - v->origin[a]) / v->spacing[a];
        double b = floor(g);
        double bmax = (double)(v->counts[a] - 2);
        if (b > bmax) b = bmax;
        if (b < 0.0) b = 0.0;
        base[a] = (int64_t)b;
        fr[a] = clampd(g - b, 0.0, 1.0);
    }
    double sumw = 0.0, acc[3] = {0.0, 0.0, 0.0};
    int64_t tsi = irr_tile_size(v), tsd = dist_tile_size(v);
    for (int c = 0; c < 8; ++c) {
        int o[3] = { c & 1, (c >> 1) & 1, (c >> 2) & 1 };
        if (wout) wout[c] = 0.0;
        int64_t p = or_probe_phys(v, base[0] + o[0], base[1] + o[1], base[2] + o[2]);
        if (!is_active(st[p])) continue;
        double xp[3];
        or_probe_pos_logical(v, base[0] + o[0], base[1] + o[1], base[2] + o[2], xp);
        if (v->offsets)   /* the probe's own (moved) position; the cage stays on the grid */
            for (int a = 0; a < 3; ++a) xp[a] += v->offsets[3 * p + a];
        /* trilinear weight */
        double wt = 1.0;
        for (int a = 0; a < 3; ++a) wt *= o[a] ? fr[a] : 1.0 - fr[a];
        /* backface weight: is the probe behind the point relative to n? */
        double dp[3];
        sub3(xp, x, dp);
        double ldp = len3(dp);
        double cw = ldp > 0.0 ? dot3(n, dp) / ldp : 1.0;
        double wb = ((1.0 + cw) * 0.5) * ((1.0 + cw) * 0.5) + 0.2;
        /* visibility: Chebyshev test of the biased point against the distance moments */
        double pv[3];
        sub3(xb, xp, pv);
        double r = len3(pv);
        double wc = 1.0;
        if (r > 0.0) {
            double dir[3] = { pv[0] / r, pv[1] / r, pv[2] / r };
            double mom[2];
            or_sample_bilinear(dist + p * tsd, v->dist_n, 2, dir, mom);
            if (r > mom[0]) {
                double var = fmax(mom[1] - mom[0] * mom[0], 0.0);
                double dr = r - mom[0];
                wc = var / (var + dr * dr);
            }
        }
        double w = wt * wb * fmax(wc, 1e-6);
        if (wout) wout[c] = w;
        /* irradiance in the lookup direction, gamma decoded to a gamma-2 curve */
        double e[3];
        or_sample_bilinear(irr + p * tsi, v->irr_n, 3, look, e);
        for (int k = 0; k < 3; ++k) acc[k] += w * pow(fmax(e[k], 0.0), 0.5 * v->gamma);
        sumw += w;
    }
    for (int k = 0; k < 3; ++k) {
        double a = sumw > 0.0 ? acc[k] / sumw : 0.0;
        M[k] = a * a;
    }
}

static void query_M(const or_volume* v, const uint8_t* st, const double* irr, const double* dist,
                    const double x[3], const double n[3], const double wo[3],
                    double M[3], double* wout) {
    query_M_look(v, st, irr, dist, x, n, wo, n, M, wout);
}

/* Second-order glossy (Sec. 4.4): at a reflection-ray hit x with normal n,
 * reached along the unit direction d, the probes are read in the mirror
 * direction r = d - 2 (d.n) n and the result is the prefiltered radiance M
 * (not pi M); the view direction of the self-shadow bias is -d. */
void or_query_glossy(const or_volume* v, const uint8_t* states, const double* irr, const double* dist,
                     int64_t n, const double* pos, const double* nrm, const double* dirs, double* out_M) {
    #pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) {
        const double* x = pos + 3*q;
        const double* nn = nrm + 3*q;
        const double* d = dirs + 3*q;
        if (nn[0] == 0.0 && nn[1] == 0.0 && nn[2] == 0.0) {
            for (int k = 0; k < 3; ++k) out_M[3*q + k] = 0.0;
            continue;
        }
        double dn = dot3(d, nn);
        double r[3] = { d[0] - 2.0 * dn * nn[0], d[1] - 2.0 * dn * nn[1], d[2] - 2.0 * dn * nn[2] };
        double lr = len3(r);
        if (lr > 0.0) { r[0] /= lr; r[1] /= lr; r[2] /= lr; }
        double wo[3] = { -d[0], -d[1], -d[2] };
        query_M_look(v, states, irr, dist, x, nn, wo, r, out_M + 3*q, NULL);
    }
}

void or_query(const or_volume* v, const uint8_t* states, const double* irr, const double* dist,
              int64_t n, const double* pos, const double* nrm, const double camera[3],
              double* out_E, double* weights_out) {
    #pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) {
        const double* x = pos + 3*q;
        const double* nn = nrm + 3*q;
        if (nn[0] == 0.0 && nn[1] == 0.0 && nn[2] == 0.0) {
            /* no surface (a background pixel): no irradiance */
            for (int k = 0; k < 3; ++k) out_E[3*q + k] = 0.0;
            if (weights_out) for (int c = 0; c < 8; ++c) weights_out[8*q + c] = 0.0;
            continue;
        }
        double wo[3];
        sub3(camera, x, wo);
        double l = len3(wo);
        if (l < 1e-6) { wo[0] = nn[0]; wo[1] = nn[1]; wo[2] = nn[2]; }
        else { wo[0] /= l; wo[1] /= l; wo[2] /= l; }
        double M[3];
        query_M(v, states, irr, dist, x, nn, wo, M, weights_out ? weights_out + 8*q : NULL);
        for (int k = 0; k < 3; ++k) out_E[3*q + k] = M_PI * M[k];
    }
}

/* Volume blending (Sec. 7.3): densest volume first, linear fall-off over the
 * last cell of each axis, stop once the accumulated weight reaches 1. */
static double volume_weight(const or_volume* v, const double x[3]) {
    double w = 1.0;
    for (int a = 0; a < 3; ++a) {
        double m = fmin(x[a] - v->blend_lo[a], v->blend_hi[a] - x[a]) / v->spacing[a];
        w *= clampd(m, 0.0, 1.0);
    }
    return w;
}

/* Cascade value M at x (Sec. 7.3): volumes densest first, each weighted by its
 * fall-off box, accumulation stops once the weights reach 1; the weighted
 * values are normalised by the weight sum (0 when no volume covers x). */
static void cascade_M(int64_t n_vol, const or_volume* vols, const uint8_t* const* states,
                      const double* const* irr, const double* const* dist,
                      const double x[3], const double n[3], const double wo[3], double M[3],
                      double* vol_weights) {
    double sum = 0.0, acc[3] = {0.0, 0.0, 0.0};
    for (int64_t k = 0; k < n_vol; ++k) {
        double vw = volume_weight(&vols[k], x);
        double take = fmin(vw, 1.0 - sum);
        if (vol_weights) vol_weights[k] = take > 0.0 ? take : 0.0;
        if (take <= 0.0) continue;
        double Mk[3];
        query_M(&vols[k], states[k], irr[k], dist[k], x, n, wo, Mk, NULL);
        for (int c = 0; c < 3; ++c) acc[c] += take * Mk[c];
        sum += take;
        if (sum >= 1.0) {
            for (int64_t j = k + 1; j < n_vol; ++j)
                if (vol_weights) vol_weights[j] = 0.0;
            break;
        }
    }
    for (int c = 0; c < 3; ++c) M[c] = sum > 0.0 ? acc[c] / sum : 0.0;
}

void or_query_cascade(int64_t n_vol, const or_volume* vols, const uint8_t* const* states,
                      const double* const* irr, const double* const* dist,
                      int64_t n, const double* pos, const double* nrm, const double camera[3],
                      double* out_E, double* vol_weights_out) {
    #pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) {
        const double* x = pos + 3*q;
        const double* nn = nrm + 3*q;
        double wo[3];
        sub3(camera, x, wo);
        double l = len3(wo);
        if (l < 1e-6) { wo[0] = nn[0]; wo[1] = nn[1]; wo[2] = nn[2]; }
        else { wo[0] /= l; wo[1] /= l; wo[2] /= l; }
        if (nn[0] == 0.0 && nn[1] == 0.0 && nn[2] == 0.0) {
            for (int c = 0; c < 3; ++c) out_E[3*q + c] = 0.0;
            if (vol_weights_out) for (int64_t k = 0; k < n_vol; ++k) vol_weights_out[q * n_vol + k] = 0.0;
            continue;
        }
        double M[3];
        cascade_M(n_vol, vols, states, irr, dist, x, nn, wo, M, vol_weights_out ? vol_weights_out + q * n_vol : NULL);
        for (int c = 0; c < 3; ++c) out_E[3*q + c] = M_PI * M[c];
    }
}

/* ------------------------------------------------------------------ */
/* Shading one probe ray (Sec. 2.3, Sec. 4.1 backface rule)             */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t n_vol;
    const or_volume* vols;
    const uint8_t* const* states;
    const double* const* irr;
    const double* const* dist;
} or_prev;   /* the previous frame's probes that hit shading samples */

static void shade_ray(const or_scene* s, const or_lights* L, const or_volume* v, const or_prev* prev,
                      const double o[3], const double d[3], double out[4]) {
    double t;
    int64_t tri;
    int back;
    if (!or_closest_hit(s, o, d, &t, &tri, &back)) {
        double c = dot3(d, L->sky_up);
        for (int k = 0; k < 3; ++k) out[k] = L->sky_a[k] + L->sky_b[k] * c;
        out[3] = v->t_max;
        return;
    }
    if (back) {
        /* backfaces: zero radiance, depth shortened by 80% */
        out[0] = out[1] = out[2] = 0.0;
        out[3] = fmin(0.2 * t, v->t_max);
        return;
    }
    double x[3] = { o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2] };
    double n[3];
    tri_unit_normal(s, tri, n);
    int32_t obj = s->tri_object[tri];
    const double* rho = s->object_albedo + 3 * (int64_t)obj;
    double Le[3] = {0.0, 0.0, 0.0};
    int32_t em = s->tri_emitter[tri];
    if (em >= 0) for (int k = 0; k < 3; ++k) Le[k] = s->emitter_radiance[3 * (int64_t)em + k];
    /* direct light from the sun with a shadow ray */
    double tol[3] = { -L->sun_dir[0], -L->sun_dir[1], -L->sun_dir[2] };
    double cosl = dot3(n, tol);
    double direct[3] = {0.0, 0.0, 0.0};
    if (cosl > 0.0 && (L->sun_irradiance[0] > 0.0 || L->sun_irradiance[1] > 0.0 || L->sun_irradiance[2] > 0.0)) {
        double off = 1e-4 * (1.0 + len3(x));
        double so[3] = { x[0] + off * n[0], x[1] + off * n[1], x[2] + off * n[2] };
        if (!or_any_hit_shadow(s, so, tol))
            for (int k = 0; k < 3; ++k) direct[k] = L->sun_irradiance[k] * cosl / M_PI;
    }
    /* indirect: the previous frame's probes queried at the hit, looking back at the probe */
    double wo[3] = { -d[0], -d[1], -d[2] };
    double M[3];
    if (prev->n_vol == 1)
        query_M(&prev->vols[0], prev->states[0], prev->irr[0], prev->dist[0], x, n, wo, M, NULL);
    else
        cascade_M(prev->n_vol, prev->vols, prev->states, prev->irr, prev->dist, x, n, wo, M, NULL);
    for (int k = 0; k < 3; ++k) out[k] = Le[k] + rho[k] * (direct[k] + M[k]);
    out[3] = fmin(t, v->t_max);
}

/* ------------------------------------------------------------------ */
/* Blend one probe (Sec. 2.3 Eq. 1; Sec. 4.2; Sec. 4.3)                 */
/* ------------------------------------------------------------------ */
static void blend_probe(const or_volume* v, const double* dirs, const double* rays,
                        int newly, double irr_scale, double vis_scale,
                        double* irr_tile, double* dist_tile) {
    int64_t R = v->rays;
    int64_t ni = v->irr_n, nd = v->dist_n;
    double a_irr = newly ? 0.0 : clampd(v->hyst_irr * irr_scale, 0.0, 1.0);
    double a_vis = newly ? 0.0 : clampd(v->hyst_vis * vis_scale, 0.0, 1.0);
    for (int64_t j = 0; j < ni; ++j) {
        for (int64_t i = 0; i < ni; ++i) {
            double nt[3];
            or_texel_dir(i, j, ni, nt);
            double sw = 0.0, m[3] = {0.0, 0.0, 0.0};
            for (int64_t r = 0; r < R; ++r) {
                double w = fmax(0.0, dot3(nt, dirs + 3*r));
                sw += w;
                for (int k = 0; k < 3; ++k) m[k] += w * rays[4*r + k];
            }
            if (!(sw > 0.0)) continue;
            double* old = TILE(irr_tile, ni + 2, 3, i + 1, j + 1);
            double enew[3], delta = 0.0;
            for (int k = 0; k < 3; ++k) {
                enew[k] = pow(m[k] / sw, 1.0 / v->gamma);
                delta = fmax(delta, fabs(enew[k] - old[k]));
            }
            double a = a_irr;
            if (delta > v->thr_low) a = fmax(0.0, a - v->thr_step);
            if (delta > v->thr_high) a = 0.0;
            for (int k = 0; k < 3; ++k) old[k] = (1.0 - a) * enew[k] + a * old[k];
        }
    }
    for (int64_t j = 0; j < nd; ++j) {
        for (int64_t i = 0; i < nd; ++i) {
            double nt[3];
            or_texel_dir(i, j, nd, nt);
            double sw = 0.0, mu = 0.0, mu2 = 0.0;
            for (int64_t r = 0; r < R; ++r) {
                double w = pow(fmax(0.0, dot3(nt, dirs + 3*r)), v->cos_power);
                double dd = rays[4*r + 3];
                sw += w;
                mu += w * dd;
                mu2 += w * dd * dd;
            }
            if (!(sw > 0.0)) continue;
            double* old = TILE(dist_tile, nd + 2, 2, i + 1, j + 1);
            old[0] = (1.0 - a_vis) * (mu / sw) + a_vis * old[0];
            old[1] = (1.0 - a_vis) * (mu2 / sw) + a_vis * old[1];
        }
    }
    or_border_copy(irr_tile, ni, 3);
    or_border_copy(dist_tile, nd, 2);
}

/* ------------------------------------------------------------------ */
/* Optional converge pass for new probes (Sec. 6.3)                     */
/* ------------------------------------------------------------------ */
static void converge_probes(const or_scene* s, const or_lights* L, const or_volume* v, int64_t frame,
                            int64_t nn, const int64_t* nl, uint8_t* states, double* irr, double* dist) {
    const int64_t R = v->rays, B = v->converge_batches;
    const int64_t ni = v->irr_n, nd = v->dist_n;
    const int64_t tsi = irr_tile_size(v), tsd = dist_tile_size(v);
    double* bdirs = (double*)malloc(sizeof(double) * 3 * (size_t)(B * R));
    for (int64_t b = 0; b < B; ++b)
        or_frame_dirs(v->seed + 0xD1B54A32D192ED03ULL * (uint64_t)(b + 1), frame, R, bdirs + 3 * b * R);
    double* ni_t = (double*)malloc(sizeof(double) * (size_t)(nn * tsi));
    double* nd_t = (double*)malloc(sizeof(double) * (size_t)(nn * tsd));
    const uint8_t* st1[1] = { states };
    const double* ir1[1] = { irr };
    const double* di1[1] = { dist };
    or_prev prev = { 1, v, st1, ir1, di1 };
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nn; ++q) {
        const int64_t p = nl[q];
        double* ti = ni_t + q * tsi;
        double* td = nd_t + q * tsd;
        memcpy(ti, irr + p * tsi, sizeof(double) * (size_t)tsi);
        memcpy(td, dist + p * tsd, sizeof(double) * (size_t)tsd);
        double* num_i = (double*)calloc((size_t)(ni * ni * 4), sizeof(double));   /* r, g, b, sum w */
        double* num_d = (double*)calloc((size_t)(nd * nd * 3), sizeof(double));   /* mu, mu2, sum w */
        double x[3];
        probe_pos_phys(v, p, x);
        for (int64_t b = 0; b < B; ++b)
            for (int64_t r = 0; r < R; ++r) {
                const double* dir = bdirs + 3 * (b * R + r);
                double ray[4];
                shade_ray(s, L, v, &prev, x, dir, ray);
                for (int64_t t = 0; t < ni * ni; ++t) {
                    double nt[3];
                    or_texel_dir(t % ni, t / ni, ni, nt);
                    const double w = fmax(0.0, dot3(nt, dir));
                    for (int k = 0; k < 3; ++k) num_i[4 * t + k] += w * ray[k];
                    num_i[4 * t + 3] += w;
                }
                for (int64_t t = 0; t < nd * nd; ++t) {
                    double nt[3];
                    or_texel_dir(t % nd, t / nd, nd, nt);
                    const double w = pow(fmax(0.0, dot3(nt, dir)), v->cos_power);
                    num_d[3 * t] += w * ray[3];
                    num_d[3 * t + 1] += w * ray[3] * ray[3];
                    num_d[3 * t + 2] += w;
                }
            }
        for (int64_t t = 0; t < ni * ni; ++t) {
            if (!(num_i[4 * t + 3] > 0.0)) continue;   /* no ray in reach: keeps its value */
            double* e = TILE(ti, ni + 2, 3, t % ni + 1, t / ni + 1);
            for (int k = 0; k < 3; ++k) e[k] = pow(num_i[4 * t + k] / num_i[4 * t + 3], 1.0 / v->gamma);
        }
        for (int64_t t = 0; t < nd * nd; ++t) {
            if (!(num_d[3 * t + 2] > 0.0)) continue;
            double* e = TILE(td, nd + 2, 2, t % nd + 1, t / nd + 1);
            e[0] = num_d[3 * t] / num_d[3 * t + 2];
            e[1] = num_d[3 * t + 1] / num_d[3 * t + 2];
        }
        or_border_copy(ti, ni, 3);
        or_border_copy(td, nd, 2);
        free(num_i);
        free(num_d);
    }
    for (int64_t q = 0; q < nn; ++q) {
        const int64_t p = nl[q];
        memcpy(irr + p * tsi, ni_t + q * tsi, sizeof(double) * (size_t)tsi);
        memcpy(dist + p * tsd, nd_t + q * tsd, sizeof(double) * (size_t)tsd);
        states[p] = advanced(states[p]);
    }
    free(ni_t);
    free(nd_t);
    free(bdirs);
}

/* ------------------------------------------------------------------ */
/* One update frame over a probe subset (Sec. 2.3, Sec. 6.3 listing)    */
/* ------------------------------------------------------------------ */
void or_update(const or_scene* s, const or_lights* L, const or_volume* v, int64_t frame,
               double irr_scale, double vis_scale,
               uint8_t* states, double* irr, double* dist,
               int64_t n_subset, const int64_t* subset, double* rays_out) {
    int64_t P = v->counts[0] * v->counts[1] * v->counts[2];
    int64_t n = subset ? n_subset : P;
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t q = 0; q < n; ++q) list[q] = subset ? subset[q] : q;
    int64_t R = v->rays;

    /* 1. classify uninitialised probes of the subset */
    if (v->state_machine) {
        int64_t nu = 0;
        int64_t* un = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        for (int64_t q = 0; q < n; ++q) if (states[list[q]] == OR_UNINIT) un[nu++] = list[q];
        if (nu) or_optimize(s, v, frame, nu, un);   /* no-op unless the optimizer is on */
        if (nu) or_classify(s, v, frame, nu, un, states, NULL, NULL);
        free(un);
        or_wake(v, n, list, states);
    }
    /* 1b. optional converge pass (Sec. 6.3): every Newly Vigilant / Newly Awake
       probe traces converge_batches batches of R rays against the atlas as it
       stands (batch b rotated by (seed + 0xD1B54A32D192ED03 (b+1), frame)),
       takes per texel the weighted average over all of them, encoded, with
       hysteresis 0, and becomes Vigilant / Awake.  The new texels are
       committed after all of them are shaded. */
    if (v->state_machine && v->converge_batches > 0) {
        int64_t nn = 0;
        int64_t* nl = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        for (int64_t q = 0; q < n; ++q) if (is_newly(states[list[q]])) nl[nn++] = list[q];
        if (nn) converge_probes(s, L, v, frame, nn, nl, states, irr, dist);
        free(nl);
    }
    /* 2. trace and shade every ray of every active probe against the old atlas */
    double* dirs = (double*)malloc(sizeof(double) * 3 * (size_t)R);
    or_frame_dirs(v->seed, frame, R, dirs);
    double* rays = (double*)calloc((size_t)(n > 0 ? n : 1) * (size_t)R * 4, sizeof(double));
    const uint8_t* st1[1] = { states };
    const double* ir1[1] = { irr };
    const double* di1[1] = { dist };
    or_prev prev = { 1, v, st1, ir1, di1 };
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < n; ++q) {
        int64_t p = list[q];
        if (!is_active(states[p])) continue;
        double x[3];
        probe_pos_phys(v, p, x);
        for (int64_t r = 0; r < R; ++r)
            shade_ray(s, L, v, &prev, x, dirs + 3*r, rays + (q * R + r) * 4);
    }
    /* 3. blend into the atlases, copy borders */
    int64_t tsi = irr_tile_size(v), tsd = dist_tile_size(v);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < n; ++q) {
        int64_t p = list[q];
        if (!is_active(states[p])) continue;
        blend_probe(v, dirs, rays + q * R * 4, is_newly(states[p]),
                    irr_scale, vis_scale, irr + p * tsi, dist + p * tsd);
    }
    if (rays_out) {
        for (int64_t q = 0; q < n; ++q)
            if (is_active(states[list[q]]))
                memcpy(rays_out + q * R * 4, rays + q * R * 4, sizeof(double) * 4 * (size_t)R);
    }
    /* 4. state advance: Newly Vigilant -> Vigilant */
    for (int64_t q = 0; q < n; ++q)
        states[list[q]] = advanced(states[list[q]]);
    free(rays);
    free(dirs);
    free(list);
}

/* ------------------------------------------------------------------ */
/* Cascades (Sec. 7.3) and the camera tracking window (Sec. 7.2)       */
/* ------------------------------------------------------------------ */

static void reset_probe(const or_volume* v, int64_t p, uint8_t* states, double* irr, double* dist) {
    states[p] = OR_UNINIT;
    memset(irr + p * irr_tile_size(v), 0, sizeof(double) * (size_t)irr_tile_size(v));
    memset(dist + p * dist_tile_size(v), 0, sizeof(double) * (size_t)dist_tile_size(v));
}

/* Moves the window by whole probe planes until the camera lies within one
 * spacing of its centre on every axis.  Each move shifts the logical grid by
 * one plane: the plane behind the camera leapfrogs to the front, keeping its
 * storage (circular buffer), and is reset to zero texels and UNINIT so it is
 * classified and converged again.  Returns the number of planes moved. */
int64_t or_tracking_scroll(or_volume* v, const double camera[3], uint8_t* states, double* irr, double* dist) {
    int64_t moved = 0;
    for (int a = 0; a < 3; ++a) {
        for (;;) {
            double centre = v->origin[a] + 0.5 * (double)(v->counts[a] - 1) * v->spacing[a];
            int dir = 0;
            if (camera[a] - centre > v->spacing[a]) dir = 1;
            else if (centre - camera[a] > v->spacing[a]) dir = -1;
            if (!dir) break;
            v->origin[a] += dir * v->spacing[a];
            v->shift[a] += dir;
            int64_t fresh = dir > 0 ? v->counts[a] - 1 : 0;   /* logical index of the new plane */
            int b = (a + 1) % 3, c = (a + 2) % 3;
            for (int64_t j = 0; j < v->counts[b]; ++j)
                for (int64_t k = 0; k < v->counts[c]; ++k) {
                    int64_t ijk[3];
                    ijk[a] = fresh; ijk[b] = j; ijk[c] = k;
                    reset_probe(v, or_probe_phys(v, ijk[0], ijk[1], ijk[2]), states, irr, dist);
                }
            moved++;
        }
    }
    return moved;
}

/* One update frame of a cascade: every volume's probes trace the same ray
 * pattern (the first volume's seed), hit shading samples the whole cascade
 * of the previous frame, and each volume blends its own probes. */
void or_update_cascade(const or_scene* s, const or_lights* L, int64_t n_vol, const or_volume* vols,
                       int64_t frame, double irr_scale, double vis_scale,
                       uint8_t* const* states, double* const* irr, double* const* dist,
                       const int64_t* n_subset, const int64_t* const* subsets, double* const* rays_out) {
    int64_t R = vols[0].rays;
    int64_t** lists = (int64_t**)malloc(sizeof(int64_t*) * (size_t)n_vol);
    int64_t* nl = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_vol);
    for (int64_t k = 0; k < n_vol; ++k) {
        const or_volume* v = &vols[k];
        int64_t P = v->counts[0] * v->counts[1] * v->counts[2];
        nl[k] = (subsets && subsets[k]) ? n_subset[k] : P;
        lists[k] = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nl[k] > 0 ? nl[k] : 1));
        for (int64_t q = 0; q < nl[k]; ++q) lists[k][q] = (subsets && subsets[k]) ? subsets[k][q] : q;
        if (v->state_machine) {
            or_volume vk = *v;
            vk.seed = vols[0].seed;
            int64_t nu = 0;
            int64_t* un = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nl[k] > 0 ? nl[k] : 1));
            for (int64_t q = 0; q < nl[k]; ++q) if (states[k][lists[k][q]] == OR_UNINIT) un[nu++] = lists[k][q];
            if (nu) or_classify(s, &vk, frame, nu, un, states[k], NULL, NULL);
            free(un);
        }
    }
    double* dirs = (double*)malloc(sizeof(double) * 3 * (size_t)R);
    or_frame_dirs(vols[0].seed, frame, R, dirs);
    or_prev prev = { n_vol, vols, (const uint8_t* const*)states, (const double* const*)irr,
                     (const double* const*)dist };
    double** rays = (double**)malloc(sizeof(double*) * (size_t)n_vol);
    for (int64_t k = 0; k < n_vol; ++k) {
        rays[k] = (double*)calloc((size_t)(nl[k] > 0 ? nl[k] : 1) * (size_t)R * 4, sizeof(double));
        const or_volume* v = &vols[k];
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t q = 0; q < nl[k]; ++q) {
            int64_t p = lists[k][q];
            if (!is_active(states[k][p])) continue;
            double x[3];
            probe_pos_phys(v, p, x);
            for (int64_t r = 0; r < R; ++r)
                shade_ray(s, L, v, &prev, x, dirs + 3*r, rays[k] + (q * R + r) * 4);
        }
    }
    for (int64_t k = 0; k < n_vol; ++k) {
        const or_volume* v = &vols[k];
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t q = 0; q < nl[k]; ++q) {
            int64_t p = lists[k][q];
            if (!is_active(states[k][p])) continue;
            blend_probe(v, dirs, rays[k] + q * R * 4, is_newly(states[k][p]), irr_scale, vis_scale,
                        irr[k] + p * irr_tile_size(v), dist[k] + p * dist_tile_size(v));
        }
        if (rays_out && rays_out[k])
            for (int64_t q = 0; q < nl[k]; ++q)
                if (is_active(states[k][lists[k][q]]))
                    memcpy(rays_out[k] + q * R * 4, rays[k] + q * R * 4, sizeof(double) * 4 * (size_t)R);
        for (int64_t q = 0; q < nl[k]; ++q)
            states[k][lists[k][q]] = advanced(states[k][lists[k][q]]);
        free(rays[k]);
        free(lists[k]);
    }
    free(rays);
    free(lists);
    free(nl);
    free(dirs);
}

/* ------------------------------------------------------------------ */
/* Differentiation: reverse mode through n_frames updates from a zero   */
/* atlas with hysteresis 0, followed by the query (Sec. 2.2-2.3, 4.2).  */
/* Parameters are the emitters' radiance and the objects' albedo;       */
/* geometry (hits, distances, Chebyshev and backface weights) is fixed. */
/* ------------------------------------------------------------------ */

/* Query adjoint: accumulates dM into texel gradients g_irr (bordered tiles
 * of the atlas `irr`).  M_c = A_c^2, A_c = sum_p w_p a_pc / sum_p w_p,
 * a_pc = b_pc^(gamma/2) with b_pc the bilinear sample; d a / d b is 0 where
 * b <= 0. */
static void query_M_adjoint(const or_volume* v, const uint8_t* st, const double* irr, const double* dist,
                            const double x[3], const double n[3], const double wo[3], const double dM[3],
                            double* g_irr) {
    double wts[8];
    double M[3];
    query_M(v, st, irr, dist, x, n, wo, M, wts);
    double D = min_spacing(v);
    double xb[3];
    for (int a = 0; a < 3; ++a) xb[a] = x[a] + (0.2 * n[a] + 0.8 * wo[a]) * (0.75 * D) * v->bias_B;
    int64_t base[3];
    for (int a = 0; a < 3; ++a) {
        double g = (xb[a] - v->origin[a]) / v->spacing[a];
        double b = floor(g);
        double bmax = (double)(v->counts[a] - 2);
        if (b > bmax) b = bmax;
        if (b < 0.0) b = 0.0;
        base[a] = (int64_t)b;
    }
    double W = 0.0;
    for (int c = 0; c < 8; ++c) W += wts[c];
    if (!(W > 0.0)) return;
    int64_t tsi = irr_tile_size(v), N = v->irr_n + 2, ni = v->irr_n;
    double A[3];
    for (int k = 0; k < 3; ++k) A[k] = sqrt(fmax(M[k], 0.0));
    /* the tile footprint of direction n */
    double u[2];
    or_oct_encode(n, u);
    double sx = 1.0 + (u[0] + 1.0) * 0.5 * (double)ni - 0.5, sy = 1.0 + (u[1] + 1.0) * 0.5 * (double)ni - 0.5;
    int64_t x0 = (int64_t)floor(sx), y0 = (int64_t)floor(sy);
    if (x0 > N - 2) x0 = N - 2;
    if (y0 > N - 2) y0 = N - 2;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    double tx = sx - (double)x0, ty = sy - (double)y0;
    double bw[4] = { (1 - tx) * (1 - ty), tx * (1 - ty), (1 - tx) * ty, tx * ty };
    int64_t bx[4] = { x0, x0 + 1, x0, x0 + 1 }, by[4] = { y0, y0, y0 + 1, y0 + 1 };
    for (int c = 0; c < 8; ++c) {
        if (!(wts[c] > 0.0)) continue;
        int o[3] = { c & 1, (c >> 1) & 1, (c >> 2) & 1 };
        int64_t p = or_probe_phys(v, base[0] + o[0], base[1] + o[1], base[2] + o[2]);
        double b[3];
        or_sample_bilinear(irr + p * tsi, ni, 3, n, b);
        for (int k = 0; k < 3; ++k) {
            if (!(b[k] > 0.0)) continue;
            double dA = dM[k] * 2.0 * A[k];                                  /* dM/dA */
            double da = dA * wts[c] / W;                                     /* dA/da_p */
            double db = da * 0.5 * v->gamma * pow(b[k], 0.5 * v->gamma - 1.0);  /* da/db */
            for (int j = 0; j < 4; ++j) g_irr[p * tsi + (by[j] * N + bx[j]) * 3 + k] += db * bw[j];
        }
    }
}

/* Folds border-texel gradients into the interior texels they copy. */
static void border_fold(double* g_tile, int64_t n, int64_t C) {
    int64_t N = n + 2;
    /* same source map as or_border_copy, transposed */
    for (int64_t k = 1; k <= n; ++k)
        for (int64_t c = 0; c < C; ++c) {
            TILE(g_tile, N, C, 1, n + 1 - k)[c] += TILE(g_tile, N, C, 0, k)[c];
            TILE(g_tile, N, C, n, n + 1 - k)[c] += TILE(g_tile, N, C, n + 1, k)[c];
            TILE(g_tile, N, C, n + 1 - k, 1)[c] += TILE(g_tile, N, C, k, 0)[c];
            TILE(g_tile, N, C, n + 1 - k, n)[c] += TILE(g_tile, N, C, k, n + 1)[c];
        }
    for (int64_t c = 0; c < C; ++c) {
        TILE(g_tile, N, C, n, n)[c] += TILE(g_tile, N, C, 0, 0)[c];
        TILE(g_tile, N, C, 1, n)[c] += TILE(g_tile, N, C, n + 1, 0)[c];
        TILE(g_tile, N, C, n, 1)[c] += TILE(g_tile, N, C, 0, n + 1)[c];
        TILE(g_tile, N, C, 1, 1)[c] += TILE(g_tile, N, C, n + 1, n + 1)[c];
    }
    for (int64_t y = 0; y < N; ++y)
        for (int64_t x = 0; x < N; ++x)
            if (x == 0 || y == 0 || x == N - 1 || y == N - 1)
                for (int64_t c = 0; c < C; ++c) TILE(g_tile, N, C, x, y)[c] = 0.0;
}

/* Texel half of the adjoint: the gradient of sum_q dE_q . E_q, E the query
 * of Sec. 2.2 at n points (E = pi M, as or_query), with respect to every
 * stored irradiance texel value (bordered tiles, the gamma-encoded values
 * the atlas holds): g_irr [P][(irr_n+2)^2][3], overwritten.  The trilinear,
 * backface and Chebyshev weights do not involve irradiance texels, so this
 * is the exact gradient.  fold != 0 adds each border texel's gradient to the
 * interior texel it copies (Sec. 7.1) and zeroes the border entries. */
void or_query_texel_grad(const or_volume* v, const uint8_t* states, const double* irr, const double* dist,
                         int64_t n, const double* pos, const double* nrm, const double camera[3],
                         const double* dE, int fold, double* g_irr) {
    int64_t P = v->counts[0] * v->counts[1] * v->counts[2], tsi = irr_tile_size(v);
    memset(g_irr, 0, sizeof(double) * (size_t)(P * tsi));
    for (int64_t q = 0; q < n; ++q) {
        const double* x = pos + 3*q;
        const double* nn = nrm + 3*q;
        if (nn[0] == 0.0 && nn[1] == 0.0 && nn[2] == 0.0) continue;   /* no surface: E = 0 */
        double wo[3];
        sub3(camera, x, wo);
        double l = len3(wo);
        if (l < 1e-6) { wo[0] = nn[0]; wo[1] = nn[1]; wo[2] = nn[2]; }
        else { wo[0] /= l; wo[1] /= l; wo[2] /= l; }
        double dM[3] = { M_PI * dE[3*q], M_PI * dE[3*q + 1], M_PI * dE[3*q + 2] };
        query_M_adjoint(v, states, irr, dist, x, nn, wo, dM, g_irr);
    }
    if (fold)
        for (int64_t p = 0; p < P; ++p) border_fold(g_irr + p * tsi, v->irr_n, 3);
}

/* Forward: n_frames updates (state machine off: every probe traces) from a
 * zero atlas with hysteresis 0, then E at the query points.  Backward: the
 * gradient of sum(dE * E) with respect to emitter radiance [n_em][3] and
 * object albedo [n_obj][3].  E_out may be NULL. */
void or_diff(const or_scene* s, const or_lights* L, const or_volume* v, int64_t first_frame, int64_t n_frames,
             int64_t n, const double* pos, const double* nrm, const double camera[3], const double* dE,
             double* E_out, double* d_emit, double* d_albedo, int64_t n_emitters, int64_t n_objects) {
    int64_t P = v->counts[0] * v->counts[1] * v->counts[2], R = v->rays;
    int64_t tsi = irr_tile_size(v), tsd = dist_tile_size(v);
    or_volume vv = *v;
    vv.hyst_irr = 0.0;
    vv.hyst_vis = 0.0;
    vv.state_machine = 0;
    /* atlases per frame: [f] is the atlas after frame f; index -1 is zero */
    double** irr = (double**)malloc(sizeof(double*) * (size_t)(n_frames + 1));
    double** dist = (double**)malloc(sizeof(double*) * (size_t)(n_frames + 1));
    uint8_t* st = (uint8_t*)malloc((size_t)P);
    memset(st, OR_VIGILANT, (size_t)P);
    for (int64_t f = 0; f <= n_frames; ++f) {
        irr[f] = (double*)calloc((size_t)(P * tsi), sizeof(double));
        dist[f] = (double*)calloc((size_t)(P * tsd), sizeof(double));
    }
    for (int64_t f = 0; f < n_frames; ++f) {
        memcpy(irr[f + 1], irr[f], sizeof(double) * (size_t)(P * tsi));
        memcpy(dist[f + 1], dist[f], sizeof(double) * (size_t)(P * tsd));
        or_update(s, L, &vv, first_frame + f, 1.0, 1.0, st, irr[f + 1], dist[f + 1], 0, NULL, NULL);
    }
    /* query of the last atlas */
    double* g = (double*)calloc((size_t)(P * tsi), sizeof(double));
    for (int64_t q = 0; q < n; ++q) {
        const double* x = pos + 3 * q;
        const double* nn = nrm + 3 * q;
        if (nn[0] == 0.0 && nn[1] == 0.0 && nn[2] == 0.0) {
            if (E_out) for (int k = 0; k < 3; ++k) E_out[3 * q + k] = 0.0;
            continue;
        }
        double wo[3];
        sub3(camera, x, wo);
        double l = len3(wo);
        if (l < 1e-6) { wo[0] = nn[0]; wo[1] = nn[1]; wo[2] = nn[2]; }
        else { wo[0] /= l; wo[1] /= l; wo[2] /= l; }
        double M[3], dM[3];
        query_M(&vv, st, irr[n_frames], dist[n_frames], x, nn, wo, M, NULL);
        for (int k = 0; k < 3; ++k) {
            if (E_out) E_out[3 * q + k] = M_PI * M[k];
            dM[k] = M_PI * dE[3 * q + k];
        }
        query_M_adjoint(&vv, st, irr[n_frames], dist[n_frames], x, nn, wo, dM, g);
    }
    for (int64_t k = 0; k < 3 * n_emitters; ++k) d_emit[k] = 0.0;
    for (int64_t k = 0; k < 3 * n_objects; ++k) d_albedo[k] = 0.0;
    double* dirs = (double*)malloc(sizeof(double) * 3 * (size_t)R);
    double* gp = (double*)calloc((size_t)(P * tsi), sizeof(double));
    for (int64_t f = n_frames - 1; f >= 0; --f) {
        /* gradients of the texels written by frame f -> ray radiance -> parameters and frame f-1 */
        or_frame_dirs(vv.seed, first_frame + f, R, dirs);
        memset(gp, 0, sizeof(double) * (size_t)(P * tsi));
        for (int64_t p = 0; p < P; ++p) {
            double* gt = g + p * tsi;
            border_fold(gt, v->irr_n, 3);
            double xp[3];
            probe_pos_phys(&vv, p, xp);
            for (int64_t r = 0; r < R; ++r) {
                const double* d = dirs + 3 * r;
                /* dL_r = sum_t W_tr / s_t * dm_t, dm = de * (1/gamma) m^(1/gamma - 1) */
                double gL[3] = {0.0, 0.0, 0.0};
                for (int64_t j = 0; j < v->irr_n; ++j)
                    for (int64_t i = 0; i < v->irr_n; ++i) {
                        double nt[3];
                        or_texel_dir(i, j, v->irr_n, nt);
                        double sw = 0.0;
                        for (int64_t rr = 0; rr < R; ++rr) sw += fmax(0.0, dot3(nt, dirs + 3 * rr));
                        if (!(sw > 0.0)) continue;
                        double w = fmax(0.0, dot3(nt, d)) / sw;
                        const double* e = irr[f + 1] + p * tsi + ((j + 1) * (v->irr_n + 2) + (i + 1)) * 3;
                        const double* gg = gt + ((j + 1) * (v->irr_n + 2) + (i + 1)) * 3;
                        for (int k = 0; k < 3; ++k) {
                            double m = pow(e[k], vv.gamma);
                            double dedm = m > 0.0 ? pow(m, 1.0 / vv.gamma - 1.0) / vv.gamma : (vv.gamma == 1.0 ? 1.0 : 0.0);
                            gL[k] += w * gg[k] * dedm;
                        }
                    }
                if (gL[0] == 0.0 && gL[1] == 0.0 && gL[2] == 0.0) continue;
                /* shading adjoint of this ray (re-traced) */
                double t;
                int64_t tri;
                int back;
                if (!or_closest_hit(s, xp, d, &t, &tri, &back) || back) continue;
                double x[3] = { xp[0] + t * d[0], xp[1] + t * d[1], xp[2] + t * d[2] };
                double nn[3];
                tri_unit_normal(s, tri, nn);
                int32_t obj = s->tri_object[tri], em = s->tri_emitter[tri];
                if (em >= 0) for (int k = 0; k < 3; ++k) d_emit[3 * em + k] += gL[k];
                double tol[3] = { -L->sun_dir[0], -L->sun_dir[1], -L->sun_dir[2] };
                double cosl = dot3(nn, tol), direct[3] = {0.0, 0.0, 0.0};
                if (cosl > 0.0 && (L->sun_irradiance[0] > 0.0 || L->sun_irradiance[1] > 0.0 || L->sun_irradiance[2] > 0.0)) {
                    double off = 1e-4 * (1.0 + len3(x));
                    double so[3] = { x[0] + off * nn[0], x[1] + off * nn[1], x[2] + off * nn[2] };
                    if (!or_any_hit_shadow(s, so, tol))
                        for (int k = 0; k < 3; ++k) direct[k] = L->sun_irradiance[k] * cosl / M_PI;
                }
                double wo[3] = { -d[0], -d[1], -d[2] }, Mp[3];
                query_M(&vv, st, irr[f], dist[f], x, nn, wo, Mp, NULL);
                const double* rho = s->object_albedo + 3 * (int64_t)obj;
                double dMp[3];
                for (int k = 0; k < 3; ++k) {
                    d_albedo[3 * obj + k] += gL[k] * (direct[k] + Mp[k]);
                    dMp[k] = gL[k] * rho[k];
                }
                if (f > 0) query_M_adjoint(&vv, st, irr[f], dist[f], x, nn, wo, dMp, gp);
            }
        }
        double* tmp = g; g = gp; gp = tmp;
    }
    for (int64_t f = 0; f <= n_frames; ++f) { free(irr[f]); free(dist[f]); }
    free(irr); free(dist); free(st); free(g); free(gp); free(dirs);
}
