// C ABI and host runtime: scene registration (BVH build + upload), volume
// allocation, the per-frame launch sequence, queries, buffer access, timing.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ddgi_internal.h"

namespace ddgi {

static thread_local std::string g_err;

static ddgi_status fail(ddgi_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

// Lets other translation units report through ddgi_last_error().
ddgi_status set_error(ddgi_status s, const std::string& msg) { return fail(s, msg); }

#define DDGI_CK(expr)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? DDGI_ERR_OOM : DDGI_ERR_CUDA,       \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// SplitMix64 (Steele, Lea, Flood 2014) for (seed, frame); three 53-bit uniforms
// make a uniformly random unit quaternion (Shoemake, Graphics Gems III 1992).
static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

FrameRot frame_rotation(uint64_t seed, int64_t frame) {
    uint64_t state = mix64(seed ^ mix64((uint64_t)frame + 0x9E3779B97F4A7C15ULL));
    double u[3];
    for (int k = 0; k < 3; ++k) {
        state += 0x9E3779B97F4A7C15ULL;
        u[k] = (double)(mix64(state) >> 11) * (1.0 / 9007199254740992.0);
    }
    const double two_pi = 6.283185307179586477;
    double a = std::sqrt(1.0 - u[0]), b = std::sqrt(u[0]);
    double qx = a * std::sin(two_pi * u[1]), qy = a * std::cos(two_pi * u[1]);
    double qz = b * std::sin(two_pi * u[2]), qw = b * std::cos(two_pi * u[2]);
    FrameRot r;
    r.m[0] = 1 - 2 * (qy * qy + qz * qz); r.m[1] = 2 * (qx * qy - qz * qw); r.m[2] = 2 * (qx * qz + qy * qw);
    r.m[3] = 2 * (qx * qy + qz * qw); r.m[4] = 1 - 2 * (qx * qx + qz * qz); r.m[5] = 2 * (qy * qz - qx * qw);
    r.m[6] = 2 * (qx * qz - qy * qw); r.m[7] = 2 * (qy * qz + qx * qw); r.m[8] = 1 - 2 * (qx * qx + qy * qy);
    return r;
}

}  // namespace ddgi

using namespace ddgi;

struct ddgi_scene_s {
    DevScene dev{};
    float4* nodes = nullptr;
    float4* tris = nullptr;
    int2* attr = nullptr;
    float4* albedo = nullptr;
    float4* emit = nullptr;
    int64_t n_nodes = 0, n_leaves = 0, n_tris = 0;
};

struct TimedStage {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    float ms = 0.0f;
    int32_t count = 0;
};

struct ddgi_volume_s {
    ddgi_volume_desc desc{};
    int64_t P = 0;
    int R = 0;
    float t_max = 0.0f;
    size_t irr_texel_bytes = 0, dist_texel_bytes = 0;
    size_t irr_bytes = 0, dist_bytes = 0;
    uint8_t* states = nullptr;
    void* irr = nullptr;
    void* dist = nullptr;
    int32_t* lists = nullptr;      // [0, P): uninit list, [P, 2P): active list
    int32_t* counts = nullptr;     // [0] uninit count, [1] active count
    uint32_t* status = nullptr;
    float4* records = nullptr;     // [P * R]
    float4* dirs = nullptr;        // [R]
    float* w_irr = nullptr;        // [irr_n^2][R]
    float* inv_s_irr = nullptr;
    float* w_dist = nullptr;       // [dist_n^2][R]
    float* inv_s_dist = nullptr;
    unsigned long long* stats = nullptr;   // [8] trace work counters
    int32_t* shadow_list = nullptr;        // [P * R] rays needing a shadow ray
    int32_t* shadow_count = nullptr;
    uint8_t* pack_irr = nullptr;           // tensor-core blend: weight tiles in operand layout
    uint8_t* pack_dist = nullptr;
    float* inv_irr_r = nullptr;            // 1 / sum of the rounded weights
    float* inv_dist_r = nullptr;
    int64_t updates = 0;
    int3 shift{0, 0, 0};
    bool timing = false;
    TimedStage stages[5];
};

static VolView make_view(const ddgi_volume_s* v) {
    VolView w{};
    const ddgi_volume_desc& d = v->desc;
    w.origin = make_float3(d.origin[0], d.origin[1], d.origin[2]);
    w.spacing = make_float3(d.spacing[0], d.spacing[1], d.spacing[2]);
    w.inv_spacing = make_float3(1.0f / d.spacing[0], 1.0f / d.spacing[1], 1.0f / d.spacing[2]);
    w.counts = make_int3(d.counts[0], d.counts[1], d.counts[2]);
    w.shift = v->shift;
    w.min_spacing = std::fmin(d.spacing[0], std::fmin(d.spacing[1], d.spacing[2]));
    w.bias = d.self_shadow_bias;
    w.gamma = d.gamma;
    w.inv_gamma = 1.0f / d.gamma;
    w.half_gamma = 0.5f * d.gamma;
    w.t_max = v->t_max;
    w.irr_n = d.irr_n;
    w.dist_n = d.dist_n;
    w.irr_tile = (d.irr_n + 2) * (d.irr_n + 2);
    w.dist_tile = (d.dist_n + 2) * (d.dist_n + 2);
    w.n_probes = (int32_t)v->P;
    w.irr_format = d.irr_format;
    w.dist_format = d.dist_format;
    w.states = v->states;
    w.irr = v->irr;
    w.dist = v->dist;
    return w;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

extern "C" {

const char* ddgi_last_error(void) { return g_err.c_str(); }

int32_t ddgi_version(void) { return 1; }

ddgi_status ddgi_scene_create(const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris,
                              const int32_t* tri_object, int32_t n_objects, const float* object_albedo,
                              const int32_t* object_flags, const int32_t* tri_emitter, int32_t n_emitters,
                              const float* emitter_radiance, ddgi_scene* out) {
    if (!out) return fail(DDGI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_verts < 0 || n_tris < 0 || n_objects < 1 || n_emitters < 0)
        return fail(DDGI_ERR_INVALID_ARG, "negative count or no objects");
    if (n_tris > 0 && (!verts || !tris || !tri_object || !tri_emitter))
        return fail(DDGI_ERR_INVALID_ARG, "NULL triangle arrays");
    if (!object_albedo || !object_flags) return fail(DDGI_ERR_INVALID_ARG, "NULL object arrays");
    if (n_emitters > 0 && !emitter_radiance) return fail(DDGI_ERR_INVALID_ARG, "NULL emitter radiance");
    std::vector<int32_t> tri_flags((size_t)n_tris);
    std::vector<int2> attr((size_t)n_tris);
    for (int64_t t = 0; t < n_tris; ++t) {
        int32_t o = tri_object[t], e = tri_emitter[t];
        if (o < 0 || o >= n_objects) return fail(DDGI_ERR_INVALID_ARG, "tri_object out of range");
        if (e < -1 || e >= n_emitters) return fail(DDGI_ERR_INVALID_ARG, "tri_emitter out of range");
        attr[t] = make_int2(o, e);
        tri_flags[t] = object_flags[o];
    }
    for (int64_t k = 0; k < 3 * n_verts; ++k)
        if (!std::isfinite(verts[k])) return fail(DDGI_ERR_INVALID_ARG, "non-finite vertex");
    BvhHost bvh;
    std::string err;
    if (!build_bvh(verts, n_verts, tris, n_tris, tri_flags.data(), bvh, err))
        return fail(DDGI_ERR_INVALID_ARG, err);
    std::vector<float4> alb((size_t)n_objects), em((size_t)(n_emitters > 0 ? n_emitters : 1));
    for (int32_t o = 0; o < n_objects; ++o) {
        float fb;
        std::memcpy(&fb, &object_flags[o], 4);
        alb[o] = make_float4(object_albedo[3 * o], object_albedo[3 * o + 1], object_albedo[3 * o + 2], fb);
    }
    for (int32_t e = 0; e < n_emitters; ++e)
        em[e] = make_float4(emitter_radiance[3 * e], emitter_radiance[3 * e + 1], emitter_radiance[3 * e + 2], 0.f);
    if (n_emitters == 0) em[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    ddgi_scene_s* s = new ddgi_scene_s();
    auto cleanup = [&]() {
        cudaFree(s->nodes); cudaFree(s->tris); cudaFree(s->attr); cudaFree(s->albedo); cudaFree(s->emit);
        delete s;
    };
    size_t nb = bvh.nodes.size() * sizeof(float4), tb = bvh.tris.size() * sizeof(float4);
    cudaError_t e = cudaSuccess;
    if (nb) e = cudaMalloc(&s->nodes, nb);
    if (e == cudaSuccess && tb) e = cudaMalloc(&s->tris, tb);
    if (e == cudaSuccess && n_tris) e = cudaMalloc(&s->attr, attr.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&s->albedo, alb.size() * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&s->emit, em.size() * sizeof(float4));
    if (e == cudaSuccess && nb) e = cudaMemcpy(s->nodes, bvh.nodes.data(), nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && tb) e = cudaMemcpy(s->tris, bvh.tris.data(), tb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n_tris)
        e = cudaMemcpy(s->attr, attr.data(), attr.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->albedo, alb.data(), alb.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->emit, em.data(), em.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cleanup();
        return fail(e == cudaErrorMemoryAllocation ? DDGI_ERR_OOM : DDGI_ERR_CUDA,
                    std::string("scene upload: ") + cudaGetErrorString(e));
    }
    s->n_nodes = (int64_t)(bvh.nodes.size() / 4);
    s->n_leaves = bvh.n_leaves;
    s->n_tris = n_tris;
    s->dev.nodes = s->nodes;
    s->dev.tris = s->tris;
    s->dev.attr = s->attr;
    s->dev.albedo = s->albedo;
    s->dev.emit = s->emit;
    s->dev.n_nodes = (int32_t)s->n_nodes;
    s->dev.n_tris = (int32_t)n_tris;
    *out = s;
    return DDGI_OK;
}

void ddgi_scene_destroy(ddgi_scene s) {
    if (!s) return;
    cudaFree(s->nodes); cudaFree(s->tris); cudaFree(s->attr); cudaFree(s->albedo); cudaFree(s->emit);
    delete s;
}

}  // extern "C"

namespace ddgi {
// Device view of a registered scene, for other translation units.
const DevScene* scene_device_view(ddgi_scene s) { return s ? &s->dev : nullptr; }
}  // namespace ddgi

extern "C" {

ddgi_status ddgi_scene_info(ddgi_scene s, int64_t* n_nodes, int64_t* n_leaves, int64_t* n_tris) {
    if (!s) return fail(DDGI_ERR_INVALID_ARG, "scene is NULL");
    if (n_nodes) *n_nodes = s->n_nodes;
    if (n_leaves) *n_leaves = s->n_leaves;
    if (n_tris) *n_tris = s->n_tris;
    return DDGI_OK;
}

ddgi_status ddgi_trace(ddgi_scene s, const float* orig_dev, const float* dir_dev, int64_t n, float* t_dev,
                       int32_t* tri_dev, int32_t* backface_dev, ddgi_stream stream) {
    if (!s) return fail(DDGI_ERR_INVALID_ARG, "scene is NULL");
    if (n < 0) return fail(DDGI_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return DDGI_OK;
    if (!orig_dev || !dir_dev || !t_dev || !tri_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned(orig_dev, 4) || !aligned(dir_dev, 4) || !aligned(t_dev, 4) || !aligned(tri_dev, 4) ||
        !aligned(backface_dev, 4))
        return fail(DDGI_ERR_INVALID_ARG, "misaligned buffer");
    DDGI_CK(launch_trace_rays(s->dev, orig_dev, dir_dev, n, t_dev, tri_dev, backface_dev, (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_raycast_gbuffer(ddgi_scene s, const float cam_pos[3], const float cam_fwd[3],
                                 const float cam_up[3], float vfov_deg, int32_t width, int32_t height,
                                 float* pos_dev, float* nrm_dev, ddgi_stream stream) {
    if (!s || !cam_pos || !cam_fwd || !cam_up) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (width <= 0 || height <= 0 || !(vfov_deg > 0.0f && vfov_deg < 180.0f))
        return fail(DDGI_ERR_INVALID_ARG, "bad image size or field of view");
    if (!pos_dev || !nrm_dev || !aligned(pos_dev, 4) || !aligned(nrm_dev, 4))
        return fail(DDGI_ERR_INVALID_ARG, "bad output buffer");
    double f[3] = {cam_fwd[0], cam_fwd[1], cam_fwd[2]}, u[3] = {cam_up[0], cam_up[1], cam_up[2]};
    double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (double& c : f) c /= fl;
    double r[3] = {f[1] * u[2] - f[2] * u[1], f[2] * u[0] - f[0] * u[2], f[0] * u[1] - f[1] * u[0]};
    double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(rl > 0.0)) return fail(DDGI_ERR_INVALID_ARG, "camera up parallel to forward");
    for (double& c : r) c /= rl;
    double uu[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    float th = (float)std::tan(vfov_deg * 3.14159265358979323846 / 360.0);
    DDGI_CK(launch_gbuffer(s->dev, make_float3(cam_pos[0], cam_pos[1], cam_pos[2]),
                           make_float3((float)f[0], (float)f[1], (float)f[2]),
                           make_float3((float)r[0], (float)r[1], (float)r[2]),
                           make_float3((float)uu[0], (float)uu[1], (float)uu[2]), th,
                           (float)width / (float)height, width, height, pos_dev, nrm_dev,
                           (cudaStream_t)stream));
    return DDGI_OK;
}

static ddgi_status check_desc(const ddgi_volume_desc* d) {
    if (!d) return fail(DDGI_ERR_INVALID_ARG, "desc is NULL");
    for (int a = 0; a < 3; ++a) {
        if (d->counts[a] < 2 || d->counts[a] > 4096) return fail(DDGI_ERR_INVALID_ARG, "counts must be in [2, 4096]");
        if (!(d->spacing[a] > 0.0f) || !std::isfinite(d->spacing[a]))
            return fail(DDGI_ERR_INVALID_ARG, "spacing must be positive");
        if (!std::isfinite(d->origin[a])) return fail(DDGI_ERR_INVALID_ARG, "origin not finite");
    }
    if ((int64_t)d->counts[0] * d->counts[1] * d->counts[2] > (1LL << 26))
        return fail(DDGI_ERR_INVALID_ARG, "too many probes");
    if (d->rays_per_probe < 1 || d->rays_per_probe > 1024)
        return fail(DDGI_ERR_INVALID_ARG, "rays_per_probe must be in [1, 1024]");
    if (d->irr_n < 1 || d->irr_n > 32 || d->dist_n < 1 || d->dist_n > 64)
        return fail(DDGI_ERR_INVALID_ARG, "irr_n in [1,32], dist_n in [1,64]");
    if (!(d->gamma > 0.0f)) return fail(DDGI_ERR_INVALID_ARG, "gamma must be positive");
    if (!(d->hysteresis_irr >= 0.0f && d->hysteresis_irr <= 1.0f && d->hysteresis_vis >= 0.0f &&
          d->hysteresis_vis <= 1.0f))
        return fail(DDGI_ERR_INVALID_ARG, "hysteresis must be in [0, 1]");
    if (!(d->dist_cos_power >= 0.0f) || !(d->self_shadow_bias >= 0.0f))
        return fail(DDGI_ERR_INVALID_ARG, "negative cosine power or bias");
    if (d->irr_format < 0 || d->irr_format > 2 || d->dist_format < 0 || d->dist_format > 1)
        return fail(DDGI_ERR_INVALID_ARG, "unknown atlas format");
    return DDGI_OK;
}

void ddgi_volume_destroy(ddgi_volume v) {
    if (!v) return;
    cudaFree(v->states); cudaFree(v->irr); cudaFree(v->dist); cudaFree(v->lists); cudaFree(v->counts);
    cudaFree(v->status); cudaFree(v->records); cudaFree(v->dirs); cudaFree(v->w_irr);
    cudaFree(v->inv_s_irr); cudaFree(v->w_dist); cudaFree(v->inv_s_dist); cudaFree(v->stats);
    cudaFree(v->shadow_list); cudaFree(v->shadow_count);
    cudaFree(v->pack_irr); cudaFree(v->pack_dist); cudaFree(v->inv_irr_r); cudaFree(v->inv_dist_r);
    for (auto& st : v->stages)
        for (auto& pr : st.pending) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    delete v;
}

ddgi_status ddgi_volume_create(const ddgi_volume_desc* desc, ddgi_volume* out) {
    if (!out) return fail(DDGI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    ddgi_status s = check_desc(desc);
    if (s != DDGI_OK) return s;
    ddgi_volume_s* v = new ddgi_volume_s();
    v->desc = *desc;
    v->P = (int64_t)desc->counts[0] * desc->counts[1] * desc->counts[2];
    v->R = desc->rays_per_probe;
    if (desc->t_max >= 0.0f) {
        v->t_max = desc->t_max;
    } else {
        double sx = desc->spacing[0], sy = desc->spacing[1], sz = desc->spacing[2];
        v->t_max = (float)(2.0 * std::sqrt(sx * sx + sy * sy + sz * sz));
    }
    v->irr_texel_bytes = desc->irr_format == DDGI_IRR_FP32 ? 12 : (desc->irr_format == DDGI_IRR_FP16 ? 8 : 4);
    v->dist_texel_bytes = desc->dist_format == DDGI_DIST_FP32 ? 8 : 4;
    int64_t ti = (int64_t)(desc->irr_n + 2) * (desc->irr_n + 2);
    int64_t td = (int64_t)(desc->dist_n + 2) * (desc->dist_n + 2);
    v->irr_bytes = (size_t)(v->P * ti) * v->irr_texel_bytes;
    v->dist_bytes = (size_t)(v->P * td) * v->dist_texel_bytes;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes > 0 ? bytes : 16);
    };
    A((void**)&v->states, (size_t)v->P);
    A(&v->irr, v->irr_bytes);
    A(&v->dist, v->dist_bytes);
    A((void**)&v->lists, sizeof(int32_t) * 2 * (size_t)v->P);
    A((void**)&v->counts, sizeof(int32_t) * 4);
    A((void**)&v->status, sizeof(uint32_t));
    A((void**)&v->records, sizeof(float4) * (size_t)v->P * v->R);
    A((void**)&v->dirs, sizeof(float4) * v->R);
    A((void**)&v->w_irr, sizeof(float) * desc->irr_n * desc->irr_n * (size_t)v->R);
    A((void**)&v->inv_s_irr, sizeof(float) * desc->irr_n * desc->irr_n);
    A((void**)&v->w_dist, sizeof(float) * desc->dist_n * desc->dist_n * (size_t)v->R);
    A((void**)&v->inv_s_dist, sizeof(float) * desc->dist_n * desc->dist_n);
    A((void**)&v->stats, sizeof(unsigned long long) * 8);
    A((void**)&v->shadow_list, sizeof(int32_t) * (size_t)v->P * v->R);
    A((void**)&v->shadow_count, sizeof(int32_t) * 4);
    A((void**)&v->pack_irr, tc_pack_irr_bytes(v->R));
    A((void**)&v->pack_dist, tc_pack_dist_bytes(v->R));
    A((void**)&v->inv_irr_r, sizeof(float) * 128);
    A((void**)&v->inv_dist_r, sizeof(float) * 256);
    if (e == cudaSuccess) e = cudaMemset(v->states, desc->state_machine ? DDGI_STATE_UNINIT : DDGI_STATE_VIGILANT, (size_t)v->P);
    if (e == cudaSuccess) e = cudaMemset(v->irr, 0, v->irr_bytes);
    if (e == cudaSuccess) e = cudaMemset(v->dist, 0, v->dist_bytes);
    if (e == cudaSuccess) e = cudaMemset(v->counts, 0, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = cudaMemset(v->status, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        ddgi_volume_destroy(v);
        return fail(e == cudaErrorMemoryAllocation ? DDGI_ERR_OOM : DDGI_ERR_CUDA,
                    std::string("volume allocation: ") + cudaGetErrorString(e));
    }
    *out = v;
    return DDGI_OK;
}

ddgi_status ddgi_volume_get_info(ddgi_volume v, ddgi_volume_info* info) {
    if (!v || !info) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    info->n_probes = v->P;
    info->irr_tile_texels = (int64_t)(v->desc.irr_n + 2) * (v->desc.irr_n + 2);
    info->dist_tile_texels = (int64_t)(v->desc.dist_n + 2) * (v->desc.dist_n + 2);
    info->irr_bytes = (int64_t)v->irr_bytes;
    info->dist_bytes = (int64_t)v->dist_bytes;
    info->irr_texel_bytes = (int64_t)v->irr_texel_bytes;
    info->dist_texel_bytes = (int64_t)v->dist_texel_bytes;
    info->t_max = v->t_max;
    return DDGI_OK;
}

static Lights make_lights(const ddgi_lights* L) {
    Lights o{};
    o.sun_dir = make_float3(L->sun_dir[0], L->sun_dir[1], L->sun_dir[2]);
    o.sun_irr = make_float3(L->sun_irradiance[0], L->sun_irradiance[1], L->sun_irradiance[2]);
    o.sky_a = make_float3(L->sky_a[0], L->sky_a[1], L->sky_a[2]);
    o.sky_b = make_float3(L->sky_b[0], L->sky_b[1], L->sky_b[2]);
    o.sky_up = make_float3(L->sky_up[0], L->sky_up[1], L->sky_up[2]);
    o.sun_on = (L->sun_irradiance[0] > 0.0f || L->sun_irradiance[1] > 0.0f || L->sun_irradiance[2] > 0.0f);
    return o;
}

// Stage timing: events recorded on the update stream around each stage.
struct StageTimer {
    ddgi_volume_s* v;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    StageTimer(ddgi_volume_s* v_, int s_, cudaStream_t st_) : v(v_), stage(s_), st(st_) {
        if (!v->timing) return;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
    }
    ~StageTimer() {
        if (!v->timing) return;
        cudaEventRecord(b, st);
        v->stages[stage].pending.emplace_back(a, b);
    }
};

ddgi_status ddgi_update(ddgi_volume v, ddgi_scene s, const ddgi_lights* lights,
                        const ddgi_update_params* params, ddgi_stream stream) {
    if (!v || !s || !lights || !params) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (!(params->irr_hyst_scale >= 0.0f) || !(params->vis_hyst_scale >= 0.0f))
        return fail(DDGI_ERR_INVALID_ARG, "negative hysteresis scale");
    if (params->blend_precision < DDGI_BLEND_FP32 || params->blend_precision > DDGI_BLEND_BF16)
        return fail(DDGI_ERR_INVALID_ARG, "unknown blend precision");
    const bool tensor = params->blend_precision != DDGI_BLEND_FP32;
    if (tensor && !tc_blend_supported(v->desc.irr_n, v->desc.dist_n))
        return fail(DDGI_ERR_UNSUPPORTED, "tensor-core blend needs irr_n^2 <= 128 and dist_n^2 <= 256");
    cudaStream_t st = (cudaStream_t)stream;
    const ddgi_volume_desc& d = v->desc;
    VolView view = make_view(v);
    int sms = sm_count();
    FrameRot rot = frame_rotation(d.seed, params->frame);
    {
        StageTimer tm(v, 4, st);
        DDGI_CK(launch_frame_setup(rot, v->R, d.irr_n, d.dist_n, d.dist_cos_power, v->dirs, v->w_irr,
                                   v->inv_s_irr, v->w_dist, v->inv_s_dist, st));
        if (tensor)
            DDGI_CK(launch_pack_weights(v->w_irr, v->w_dist, v->R, d.irr_n, d.dist_n,
                                        params->blend_precision == DDGI_BLEND_BF16, v->pack_irr, v->pack_dist,
                                        v->inv_irr_r, v->inv_dist_r, st));
    }
    DDGI_CK(cudaMemsetAsync(v->counts, 0, sizeof(int32_t) * 2, st));
    if (d.state_machine) {
        {
            StageTimer tm(v, 1, st);
            DDGI_CK(launch_build_list(v->states, (int)v->P, 0, v->lists, v->counts + 0, st));
        }
        StageTimer tm(v, 0, st);
        DDGI_CK(launch_classify(s->dev, view, v->dirs, v->R, v->lists, v->counts + 0, sms * 8, st));
    }
    {
        StageTimer tm(v, 1, st);
        DDGI_CK(launch_build_list(v->states, (int)v->P, 1, v->lists + v->P, v->counts + 1, st));
    }
    {
        StageTimer tm(v, 2, st);
        DDGI_CK(launch_trace_wavefront(s->dev, view, make_lights(lights), v->dirs, v->R, v->lists + v->P,
                                       v->counts + 1, v->records, v->shadow_list, v->shadow_count, sms * 8,
                                       st));
    }
    BlendParams bp{};
    bp.hyst_irr = std::fmin(1.0f, std::fmax(0.0f, d.hysteresis_irr * params->irr_hyst_scale));
    bp.hyst_vis = std::fmin(1.0f, std::fmax(0.0f, d.hysteresis_vis * params->vis_hyst_scale));
    bp.thr_low = d.thr_low;
    bp.thr_high = d.thr_high;
    bp.thr_step = d.thr_step;
    bp.R = v->R;
    {
        StageTimer tm(v, 3, st);
        if (tensor)
            DDGI_CK(launch_blend_tc(view, bp, params->blend_precision == DDGI_BLEND_BF16, v->pack_irr, v->pack_dist,
                                    v->inv_irr_r, v->inv_dist_r, v->records, v->lists + v->P, v->counts + 1,
                                    v->status, sms, st));
        else
            DDGI_CK(launch_blend(view, bp, v->w_irr, v->inv_s_irr, v->w_dist, v->inv_s_dist, v->records,
                                 v->lists + v->P, v->counts + 1, v->status, sms * 4, st));
    }
    v->updates++;
    return DDGI_OK;
}

ddgi_status ddgi_trace_stats(ddgi_volume v, ddgi_scene s, const ddgi_lights* lights, uint64_t stats[7],
                             ddgi_stream stream) {
    if (!v || !s || !lights || !stats) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (v->updates == 0) return fail(DDGI_ERR_INVALID_ARG, "no update has run on this volume");
    cudaStream_t st = (cudaStream_t)stream;
    DDGI_CK(cudaMemsetAsync(v->stats, 0, sizeof(unsigned long long) * 8, st));
    DDGI_CK(launch_trace_shade_count(s->dev, make_view(v), make_lights(lights), v->dirs, v->R,
                                     v->lists + v->P, v->counts + 1, v->stats, sm_count() * 16, st));
    unsigned long long h[8];
    DDGI_CK(cudaMemcpyAsync(h, v->stats, sizeof(h), cudaMemcpyDeviceToHost, st));
    DDGI_CK(cudaStreamSynchronize(st));
    for (int k = 0; k < 7; ++k) stats[k] = h[k];
    return DDGI_OK;
}

ddgi_status ddgi_query(ddgi_volume v, const float* pos_dev, const float* nrm_dev, int64_t n,
                       const float camera_pos[3], float* out_dev, ddgi_stream stream) {
    if (!v || !camera_pos) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (n < 0) return fail(DDGI_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return DDGI_OK;
    if (!pos_dev || !nrm_dev || !out_dev || !aligned(pos_dev, 4) || !aligned(nrm_dev, 4) || !aligned(out_dev, 4))
        return fail(DDGI_ERR_INVALID_ARG, "bad buffer");
    DDGI_CK(launch_query(make_view(v), pos_dev, nrm_dev, n,
                         make_float3(camera_pos[0], camera_pos[1], camera_pos[2]), out_dev,
                         (cudaStream_t)stream));
    return DDGI_OK;
}

static ddgi_status buffer_of(ddgi_volume v, int32_t which, void** p, size_t* bytes) {
    if (which == 0) { *p = v->irr; *bytes = v->irr_bytes; }
    else if (which == 1) { *p = v->dist; *bytes = v->dist_bytes; }
    else if (which == 2) { *p = v->states; *bytes = (size_t)v->P; }
    else return fail(DDGI_ERR_INVALID_ARG, "which must be 0, 1 or 2");
    return DDGI_OK;
}

ddgi_status ddgi_get_buffer(ddgi_volume v, int32_t which, void* dst_dev, size_t bytes, ddgi_stream stream) {
    if (!v || !dst_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    void* p;
    size_t nb;
    ddgi_status s = buffer_of(v, which, &p, &nb);
    if (s != DDGI_OK) return s;
    if (bytes != nb) return fail(DDGI_ERR_INVALID_ARG, "size mismatch: expected " + std::to_string(nb));
    DDGI_CK(cudaMemcpyAsync(dst_dev, p, nb, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_set_buffer(ddgi_volume v, int32_t which, const void* src_dev, size_t bytes, ddgi_stream stream) {
    if (!v || !src_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    void* p;
    size_t nb;
    ddgi_status s = buffer_of(v, which, &p, &nb);
    if (s != DDGI_OK) return s;
    if (bytes != nb) return fail(DDGI_ERR_INVALID_ARG, "size mismatch: expected " + std::to_string(nb));
    DDGI_CK(cudaMemcpyAsync(p, src_dev, nb, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_get_ray_records(ddgi_volume v, float* records_dev, int32_t* probe_ids_dev, int64_t* n_active,
                                 ddgi_stream stream) {
    if (!v || !records_dev || !probe_ids_dev || !n_active) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    int32_t cnt = 0;
    DDGI_CK(cudaMemcpyAsync(&cnt, v->counts + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    DDGI_CK(cudaStreamSynchronize(st));
    *n_active = cnt;
    if (cnt > 0) {
        DDGI_CK(cudaMemcpyAsync(records_dev, v->records, sizeof(float4) * (size_t)cnt * v->R,
                                cudaMemcpyDeviceToDevice, st));
        DDGI_CK(cudaMemcpyAsync(probe_ids_dev, v->lists + v->P, sizeof(int32_t) * (size_t)cnt,
                                cudaMemcpyDeviceToDevice, st));
    }
    return DDGI_OK;
}

ddgi_status ddgi_enable_timing(ddgi_volume v, int32_t enable) {
    if (!v) return fail(DDGI_ERR_INVALID_ARG, "volume is NULL");
    v->timing = enable != 0;
    return DDGI_OK;
}

ddgi_status ddgi_read_timings(ddgi_volume v, float ms[5], int32_t counts[5]) {
    if (!v || !ms || !counts) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    for (int k = 0; k < 5; ++k) {
        float total = 0.0f;
        int32_t c = 0;
        for (auto& pr : v->stages[k].pending) {
            DDGI_CK(cudaEventSynchronize(pr.second));
            float t = 0.0f;
            DDGI_CK(cudaEventElapsedTime(&t, pr.first, pr.second));
            total += t;
            c++;
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        v->stages[k].pending.clear();
        ms[k] = total;
        counts[k] = c;
    }
    return DDGI_OK;
}

ddgi_status ddgi_poll_status(ddgi_volume v, ddgi_stream stream) {
    if (!v) return fail(DDGI_ERR_INVALID_ARG, "volume is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t w = 0;
    DDGI_CK(cudaMemcpyAsync(&w, v->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    DDGI_CK(cudaMemsetAsync(v->status, 0, sizeof(uint32_t), st));
    DDGI_CK(cudaStreamSynchronize(st));
    if (w & 2u) return fail(DDGI_ERR_TIMEOUT, "a bounded device wait gave up");
    if (w & 1u) return fail(DDGI_ERR_NUMERIC, "non-finite texel value produced");
    return DDGI_OK;
}

}  // extern "C"
