// C ABI and host runtime: scene registration (BVH build + upload), volume
// allocation, the per-frame launch sequence, queries, buffer access, timing.
#include <algorithm>
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

std::vector<int32_t> ray_order_morton(int R) {
    auto spread = [](uint32_t v) {
        v &= 0x3FFu;
        v = (v | (v << 16)) & 0x030000FFu;
        v = (v | (v << 8)) & 0x0300F00Fu;
        v = (v | (v << 4)) & 0x030C30C3u;
        v = (v | (v << 2)) & 0x09249249u;
        return v;
    };
    std::vector<std::pair<uint32_t, int32_t>> keys((size_t)R);
    const double inv_phi = 0.61803398874989484820, two_pi = 6.283185307179586477;
    for (int i = 0; i < R; ++i) {
        double a = (double)i * inv_phi;
        double phi = two_pi * (a - std::floor(a));
        double z = 1.0 - (2.0 * i + 1.0) / (double)R;
        double r = std::sqrt(std::fmax(0.0, 1.0 - z * z));
        double x = std::cos(phi) * r, y = std::sin(phi) * r;
        double l1 = std::fabs(x) + std::fabs(y) + std::fabs(z);
        double px = x / l1, py = y / l1;
        if (z < 0.0) {
            double qx = (1.0 - std::fabs(py)) * (px >= 0.0 ? 1.0 : -1.0);
            double qy = (1.0 - std::fabs(px)) * (py >= 0.0 ? 1.0 : -1.0);
            px = qx;
            py = qy;
        }
        uint32_t ux = (uint32_t)std::fmin(1023.0, (px + 1.0) * 512.0);
        uint32_t uy = (uint32_t)std::fmin(1023.0, (py + 1.0) * 512.0);
        keys[i] = {spread(ux) | (spread(uy) << 1), i};
    }
    std::sort(keys.begin(), keys.end());
    std::vector<int32_t> perm((size_t)R);
    for (int i = 0; i < R; ++i) perm[i] = keys[i].second;
    return perm;
}

}  // namespace ddgi

using namespace ddgi;

struct ddgi_scene_s {
    DevScene dev{};
    float4* nodes = nullptr;
    float4* nodes4 = nullptr;
    float4* tris = nullptr;
    int2* attr = nullptr;
    float4* albedo = nullptr;
    float4* emit = nullptr;
    int64_t n_nodes = 0, n_leaves = 0, n_tris = 0;
    int32_t n_objects = 0, n_emitters = 0;
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
    int32_t* counts = nullptr;     // [0] uninit count, [1] active count, [2] new-probe count, [4..9] trace counters
                                   // (shadow_count below), all cleared by one memset per frame
    uint32_t* status = nullptr;
    float4* records = nullptr;     // [P * R]
    float4* dirs = nullptr;        // [R]
    double* sf64 = nullptr;        // [R][3] unrotated ray pattern sf(i, R), double (frame setup)
    float* w_irr = nullptr;        // [irr_n^2][R]
    float* inv_s_irr = nullptr;
    float* w_dist = nullptr;       // [dist_n^2][R]
    float* inv_s_dist = nullptr;
    unsigned long long* stats = nullptr;   // [8] trace work counters
    int32_t* shadow_list = nullptr;        // [P * R] rays needing a shadow ray
    int32_t* hit_list = nullptr;           // [P * R] rays with a front hit to shade
    int4* class_scratch = nullptr;         // [P] classification sums (zeroed between uses)
    int32_t* shadow_count = nullptr;
    int32_t* perm = nullptr;               // [R] ray order within a probe's warps
    std::vector<void*> snap_irr, snap_dist;   // differentiable forward: atlas after each frame
    // its FP64 instantiation: atlases after each frame, ray records, texel
    // gradients of two frames, per-ray radiance gradients, weight row sums
    std::vector<double*> snap64_irr, snap64_dist;
    double *rec64 = nullptr, *g64 = nullptr, *g64_prev = nullptr, *gL64 = nullptr, *sw64 = nullptr;
    float* g_irr = nullptr;                // adjoint: texel gradients of two frames
    float* g_prev = nullptr;
    uint8_t* pack_w = nullptr;             // tensor-core blend: weight tiles in operand layout
    float* inv_irr_r = nullptr;            // 1 / sum of the rounded weights
    float* inv_dist_r = nullptr;
    int64_t updates = 0;
    int3 shift{0, 0, 0};
    float4* offsets = nullptr;             // [P] probe offsets (position optimizer)
    float4* opt_dirs = nullptr;            // [3R] rays (and their constants) of an optimizer iteration
    bool uninit_possible = true;           // some probe may still be UNINIT
    float* dyn_boxes = nullptr;            // [DDGI_MAX_DYNAMIC_BOXES][6] extended boxes (device)
    int32_t n_dyn = 0;
    bool awake_possible = false;           // some probe may be Awake
    int64_t list_begin = -1, list_end = -1; // range of the active list built last, if still valid
    // ddgi_frame_host: device staging of host G-buffers, copy streams, events
    float* stage = nullptr;                // [3][stage_cap][3] float: positions, normals, results
    int64_t stage_cap = 0;
    cudaStream_t copy_in = nullptr, copy_out = nullptr;
    cudaEvent_t ev_entry = nullptr, ev_in = nullptr, ev_out = nullptr;
    cudaEvent_t ev_chunk[4] = {nullptr, nullptr, nullptr, nullptr};
    // optional converge pass (Sec. 6.3): its batch's frame tables and the sums
    float4* conv_dirs = nullptr;
    float *conv_w_irr = nullptr, *conv_inv_irr = nullptr, *conv_w_dist = nullptr, *conv_inv_dist = nullptr;
    float4* conv_acc_irr = nullptr;
    float2* conv_acc_dist = nullptr;
    float* conv_den = nullptr;
    // the frame's texel weights run on a side stream, overlapping the trace
    cudaStream_t setup_st = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_weights = nullptr;
    bool timing = false;
    TimedStage stages[8];
};

static VolView make_view(const ddgi_volume_s* v) {
    VolView w{};
    const ddgi_volume_desc& d = v->desc;
    w.origin = make_float3(d.origin[0], d.origin[1], d.origin[2]);
    w.spacing = make_float3(d.spacing[0], d.spacing[1], d.spacing[2]);
    w.inv_spacing = make_float3(1.0f / d.spacing[0], 1.0f / d.spacing[1], 1.0f / d.spacing[2]);
    w.counts = make_int3(d.counts[0], d.counts[1], d.counts[2]);
    set_view_divisors(w);
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
    // offsets only when the position optimizer is on: the query then reads them
    w.offsets = d.optimizer_iters > 0 ? v->offsets : nullptr;
    w.offset_limit = d.offset_limit;
    return w;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }
// Caller-owned device buffers start on 16-byte boundaries (the base of any
// cudaMalloc or torch allocation does); NULL passes, callers check it apart.
static bool dev16(const void* p) { return aligned(p, 16); }
static const char* kMisaligned = "device buffers must be 16-byte aligned";

extern "C" {

const char* ddgi_last_error(void) { return g_err.c_str(); }

int32_t ddgi_version(void) { return 1; }

int32_t ddgi_texel_bytes(int32_t which, int32_t format) {
    if (which == 0) {
        if (format == DDGI_IRR_FP32) return 16;
        if (format == DDGI_IRR_FP16) return 8;
        if (format == DDGI_IRR_RGB9E5) return 4;
    } else if (which == 1) {
        if (format == DDGI_DIST_FP32) return 8;
        if (format == DDGI_DIST_FP16) return 4;
    }
    return 0;
}

ddgi_status ddgi_scene_create(const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris,
                              const int32_t* tri_object, int32_t n_objects, const float* object_albedo,
                              const int32_t* object_flags, const int32_t* tri_emitter, int32_t n_emitters,
                              const float* emitter_radiance, ddgi_scene* out) {
    if (!out) return fail(DDGI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_verts < 0 || n_tris < 0 || n_objects < 1 || n_emitters < 0)
        return fail(DDGI_ERR_INVALID_ARG, "negative count or no objects");
    if (n_tris > DDGI_MAX_TRIS) return fail(DDGI_ERR_INVALID_ARG, "more than DDGI_MAX_TRIS triangles");
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
    // the 4-wide walk pushes without a bound test; the collapse keeps its
    // stack within kStackSize4 by construction, checked here
    if (wide_stack_bound(bvh.nodes4) > kStackSize4) return fail(DDGI_ERR_INVALID_ARG, "BVH too deep for the traversal");
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
        cudaFree(s->nodes); cudaFree(s->nodes4); cudaFree(s->tris); cudaFree(s->attr); cudaFree(s->albedo); cudaFree(s->emit);
        delete s;
    };
    size_t nb = bvh.nodes.size() * sizeof(float4), tb = bvh.tris.size() * sizeof(float4);
    size_t nb4 = bvh.nodes4.size() * sizeof(float4);
    cudaError_t e = cudaSuccess;
    if (nb) e = cudaMalloc(&s->nodes, nb);
    if (e == cudaSuccess && nb4) e = cudaMalloc(&s->nodes4, nb4);
    if (e == cudaSuccess && tb) e = cudaMalloc(&s->tris, tb);
    if (e == cudaSuccess && n_tris) e = cudaMalloc(&s->attr, attr.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&s->albedo, alb.size() * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&s->emit, em.size() * sizeof(float4));
    if (e == cudaSuccess && nb) e = cudaMemcpy(s->nodes, bvh.nodes.data(), nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nb4) e = cudaMemcpy(s->nodes4, bvh.nodes4.data(), nb4, cudaMemcpyHostToDevice);
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
    s->dev.nodes4 = s->nodes4;
    s->dev.n_nodes4 = (int32_t)(bvh.nodes4.size() / 8);
    s->dev.tris = s->tris;
    s->dev.attr = s->attr;
    s->dev.albedo = s->albedo;
    s->dev.emit = s->emit;
    s->dev.n_nodes = (int32_t)s->n_nodes;
    s->dev.n_tris = (int32_t)n_tris;
    s->n_objects = n_objects;
    s->n_emitters = n_emitters;
    *out = s;
    return DDGI_OK;
}

void ddgi_scene_destroy(ddgi_scene s) {
    if (!s) return;
    cudaFree(s->nodes); cudaFree(s->nodes4); cudaFree(s->tris); cudaFree(s->attr); cudaFree(s->albedo); cudaFree(s->emit);
    delete s;
}

}  // extern "C"

namespace ddgi {
// Device view of a registered scene, for other translation units.
const DevScene* scene_device_view(ddgi_scene s) { return s ? &s->dev : nullptr; }
}  // namespace ddgi

extern "C" {

ddgi_status ddgi_bvh_check(const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris,
                           int64_t stats[9]) {
    if (!stats) return fail(DDGI_ERR_INVALID_ARG, "stats is NULL");
    if (n_verts < 0 || n_tris < 0 || n_tris > DDGI_MAX_TRIS) return fail(DDGI_ERR_INVALID_ARG, "bad count");
    if (n_tris > 0 && (!verts || !tris)) return fail(DDGI_ERR_INVALID_ARG, "NULL triangle arrays");
    BvhHost bvh;
    std::string err;
    if (!build_bvh(verts, n_verts, tris, n_tris, nullptr, bvh, err)) return fail(DDGI_ERR_INVALID_ARG, err);
    for (int k = 0; k < 9; ++k) stats[k] = 0;
    const int64_t n4 = (int64_t)(bvh.nodes4.size() / 8);
    stats[0] = (int64_t)(bvh.nodes.size() / 4);
    stats[1] = n4;
    stats[2] = bvh.n_leaves;
    stats[3] = bvh.max_depth;
    stats[4] = bvh.max_depth4;
    stats[8] = n_tris;
    if (n4 == 0) return DDGI_OK;
    struct Item {
        int32_t ref;
        float lo[3], hi[3];
    };
    std::vector<int32_t> seen((size_t)n_tris, 0);
    std::vector<Item> stack;
    stack.push_back({0, {-INFINITY, -INFINITY, -INFINITY}, {INFINITY, INFINITY, INFINITY}});
    int64_t bad = 0, deepest = 0;
    while (!stack.empty()) {
        Item it = stack.back();
        stack.pop_back();
        if (it.ref >= 0) {
            if (it.ref >= n4) { bad++; continue; }
            const float4* N = &bvh.nodes4[8 * (size_t)it.ref];
            int32_t ref[4];
            std::memcpy(ref, &N[6], sizeof(ref));
            const float* lo[3] = {&N[0].x, &N[2].x, &N[4].x};
            const float* hi[3] = {&N[1].x, &N[3].x, &N[5].x};
            for (int c = 0; c < 4; ++c) {
                if (ref[c] == kRefDone) {
                    stats[6]++;
                    continue;
                }
                Item k;
                k.ref = ref[c];
                for (int a = 0; a < 3; ++a) {
                    k.lo[a] = lo[a][c];
                    k.hi[a] = hi[a][c];
                    if (k.lo[a] < it.lo[a] || k.hi[a] > it.hi[a] || k.lo[a] > k.hi[a]) bad++;
                }
                stack.push_back(k);
            }
            deepest = std::max<int64_t>(deepest, (int64_t)stack.size());
        } else {
            const int code = ~it.ref;
            const int first = code >> kLeafBits, cnt = (code & ((1 << kLeafBits) - 1)) + 1;
            if (first < 0 || (int64_t)first + cnt > n_tris) { bad++; continue; }
            for (int k = first; k < first + cnt; ++k) {
                seen[(size_t)k]++;
                const float* p[3] = {&bvh.tris[3 * (size_t)k].x, &bvh.tris[3 * (size_t)k + 1].x,
                                     &bvh.tris[3 * (size_t)k + 2].x};
                for (int q = 0; q < 3; ++q)
                    for (int a = 0; a < 3; ++a)
                        if (p[q][a] < it.lo[a] || p[q][a] > it.hi[a]) bad++;
            }
        }
    }
    for (int32_t c : seen)
        if (c != 1) bad++;
    stats[5] = deepest;
    stats[7] = bad;
    return DDGI_OK;
}

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
    if (!dev16(orig_dev) || !dev16(dir_dev) || !dev16(t_dev) || !dev16(tri_dev) ||
        !dev16(backface_dev))
        return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
    DDGI_CK(launch_trace_rays(s->dev, orig_dev, dir_dev, n, t_dev, tri_dev, backface_dev, (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_raycast_gbuffer(ddgi_scene s, const float cam_pos[3], const float cam_fwd[3],
                                 const float cam_up[3], float vfov_deg, int32_t width, int32_t height,
                                 float* pos_dev, float* nrm_dev, ddgi_stream stream) {
    if (!s || !cam_pos || !cam_fwd || !cam_up) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (width <= 0 || height <= 0 || !(vfov_deg > 0.0f && vfov_deg < 180.0f))
        return fail(DDGI_ERR_INVALID_ARG, "bad image size or field of view");
    if (!pos_dev || !nrm_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL output buffer");
    if (!dev16(pos_dev) || !dev16(nrm_dev)) return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
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
    if (d->optimizer_iters < 0 || d->optimizer_iters > 16)
        return fail(DDGI_ERR_INVALID_ARG, "optimizer_iters must be in [0, 16]");
    if (!(d->offset_limit >= 0.0f && d->offset_limit < 0.5f))
        return fail(DDGI_ERR_INVALID_ARG, "offset_limit must be in [0, 0.5)");
    if (d->converge_batches < 0 || d->converge_batches > 64)
        return fail(DDGI_ERR_INVALID_ARG, "converge_batches must be in [0, 64]");
    if ((int64_t)d->counts[0] * d->counts[1] * d->counts[2] * d->rays_per_probe >= (1LL << 31))
        return fail(DDGI_ERR_INVALID_ARG, "probes x rays_per_probe must stay below 2^31");
    return DDGI_OK;
}

void ddgi_volume_destroy(ddgi_volume v) {
    if (!v) return;
    cudaFree(v->states); cudaFree(v->irr); cudaFree(v->dist); cudaFree(v->lists); cudaFree(v->counts);
    cudaFree(v->status); cudaFree(v->records); cudaFree(v->dirs); cudaFree(v->sf64); cudaFree(v->w_irr);
    cudaFree(v->inv_s_irr); cudaFree(v->w_dist); cudaFree(v->inv_s_dist); cudaFree(v->stats);
    cudaFree(v->shadow_list); cudaFree(v->hit_list); cudaFree(v->class_scratch); cudaFree(v->perm);
    for (void* p : v->snap_irr) cudaFree(p);
    for (void* p : v->snap_dist) cudaFree(p);
    cudaFree(v->g_irr); cudaFree(v->g_prev);
    cudaFree(v->pack_w); cudaFree(v->inv_irr_r); cudaFree(v->inv_dist_r);
    cudaFree(v->offsets); cudaFree(v->opt_dirs); cudaFree(v->dyn_boxes);
    for (double* q : v->snap64_irr) cudaFree(q);
    for (double* q : v->snap64_dist) cudaFree(q);
    cudaFree(v->rec64); cudaFree(v->g64); cudaFree(v->g64_prev); cudaFree(v->gL64); cudaFree(v->sw64);
    cudaFree(v->stage);
    cudaFree(v->conv_dirs); cudaFree(v->conv_w_irr); cudaFree(v->conv_inv_irr); cudaFree(v->conv_w_dist);
    cudaFree(v->conv_inv_dist); cudaFree(v->conv_acc_irr); cudaFree(v->conv_acc_dist); cudaFree(v->conv_den);
    if (v->setup_st) cudaStreamDestroy(v->setup_st);
    if (v->ev_fork) cudaEventDestroy(v->ev_fork);
    if (v->ev_weights) cudaEventDestroy(v->ev_weights);
    if (v->copy_in) cudaStreamDestroy(v->copy_in);
    if (v->copy_out) cudaStreamDestroy(v->copy_out);
    for (cudaEvent_t e : {v->ev_entry, v->ev_in, v->ev_out, v->ev_chunk[0], v->ev_chunk[1], v->ev_chunk[2],
                          v->ev_chunk[3]})
        if (e) cudaEventDestroy(e);
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
    v->irr_texel_bytes = (size_t)ddgi_texel_bytes(0, desc->irr_format);
    v->dist_texel_bytes = (size_t)ddgi_texel_bytes(1, desc->dist_format);
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
    A((void**)&v->counts, sizeof(int32_t) * kCounterInts);
    A((void**)&v->status, sizeof(uint32_t));
    A((void**)&v->records, sizeof(float4) * (size_t)v->P * v->R);
    A((void**)&v->dirs, sizeof(float4) * 3 * v->R);
    A((void**)&v->sf64, sizeof(double) * 3 * v->R);
    if (e == cudaSuccess) e = launch_sf_table(v->R, v->sf64, 0);
    A((void**)&v->offsets, sizeof(float4) * (size_t)v->P);
    if (desc->optimizer_iters > 0) {
        A((void**)&v->opt_dirs, sizeof(float4) * 3 * v->R);
    }
    if (desc->converge_batches > 0) {
        const size_t ti = (size_t)desc->irr_n * desc->irr_n, td = (size_t)desc->dist_n * desc->dist_n;
        A((void**)&v->conv_dirs, sizeof(float4) * 3 * v->R);
        A((void**)&v->conv_w_irr, sizeof(float) * ti * (size_t)v->R);
        A((void**)&v->conv_inv_irr, sizeof(float) * ti);
        A((void**)&v->conv_w_dist, sizeof(float) * td * (size_t)v->R);
        A((void**)&v->conv_inv_dist, sizeof(float) * td);
        A((void**)&v->conv_acc_irr, sizeof(float4) * ti * (size_t)v->P);
        A((void**)&v->conv_acc_dist, sizeof(float2) * td * (size_t)v->P);
        A((void**)&v->conv_den, sizeof(float) * (ti + td));
    }
    A((void**)&v->w_irr, sizeof(float) * desc->irr_n * desc->irr_n * (size_t)v->R);
    A((void**)&v->inv_s_irr, sizeof(float) * desc->irr_n * desc->irr_n);
    A((void**)&v->w_dist, sizeof(float) * desc->dist_n * desc->dist_n * (size_t)v->R);
    A((void**)&v->inv_s_dist, sizeof(float) * desc->dist_n * desc->dist_n);
    A((void**)&v->stats, sizeof(unsigned long long) * 8);
    A((void**)&v->shadow_list, sizeof(int32_t) * (size_t)v->P * v->R);
    A((void**)&v->hit_list, sizeof(int32_t) * (size_t)v->P * v->R);
    A((void**)&v->class_scratch, sizeof(int4) * (size_t)v->P);
    if (e == cudaSuccess) e = cudaMemset(v->class_scratch, 0, sizeof(int4) * (size_t)v->P);
    A((void**)&v->perm, sizeof(int32_t) * v->R);
    if (e == cudaSuccess) {
        std::vector<int32_t> perm = ray_order_morton(v->R);
        e = cudaMemcpy(v->perm, perm.data(), sizeof(int32_t) * v->R, cudaMemcpyHostToDevice);
    }
    A((void**)&v->pack_w, tc_pack_bytes(v->R));
    A((void**)&v->inv_irr_r, sizeof(float) * 128);
    A((void**)&v->inv_dist_r, sizeof(float) * 256);
    if (e == cudaSuccess) e = cudaMemset(v->states, desc->state_machine ? DDGI_STATE_UNINIT : DDGI_STATE_VIGILANT, (size_t)v->P);
    if (e == cudaSuccess) e = cudaMemset(v->irr, 0, v->irr_bytes);
    if (e == cudaSuccess) e = cudaMemset(v->dist, 0, v->dist_bytes);
    if (e == cudaSuccess) e = cudaMemset(v->offsets, 0, sizeof(float4) * (size_t)v->P);
    if (e == cudaSuccess) e = cudaMemset(v->counts, 0, sizeof(int32_t) * kCounterInts);
    v->shadow_count = v->counts + 4;
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

static ddgi_status update_impl(ddgi_volume v, ddgi_scene s, const ddgi_lights* lights,
                               const ddgi_update_params* params, int64_t begin, int64_t end, ddgi_stream stream);

ddgi_status ddgi_update(ddgi_volume v, ddgi_scene s, const ddgi_lights* lights,
                        const ddgi_update_params* params, ddgi_stream stream) {
    if (!v) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    return update_impl(v, s, lights, params, 0, v->P, stream);
}

ddgi_status ddgi_set_dynamic_boxes(ddgi_volume v, const float* boxes_host, int32_t n) {
    if (!v) return fail(DDGI_ERR_INVALID_ARG, "volume is NULL");
    if (n < 0 || n > DDGI_MAX_DYNAMIC_BOXES) return fail(DDGI_ERR_INVALID_ARG, "n must be in [0, DDGI_MAX_DYNAMIC_BOXES]");
    if (n > 0 && !boxes_host) return fail(DDGI_ERR_INVALID_ARG, "boxes_host is NULL");
    if (n > 0 && !v->desc.state_machine) return fail(DDGI_ERR_INVALID_ARG, "dynamic objects need the state machine");
    const ddgi_volume_desc& d = v->desc;
    const float bias = 0.75f * std::fmin(d.spacing[0], std::fmin(d.spacing[1], d.spacing[2])) * d.self_shadow_bias;
    std::vector<float> ext((size_t)6 * n);
    for (int32_t b = 0; b < n; ++b)
        for (int a = 0; a < 3; ++a) {
            const float lo = boxes_host[6 * b + a], hi = boxes_host[6 * b + 3 + a];
            if (!std::isfinite(lo) || !std::isfinite(hi) || lo > hi)
                return fail(DDGI_ERR_INVALID_ARG, "box with lo > hi or a non-finite bound");
            ext[6 * b + a] = lo - (d.spacing[a] + bias);
            ext[6 * b + 3 + a] = hi + (d.spacing[a] + bias);
        }
    if (!v->dyn_boxes) DDGI_CK(cudaMalloc(&v->dyn_boxes, sizeof(float) * 6 * DDGI_MAX_DYNAMIC_BOXES));
    if (n > 0) DDGI_CK(cudaMemcpy(v->dyn_boxes, ext.data(), sizeof(float) * 6 * (size_t)n, cudaMemcpyHostToDevice));
    v->n_dyn = n;
    return DDGI_OK;
}

ddgi_status ddgi_update_range(ddgi_volume v, ddgi_scene s, const ddgi_lights* lights,
                              const ddgi_update_params* params, int64_t probe_begin, int64_t probe_end,
                              ddgi_stream stream) {
    if (!v) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (probe_begin < 0 || probe_end > v->P || probe_begin > probe_end)
        return fail(DDGI_ERR_INVALID_ARG, "probe range out of bounds");
    return update_impl(v, s, lights, params, probe_begin, probe_end, stream);
}

static ddgi_status update_impl(ddgi_volume v, ddgi_scene s, const ddgi_lights* lights,
                               const ddgi_update_params* params, int64_t begin, int64_t end, ddgi_stream stream) {
    if (!v || !s || !lights || !params) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (!(params->irr_hyst_scale >= 0.0f) || !(params->vis_hyst_scale >= 0.0f))
        return fail(DDGI_ERR_INVALID_ARG, "negative hysteresis scale");
    if (params->blend_precision < DDGI_BLEND_FP32 || params->blend_precision > DDGI_BLEND_TF32X3)
        return fail(DDGI_ERR_INVALID_ARG, "unknown blend precision");
    const bool tensor = params->blend_precision != DDGI_BLEND_FP32;
    if (tensor && !tc_blend_supported(v->desc.irr_n, v->desc.dist_n))
        return fail(DDGI_ERR_UNSUPPORTED, "tensor-core blend needs irr_n^2 <= 128 and dist_n^2 <= 256");
    cudaStream_t st = (cudaStream_t)stream;
    const ddgi_volume_desc& d = v->desc;
    VolView view = make_view(v);
    int sms = sm_count();
    FrameRot rot = frame_rotation(d.seed, params->frame);
    // the active list can be kept from the previous frame when no state can
    // have changed in between: no uninitialised probe, no dynamic object
    // waking or putting probes to sleep, same probe range
    const bool keep_list = d.state_machine && !v->uninit_possible && v->n_dyn == 0 && !v->awake_possible &&
                           v->list_begin == begin && v->list_end == end;
    {
        StageTimer tm(v, 4, st);
        if (!v->setup_st) {
            DDGI_CK(cudaStreamCreateWithFlags(&v->setup_st, cudaStreamNonBlocking));
            DDGI_CK(cudaEventCreateWithFlags(&v->ev_fork, cudaEventDisableTiming));
            DDGI_CK(cudaEventCreateWithFlags(&v->ev_weights, cudaEventDisableTiming));
        }
        // the texel weights (and their tensor-core packing) on the side stream,
        // after all earlier work on the stream (the previous blend read them);
        // the directions on the stream.  The directions launch also clears the
        // trace counters, and the list counts unless the active list is kept.
        DDGI_CK(cudaEventRecord(v->ev_fork, st));
        DDGI_CK(cudaStreamWaitEvent(v->setup_st, v->ev_fork, 0));
        DDGI_CK(launch_frame_setup_split(rot, v->R, d.irr_n, d.dist_n, d.dist_cos_power, v->sf64, v->dirs, v->w_irr,
                                         v->inv_s_irr, v->w_dist, v->inv_s_dist,
                                         keep_list ? v->counts + 4 : v->counts,
                                         keep_list ? kCounterInts - 4 : kCounterInts, st, v->setup_st));
        if (tensor)
            DDGI_CK(launch_pack_weights(v->w_irr, v->w_dist, v->R, d.irr_n, d.dist_n, params->blend_precision,
                                        v->pack_w, v->inv_irr_r, v->inv_dist_r, v->setup_st));
        DDGI_CK(cudaEventRecord(v->ev_weights, v->setup_st));
    }
    // uninitialised probes (none after a full-range update, until states are
    // set again): position optimizer iterations, then classification
    bool states_changed = false;   // classification or waking ran: new probes may exist
    if (d.state_machine && v->uninit_possible) {
        states_changed = true;
        {
            StageTimer tm(v, 1, st);
            DDGI_CK(launch_build_list_range(v->states, (int)begin, (int)end, 0, v->lists, v->counts + 0, st));
        }
        StageTimer tm(v, 0, st);
        for (int k = 0; k < d.optimizer_iters; ++k) {
            // iteration k traces the rays of frame + k, as if spread over frames
            DDGI_CK(launch_frame_dirs(frame_rotation(d.seed, params->frame + k), v->R, d.irr_n, d.dist_n, v->sf64,
                                      v->opt_dirs, st));
            DDGI_CK(launch_optimize(s->dev, view, v->opt_dirs, v->R, v->lists, v->counts + 0, sms * 8, st));
        }
        DDGI_CK(launch_classify(s->dev, view, v->dirs, v->R, v->perm, v->lists, v->counts + 0, v->class_scratch,
                                sms * 8, st));
        if (begin == 0 && end == v->P) v->uninit_possible = false;
    }
    // dynamic objects wake sleeping probes (and awake probes fall asleep
    // again once none is near: one more pass after the boxes are cleared)
    if (d.state_machine && (v->n_dyn > 0 || v->awake_possible)) {
        states_changed = true;
        StageTimer tm(v, 1, st);
        DDGI_CK(launch_wake(view, v->dyn_boxes, v->n_dyn, (int)begin, (int)end, st));
        v->awake_possible = v->n_dyn > 0;
    }
    // optional converge pass (Sec. 6.3): new probes (only when states changed)
    // trace converge_batches batches of R rays against the atlas as it stands,
    // take the encoded weighted average over all of them and advance to
    // Vigilant / Awake before the regular trace
    if (d.state_machine && d.converge_batches > 0 && states_changed) {
        StageTimer tm(v, 1, st);
        DDGI_CK(cudaMemsetAsync(v->counts + 2, 0, sizeof(int32_t), st));
        DDGI_CK(launch_build_list_range(v->states, (int)begin, (int)end, 2, v->lists, v->counts + 2, st));
        for (int b = 0; b < d.converge_batches; ++b) {
            const FrameRot rb = frame_rotation(d.seed + 0xD1B54A32D192ED03ULL * (uint64_t)(b + 1), params->frame);
            DDGI_CK(launch_frame_setup(rb, v->R, d.irr_n, d.dist_n, d.dist_cos_power, v->sf64, v->conv_dirs,
                                       v->conv_w_irr, v->conv_inv_irr, v->conv_w_dist, v->conv_inv_dist,
                                       v->counts + 4, kCounterInts - 4, st));
            DDGI_CK(launch_trace_wavefront(s->dev, view, make_lights(lights), v->conv_dirs, v->R, v->perm, v->lists,
                                           v->counts + 2, v->records, v->shadow_list, v->hit_list, v->shadow_count,
                                           sms * 8, st, nullptr));
            DDGI_CK(launch_converge_accum(v->R, d.irr_n, d.dist_n, v->conv_w_irr, v->conv_w_dist, v->records,
                                          v->counts + 2, v->conv_acc_irr, v->conv_acc_dist, v->conv_den, b == 0,
                                          sms * 8, st));
        }
        DDGI_CK(launch_converge_finish(view, v->lists, v->counts + 2, v->conv_acc_irr, v->conv_acc_dist,
                                       v->conv_den, v->status, sms * 8, st));
        // the regular trace starts its counters from zero
        DDGI_CK(cudaMemsetAsync(v->counts + 4, 0, sizeof(int32_t) * (kCounterInts - 4), st));
    }
    if (!keep_list) {
        StageTimer tm(v, 1, st);
        DDGI_CK(launch_build_list_range(v->states, (int)begin, (int)end, 1, v->lists + v->P, v->counts + 1, st));
        // reusable next frame only if nothing below changes which probes are active
        v->list_begin = begin;
        v->list_end = end;
    }
    {
        StageTimer tm(v, 2, st);
        // per-pass events (stages 5, 6, 7) when timing is on
        cudaEvent_t marks[4] = {nullptr, nullptr, nullptr, nullptr};
        if (v->timing)
            for (auto& m : marks) DDGI_CK(cudaEventCreate(&m));
        DDGI_CK(launch_trace_wavefront(s->dev, view, make_lights(lights), v->dirs, v->R, v->perm, v->lists + v->P,
                                       v->counts + 1, v->records, v->shadow_list, v->hit_list, v->shadow_count, sms * 8,
                                       st, v->timing ? marks : nullptr));
        if (v->timing) {
            v->stages[5].pending.emplace_back(marks[0], marks[1]);
            v->stages[6].pending.emplace_back(marks[1], marks[2]);
            v->stages[7].pending.emplace_back(marks[2], marks[3]);
        }
    }
    BlendParams bp{};
    bp.hyst_irr = std::fmin(1.0f, std::fmax(0.0f, d.hysteresis_irr * params->irr_hyst_scale));
    bp.hyst_vis = std::fmin(1.0f, std::fmax(0.0f, d.hysteresis_vis * params->vis_hyst_scale));
    bp.thr_low = d.thr_low;
    bp.thr_high = d.thr_high;
    bp.thr_step = d.thr_step;
    bp.R = v->R;
    DDGI_CK(cudaStreamWaitEvent(st, v->ev_weights, 0));   // the frame's weights are ready
    {
        StageTimer tm(v, 3, st);
        if (tensor)
            DDGI_CK(launch_blend_tc(view, bp, params->blend_precision, v->pack_w, v->inv_irr_r, v->inv_dist_r,
                                    v->records, v->lists + v->P, v->counts + 1, v->status, sms, st));
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
    // the counting passes write their hit records to scratch, leaving the
    // update's records untouched
    float4* scratch = nullptr;
    DDGI_CK(cudaMalloc(&scratch, sizeof(float4) * (size_t)v->P * v->R));
    DDGI_CK(cudaMemsetAsync(v->stats, 0, sizeof(unsigned long long) * 8, st));
    cudaError_t e = launch_trace_count(s->dev, make_view(v), make_lights(lights), v->dirs, v->R, v->perm,
                                       v->lists + v->P, v->counts + 1, scratch, v->shadow_list, v->hit_list,
                                       v->shadow_count, v->stats, sm_count() * 8, st);
    unsigned long long h[8];
    int32_t n[4] = {0, 0, 0, 0};
    int32_t n_active = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, v->stats, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n, v->shadow_count, sizeof(n), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n_active, v->counts + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(scratch);
    DDGI_CK(e);
    stats[0] = (uint64_t)n_active * (uint64_t)v->R;
    stats[1] = h[1];
    stats[2] = h[2];
    stats[3] = (uint64_t)n[0];
    stats[4] = h[4];
    stats[5] = h[5];
    stats[6] = (uint64_t)n[1];
    return DDGI_OK;
}

ddgi_status ddgi_query_glossy(ddgi_volume v, const float* pos_dev, const float* nrm_dev, const float* dir_dev,
                              int64_t n, float* out_dev, ddgi_stream stream) {
    if (!v) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (n < 0) return fail(DDGI_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return DDGI_OK;
    if (!pos_dev || !nrm_dev || !dir_dev || !out_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL buffer");
    if (!dev16(pos_dev) || !dev16(nrm_dev) || !dev16(dir_dev) || !dev16(out_dev))
        return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
    DDGI_CK(launch_query_glossy(make_view(v), pos_dev, nrm_dev, dir_dev, n, out_dev, (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_query(ddgi_volume v, const float* pos_dev, const float* nrm_dev, int64_t n,
                       const float camera_pos[3], float* out_dev, ddgi_stream stream) {
    if (!v || !camera_pos) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (n < 0) return fail(DDGI_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return DDGI_OK;
    if (!pos_dev || !nrm_dev || !out_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL buffer");
    if (!dev16(pos_dev) || !dev16(nrm_dev) || !dev16(out_dev)) return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
    DDGI_CK(launch_query(make_view(v), pos_dev, nrm_dev, n,
                         make_float3(camera_pos[0], camera_pos[1], camera_pos[2]), out_dev,
                         (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_frame_host(ddgi_volume v, ddgi_scene s, const ddgi_lights* lights,
                            const ddgi_update_params* params, const float* pos_host, const float* nrm_host,
                            int64_t n, const float camera_pos[3], float* out_host, ddgi_stream stream) {
    if (!v || !camera_pos) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (n < 0) return fail(DDGI_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!pos_host || !nrm_host || !out_host)) return fail(DDGI_ERR_INVALID_ARG, "NULL host array");
    cudaStream_t st = (cudaStream_t)stream;
    constexpr int kChunks = 4;
    if (!v->copy_in) {
        DDGI_CK(cudaStreamCreateWithFlags(&v->copy_in, cudaStreamNonBlocking));
        DDGI_CK(cudaStreamCreateWithFlags(&v->copy_out, cudaStreamNonBlocking));
        for (cudaEvent_t* e : {&v->ev_entry, &v->ev_in, &v->ev_out, &v->ev_chunk[0], &v->ev_chunk[1],
                               &v->ev_chunk[2], &v->ev_chunk[3]})
            DDGI_CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    if (n > v->stage_cap) {   // earlier frames may still read the old staging
        DDGI_CK(cudaStreamSynchronize(st));
        cudaFree(v->stage);
        v->stage = nullptr;
        v->stage_cap = 0;
        DDGI_CK(cudaMalloc(&v->stage, sizeof(float) * 9 * (size_t)n));
        v->stage_cap = n;
    }
    const size_t row = sizeof(float) * 3;
    float* pos_d = v->stage;
    float* nrm_d = v->stage + 3 * v->stage_cap;
    float* out_d = v->stage + 6 * v->stage_cap;
    // inputs: after everything enqueued on the stream so far (the previous
    // frame's query read the staging), alongside the probe update
    if (n > 0) {
        DDGI_CK(cudaEventRecord(v->ev_entry, st));
        DDGI_CK(cudaStreamWaitEvent(v->copy_in, v->ev_entry, 0));
        DDGI_CK(cudaMemcpyAsync(pos_d, pos_host, row * (size_t)n, cudaMemcpyHostToDevice, v->copy_in));
        DDGI_CK(cudaMemcpyAsync(nrm_d, nrm_host, row * (size_t)n, cudaMemcpyHostToDevice, v->copy_in));
        DDGI_CK(cudaEventRecord(v->ev_in, v->copy_in));
    }
    ddgi_status r = update_impl(v, s, lights, params, 0, v->P, stream);
    if (r != DDGI_OK || n == 0) {   // the stream still orders after the input copies
        if (n > 0) DDGI_CK(cudaStreamWaitEvent(st, v->ev_in, 0));
        return r;
    }
    DDGI_CK(cudaStreamWaitEvent(st, v->ev_in, 0));
    const float3 cam = make_float3(camera_pos[0], camera_pos[1], camera_pos[2]);
    const VolView view = make_view(v);
    // page-locked, device-mapped result memory: the query writes it directly
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, out_host) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer != nullptr) {
        DDGI_CK(launch_query(view, pos_d, nrm_d, n, cam, (float*)pa.devicePointer, st, true));
        return DDGI_OK;
    }
    (void)cudaGetLastError();   // an unregistered pointer is not an error here
    // otherwise the query runs in chunks; each chunk's result copy overlaps
    // the next chunk's query
    const int64_t chunk = (n + kChunks - 1) / kChunks;
    for (int c = 0; c < kChunks; ++c) {
        const int64_t a = c * chunk, b = std::min(n, a + chunk);
        if (a >= b) break;
        DDGI_CK(launch_query(view, pos_d + 3 * a, nrm_d + 3 * a, b - a, cam, out_d + 3 * a, st));
        DDGI_CK(cudaEventRecord(v->ev_chunk[c], st));
        DDGI_CK(cudaStreamWaitEvent(v->copy_out, v->ev_chunk[c], 0));
        DDGI_CK(cudaMemcpyAsync(out_host + 3 * a, out_d + 3 * a, row * (size_t)(b - a), cudaMemcpyDeviceToHost,
                                v->copy_out));
    }
    DDGI_CK(cudaEventRecord(v->ev_out, v->copy_out));
    DDGI_CK(cudaStreamWaitEvent(st, v->ev_out, 0));
    return DDGI_OK;
}

static ddgi_status buffer_of(ddgi_volume v, int32_t which, void** p, size_t* bytes) {
    if (which == 0) { *p = v->irr; *bytes = v->irr_bytes; }
    else if (which == 1) { *p = v->dist; *bytes = v->dist_bytes; }
    else if (which == 2) { *p = v->states; *bytes = (size_t)v->P; }
    else if (which == 3) { *p = v->offsets; *bytes = sizeof(float4) * (size_t)v->P; }
    else return fail(DDGI_ERR_INVALID_ARG, "which must be 0, 1, 2 or 3");
    return DDGI_OK;
}

ddgi_status ddgi_get_buffer(ddgi_volume v, int32_t which, void* dst_dev, size_t bytes, ddgi_stream stream) {
    if (!v || !dst_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (!dev16(dst_dev)) return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
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
    if (!dev16(src_dev)) return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
    void* p;
    size_t nb;
    ddgi_status s = buffer_of(v, which, &p, &nb);
    if (s != DDGI_OK) return s;
    if (bytes != nb) return fail(DDGI_ERR_INVALID_ARG, "size mismatch: expected " + std::to_string(nb));
    DDGI_CK(cudaMemcpyAsync(p, src_dev, nb, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    if (which == 2) {   // restored states may hold UNINIT or Awake probes and change the active set
        v->uninit_possible = true;
        v->awake_possible = true;
        v->list_begin = v->list_end = -1;
    }
    return DDGI_OK;
}

ddgi_status ddgi_get_ray_records(ddgi_volume v, float* records_dev, int32_t* probe_ids_dev, int64_t* n_active,
                                 ddgi_stream stream) {
    if (!v || !records_dev || !probe_ids_dev || !n_active) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (!dev16(records_dev) || !dev16(probe_ids_dev)) return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
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

ddgi_status ddgi_read_timings(ddgi_volume v, float ms[8], int32_t counts[8]) {
    if (!v || !ms || !counts) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    for (int k = 0; k < 8; ++k) {
        float total = 0.0f;
        int32_t c = 0;
        for (auto& pr : v->stages[k].pending) {
            DDGI_CK(cudaEventSynchronize(pr.second));
            float t = 0.0f;
            DDGI_CK(cudaEventElapsedTime(&t, pr.first, pr.second));
            total += t;
            c++;
            // the pass marks share events (stage 6 starts where stage 5 ends,
            // 7 where 6 ends): each is destroyed once, as a pair's start
            cudaEventDestroy(pr.first);
            if (k < 5 || k == 7) cudaEventDestroy(pr.second);
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

// ===========================================================================
// Cascades (Sec. 7.3) with camera tracking windows (Sec. 7.2): one batched
// launch sequence over every volume per frame, optionally replayed as a
// CUDA graph, launch shapes from an autotuner.
// ===========================================================================

#include <fstream>
#include <sstream>

namespace {

constexpr int kMaxPlanes = 256;

struct FrameParams {
    VolView views[kMaxVolumes];
    FrameRot rot;
    int4 planes[kMaxPlanes];
    int32_t n_planes;
    int32_t pad[3];
};

struct GraphKey {
    int32_t precision = -1, trace_mult = 0, blend_probes = 0;
    float irr_scale = 0.f, vis_scale = 0.f;
    ddgi_lights lights{};
    bool operator==(const GraphKey& o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

}  // namespace

struct ddgi_cascade_s {
    int n = 0;
    ddgi_volume_desc desc[kMaxVolumes]{};
    int64_t P[kMaxVolumes]{};
    int64_t total = 0;
    int R = 0;
    float t_max[kMaxVolumes]{};
    size_t irr_bytes[kMaxVolumes]{}, dist_bytes[kMaxVolumes]{};
    uint8_t* states[kMaxVolumes]{};
    void* irr[kMaxVolumes]{};
    void* dist[kMaxVolumes]{};
    double origin[kMaxVolumes][3]{};
    int shift[kMaxVolumes][3]{};
    int32_t* lists = nullptr;
    int32_t* counts = nullptr;
    uint32_t* status = nullptr;
    float4* records = nullptr;
    int32_t* shadow_list = nullptr;
    int32_t* hit_list = nullptr;
    int4* class_scratch = nullptr;   // [total] classification sums (zeroed between uses)
    int32_t* shadow_count = nullptr;
    int32_t* perm = nullptr;
    float4* dirs = nullptr;
    double* sf64 = nullptr;   // [R][3] unrotated ray pattern, double
    float *w_irr = nullptr, *inv_s_irr = nullptr, *w_dist = nullptr, *inv_s_dist = nullptr;
    uint8_t* pack_w = nullptr;
    float *inv_irr_r = nullptr, *inv_dist_r = nullptr;
    FrameParams* d_params = nullptr;
    FrameParams* h_params[2]{};
    cudaEvent_t slot_done[2]{};
    bool slot_used[2]{};
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph[2]{};
    GraphKey graph_key[2];
    int64_t updates = 0;
    int trace_mult = 8;
    int blend_probes = 8;
};

namespace {

void cascade_free(ddgi_cascade_s* c) {
    for (int k = 0; k < c->n; ++k) { cudaFree(c->states[k]); cudaFree(c->irr[k]); cudaFree(c->dist[k]); }
    cudaFree(c->lists); cudaFree(c->counts); cudaFree(c->status); cudaFree(c->records);
    cudaFree(c->shadow_list); cudaFree(c->hit_list); cudaFree(c->class_scratch); cudaFree(c->perm); cudaFree(c->dirs);
    cudaFree(c->sf64);
    cudaFree(c->w_irr);
    cudaFree(c->inv_s_irr); cudaFree(c->w_dist); cudaFree(c->inv_s_dist); cudaFree(c->pack_w);
    cudaFree(c->inv_irr_r); cudaFree(c->inv_dist_r); cudaFree(c->d_params);
    for (int s = 0; s < 2; ++s) {
        if (c->h_params[s]) cudaFreeHost(c->h_params[s]);
        if (c->slot_done[s]) cudaEventDestroy(c->slot_done[s]);
        if (c->graph[s]) cudaGraphExecDestroy(c->graph[s]);
    }
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    delete c;
}

// Host side of the tracking window (Sec. 7.2), the same rule as the oracle:
// move by whole planes until the camera is within one spacing of the centre
// on every axis; each move records the physical plane that leapfrogs.
void cascade_scroll(ddgi_cascade_s* c, int k, const float cam[3], FrameParams* fp) {
    const ddgi_volume_desc& d = c->desc[k];
    for (int a = 0; a < 3; ++a) {
        int moves = 0;
        for (;;) {
            double centre = c->origin[k][a] + 0.5 * (double)(d.counts[a] - 1) * (double)d.spacing[a];
            int dir = 0;
            if ((double)cam[a] - centre > (double)d.spacing[a]) dir = 1;
            else if (centre - (double)cam[a] > (double)d.spacing[a]) dir = -1;
            if (!dir) break;
            c->origin[k][a] += dir * (double)d.spacing[a];
            c->shift[k][a] += dir;
            int fresh = dir > 0 ? d.counts[a] - 1 : 0;
            int phys = ((fresh + c->shift[k][a]) % d.counts[a] + d.counts[a]) % d.counts[a];
            if (moves < d.counts[a] && fp->n_planes < kMaxPlanes) fp->planes[fp->n_planes++] = make_int4(k, a, phys, 0);
            ++moves;
        }
    }
}

VolView cascade_view(const ddgi_cascade_s* c, int k, const float cam[3]) {
    const ddgi_volume_desc& d = c->desc[k];
    VolView w{};
    w.origin = make_float3((float)c->origin[k][0], (float)c->origin[k][1], (float)c->origin[k][2]);
    w.spacing = make_float3(d.spacing[0], d.spacing[1], d.spacing[2]);
    w.inv_spacing = make_float3(1.0f / d.spacing[0], 1.0f / d.spacing[1], 1.0f / d.spacing[2]);
    w.counts = make_int3(d.counts[0], d.counts[1], d.counts[2]);
    set_view_divisors(w);
    // reduced to [0, count): the device indexes with one conditional add / subtract
    w.shift = make_int3(((c->shift[k][0] % d.counts[0]) + d.counts[0]) % d.counts[0],
                        ((c->shift[k][1] % d.counts[1]) + d.counts[1]) % d.counts[1],
                        ((c->shift[k][2] % d.counts[2]) + d.counts[2]) % d.counts[2]);
    w.min_spacing = std::fmin(d.spacing[0], std::fmin(d.spacing[1], d.spacing[2]));
    w.bias = d.self_shadow_bias;
    w.gamma = d.gamma;
    w.inv_gamma = 1.0f / d.gamma;
    w.half_gamma = 0.5f * d.gamma;
    w.t_max = c->t_max[k];
    w.irr_n = d.irr_n;
    w.dist_n = d.dist_n;
    w.irr_tile = (d.irr_n + 2) * (d.irr_n + 2);
    w.dist_tile = (d.dist_n + 2) * (d.dist_n + 2);
    w.n_probes = (int32_t)c->P[k];
    w.irr_format = d.irr_format;
    w.dist_format = d.dist_format;
    w.states = c->states[k];
    w.irr = c->irr[k];
    w.dist = c->dist[k];
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        if (d.tracking) {   // tracking: fall-off box tightened by one cell and centred on the camera
            double h = (0.5 * (double)(d.counts[a] - 1) - 1.0) * (double)d.spacing[a];
            lo[a] = (float)((double)cam[a] - h);
            hi[a] = (float)((double)cam[a] + h);
        } else {
            lo[a] = (float)c->origin[k][a];
            hi[a] = (float)(c->origin[k][a] + (double)(d.counts[a] - 1) * (double)d.spacing[a]);
        }
    }
    w.blend_lo = make_float3(lo[0], lo[1], lo[2]);
    w.blend_hi = make_float3(hi[0], hi[1], hi[2]);
    return w;
}

ddgi_status cascade_enqueue(ddgi_cascade_s* c, const DevScene& sc, const Lights& L, const BlendParams& bp,
                            int precision, int slot, cudaStream_t st) {
    const ddgi_volume_desc& d0 = c->desc[0];
    const bool tensor = precision != DDGI_BLEND_FP32;
    int sms = sm_count();
    VolSet vs{};
    vs.table = c->d_params->views;
    vs.n = c->n;
    DDGI_CK(cudaMemcpyAsync(c->d_params, c->h_params[slot], sizeof(FrameParams), cudaMemcpyHostToDevice, st));
    DDGI_CK(launch_reset_planes(vs, c->d_params->planes, &c->d_params->n_planes, kMaxPlanes, st));
    // frame setup; also clears the lists and trace counters
    DDGI_CK(launch_frame_setup_dev(&c->d_params->rot, c->R, d0.irr_n, d0.dist_n, d0.dist_cos_power, c->sf64, c->dirs,
                                   c->w_irr, c->inv_s_irr, c->w_dist, c->inv_s_dist, c->counts, kCounterInts, st));
    if (tensor)
        DDGI_CK(launch_pack_weights(c->w_irr, c->w_dist, c->R, d0.irr_n, d0.dist_n, precision, c->pack_w,
                                    c->inv_irr_r, c->inv_dist_r, st));
    DDGI_CK(launch_build_list_multi(vs, (int)c->total, 0, c->lists, c->counts + 0, st));
    DDGI_CK(launch_classify_multi(sc, vs, c->dirs, c->R, c->perm, c->lists, c->counts + 0, c->class_scratch,
                                  sms * 8, st));
    DDGI_CK(launch_build_list_multi(vs, (int)c->total, 1, c->lists + c->total, c->counts + 1, st));
    DDGI_CK(launch_trace_wavefront_multi(sc, vs, L, c->dirs, c->R, c->perm, c->lists + c->total, c->counts + 1,
                                         c->records, c->shadow_list, c->hit_list, c->shadow_count, sms * c->trace_mult,
                                         st, query_fast_view(c->h_params[slot]->views[0])));
    if (tensor)
        DDGI_CK(launch_blend_tc_set(vs, true, bp, precision, d0.irr_n, d0.dist_n, c->pack_w, c->inv_irr_r,
                                    c->inv_dist_r, c->records, c->lists + c->total, c->counts + 1, c->status, sms, st));
    else
        DDGI_CK(launch_blend_set(vs, true, bp, d0.irr_n, d0.dist_n, c->w_irr, c->inv_s_irr, c->w_dist, c->inv_s_dist,
                                 c->records,
                                 c->lists + c->total, c->counts + 1, c->status, sms * 4, c->blend_probes, st));
    return DDGI_OK;
}

}  // namespace

extern "C" {

ddgi_status ddgi_cascade_create(const ddgi_volume_desc* descs, int32_t n, ddgi_cascade* out) {
    if (!out) return fail(DDGI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!descs || n < 1 || n > kMaxVolumes) return fail(DDGI_ERR_INVALID_ARG, "need 1..8 volume descriptors");
    int64_t all_rays = 0;   // the lists index rays of all volumes with 32-bit ints
    for (int k = 0; k < n; ++k) {
        ddgi_status s = check_desc(&descs[k]);
        if (s != DDGI_OK) return s;
        all_rays += (int64_t)descs[k].counts[0] * descs[k].counts[1] * descs[k].counts[2] * descs[k].rays_per_probe;
        if (all_rays >= (1LL << 31)) return fail(DDGI_ERR_INVALID_ARG, "probes x rays_per_probe must stay below 2^31");
        if (descs[k].optimizer_iters != 0)
            return fail(DDGI_ERR_UNSUPPORTED, "cascades have no probe position optimizer");
        if (descs[k].converge_batches != 0)
            return fail(DDGI_ERR_UNSUPPORTED, "cascades have no converge pass");
        const ddgi_volume_desc &a = descs[0], &b = descs[k];
        if (b.rays_per_probe != a.rays_per_probe || b.irr_n != a.irr_n || b.dist_n != a.dist_n ||
            b.irr_format != a.irr_format || b.dist_format != a.dist_format || b.gamma != a.gamma ||
            b.hysteresis_irr != a.hysteresis_irr || b.hysteresis_vis != a.hysteresis_vis ||
            b.dist_cos_power != a.dist_cos_power || b.thr_low != a.thr_low || b.thr_high != a.thr_high ||
            b.thr_step != a.thr_step)
            return fail(DDGI_ERR_INVALID_ARG,
                        "cascade volumes must share rays, tile sizes, formats, gamma, hysteresis and thresholds");
    }
    ddgi_cascade_s* c = new ddgi_cascade_s();
    c->n = n;
    c->R = descs[0].rays_per_probe;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes > 0 ? bytes : 16);
    };
    for (int k = 0; k < n; ++k) {
        const ddgi_volume_desc& d = descs[k];
        c->desc[k] = d;
        c->P[k] = (int64_t)d.counts[0] * d.counts[1] * d.counts[2];
        c->total += c->P[k];
        double sx = d.spacing[0], sy = d.spacing[1], sz = d.spacing[2];
        c->t_max[k] = d.t_max >= 0.0f ? d.t_max : (float)(2.0 * std::sqrt(sx * sx + sy * sy + sz * sz));
        size_t tb = (size_t)ddgi_texel_bytes(0, d.irr_format);
        size_t db = (size_t)ddgi_texel_bytes(1, d.dist_format);
        c->irr_bytes[k] = (size_t)c->P[k] * (d.irr_n + 2) * (d.irr_n + 2) * tb;
        c->dist_bytes[k] = (size_t)c->P[k] * (d.dist_n + 2) * (d.dist_n + 2) * db;
        for (int a = 0; a < 3; ++a) c->origin[k][a] = d.origin[a];
        A((void**)&c->states[k], (size_t)c->P[k]);
        A(&c->irr[k], c->irr_bytes[k]);
        A(&c->dist[k], c->dist_bytes[k]);
        if (e == cudaSuccess)
            e = cudaMemset(c->states[k], d.state_machine ? DDGI_STATE_UNINIT : DDGI_STATE_VIGILANT, (size_t)c->P[k]);
        if (e == cudaSuccess) e = cudaMemset(c->irr[k], 0, c->irr_bytes[k]);
        if (e == cudaSuccess) e = cudaMemset(c->dist[k], 0, c->dist_bytes[k]);
    }
    if (c->total > (int64_t)kEntryMask) {
        cascade_free(c);
        return fail(DDGI_ERR_INVALID_ARG, "cascade has too many probes");
    }
    const ddgi_volume_desc& d0 = descs[0];
    A((void**)&c->lists, sizeof(int32_t) * 2 * (size_t)c->total);
    A((void**)&c->counts, sizeof(int32_t) * kCounterInts);
    c->shadow_count = c->counts + 4;
    A((void**)&c->status, sizeof(uint32_t));
    A((void**)&c->records, sizeof(float4) * (size_t)c->total * c->R);
    A((void**)&c->shadow_list, sizeof(int32_t) * (size_t)c->total * c->R);
    A((void**)&c->hit_list, sizeof(int32_t) * (size_t)c->total * c->R);
    A((void**)&c->class_scratch, sizeof(int4) * (size_t)c->total);
    if (e == cudaSuccess) e = cudaMemset(c->class_scratch, 0, sizeof(int4) * (size_t)c->total);
    A((void**)&c->dirs, sizeof(float4) * 3 * c->R);
    A((void**)&c->sf64, sizeof(double) * 3 * c->R);
    if (e == cudaSuccess) e = launch_sf_table(c->R, c->sf64, 0);
    A((void**)&c->perm, sizeof(int32_t) * c->R);
    if (e == cudaSuccess) {
        std::vector<int32_t> perm = ray_order_morton(c->R);
        e = cudaMemcpy(c->perm, perm.data(), sizeof(int32_t) * c->R, cudaMemcpyHostToDevice);
    }
    A((void**)&c->w_irr, sizeof(float) * d0.irr_n * d0.irr_n * (size_t)c->R);
    A((void**)&c->inv_s_irr, sizeof(float) * d0.irr_n * d0.irr_n);
    A((void**)&c->w_dist, sizeof(float) * d0.dist_n * d0.dist_n * (size_t)c->R);
    A((void**)&c->inv_s_dist, sizeof(float) * d0.dist_n * d0.dist_n);
    A((void**)&c->pack_w, tc_pack_bytes(c->R));
    A((void**)&c->inv_irr_r, sizeof(float) * 128);
    A((void**)&c->inv_dist_r, sizeof(float) * 256);
    A((void**)&c->d_params, sizeof(FrameParams));
    for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
        e = cudaMallocHost((void**)&c->h_params[s], sizeof(FrameParams));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->slot_done[s], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = prepare_blend_kernels(c->R);
    if (e == cudaSuccess) e = prepare_blend_tc_kernels();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cascade_free(c);
        return fail(e == cudaErrorMemoryAllocation ? DDGI_ERR_OOM : DDGI_ERR_CUDA,
                    std::string("cascade allocation: ") + cudaGetErrorString(e));
    }
    *out = c;
    return DDGI_OK;
}

void ddgi_cascade_destroy(ddgi_cascade c) {
    if (!c) return;
    cudaDeviceSynchronize();
    cascade_free(c);
}

ddgi_status ddgi_cascade_update(ddgi_cascade c, ddgi_scene s, const ddgi_lights* lights,
                                const ddgi_cascade_params* params, ddgi_stream stream) {
    if (!c || !s || !lights || !params) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (!(params->irr_hyst_scale >= 0.0f) || !(params->vis_hyst_scale >= 0.0f))
        return fail(DDGI_ERR_INVALID_ARG, "negative hysteresis scale");
    if (params->blend_precision < DDGI_BLEND_FP32 || params->blend_precision > DDGI_BLEND_TF32X3)
        return fail(DDGI_ERR_INVALID_ARG, "unknown blend precision");
    if (params->blend_precision != DDGI_BLEND_FP32 && !tc_blend_supported(c->desc[0].irr_n, c->desc[0].dist_n))
        return fail(DDGI_ERR_UNSUPPORTED, "tensor-core blend needs irr_n^2 <= 128 and dist_n^2 <= 256");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(params->camera_pos[a])) return fail(DDGI_ERR_INVALID_ARG, "camera not finite");
    cudaStream_t st = (cudaStream_t)stream;
    const int slot = (int)(params->frame & 1);
    // the pinned slot may still be read by the copy of an earlier frame
    if (c->slot_used[slot]) DDGI_CK(cudaEventSynchronize(c->slot_done[slot]));
    FrameParams* fp = c->h_params[slot];
    fp->n_planes = 0;
    for (int k = 0; k < c->n; ++k)
        if (c->desc[k].tracking) cascade_scroll(c, k, params->camera_pos, fp);
    for (int k = 0; k < c->n; ++k) fp->views[k] = cascade_view(c, k, params->camera_pos);
    fp->rot = frame_rotation(c->desc[0].seed, params->frame);

    const ddgi_volume_desc& d0 = c->desc[0];
    BlendParams bp{};
    bp.hyst_irr = std::fmin(1.0f, std::fmax(0.0f, d0.hysteresis_irr * params->irr_hyst_scale));
    bp.hyst_vis = std::fmin(1.0f, std::fmax(0.0f, d0.hysteresis_vis * params->vis_hyst_scale));
    bp.thr_low = d0.thr_low;
    bp.thr_high = d0.thr_high;
    bp.thr_step = d0.thr_step;
    bp.R = c->R;
    Lights L = make_lights(lights);

    if (params->use_graph) {
        GraphKey key;
        key.precision = params->blend_precision;
        key.trace_mult = c->trace_mult;
        key.blend_probes = c->blend_probes;
        key.irr_scale = params->irr_hyst_scale;
        key.vis_scale = params->vis_hyst_scale;
        key.lights = *lights;
        if (!c->graph[slot] || !(c->graph_key[slot] == key)) {
            if (c->graph[slot]) {
                cudaGraphExecDestroy(c->graph[slot]);
                c->graph[slot] = nullptr;
            }
            cudaGraph_t g = nullptr;
            DDGI_CK(cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeRelaxed));
            ddgi_status rs = cascade_enqueue(c, s->dev, L, bp, params->blend_precision, slot, c->capture_stream);
            cudaError_t ce = cudaStreamEndCapture(c->capture_stream, &g);
            if (rs != DDGI_OK) {
                if (g) cudaGraphDestroy(g);
                return rs;
            }
            if (ce != cudaSuccess) return fail(DDGI_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&c->graph[slot], g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) return fail(DDGI_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
            c->graph_key[slot] = key;
        }
        DDGI_CK(cudaGraphLaunch(c->graph[slot], st));
    } else {
        ddgi_status rs = cascade_enqueue(c, s->dev, L, bp, params->blend_precision, slot, st);
        if (rs != DDGI_OK) return rs;
    }
    DDGI_CK(cudaEventRecord(c->slot_done[slot], st));
    c->slot_used[slot] = true;
    c->updates++;
    return DDGI_OK;
}

ddgi_status ddgi_cascade_query(ddgi_cascade c, const float* pos_dev, const float* nrm_dev, int64_t n,
                               const float camera_pos[3], float* out_dev, ddgi_stream stream) {
    if (!c || !camera_pos) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (c->updates == 0) return fail(DDGI_ERR_INVALID_ARG, "no cascade update has run");
    if (n < 0) return fail(DDGI_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return DDGI_OK;
    if (!pos_dev || !nrm_dev || !out_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL buffer");
    if (!dev16(pos_dev) || !dev16(nrm_dev) || !dev16(out_dev)) return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
    VolSet vs{};
    vs.table = c->d_params->views;
    vs.n = c->n;
    DDGI_CK(launch_query_cascade(vs, pos_dev, nrm_dev, n, make_float3(camera_pos[0], camera_pos[1], camera_pos[2]),
                                 out_dev, (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_cascade_get_buffer(ddgi_cascade c, int32_t vol, int32_t which, void* dst_dev, size_t bytes,
                                    ddgi_stream stream) {
    if (!c || !dst_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (!dev16(dst_dev)) return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
    if (vol < 0 || vol >= c->n) return fail(DDGI_ERR_INVALID_ARG, "volume index out of range");
    void* p;
    size_t nb;
    if (which == 0) { p = c->irr[vol]; nb = c->irr_bytes[vol]; }
    else if (which == 1) { p = c->dist[vol]; nb = c->dist_bytes[vol]; }
    else if (which == 2) { p = c->states[vol]; nb = (size_t)c->P[vol]; }
    else return fail(DDGI_ERR_INVALID_ARG, "which must be 0, 1 or 2");
    if (bytes != nb) return fail(DDGI_ERR_INVALID_ARG, "size mismatch: expected " + std::to_string(nb));
    DDGI_CK(cudaMemcpyAsync(dst_dev, p, nb, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_cascade_get_ray_records(ddgi_cascade c, float* records_dev, int32_t* entries_dev,
                                         int64_t* n_active, ddgi_stream stream) {
    if (!c || !records_dev || !entries_dev || !n_active) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (!dev16(records_dev) || !dev16(entries_dev)) return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
    if (c->updates == 0) return fail(DDGI_ERR_INVALID_ARG, "no update has run on this cascade");
    cudaStream_t st = (cudaStream_t)stream;
    int32_t cnt = 0;
    DDGI_CK(cudaMemcpyAsync(&cnt, c->counts + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    DDGI_CK(cudaStreamSynchronize(st));
    *n_active = cnt;
    if (cnt > 0) {
        DDGI_CK(cudaMemcpyAsync(records_dev, c->records, sizeof(float4) * (size_t)cnt * c->R,
                                cudaMemcpyDeviceToDevice, st));
        DDGI_CK(cudaMemcpyAsync(entries_dev, c->lists + c->total, sizeof(int32_t) * (size_t)cnt,
                                cudaMemcpyDeviceToDevice, st));
    }
    return DDGI_OK;
}

ddgi_status ddgi_cascade_get_window(ddgi_cascade c, int32_t vol, double origin[3], int32_t shift[3]) {
    if (!c || !origin || !shift) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (vol < 0 || vol >= c->n) return fail(DDGI_ERR_INVALID_ARG, "volume index out of range");
    for (int a = 0; a < 3; ++a) {
        origin[a] = c->origin[vol][a];
        shift[a] = c->shift[vol][a];
    }
    return DDGI_OK;
}

ddgi_status ddgi_cascade_set_tuning(ddgi_cascade c, int32_t trace_blocks_per_sm, int32_t blend_probes_per_cta) {
    if (!c) return fail(DDGI_ERR_INVALID_ARG, "cascade is NULL");
    if (trace_blocks_per_sm < 1 || trace_blocks_per_sm > 32)
        return fail(DDGI_ERR_INVALID_ARG, "trace_blocks_per_sm must be in [1, 32]");
    if (blend_probes_per_cta != 4 && blend_probes_per_cta != 8 && blend_probes_per_cta != 16)
        return fail(DDGI_ERR_INVALID_ARG, "blend_probes_per_cta must be 4, 8 or 16");
    c->trace_mult = trace_blocks_per_sm;
    c->blend_probes = blend_probes_per_cta;
    return DDGI_OK;
}

ddgi_status ddgi_cascade_get_tuning(ddgi_cascade c, int32_t* trace_blocks_per_sm, int32_t* blend_probes_per_cta) {
    if (!c || !trace_blocks_per_sm || !blend_probes_per_cta) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    *trace_blocks_per_sm = c->trace_mult;
    *blend_probes_per_cta = c->blend_probes;
    return DDGI_OK;
}

ddgi_status ddgi_cascade_poll_status(ddgi_cascade c, ddgi_stream stream) {
    if (!c) return fail(DDGI_ERR_INVALID_ARG, "cascade is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t w = 0;
    DDGI_CK(cudaMemcpyAsync(&w, c->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    DDGI_CK(cudaMemsetAsync(c->status, 0, sizeof(uint32_t), st));
    DDGI_CK(cudaStreamSynchronize(st));
    if (w & 2u) return fail(DDGI_ERR_TIMEOUT, "a bounded device wait gave up");
    if (w & 1u) return fail(DDGI_ERR_NUMERIC, "non-finite texel value produced");
    return DDGI_OK;
}

// Autotuner: times the cascade update under each candidate launch shape
// (trace blocks per SM x SIMT blend probes per CTA) and keeps the fastest.
// Results are cached in a small JSON file keyed by GPU name and workload
// signature; a cached entry is used without timing.  Timing advances the
// volumes by the frames it runs (all with params->frame's ray pattern).
ddgi_status ddgi_cascade_autotune(ddgi_cascade c, ddgi_scene s, const ddgi_lights* lights,
                                  const ddgi_cascade_params* params, const char* cache_path, int32_t* from_cache,
                                  ddgi_stream stream) {
    if (!c || !s || !lights || !params) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaDeviceProp prop{};
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::ostringstream key;
    key << prop.name << "|n=" << c->n << "|P=" << c->total << "|R=" << c->R << "|tris=" << s->n_tris
        << "|prec=" << params->blend_precision;
    std::string k = key.str();
    std::string cache;
    if (cache_path) {
        std::ifstream f(cache_path);
        if (f) { std::stringstream ss; ss << f.rdbuf(); cache = ss.str(); }
        size_t at = cache.find("\"" + k + "\"");
        if (at != std::string::npos) {
            int tm = 0, bp = 0;
            size_t a = cache.find("\"trace_blocks_per_sm\":", at), b = cache.find("\"blend_probes_per_cta\":", at);
            if (a != std::string::npos && b != std::string::npos) {
                tm = std::atoi(cache.c_str() + a + 22);
                bp = std::atoi(cache.c_str() + b + 23);
                if (ddgi_cascade_set_tuning(c, tm, bp) == DDGI_OK) {
                    if (from_cache) *from_cache = 1;
                    return DDGI_OK;
                }
            }
        }
    }
    const int trace_opts[] = {2, 4, 8, 16};
    const int blend_opts[] = {4, 8, 16};
    ddgi_cascade_params p = *params;
    p.use_graph = 0;
    // one untimed frame: classification and first allocations of work
    ddgi_status r = ddgi_cascade_update(c, s, lights, &p, stream);
    if (r != DDGI_OK) return r;
    cudaEvent_t e0, e1;
    DDGI_CK(cudaEventCreate(&e0));
    DDGI_CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_t = c->trace_mult, best_b = c->blend_probes;
    for (int tmul : trace_opts) {
        for (int bpp : blend_opts) {
            if (params->blend_precision != DDGI_BLEND_FP32 && bpp != 8) continue;   // tensor blend: fixed tiles
            c->trace_mult = tmul;
            c->blend_probes = bpp;
            float tot = 0.0f;
            for (int rep = 0; rep < 2; ++rep) {
                DDGI_CK(cudaEventRecord(e0, st));
                r = ddgi_cascade_update(c, s, lights, &p, stream);
                if (r != DDGI_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return r; }
                DDGI_CK(cudaEventRecord(e1, st));
                DDGI_CK(cudaEventSynchronize(e1));
                float ms = 0.0f;
                DDGI_CK(cudaEventElapsedTime(&ms, e0, e1));
                tot += ms;
            }
            if (tot < best) { best = tot; best_t = tmul; best_b = bpp; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->trace_mult = best_t;
    c->blend_probes = best_b;
    if (from_cache) *from_cache = 0;
    if (cache_path) {
        std::ostringstream entry;
        entry << "\"" << k << "\": {\"trace_blocks_per_sm\": " << best_t << ", \"blend_probes_per_cta\": " << best_b
              << ", \"ms\": " << best / 2.0f << "}";
        std::string body;
        size_t l = cache.find('{'), rb = cache.rfind('}');
        if (l != std::string::npos && rb != std::string::npos && rb > l) {
            std::string inner = cache.substr(l + 1, rb - l - 1);
            bool empty = inner.find_first_not_of(" \n\t\r") == std::string::npos;
            body = "{" + inner + (empty ? "" : ",\n ") + entry.str() + "}\n";
        } else {
            body = "{\n " + entry.str() + "}\n";
        }
        std::ofstream f(cache_path);
        if (f) f << body;
    }
    return DDGI_OK;
}

}  // extern "C"


// ===========================================================================
// Differentiation: forward through n frames of the update from a zero atlas
// (hysteresis 0, every probe tracing) and the query; reverse pass to the
// emitters' radiance and the objects' albedo.  Geometry is fixed.
// ===========================================================================

namespace ddgi {
cudaError_t launch_query_adjoint(const VolView& v, const float* pos, const float* nrm, int64_t n, float3 cam,
                                 const float* dE, float* g_irr, cudaStream_t st);
cudaError_t launch_border_fold(float* g_irr, int P, int n, cudaStream_t st);
cudaError_t launch_blend_adjoint(const VolView& v_after, const float* w_irr, const float* inv_s, const float* g_irr,
                                 int P, int R, float4* gL, cudaStream_t st);
cudaError_t launch_shade_adjoint(const DevScene& s, const VolView& v_before, const Lights& L, const float4* dirs,
                                 int P, int R, const float4* gL, float* d_emit, float* d_albedo, float* g_prev,
                                 int with_prev, cudaStream_t st);
cudaError_t launch_set_materials(float4* albedo, int n_obj, const float* alb, float4* emit, int n_em, const float* em,
                                 cudaStream_t st);
}  // namespace ddgi

static ddgi_status diff_check(ddgi_volume v, int32_t n_frames) {
    const ddgi_volume_desc& d = v->desc;
    if (n_frames < 1 || n_frames > 8) return fail(DDGI_ERR_INVALID_ARG, "n_frames must be in [1, 8]");
    if (d.hysteresis_irr != 0.0f || d.hysteresis_vis != 0.0f || d.state_machine != 0 ||
        d.irr_format != DDGI_IRR_FP32 || d.dist_format != DDGI_DIST_FP32)
        return fail(DDGI_ERR_UNSUPPORTED,
                    "differentiation needs hysteresis 0, the state machine off and FP32 atlases");
    return DDGI_OK;
}

extern "C" {

ddgi_status ddgi_scene_set_materials(ddgi_scene s, const float* albedo_dev, const float* emit_dev,
                                     ddgi_stream stream) {
    if (!s) return fail(DDGI_ERR_INVALID_ARG, "scene is NULL");
    if (!dev16(albedo_dev) || !dev16(emit_dev)) return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
    DDGI_CK(launch_set_materials(s->albedo, albedo_dev ? s->n_objects : 0, albedo_dev, s->emit,
                                 emit_dev ? s->n_emitters : 0, emit_dev, (cudaStream_t)stream));
    return DDGI_OK;
}

ddgi_status ddgi_diff_forward(ddgi_volume v, ddgi_scene s, const ddgi_lights* lights, int64_t first_frame,
                              int32_t n_frames, const float* pos_dev, const float* nrm_dev, int64_t n,
                              const float camera_pos[3], float* out_dev, ddgi_stream stream) {
    if (!v || !s || !lights || !camera_pos) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (!dev16(pos_dev) || !dev16(nrm_dev) || !dev16(out_dev)) return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
    ddgi_status r = diff_check(v, n_frames);
    if (r != DDGI_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    while ((int)v->snap_irr.size() < n_frames + 1) {
        void *a = nullptr, *b = nullptr;
        DDGI_CK(cudaMalloc(&a, v->irr_bytes));
        DDGI_CK(cudaMalloc(&b, v->dist_bytes));
        v->snap_irr.push_back(a);
        v->snap_dist.push_back(b);
    }
    DDGI_CK(cudaMemsetAsync(v->irr, 0, v->irr_bytes, st));
    DDGI_CK(cudaMemsetAsync(v->dist, 0, v->dist_bytes, st));
    DDGI_CK(cudaMemsetAsync(v->states, DDGI_STATE_VIGILANT, (size_t)v->P, st));
    v->list_begin = v->list_end = -1;   // every probe active now: rebuild the list
    DDGI_CK(cudaMemsetAsync(v->snap_irr[0], 0, v->irr_bytes, st));
    DDGI_CK(cudaMemsetAsync(v->snap_dist[0], 0, v->dist_bytes, st));
    for (int f = 0; f < n_frames; ++f) {
        ddgi_update_params p{};
        p.frame = first_frame + f;
        p.irr_hyst_scale = 1.0f;
        p.vis_hyst_scale = 1.0f;
        p.blend_precision = DDGI_BLEND_FP32;
        r = ddgi_update(v, s, lights, &p, stream);
        if (r != DDGI_OK) return r;
        DDGI_CK(cudaMemcpyAsync(v->snap_irr[f + 1], v->irr, v->irr_bytes, cudaMemcpyDeviceToDevice, st));
        DDGI_CK(cudaMemcpyAsync(v->snap_dist[f + 1], v->dist, v->dist_bytes, cudaMemcpyDeviceToDevice, st));
    }
    return ddgi_query(v, pos_dev, nrm_dev, n, camera_pos, out_dev, stream);
}

ddgi_status ddgi_diff_backward(ddgi_volume v, ddgi_scene s, const ddgi_lights* lights, int64_t first_frame,
                               int32_t n_frames, const float* pos_dev, const float* nrm_dev, int64_t n,
                               const float camera_pos[3], const float* dE_dev, float* d_albedo_dev,
                               float* d_emit_dev, ddgi_stream stream) {
    if (!v || !s || !lights || !camera_pos || !d_albedo_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (s->n_emitters > 0 && !d_emit_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL emitter gradient");
    if (n > 0 && (!pos_dev || !nrm_dev || !dE_dev)) return fail(DDGI_ERR_INVALID_ARG, "NULL buffer");
    if (!dev16(pos_dev) || !dev16(nrm_dev) || !dev16(dE_dev) || !dev16(d_albedo_dev) || !dev16(d_emit_dev))
        return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
    ddgi_status r = diff_check(v, n_frames);
    if (r != DDGI_OK) return r;
    if ((int)v->snap_irr.size() < n_frames + 1)
        return fail(DDGI_ERR_INVALID_ARG, "ddgi_diff_forward with these frames has not run");
    cudaStream_t st = (cudaStream_t)stream;
    const ddgi_volume_desc& d = v->desc;
    size_t gbytes = (size_t)v->P * (d.irr_n + 2) * (d.irr_n + 2) * 3 * sizeof(float);
    if (!v->g_irr) DDGI_CK(cudaMalloc((void**)&v->g_irr, gbytes));
    if (!v->g_prev) DDGI_CK(cudaMalloc((void**)&v->g_prev, gbytes));
    DDGI_CK(cudaMemsetAsync(v->g_irr, 0, gbytes, st));
    DDGI_CK(cudaMemsetAsync(d_albedo_dev, 0, sizeof(float) * 3 * (size_t)s->n_objects, st));
    if (s->n_emitters > 0) DDGI_CK(cudaMemsetAsync(d_emit_dev, 0, sizeof(float) * 3 * (size_t)s->n_emitters, st));
    auto snap_view = [&](int k) {
        VolView w = make_view(v);
        w.irr = v->snap_irr[k];
        w.dist = v->snap_dist[k];
        return w;
    };
    Lights L = make_lights(lights);
    float3 cam = make_float3(camera_pos[0], camera_pos[1], camera_pos[2]);
    DDGI_CK(launch_query_adjoint(snap_view(n_frames), pos_dev, nrm_dev, n, cam, dE_dev, v->g_irr, st));
    float* g = v->g_irr;
    float* gp = v->g_prev;
    for (int f = n_frames - 1; f >= 0; --f) {
        DDGI_CK(launch_border_fold(g, (int)v->P, d.irr_n, st));
        FrameRot rot = frame_rotation(d.seed, first_frame + f);
        DDGI_CK(launch_frame_setup(rot, v->R, d.irr_n, d.dist_n, d.dist_cos_power, v->sf64, v->dirs, v->w_irr,
                                   v->inv_s_irr, v->w_dist, v->inv_s_dist, nullptr, 0, st));
        DDGI_CK(launch_blend_adjoint(snap_view(f + 1), v->w_irr, v->inv_s_irr, g, (int)v->P, v->R, v->records, st));
        DDGI_CK(cudaMemsetAsync(gp, 0, gbytes, st));
        DDGI_CK(launch_shade_adjoint(s->dev, snap_view(f), L, v->dirs, (int)v->P, v->R, v->records, d_emit_dev,
                                     d_albedo_dev, gp, f > 0, st));
        float* t = g;
        g = gp;
        gp = t;
    }
    return DDGI_OK;
}

static Diff64Volume diff64_volume(const ddgi_volume_s* v) {
    const ddgi_volume_desc& d = v->desc;
    Diff64Volume dv{};
    for (int a = 0; a < 3; ++a) {
        dv.origin[a] = d.origin[a];
        dv.spacing[a] = d.spacing[a];
        dv.counts[a] = d.counts[a];
    }
    dv.R = v->R;
    dv.irr_n = d.irr_n;
    dv.dist_n = d.dist_n;
    dv.bias = d.self_shadow_bias;
    dv.gamma = d.gamma;
    dv.t_max = v->t_max;
    dv.cos_power = d.dist_cos_power;
    return dv;
}

static size_t irr64_bytes(const ddgi_volume_s* v) {
    return sizeof(double) * 3 * (size_t)(v->desc.irr_n + 2) * (v->desc.irr_n + 2) * (size_t)v->P;
}
static size_t dist64_bytes(const ddgi_volume_s* v) {
    return sizeof(double) * 2 * (size_t)(v->desc.dist_n + 2) * (v->desc.dist_n + 2) * (size_t)v->P;
}

ddgi_status ddgi_diff_forward_f64(ddgi_volume v, ddgi_scene s, const ddgi_lights* lights, int64_t first_frame,
                                  int32_t n_frames, const double* albedo_dev, const double* emit_dev,
                                  const float* pos_dev, const float* nrm_dev, int64_t n, const float camera_pos[3],
                                  double* out_dev, ddgi_stream stream) {
    if (!v || !s || !lights || !camera_pos || !albedo_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (s->n_emitters > 0 && !emit_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL emitter radiance");
    if (n < 0) return fail(DDGI_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!pos_dev || !nrm_dev || !out_dev)) return fail(DDGI_ERR_INVALID_ARG, "NULL buffer");
    if (!dev16(albedo_dev) || !dev16(emit_dev) || !dev16(pos_dev) || !dev16(nrm_dev) || !dev16(out_dev))
        return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
    if (v->desc.optimizer_iters != 0) return fail(DDGI_ERR_UNSUPPORTED, "no probe offsets in the FP64 path");
    ddgi_status r = diff_check(v, n_frames);
    if (r != DDGI_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    while ((int)v->snap64_irr.size() < n_frames + 1) {
        double *a = nullptr, *b = nullptr;
        DDGI_CK(cudaMalloc(&a, irr64_bytes(v)));
        DDGI_CK(cudaMalloc(&b, dist64_bytes(v)));
        v->snap64_irr.push_back(a);
        v->snap64_dist.push_back(b);
    }
    if (!v->rec64) DDGI_CK(cudaMalloc(&v->rec64, sizeof(double) * 4 * (size_t)v->P * v->R));
    const Diff64Volume dv = diff64_volume(v);
    const ddgi_volume_desc& d = v->desc;
    const Lights L = make_lights(lights);
    DDGI_CK(cudaMemsetAsync(v->snap64_irr[0], 0, irr64_bytes(v), st));
    DDGI_CK(cudaMemsetAsync(v->snap64_dist[0], 0, dist64_bytes(v), st));
    for (int f = 0; f < n_frames; ++f) {
        DDGI_CK(launch_frame_dirs(frame_rotation(d.seed, first_frame + f), v->R, d.irr_n, d.dist_n, v->sf64, v->dirs,
                                  st));
        // a texel no ray reaches keeps its value: start from the previous atlas
        DDGI_CK(cudaMemcpyAsync(v->snap64_irr[f + 1], v->snap64_irr[f], irr64_bytes(v), cudaMemcpyDeviceToDevice, st));
        DDGI_CK(cudaMemcpyAsync(v->snap64_dist[f + 1], v->snap64_dist[f], dist64_bytes(v), cudaMemcpyDeviceToDevice,
                                st));
        DDGI_CK(launch_diff64_frame(dv, s->dev, L, v->dirs, albedo_dev, emit_dev, v->snap64_irr[f],
                                    v->snap64_dist[f], f > 0, v->rec64, v->snap64_irr[f + 1], v->snap64_dist[f + 1],
                                    st));
    }
    return launch_diff64_query(dv, v->snap64_irr[n_frames], v->snap64_dist[n_frames], pos_dev, nrm_dev, n,
                               make_float3(camera_pos[0], camera_pos[1], camera_pos[2]), out_dev, st) == cudaSuccess
               ? DDGI_OK
               : fail(DDGI_ERR_CUDA, "FP64 query launch failed");
}

ddgi_status ddgi_diff_backward_f64(ddgi_volume v, ddgi_scene s, const ddgi_lights* lights, int64_t first_frame,
                                   int32_t n_frames, const double* albedo_dev, const float* pos_dev,
                                   const float* nrm_dev, int64_t n, const float camera_pos[3], const double* dE_dev,
                                   double* d_albedo_dev, double* d_emit_dev, ddgi_stream stream) {
    if (!v || !s || !lights || !camera_pos || !albedo_dev || !d_albedo_dev)
        return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (s->n_emitters > 0 && !d_emit_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL emitter gradient");
    if (n > 0 && (!pos_dev || !nrm_dev || !dE_dev)) return fail(DDGI_ERR_INVALID_ARG, "NULL buffer");
    if (!dev16(albedo_dev) || !dev16(pos_dev) || !dev16(nrm_dev) || !dev16(dE_dev) || !dev16(d_albedo_dev) ||
        !dev16(d_emit_dev))
        return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
    ddgi_status r = diff_check(v, n_frames);
    if (r != DDGI_OK) return r;
    if ((int)v->snap64_irr.size() < n_frames + 1 || !v->rec64)
        return fail(DDGI_ERR_INVALID_ARG, "ddgi_diff_forward_f64 with these frames has not run");
    cudaStream_t st = (cudaStream_t)stream;
    if (!v->g64) DDGI_CK(cudaMalloc(&v->g64, irr64_bytes(v)));
    if (!v->g64_prev) DDGI_CK(cudaMalloc(&v->g64_prev, irr64_bytes(v)));
    if (!v->gL64) DDGI_CK(cudaMalloc(&v->gL64, sizeof(double) * 4 * (size_t)v->P * v->R));
    if (!v->sw64) DDGI_CK(cudaMalloc(&v->sw64, sizeof(double) * 128));
    const Diff64Volume dv = diff64_volume(v);
    const ddgi_volume_desc& d = v->desc;
    const Lights L = make_lights(lights);
    DDGI_CK(cudaMemsetAsync(v->g64, 0, irr64_bytes(v), st));
    DDGI_CK(cudaMemsetAsync(d_albedo_dev, 0, sizeof(double) * 3 * (size_t)s->n_objects, st));
    if (s->n_emitters > 0) DDGI_CK(cudaMemsetAsync(d_emit_dev, 0, sizeof(double) * 3 * (size_t)s->n_emitters, st));
    const float3 cam = make_float3(camera_pos[0], camera_pos[1], camera_pos[2]);
    DDGI_CK(launch_diff64_query_adjoint(dv, v->snap64_irr[n_frames], v->snap64_dist[n_frames], pos_dev, nrm_dev, n,
                                        cam, dE_dev, v->g64, st));
    double* g = v->g64;
    double* gp = v->g64_prev;
    for (int f = n_frames - 1; f >= 0; --f) {
        DDGI_CK(launch_frame_dirs(frame_rotation(d.seed, first_frame + f), v->R, d.irr_n, d.dist_n, v->sf64, v->dirs,
                                  st));
        DDGI_CK(cudaMemsetAsync(gp, 0, irr64_bytes(v), st));
        DDGI_CK(launch_diff64_frame_adjoint(dv, s->dev, L, v->dirs, albedo_dev, v->snap64_irr[f], v->snap64_dist[f],
                                            v->snap64_irr[f + 1], f > 0, v->sw64, g, v->gL64, d_emit_dev,
                                            d_albedo_dev, gp, st));
        std::swap(g, gp);
    }
    return DDGI_OK;
}

ddgi_status ddgi_query_backward(ddgi_volume v, const float* pos_dev, const float* nrm_dev, int64_t n,
                                const float camera_pos[3], const float* dE_dev, int32_t fold_borders,
                                float* g_irr_dev, ddgi_stream stream) {
    if (!v || !camera_pos || !g_irr_dev) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (n < 0) return fail(DDGI_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!pos_dev || !nrm_dev || !dE_dev)) return fail(DDGI_ERR_INVALID_ARG, "NULL buffer");
    if (!dev16(pos_dev) || !dev16(nrm_dev) || !dev16(dE_dev) || !dev16(g_irr_dev))
        return fail(DDGI_ERR_INVALID_ARG, kMisaligned);
    const ddgi_volume_desc& d = v->desc;
    const int N = d.irr_n + 2;
    cudaStream_t st = (cudaStream_t)stream;
    DDGI_CK(cudaMemsetAsync(g_irr_dev, 0, sizeof(float) * 3 * (size_t)N * N * (size_t)v->P, st));
    if (n > 0)
        DDGI_CK(launch_query_adjoint(make_view(v), pos_dev, nrm_dev, n,
                                     make_float3(camera_pos[0], camera_pos[1], camera_pos[2]), dE_dev, g_irr_dev,
                                     st));
    if (fold_borders) DDGI_CK(launch_border_fold(g_irr_dev, (int)v->P, d.irr_n, st));
    return DDGI_OK;
}

// ---------------------------------------------------------------------------
// Volume save / load: a versioned host blob (header, then states, atlases and
// probe offsets as stored on the device), guarded by an FNV-1a checksum.
// ---------------------------------------------------------------------------

namespace {

constexpr char kBlobMagic[8] = {'D', 'D', 'G', 'I', 'V', 'O', 'L', '1'};
constexpr uint32_t kBlobVersion = 1;

struct BlobHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;          // sizeof(BlobHeader)
    uint32_t desc_bytes;            // sizeof(ddgi_volume_desc)
    uint32_t reserved;
    ddgi_volume_desc desc;          // the descriptor of the saved volume
    int64_t n_probes;
    int64_t states_bytes, irr_bytes, dist_bytes, offsets_bytes;
    int64_t updates;                // updates run on the volume before the save
    uint64_t checksum;              // FNV-1a over the payload that follows the header
};

uint64_t fnv1a(const uint8_t* p, size_t n, uint64_t h = 1469598103934665603ull) {
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

size_t blob_bytes(const ddgi_volume_s* v) {
    return sizeof(BlobHeader) + (size_t)v->P + v->irr_bytes + v->dist_bytes + sizeof(float4) * (size_t)v->P;
}

// The descriptor fields that fix what the stored bytes mean: the grid and
// its placement, tile sizes, storage formats and the gamma encoding.
bool blob_compatible(const ddgi_volume_desc& a, const ddgi_volume_desc& b, std::string* why) {
    for (int k = 0; k < 3; ++k) {
        if (a.counts[k] != b.counts[k]) { *why = "probe counts differ"; return false; }
        if (a.origin[k] != b.origin[k] || a.spacing[k] != b.spacing[k]) { *why = "grid placement differs"; return false; }
    }
    if (a.irr_n != b.irr_n || a.dist_n != b.dist_n) { *why = "tile sizes differ"; return false; }
    if (a.irr_format != b.irr_format || a.dist_format != b.dist_format) { *why = "storage formats differ"; return false; }
    if (a.gamma != b.gamma) { *why = "gamma encodings differ"; return false; }
    return true;
}

}  // namespace

ddgi_status ddgi_volume_save(ddgi_volume v, void* host_buf, size_t* bytes, ddgi_stream stream) {
    if (!v || !bytes) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    const size_t need = blob_bytes(v);
    if (!host_buf) {
        *bytes = need;
        return DDGI_OK;
    }
    if (*bytes < need) {
        *bytes = need;
        return fail(DDGI_ERR_INVALID_ARG, "buffer too small: " + std::to_string(need) + " bytes needed");
    }
    BlobHeader h{};
    std::memcpy(h.magic, kBlobMagic, sizeof(kBlobMagic));
    h.version = kBlobVersion;
    h.header_bytes = sizeof(BlobHeader);
    h.desc_bytes = sizeof(ddgi_volume_desc);
    h.desc = v->desc;
    h.n_probes = v->P;
    h.states_bytes = v->P;
    h.irr_bytes = (int64_t)v->irr_bytes;
    h.dist_bytes = (int64_t)v->dist_bytes;
    h.offsets_bytes = (int64_t)(sizeof(float4) * (size_t)v->P);
    h.updates = v->updates;
    uint8_t* out = (uint8_t*)host_buf + sizeof(BlobHeader);
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t* q = out;
    DDGI_CK(cudaMemcpyAsync(q, v->states, (size_t)h.states_bytes, cudaMemcpyDeviceToHost, st));
    q += h.states_bytes;
    DDGI_CK(cudaMemcpyAsync(q, v->irr, (size_t)h.irr_bytes, cudaMemcpyDeviceToHost, st));
    q += h.irr_bytes;
    DDGI_CK(cudaMemcpyAsync(q, v->dist, (size_t)h.dist_bytes, cudaMemcpyDeviceToHost, st));
    q += h.dist_bytes;
    DDGI_CK(cudaMemcpyAsync(q, v->offsets, (size_t)h.offsets_bytes, cudaMemcpyDeviceToHost, st));
    DDGI_CK(cudaStreamSynchronize(st));
    h.checksum = fnv1a(out, need - sizeof(BlobHeader));
    std::memcpy(host_buf, &h, sizeof(BlobHeader));
    *bytes = need;
    return DDGI_OK;
}

ddgi_status ddgi_volume_load(ddgi_volume v, const void* host_buf, size_t bytes, ddgi_stream stream) {
    if (!v || !host_buf) return fail(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (bytes < sizeof(BlobHeader)) return fail(DDGI_ERR_INVALID_ARG, "blob shorter than its header");
    BlobHeader h;
    std::memcpy(&h, host_buf, sizeof(BlobHeader));
    if (std::memcmp(h.magic, kBlobMagic, sizeof(kBlobMagic)) != 0) return fail(DDGI_ERR_INVALID_ARG, "not a volume blob");
    if (h.version != kBlobVersion) return fail(DDGI_ERR_UNSUPPORTED, "blob version " + std::to_string(h.version));
    if (h.header_bytes != sizeof(BlobHeader) || h.desc_bytes != sizeof(ddgi_volume_desc))
        return fail(DDGI_ERR_INVALID_ARG, "blob header layout differs from this library's");
    std::string why;
    if (!blob_compatible(h.desc, v->desc, &why)) return fail(DDGI_ERR_INVALID_ARG, "blob does not fit the volume: " + why);
    if (h.n_probes != v->P || h.states_bytes != v->P || h.irr_bytes != (int64_t)v->irr_bytes ||
        h.dist_bytes != (int64_t)v->dist_bytes || h.offsets_bytes != (int64_t)(sizeof(float4) * (size_t)v->P))
        return fail(DDGI_ERR_INVALID_ARG, "blob sizes do not fit the volume");
    const size_t need = blob_bytes(v);
    if (bytes != need) return fail(DDGI_ERR_INVALID_ARG, "blob size " + std::to_string(bytes) + ", expected " +
                                                             std::to_string(need));
    const uint8_t* in = (const uint8_t*)host_buf + sizeof(BlobHeader);
    if (fnv1a(in, need - sizeof(BlobHeader)) != h.checksum) return fail(DDGI_ERR_INVALID_ARG, "blob checksum mismatch");
    cudaStream_t st = (cudaStream_t)stream;
    const uint8_t* q = in;
    DDGI_CK(cudaMemcpyAsync(v->states, q, (size_t)h.states_bytes, cudaMemcpyHostToDevice, st));
    q += h.states_bytes;
    DDGI_CK(cudaMemcpyAsync(v->irr, q, (size_t)h.irr_bytes, cudaMemcpyHostToDevice, st));
    q += h.irr_bytes;
    DDGI_CK(cudaMemcpyAsync(v->dist, q, (size_t)h.dist_bytes, cudaMemcpyHostToDevice, st));
    q += h.dist_bytes;
    DDGI_CK(cudaMemcpyAsync(v->offsets, q, (size_t)h.offsets_bytes, cudaMemcpyHostToDevice, st));
    // the host buffer may be released once the call returns
    DDGI_CK(cudaStreamSynchronize(st));
    v->updates = h.updates;
    v->uninit_possible = true;      // the loaded states decide; the next update rebuilds its lists
    v->awake_possible = true;
    v->list_begin = v->list_end = -1;
    return DDGI_OK;
}

}  // extern "C"
