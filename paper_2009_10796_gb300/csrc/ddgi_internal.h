// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "ddgi.h"

namespace ddgi {

// ---------------------------------------------------------------------------
// Scene on the device.
//   nodes: 4 float4 per BVH2 node:
//     [0] child0 (lo.x, hi.x, lo.y, hi.y)  [1] child1 (lo.x, hi.x, lo.y, hi.y)
//     [2] (c0 lo.z, c0 hi.z, c1 lo.z, c1 hi.z)
//     [3] int bits (child0, child1, count0, count1); child >= 0 is an inner
//         node, child < 0 a leaf whose triangles start at ~child.
//   tris: 3 float4 per triangle in BVH order:
//     v0 (w = original index bits), v1 (w = flags bits: bit0 casts shadow), v2.
//   attr: per original triangle (object, emitter).
// ---------------------------------------------------------------------------
struct DevScene {
    const float4* nodes;     // binary hierarchy, 4 float4 per node
    const float4* nodes4;    // the same collapsed to 4-wide nodes, 8 float4 per node
    const float4* tris;
    const int2*   attr;
    const float4* albedo;    // per object (r, g, b, flags bits)
    const float4* emit;      // per emitter (r, g, b, 0)
    int32_t n_nodes;
    int32_t n_nodes4;
    int32_t n_tris;
};

struct Lights {
    float3 sun_dir, sun_irr, sky_a, sky_b, sky_up;
    int32_t sun_on;
};

// Volume view passed by value to kernels.
// Division by an invariant divisor d >= 1 of dividends below 2^31
// (Granlund and Montgomery, PLDI 1994, Sec. 4): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(m, n) + n) >> l; the
// sum stays below 2^32 for such n.
struct FastDiv {
    uint32_t m;
    int32_t l;
};

inline FastDiv make_fast_div(uint32_t d) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    FastDiv f;
    f.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
    f.l = l;
    return f;
}

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t fast_div(uint32_t n, FastDiv f) { return (__umulhi(f.m, n) + n) >> f.l; }
#endif

struct VolView {
    float3 origin;
    float3 spacing;
    float3 inv_spacing;
    int3   counts;
    int3   shift;           // circular window shift, each component in [0, count)
    float  min_spacing;
    float  bias;            // self-shadow bias B
    float  gamma;
    float  inv_gamma;
    float  half_gamma;
    float  t_max;
    int32_t irr_n, dist_n;
    int32_t irr_tile, dist_tile;   // texels per bordered tile
    int32_t n_probes;
    int32_t irr_format, dist_format;
    uint8_t* states;
    void*    irr;
    void*    dist;
    float3   blend_lo;      // cascade fall-off box (Sec. 7.3): outermost planes, or
    float3   blend_hi;      // camera-centred for a tracking window
    float4*  offsets;       // [P] probe offsets from the grid (Sec. 5), or nullptr
    float    offset_limit;  // largest offset per axis, fraction of the spacing
    FastDiv  div_x, div_xy; // by counts.x and counts.x * counts.y (set_view_divisors)
};

inline void set_view_divisors(VolView& w) {
    w.div_x = make_fast_div((uint32_t)w.counts.x);
    w.div_xy = make_fast_div((uint32_t)w.counts.x * (uint32_t)w.counts.y);
}

// Views the specialised (FAST) probe query serves: FP32 atlases, gamma 5 and
// no probe offsets; its kernels skip the per-probe format, gamma and offset
// tests and otherwise compute the same operations in the same order.
inline bool query_fast_view(const VolView& w) {
    return w.irr_format == DDGI_IRR_FP32 && w.dist_format == DDGI_DIST_FP32 && w.half_gamma == 2.5f &&
           w.offsets == nullptr;
}

// Largest BVH leaf (triangles); the traversal packs a leaf's first triangle
// and count - 1 into one int (kLeafBits bits of count), so scenes stay below
// 2^(31 - kLeafBits) triangles.
constexpr int kMaxLeafTris = 8;
constexpr int kLeafBits = 3;
static_assert(kMaxLeafTris <= (1 << kLeafBits), "leaf count must fit its bits");

// Child references of 4-wide nodes: node index (>= 0), leaf code (< 0), or
// kRefDone for an empty slot.  Nodes deeper than kWideFullDepth take two
// children, so a traversal stack of kStackSize4 entries cannot overflow
// (at most 3 pushes per level down to that depth, 1 below, 63 levels).
constexpr int kRefDone = (int)0x80000000;
constexpr int kWideFullDepth = 20;
constexpr int kStackSize4 = 128;
static_assert(3 * kWideFullDepth + 63 <= kStackSize4, "4-wide traversal stack bound");

// Host-side, once-per-device setup of a kernel (shared-memory opt-in and
// the like), safe when several host threads launch at once: f() runs under
// the flags' mutex until it succeeds once on the current device.
constexpr int kMaxHostDevices = 64;
struct DeviceOnce {
    std::mutex m;
    bool done[kMaxHostDevices] = {};
};

template <typename F>
inline cudaError_t once_per_device(DeviceOnce& once, F&& f) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxHostDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(once.m);
    if (once.done[dev]) return cudaSuccess;
    e = f();
    if (e == cudaSuccess) once.done[dev] = true;
    return e;
}

// Volumes a kernel works on: one view by value (a single volume) or a device
// table of up to kMaxVolumes views (a cascade).  Probe lists hold entries
// (volume << 24) | probe, so a single volume's entries are its probe indices.
constexpr int kMaxVolumes = 8;
constexpr int kEntryShift = 24;
constexpr int32_t kEntryMask = (1 << kEntryShift) - 1;

struct VolSet {
    VolView single;           // the volume when table == nullptr
    const VolView* table;     // device array [n] for cascades
    int32_t n;
};

template <bool MULTI>
__device__ __forceinline__ const VolView& vol_of(const VolSet& s, int k) {
    if (MULTI) return s.table[k];
    return s.single;
}

inline VolSet single_set(const VolView& v) {
    VolSet s{};
    s.single = v;
    s.table = nullptr;
    s.n = 1;
    return s;
}

struct BlendParams {
    float hyst_irr, hyst_vis;      // already scaled and clamped
    float thr_low, thr_high, thr_step;
    int32_t R;
    // set by the tiled blend's launcher: by the texel counts n^2 and the
    // tile widths n of irradiance and distance
    FastDiv div_ti, div_td, div_ni, div_nd;
};

struct FrameRot { double m[9]; };

// Host-side BVH build result.
struct BvhHost {
    std::vector<float4> nodes;   // 4 per node
    std::vector<float4> nodes4;  // 8 per 4-wide node
    int32_t max_depth4 = 0;
    std::vector<float4> tris;    // 3 per triangle
    int64_t n_leaves = 0;
    int32_t max_depth = 0;
};

// bvh_build.cpp
// Deepest stack of a depth-first walk of the 4-wide form that pushes every
// child: a bound on the traversal stack (pushes fewer children, keeps one).
int64_t wide_stack_bound(const std::vector<float4>& n4);
bool build_bvh(const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris,
               const int32_t* tri_flags, BvhHost& out, std::string& err);

// Host rotation generator: SplitMix64 stream for (seed, frame), Shoemake quaternion.
FrameRot frame_rotation(uint64_t seed, int64_t frame);

// ---------------------------------------------------------------------------
// Kernel launchers (k_*.cu)
// ---------------------------------------------------------------------------
// Per-frame direction buffers hold 3R float4: the R ray directions (w = 0),
// then for ray i the two packed ray constants of dir_pre_pack at R + 2i.
// Frame ray pattern and texel weights in one launch.  sf64: [R][3] double,
// the unrotated pattern written once by launch_sf_table; the first n_zero
// ints at zero (counters) are cleared by the same launch.
cudaError_t launch_sf_table(int R, double* sf64, cudaStream_t st);
// Optional converge pass for new probes (Sec. 6.3): one batch's weighted
// sums per list slot (init: first batch), then the texels and state advance.
// acc_irr [n][irr_n^2], acc_dist [n][dist_n^2], den [irr_n^2 + dist_n^2].
cudaError_t launch_converge_accum(int R, int irr_n, int dist_n, const float* w_irr, const float* w_dist,
                                  const float4* records, const int32_t* count, float4* acc_irr, float2* acc_dist,
                                  float* den, bool init, int grid, cudaStream_t st);
cudaError_t launch_converge_finish(const VolView& v, const int32_t* list, const int32_t* count,
                                   const float4* acc_irr, const float2* acc_dist, const float* den, uint32_t* status,
                                   int grid, cudaStream_t st);
cudaError_t launch_frame_setup(const FrameRot& rot, int R, int irr_n, int dist_n, float cos_power,
                               const double* sf64, float4* dirs, float* w_irr, float* inv_s_irr, float* w_dist,
                               float* inv_s_dist, int32_t* zero, int n_zero, cudaStream_t st);
// The same as two launches: the texel weights on st_weights, the directions
// (and the counter clear) on st_dirs, so the weights can overlap the trace.
cudaError_t launch_frame_setup_split(const FrameRot& rot, int R, int irr_n, int dist_n, float cos_power,
                                     const double* sf64, float4* dirs, float* w_irr, float* inv_s_irr,
                                     float* w_dist, float* inv_s_dist, int32_t* zero, int n_zero,
                                     cudaStream_t st_dirs, cudaStream_t st_weights);
cudaError_t launch_frame_setup_dev(const FrameRot* rot_dev, int R, int irr_n, int dist_n, float cos_power,
                                   const double* sf64, float4* dirs, float* w_irr, float* inv_s_irr, float* w_dist,
                                   float* inv_s_dist, int32_t* zero, int n_zero, cudaStream_t st);
cudaError_t launch_build_list(const uint8_t* states, int P, int which, int32_t* list,
                              int32_t* count, cudaStream_t st);
// probes [begin, end) only (a shard of the grid)
cudaError_t launch_build_list_range(const uint8_t* states, int begin, int end, int which, int32_t* list,
                                    int32_t* count, cudaStream_t st);
cudaError_t launch_build_list_multi(const VolSet& vs, int total, int which, int32_t* list, int32_t* count,
                                    cudaStream_t st);
// perm (may be NULL = identity): ray order of a probe's warps, a permutation
// of [0, R) that groups nearby directions (ray_order_morton)
// One position-optimizer iteration (Sec. 5) over the UNINIT list, rays `dirs`.
cudaError_t launch_optimize(const DevScene& s, const VolView& v, const float4* dirs, int R, const int32_t* list,
                            const int32_t* count, int grid, cudaStream_t st);
// Frame ray directions only (float4 for the trace, double for the weights).
// The frame directions and ray constants alone (position-optimizer rays).
cudaError_t launch_frame_dirs(const FrameRot& rot, int R, int irr_n, int dist_n, const double* sf64, float4* dirs,
                              cudaStream_t st);
// Classification of the listed (uninitialised) probes.  scratch: one zeroed
// int4 per list entry, left zeroed (batch-split kernel), or nullptr (one
// warp per probe, no scratch: the allocation-free update).
cudaError_t launch_classify(const DevScene& s, const VolView& v, const float4* dirs, int R, const int32_t* perm,
                            const int32_t* list, const int32_t* count, int4* scratch, int grid, cudaStream_t st);
cudaError_t launch_classify_multi(const DevScene& s, const VolSet& vs, const float4* dirs, int R,
                                  const int32_t* perm, const int32_t* list, const int32_t* count, int4* scratch,
                                  int grid, cudaStream_t st);
cudaError_t launch_trace_shade(const DevScene& s, const VolView& v, const Lights& L,
                               const float4* dirs, int R, const int32_t* active,
                               const int32_t* count, float4* records, int grid, cudaStream_t st);
// Per-volume device counters, one block cleared by one memset per frame:
// [0] uninitialised-list count, [1] active-list count, [4..9] the trace's
// counters (shadow_count below).
constexpr int kCounterInts = 10;

// Wavefront trace: persistent primary pass (closest hits; final records of
// misses and back faces; lists of shadow rays and of front hits), persistent
// shadow pass, then shading of the front hits.  shadow_list and hit_list
// hold one int32 per ray (active probes x R); shadow_count is 6 int32 of
// device scratch, 8-byte aligned, zeroed by the caller: shadow rays, front
// hits, the 64-bit work counters of the primary and the shadow pass.
// marks: 4 events recorded around the three passes, or nullptr.
cudaError_t launch_trace_wavefront(const DevScene& s, const VolView& v, const Lights& L, const float4* dirs,
                                   int R, const int32_t* perm, const int32_t* active, const int32_t* count,
                                   float4* records, int32_t* shadow_list, int32_t* hit_list, int32_t* shadow_count,
                                   int grid, cudaStream_t st, cudaEvent_t* marks);
// Measurement build of the primary and shadow passes: adds 4-wide node
// visits and triangle tests to stats[1], [2] (primary) and [4], [5] (shadow);
// the shadow-ray and front-hit counts are left in shadow_count[0], [1].
cudaError_t launch_trace_count(const DevScene& s, const VolView& v, const Lights& L, const float4* dirs, int R,
                               const int32_t* perm, const int32_t* active, const int32_t* count, float4* records,
                               int32_t* shadow_list, int32_t* hit_list, int32_t* shadow_count,
                               unsigned long long* stats, int grid, cudaStream_t st);
cudaError_t launch_trace_wavefront_multi(const DevScene& s, const VolSet& vs, const Lights& L,
                                         const float4* dirs, int R, const int32_t* perm, const int32_t* active,
                                         const int32_t* count, float4* records, int32_t* shadow_list,
                                         int32_t* hit_list, int32_t* shadow_count, int grid, cudaStream_t st,
                                         bool fast_query);
// Morton order of the octahedral positions of the unrotated spherical-
// Fibonacci directions (host; a rotation keeps neighbouring directions together)
std::vector<int32_t> ray_order_morton(int R);
cudaError_t launch_blend(const VolView& v, const BlendParams& bp, const float* w_irr,
                         const float* inv_s_irr, const float* w_dist, const float* inv_s_dist,
                         const float4* records, const int32_t* active, const int32_t* count,
                         uint32_t* status, int grid, cudaStream_t st);
// blend over a volume set sharing irr_n / dist_n; probes_per_cta in
// {4, 8, 16} (autotuned)
cudaError_t launch_blend_set(const VolSet& vs, bool multi, const BlendParams& bp, int irr_n, int dist_n,
                             const float* w_irr,
                             const float* inv_s_irr, const float* w_dist, const float* inv_s_dist,
                             const float4* records, const int32_t* active, const int32_t* count,
                             uint32_t* status, int grid, int probes_per_cta, cudaStream_t st);
cudaError_t prepare_blend_kernels(int R);
// tensor-core blend (k_blend_tc.cu)
// (precision: DDGI_BLEND_TF32, _BF16 or _TF32X3; one packed weight buffer
// of tc_pack_bytes(R), written per frame by launch_pack_weights)
int tc_blend_chunks(int R);
size_t tc_pack_bytes(int R);
bool tc_blend_supported(int irr_n, int dist_n);
cudaError_t launch_pack_weights(const float* w_irr, const float* w_dist, int R, int irr_n, int dist_n, int precision,
                                uint8_t* pack, float* inv_irr, float* inv_dist, cudaStream_t st);
cudaError_t launch_blend_tc(const VolView& v, const BlendParams& bp, int precision, const uint8_t* pack,
                            const float* inv_irr, const float* inv_dist, const float4* records, const int32_t* active,
                            const int32_t* count, uint32_t* status, int grid, cudaStream_t st);
cudaError_t launch_blend_tc_set(const VolSet& vs, bool multi, const BlendParams& bp, int precision, int irr_n,
                                int dist_n, const uint8_t* pack, const float* inv_irr, const float* inv_dist,
                                const float4* records, const int32_t* active, const int32_t* count, uint32_t* status,
                                int grid, cudaStream_t st);
cudaError_t prepare_blend_tc_kernels();
// FP64 differentiable path (k_diff64.cu): the volume's grid and parameters
// in double; atlases [P][(n+2)^2][3] / [P][(m+2)^2][2] and ray records
// [P*R][4] in double.
struct Diff64Volume {
    double origin[3], spacing[3];
    int counts[3];
    int R, irr_n, dist_n;
    double bias, gamma, t_max, cos_power;
};
cudaError_t launch_diff64_frame(const Diff64Volume& dv, const DevScene& s, const Lights& L, const float4* dirs,
                                const double* albedo, const double* emit, const double* irr_prev,
                                const double* dist_prev, int with_prev, double* rec, double* irr_out,
                                double* dist_out, cudaStream_t st);
cudaError_t launch_diff64_query(const Diff64Volume& dv, const double* irr, const double* dist, const float* pos,
                                const float* nrm, int64_t n, float3 cam, double* out, cudaStream_t st);
cudaError_t launch_diff64_query_adjoint(const Diff64Volume& dv, const double* irr, const double* dist,
                                        const float* pos, const float* nrm, int64_t n, float3 cam, const double* dE,
                                        double* g_irr, cudaStream_t st);
cudaError_t launch_diff64_frame_adjoint(const Diff64Volume& dv, const DevScene& s, const Lights& L,
                                        const float4* dirs, const double* albedo, const double* irr_before,
                                        const double* dist_before, const double* irr_after, int with_prev,
                                        double* sw_irr, double* g_irr, double* gL, double* d_emit, double* d_albedo,
                                        double* g_prev, cudaStream_t st);
cudaError_t launch_query_glossy(const VolView& v, const float* pos, const float* nrm, const float* dirs, int64_t n,
                                float* out, cudaStream_t st);
// Dynamic-object wake-up over probes [begin, end); boxes [n][6] device, extended.
cudaError_t launch_wake(const VolView& v, const float* boxes, int n_boxes, int begin, int end, cudaStream_t st);
cudaError_t launch_query(const VolView& v, const float* pos, const float* nrm, int64_t n,
                         float3 camera, float* out, cudaStream_t st,
                         bool out_host = false);
cudaError_t launch_query_cascade(const VolSet& vs, const float* pos, const float* nrm, int64_t n, float3 camera,
                                 float* out, cudaStream_t st);
// Resets probe planes that a tracking window leapfrogged: planes[i] =
// (volume, axis, physical plane index); count on the device.
cudaError_t launch_reset_planes(const VolSet& vs, const int4* planes, const int32_t* count, int max_planes,
                                cudaStream_t st);
cudaError_t launch_trace_rays(const DevScene& s, const float* orig, const float* dir, int64_t n,
                              float* t, int32_t* tri, int32_t* backface, cudaStream_t st);
cudaError_t launch_gbuffer(const DevScene& s, float3 pos, float3 fwd, float3 right, float3 up,
                           float tan_half, float aspect, int w, int h, float* out_pos,
                           float* out_nrm, cudaStream_t st);

int sm_count();

// Records an error message for ddgi_last_error() and returns the status.
ddgi_status set_error(ddgi_status s, const std::string& msg);

// Device view of a registered scene (NULL for a NULL handle).
const DevScene* scene_device_view(ddgi_scene s);

}  // namespace ddgi
