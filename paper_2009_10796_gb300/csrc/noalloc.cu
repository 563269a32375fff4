// Allocation-free probe update.
//
// Some callers cannot allocate device memory once they are running: a
// renderer that budgets all of its GPU memory up front and forbids cudaMalloc
// inside its frame loop (an allocation can synchronise the device and breaks a
// pre-planned memory pool), or a plug-in whose host owns every device buffer.
// ddgi_update_noalloc serves them: the caller passes the probe states and
// atlases it owns, and every scratch buffer of the update (ray pattern, texel
// weight tables, probe lists, counters, ray records) lives in the file-scope
// device arrays below, whose sizes fix the largest volume this entry point
// accepts.  Every GPU that loads the library holds these arrays (about 17 MiB)
// until the process exits; they come into being when this file's module is
// loaded on a device, which the first call on that device triggers.
// Device-side errors (a non-finite texel) accumulate in a status word of the
// same kind until ddgi_update_noalloc_poll_status reads and clears it.
#include <cmath>
#include <mutex>

#include "ddgi_internal.h"

namespace ddgi {
namespace {

constexpr int kNaMaxRays = 512;               // rays per probe
constexpr int kNaMaxIrrTexels = 8 * 8;        // interior irradiance texels (irr_n <= 8)
constexpr int kNaMaxDistTexels = 16 * 16;     // interior distance texels (dist_n <= 16)
constexpr int kNaMaxProbes = 32768;           // probes in the volume
constexpr int64_t kNaMaxRecords = 1 << 20;    // probes x rays (16 MiB of ray records)

static __device__ __align__(256) float4 g_na_records[kNaMaxRecords];
static __device__ __align__(256) float4 g_na_dirs[3 * kNaMaxRays];   // directions, then ray constants
static __device__ __align__(256) double g_na_sf64[3 * kNaMaxRays];   // unrotated ray pattern
static __device__ __align__(256) float g_na_w_irr[kNaMaxIrrTexels * kNaMaxRays];
static __device__ __align__(256) float g_na_inv_s_irr[kNaMaxIrrTexels];
static __device__ __align__(256) float g_na_w_dist[kNaMaxDistTexels * kNaMaxRays];
static __device__ __align__(256) float g_na_inv_s_dist[kNaMaxDistTexels];
static __device__ __align__(256) int32_t g_na_lists[2 * kNaMaxProbes];
static __device__ __align__(256) int32_t g_na_counts[4];
static __device__ __align__(256) uint32_t g_na_status[4];

struct NaScratch {
    float4* records;
    float4* dirs;
    double* sf64;
    float* w_irr;
    float* inv_s_irr;
    float* w_dist;
    float* inv_s_dist;
    int32_t* lists;
    int32_t* counts;
    uint32_t* status;
};

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
bool g_na_ready[kNaMaxDevices];
NaScratch g_na_scratch[kNaMaxDevices];

// In host code the array names are host-side stand-ins, not device addresses:
// the device addresses are looked up once per device, with that device
// current, and cached.
cudaError_t scratch_for_current_device(NaScratch* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ready[dev]) {
        NaScratch s{};
        if ((e = cudaGetSymbolAddress((void**)&s.records, g_na_records)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void**)&s.dirs, g_na_dirs)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void**)&s.sf64, g_na_sf64)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void**)&s.w_irr, g_na_w_irr)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void**)&s.inv_s_irr, g_na_inv_s_irr)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void**)&s.w_dist, g_na_w_dist)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void**)&s.inv_s_dist, g_na_inv_s_dist)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void**)&s.lists, g_na_lists)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void**)&s.counts, g_na_counts)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void**)&s.status, g_na_status)) != cudaSuccess) return e;
        g_na_scratch[dev] = s;
        g_na_ready[dev] = true;
    }
    *out = g_na_scratch[dev];
    return cudaSuccess;
}

ddgi_status na_fail(cudaError_t e, const char* what) {
    return set_error(DDGI_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace
}  // namespace ddgi

using namespace ddgi;

extern "C" ddgi_status ddgi_update_noalloc(ddgi_scene scene, const ddgi_volume_desc* d,
                                           const ddgi_lights* lights, const ddgi_update_params* params,
                                           uint8_t* states_dev, void* irr_dev, void* dist_dev,
                                           ddgi_stream stream) {
    const DevScene* sv = scene_device_view(scene);
    if (!sv || !d || !lights || !params || !states_dev || !irr_dev || !dist_dev)
        return set_error(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (((uintptr_t)states_dev % 16) != 0 || ((uintptr_t)irr_dev % 16) != 0 || ((uintptr_t)dist_dev % 16) != 0)
        return set_error(DDGI_ERR_INVALID_ARG, "device buffers must be 16-byte aligned");
    for (int a = 0; a < 3; ++a) {
        if (d->counts[a] < 2) return set_error(DDGI_ERR_INVALID_ARG, "counts must be >= 2");
        if (!(d->spacing[a] > 0.0f) || !std::isfinite(d->spacing[a]) || !std::isfinite(d->origin[a]))
            return set_error(DDGI_ERR_INVALID_ARG, "spacing must be positive and origin finite");
    }
    int64_t P = (int64_t)d->counts[0] * d->counts[1] * d->counts[2];
    int R = d->rays_per_probe;
    if (P > kNaMaxProbes)
        return set_error(DDGI_ERR_INVALID_ARG, "ddgi_update_noalloc: more than 32768 probes");
    if (R < 1 || R > kNaMaxRays)
        return set_error(DDGI_ERR_INVALID_ARG, "ddgi_update_noalloc: rays_per_probe must be in [1, 512]");
    if (P * R > kNaMaxRecords)
        return set_error(DDGI_ERR_INVALID_ARG, "ddgi_update_noalloc: probes x rays exceeds 1048576");
    if (d->irr_n < 1 || d->irr_n * d->irr_n > kNaMaxIrrTexels || d->dist_n < 1 ||
        d->dist_n * d->dist_n > kNaMaxDistTexels)
        return set_error(DDGI_ERR_INVALID_ARG, "ddgi_update_noalloc: irr_n must be in [1, 8], dist_n in [1, 16]");
    if (d->irr_format < 0 || d->irr_format > 2 || d->dist_format < 0 || d->dist_format > 1)
        return set_error(DDGI_ERR_INVALID_ARG, "unknown atlas format");
    if (d->optimizer_iters != 0)
        return set_error(DDGI_ERR_UNSUPPORTED, "ddgi_update_noalloc: no probe position optimizer (no offset storage)");
    if (d->converge_batches != 0)
        return set_error(DDGI_ERR_UNSUPPORTED, "ddgi_update_noalloc: no converge pass (no storage for its sums)");
    if (!(d->gamma > 0.0f) || !(d->hysteresis_irr >= 0.0f && d->hysteresis_irr <= 1.0f) ||
        !(d->hysteresis_vis >= 0.0f && d->hysteresis_vis <= 1.0f) || !(d->dist_cos_power >= 0.0f) ||
        !(d->self_shadow_bias >= 0.0f))
        return set_error(DDGI_ERR_INVALID_ARG, "bad gamma, hysteresis, cosine power or bias");
    if (!(params->irr_hyst_scale >= 0.0f) || !(params->vis_hyst_scale >= 0.0f))
        return set_error(DDGI_ERR_INVALID_ARG, "negative hysteresis scale");
    if (params->blend_precision != DDGI_BLEND_FP32)
        return set_error(DDGI_ERR_UNSUPPORTED, "ddgi_update_noalloc blends in FP32 only");

    NaScratch s;
    cudaError_t e = scratch_for_current_device(&s);
    if (e != cudaSuccess) return na_fail(e, "scratch address lookup");

    VolView v{};
    v.origin = make_float3(d->origin[0], d->origin[1], d->origin[2]);
    v.spacing = make_float3(d->spacing[0], d->spacing[1], d->spacing[2]);
    v.inv_spacing = make_float3(1.0f / d->spacing[0], 1.0f / d->spacing[1], 1.0f / d->spacing[2]);
    v.counts = make_int3(d->counts[0], d->counts[1], d->counts[2]);
    set_view_divisors(v);
    v.shift = make_int3(0, 0, 0);
    v.min_spacing = std::fmin(d->spacing[0], std::fmin(d->spacing[1], d->spacing[2]));
    v.bias = d->self_shadow_bias;
    v.gamma = d->gamma;
    v.inv_gamma = 1.0f / d->gamma;
    v.half_gamma = 0.5f * d->gamma;
    if (d->t_max >= 0.0f) {
        v.t_max = d->t_max;
    } else {
        double sx = d->spacing[0], sy = d->spacing[1], sz = d->spacing[2];
        v.t_max = (float)(2.0 * std::sqrt(sx * sx + sy * sy + sz * sz));
    }
    v.irr_n = d->irr_n;
    v.dist_n = d->dist_n;
    v.irr_tile = (d->irr_n + 2) * (d->irr_n + 2);
    v.dist_tile = (d->dist_n + 2) * (d->dist_n + 2);
    v.n_probes = (int32_t)P;
    v.irr_format = d->irr_format;
    v.dist_format = d->dist_format;
    v.states = states_dev;
    v.irr = irr_dev;
    v.dist = dist_dev;

    Lights L{};
    L.sun_dir = make_float3(lights->sun_dir[0], lights->sun_dir[1], lights->sun_dir[2]);
    L.sun_irr = make_float3(lights->sun_irradiance[0], lights->sun_irradiance[1], lights->sun_irradiance[2]);
    L.sky_a = make_float3(lights->sky_a[0], lights->sky_a[1], lights->sky_a[2]);
    L.sky_b = make_float3(lights->sky_b[0], lights->sky_b[1], lights->sky_b[2]);
    L.sky_up = make_float3(lights->sky_up[0], lights->sky_up[1], lights->sky_up[2]);
    L.sun_on = (lights->sun_irradiance[0] > 0.0f || lights->sun_irradiance[1] > 0.0f ||
                lights->sun_irradiance[2] > 0.0f);

    BlendParams bp{};
    bp.hyst_irr = std::fmin(1.0f, std::fmax(0.0f, d->hysteresis_irr * params->irr_hyst_scale));
    bp.hyst_vis = std::fmin(1.0f, std::fmax(0.0f, d->hysteresis_vis * params->vis_hyst_scale));
    bp.thr_low = d->thr_low;
    bp.thr_high = d->thr_high;
    bp.thr_step = d->thr_step;
    bp.R = R;

    cudaStream_t st = (cudaStream_t)stream;
    int sms = sm_count();
    FrameRot rot = frame_rotation(d->seed, params->frame);
    // the arrays keep the previous call's contents: the frame setup clears the
    // counters; the status word keeps its flags until it is polled
    if ((e = launch_sf_table(R, s.sf64, st)) != cudaSuccess) return na_fail(e, "ray pattern");
    if ((e = launch_frame_setup(rot, R, d->irr_n, d->dist_n, d->dist_cos_power, s.sf64, s.dirs, s.w_irr,
                                s.inv_s_irr, s.w_dist, s.inv_s_dist, s.counts, 4, st)) != cudaSuccess)
        return na_fail(e, "frame setup");
    if (d->state_machine) {
        if ((e = launch_build_list(states_dev, (int)P, 0, s.lists, s.counts + 0, st)) != cudaSuccess)
            return na_fail(e, "uninitialised list");
        if ((e = launch_classify(*sv, v, s.dirs, R, nullptr, s.lists, s.counts + 0, nullptr, sms * 8, st)) != cudaSuccess)
            return na_fail(e, "classify");
    }
    if ((e = launch_build_list(states_dev, (int)P, 1, s.lists + P, s.counts + 1, st)) != cudaSuccess)
        return na_fail(e, "active list");
    if ((e = launch_trace_shade(*sv, v, L, s.dirs, R, s.lists + P, s.counts + 1, s.records, sms * 16, st)) !=
        cudaSuccess)
        return na_fail(e, "trace and shade");
    if ((e = launch_blend(v, bp, s.w_irr, s.inv_s_irr, s.w_dist, s.inv_s_dist, s.records, s.lists + P,
                          s.counts + 1, s.status, sms * 4, st)) != cudaSuccess)
        return na_fail(e, "blend");
    return DDGI_OK;
}

extern "C" ddgi_status ddgi_update_noalloc_poll_status(ddgi_stream stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(e, "current device");
    if (dev < 0 || dev >= kNaMaxDevices) return set_error(DDGI_ERR_INVALID_ARG, "device index out of range");
    NaScratch s;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ready[dev]) return DDGI_OK;   // no call on this device yet: nothing was flagged
        s = g_na_scratch[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t w = 0;
    if ((e = cudaMemcpyAsync(&w, s.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return na_fail(e, "read status");
    if ((e = cudaMemsetAsync(s.status, 0, sizeof(uint32_t), st)) != cudaSuccess) return na_fail(e, "clear status");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return na_fail(e, "synchronise");
    if (w & 2u) return set_error(DDGI_ERR_TIMEOUT, "a bounded device wait gave up");
    if (w & 1u) return set_error(DDGI_ERR_NUMERIC, "non-finite texel value produced");
    return DDGI_OK;
}
