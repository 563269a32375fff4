// Per-frame ray pattern and the probe blend (Sec. 2.3 Eq. 1, Sec. 4.2, 4.3, 7.1).
//
// k_frame_setup computes, once per frame and shared by every probe, the ray
// directions w_i = R_t sf(i, R) and the texel weight matrices
//   W_irr[t][i]  = max(0, n_t . w_i)              (cosine weight)
//   W_dist[t][i] = max(0, n_t . w_i)^p            (power-cosine weight)
// with 1 / sum_i W per texel, in double precision, rounded once to float.
//
// k_blend_simt is the plain FP32 blend.  A CTA owns a group of kProbes
// active probes: their ray records are staged in shared memory (padded
// stride, conflict-free across probes), each thread computes (texel, probe)
// dot products over the R rays, and the epilogue normalises, gamma-encodes,
// applies the per-texel hysteresis thresholds, lerps with the old texel and
// writes the texel plus the border texels that copy it (the octahedral
// border copy of Sec. 7.1 fused into the blend).  The probe's state advances
// Newly Vigilant -> Vigilant after its texels are written.
#include "blend_epilogue.cuh"

namespace ddgi {

namespace {

__device__ double sf_component(int i, int n, int axis) {
    const double inv_phi = 0.61803398874989484820;
    double a = (double)i * inv_phi;
    double phi = 6.283185307179586477 * (a - floor(a));
    double z = 1.0 - (2.0 * i + 1.0) / (double)n;
    double r = sqrt(fmax(0.0, 1.0 - z * z));
    return axis == 0 ? cos(phi) * r : (axis == 1 ? sin(phi) * r : z);
}

__device__ void frame_dir(const FrameRot& rot, int i, int n, double out[3]) {
    double s0 = sf_component(i, n, 0), s1 = sf_component(i, n, 1), s2 = sf_component(i, n, 2);
    for (int a = 0; a < 3; ++a) out[a] = rot.m[3 * a] * s0 + rot.m[3 * a + 1] * s1 + rot.m[3 * a + 2] * s2;
}

__device__ void texel_dir(int t, int n, double v[3]) {
    int i = t % n, j = t / n;
    double ux = 2.0 * (i + 0.5) / n - 1.0, uy = 2.0 * (j + 0.5) / n - 1.0;
    double x = ux, y = uy, z = 1.0 - fabs(ux) - fabs(uy);
    if (z < 0.0) {
        x = (1.0 - fabs(uy)) * (ux >= 0.0 ? 1.0 : -1.0);
        y = (1.0 - fabs(ux)) * (uy >= 0.0 ? 1.0 : -1.0);
    }
    double l = sqrt(x * x + y * y + z * z);
    v[0] = x / l;
    v[1] = y / l;
    v[2] = z / l;
}

}  // namespace

// grid: irr_n^2 + dist_n^2 + 1 blocks; block b < irr_n^2 handles irradiance
// texel b, the next dist_n^2 blocks distance texels, the last one the rays.
template <bool ROT_DEV>
__global__ void __launch_bounds__(256) k_frame_setup(FrameRot rot_arg, const FrameRot* rot_dev, int R, int irr_n,
                                                     int dist_n, double cos_power, float4* dirs, float* w_irr,
                                                     float* inv_s_irr, float* w_dist,
                                                     float* inv_s_dist) {
    __shared__ double red[256];
    // ROT_DEV: the rotation is read from device memory (per-frame parameters
    // written before a captured graph replays)
    const FrameRot rot = ROT_DEV ? *rot_dev : rot_arg;
    int b = blockIdx.x;
    int ti = irr_n * irr_n, td = dist_n * dist_n;
    if (b == ti + td) {
        for (int i = threadIdx.x; i < R; i += blockDim.x) {
            double w[3];
            frame_dir(rot, i, R, w);
            dirs[i] = make_float4((float)w[0], (float)w[1], (float)w[2], 0.0f);
        }
        return;
    }
    bool is_irr = b < ti;
    int t = is_irr ? b : b - ti;
    double nt[3];
    texel_dir(t, is_irr ? irr_n : dist_n, nt);
    double acc = 0.0;
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
        double w[3];
        frame_dir(rot, i, R, w);
        double c = fmax(0.0, nt[0] * w[0] + nt[1] * w[1] + nt[2] * w[2]);
        double wt = is_irr ? c : pow(c, cos_power);
        acc += wt;
        if (is_irr) w_irr[(int64_t)t * R + i] = (float)wt;
        else w_dist[(int64_t)t * R + i] = (float)wt;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        float inv = red[0] > 0.0 ? (float)(1.0 / red[0]) : -1.0f;   // -1: no ray in reach
        if (is_irr) inv_s_irr[t] = inv;
        else inv_s_dist[t] = inv;
    }
}

template <bool MULTI, int kProbes>
__global__ void __launch_bounds__(256) k_blend_simt(VolSet vs, BlendParams bp,
                                                    const float* __restrict__ w_irr,
                                                    const float* __restrict__ inv_s_irr,
                                                    const float* __restrict__ w_dist,
                                                    const float* __restrict__ inv_s_dist,
                                                    const float4* __restrict__ records,
                                                    const int32_t* __restrict__ active,
                                                    const int32_t* __restrict__ count,
                                                    uint32_t* status) {
    extern __shared__ float4 srec[];   // kProbes x (R + 1) records
    __shared__ int s_probe[kProbes];
    __shared__ int s_newly[kProbes];
    const int R = bp.R;
    const int stride = R + 1;
    const int n_act = *count;
    const VolView& v0 = vol_of<MULTI>(vs, 0);   // cascades share R and tile sizes
    const int ni = v0.irr_n, nd = v0.dist_n;
    const int ti = ni * ni, td = nd * nd;
    for (int g0 = blockIdx.x * kProbes; g0 < n_act; g0 += gridDim.x * kProbes) {
        const int np = min(kProbes, n_act - g0);
        if (threadIdx.x < np) {
            int e = active[g0 + threadIdx.x];
            s_probe[threadIdx.x] = e;
            s_newly[threadIdx.x] =
                vol_of<MULTI>(vs, e >> kEntryShift).states[e & kEntryMask] == DDGI_STATE_NEWLY_VIGILANT;
        }
        for (int k = threadIdx.x; k < np * R; k += blockDim.x) {
            int pp = k / R, i = k - pp * R;
            srec[pp * stride + i] = records[(int64_t)(g0 + pp) * R + i];
        }
        __syncthreads();
        // irradiance texels: cosine-weighted average, gamma encode, thresholds, lerp
        for (int q = threadIdx.x; q < ti * np; q += blockDim.x) {
            int t = q / np, pp = q - t * np;
            const float* wr = w_irr + (int64_t)t * R;
            const float4* rr = srec + pp * stride;
            float ar = 0.0f, ag = 0.0f, ab = 0.0f;
            for (int i = 0; i < R; ++i) {
                float w = __ldg(wr + i);
                float4 L = rr[i];
                ar = fmaf(w, L.x, ar);
                ag = fmaf(w, L.y, ag);
                ab = fmaf(w, L.z, ab);
            }
            const int e = s_probe[pp];
            blend_irr_texel(vol_of<MULTI>(vs, e >> kEntryShift), bp, e & kEntryMask, t, ar, ag, ab,
                            __ldg(inv_s_irr + t), s_newly[pp] != 0, status);
        }
        // distance texels: power-cosine weighted mean distance and mean squared distance
        for (int q = threadIdx.x; q < td * np; q += blockDim.x) {
            int t = q / np, pp = q - t * np;
            const float* wr = w_dist + (int64_t)t * R;
            const float4* rr = srec + pp * stride;
            float m1 = 0.0f, m2 = 0.0f;
            for (int i = 0; i < R; ++i) {
                float w = __ldg(wr + i);
                float d = rr[i].w;
                float wd = w * d;
                m1 += wd;
                m2 = fmaf(wd, d, m2);
            }
            const int e = s_probe[pp];
            blend_dist_texel(vol_of<MULTI>(vs, e >> kEntryShift), bp, e & kEntryMask, t, m1, m2,
                             __ldg(inv_s_dist + t), s_newly[pp] != 0, status);
        }
        __syncthreads();
        if (threadIdx.x < np && s_newly[threadIdx.x]) {
            const int e = s_probe[threadIdx.x];
            vol_of<MULTI>(vs, e >> kEntryShift).states[e & kEntryMask] = DDGI_STATE_VIGILANT;
        }
        __syncthreads();
    }
}

cudaError_t launch_frame_setup(const FrameRot& rot, int R, int irr_n, int dist_n, float cos_power,
                               float4* dirs, float* w_irr, float* inv_s_irr, float* w_dist,
                               float* inv_s_dist, cudaStream_t st) {
    int blocks = irr_n * irr_n + dist_n * dist_n + 1;
    k_frame_setup<false><<<blocks, 256, 0, st>>>(rot, nullptr, R, irr_n, dist_n, (double)cos_power, dirs, w_irr,
                                                 inv_s_irr, w_dist, inv_s_dist);
    return cudaGetLastError();
}

cudaError_t launch_frame_setup_dev(const FrameRot* rot_dev, int R, int irr_n, int dist_n, float cos_power,
                                   float4* dirs, float* w_irr, float* inv_s_irr, float* w_dist,
                                   float* inv_s_dist, cudaStream_t st) {
    int blocks = irr_n * irr_n + dist_n * dist_n + 1;
    k_frame_setup<true><<<blocks, 256, 0, st>>>(FrameRot{}, rot_dev, R, irr_n, dist_n, (double)cos_power, dirs,
                                                w_irr, inv_s_irr, w_dist, inv_s_dist);
    return cudaGetLastError();
}

template <bool MULTI, int PGS>
static cudaError_t blend_simt(const VolSet& vs, const BlendParams& bp, const float* w_irr, const float* inv_s_irr,
                              const float* w_dist, const float* inv_s_dist, const float4* records,
                              const int32_t* active, const int32_t* count, uint32_t* status, int grid,
                              cudaStream_t st) {
    size_t smem = (size_t)PGS * (bp.R + 1) * sizeof(float4);
    static int configured_smem = 0;
    if ((int)smem > configured_smem) {
        cudaError_t e = cudaFuncSetAttribute(k_blend_simt<MULTI, PGS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured_smem = (int)smem;
    }
    k_blend_simt<MULTI, PGS><<<grid, 256, smem, st>>>(vs, bp, w_irr, inv_s_irr, w_dist, inv_s_dist, records,
                                                      active, count, status);
    return cudaGetLastError();
}

cudaError_t launch_blend(const VolView& v, const BlendParams& bp, const float* w_irr, const float* inv_s_irr,
                         const float* w_dist, const float* inv_s_dist, const float4* records,
                         const int32_t* active, const int32_t* count, uint32_t* status, int grid,
                         cudaStream_t st) {
    return blend_simt<false, 8>(single_set(v), bp, w_irr, inv_s_irr, w_dist, inv_s_dist, records, active, count,
                                status, grid, st);
}

cudaError_t launch_blend_set(const VolSet& vs, bool multi, const BlendParams& bp, const float* w_irr,
                             const float* inv_s_irr, const float* w_dist, const float* inv_s_dist,
                             const float4* records, const int32_t* active, const int32_t* count,
                             uint32_t* status, int grid, int probes_per_cta, cudaStream_t st) {
#define DDGI_BLEND_CASE(M, P)                                                                                 \
    if (multi == M && probes_per_cta == P)                                                                   \
        return blend_simt<M, P>(vs, bp, w_irr, inv_s_irr, w_dist, inv_s_dist, records, active, count, status, \
                                grid, st);
    DDGI_BLEND_CASE(false, 4)
    DDGI_BLEND_CASE(false, 8)
    DDGI_BLEND_CASE(false, 16)
    DDGI_BLEND_CASE(true, 4)
    DDGI_BLEND_CASE(true, 8)
    DDGI_BLEND_CASE(true, 16)
#undef DDGI_BLEND_CASE
    return cudaErrorInvalidValue;
}

// Sets the shared-memory opt-in of every SIMT blend instantiation for R rays
// (outside any stream capture).
cudaError_t prepare_blend_kernels(int R) {
    cudaError_t e = cudaSuccess;
#define DDGI_PREP(M, P)                                                                                   \
    if (e == cudaSuccess)                                                                                \
        e = cudaFuncSetAttribute(k_blend_simt<M, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                                 (int)((size_t)P * (R + 1) * sizeof(float4)) > 48 * 1024                    \
                                     ? (int)((size_t)P * (R + 1) * sizeof(float4))                          \
                                     : 48 * 1024);
    DDGI_PREP(false, 4)
    DDGI_PREP(false, 8)
    DDGI_PREP(false, 16)
    DDGI_PREP(true, 4)
    DDGI_PREP(true, 8)
    DDGI_PREP(true, 16)
#undef DDGI_PREP
    return e;
}

}  // namespace ddgi
