// Probe-ray kernels of the update (Sec. 2.3 and Sec. 6.3):
//   k_classify     distance-only trace of UNINIT probes -> OFF / NEWLY_VIGILANT / SLEEPING
//   k_trace_shade  closest hit + shading of every ray of every active probe
// plus two utility kernels over arbitrary rays (raw closest hit, camera G-buffer).
//
// Work layout: rays of one probe are consecutive work items, so a warp
// traces 32 rays of the same probe (same origin, directions spread by the
// spherical-Fibonacci pattern).  Kernels are persistent: the grid is sized to
// the machine and threads stride over the device-side work count, so the host
// never waits for the active-probe count.
#include "traverse.cuh"

namespace ddgi {

__global__ void __launch_bounds__(256) k_classify(DevScene s, VolView v, const float4* __restrict__ dirs,
                                                  int R, const int32_t* __restrict__ list,
                                                  const int32_t* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int n = *count;
    for (int q = warp; q < n; q += nwarps) {
        int p = list[q];
        float3 o = probe_pos_phys(v, p);
        int bf = 0;
        float dmin = INFINITY;
        for (int i = lane; i < R; i += 32) {
            float4 d4 = __ldg(dirs + i);
            float3 d = f3(d4.x, d4.y, d4.z);
            RayPre r = ray_pre(o, d);
            Hit h = traverse<false>(s, r);
            if (h.orig >= 0) {
                const float4* T = s.tris + 3 * (int64_t)h.k;
                float4 p0 = __ldg(T), p1 = __ldg(T + 1), p2 = __ldg(T + 2);
                float3 ng = cross(f3(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z),
                                  f3(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z));
                if (dot(d, ng) > 0.0f) bf++;
                else dmin = fminf(dmin, h.t);
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            bf += __shfl_xor_sync(0xffffffffu, bf, off);
            dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, off));
        }
        if (lane == 0) {
            uint8_t st;
            if (4 * bf > R) st = DDGI_STATE_OFF;
            else if (dmin < v.min_spacing) st = DDGI_STATE_NEWLY_VIGILANT;
            else st = DDGI_STATE_SLEEPING;
            v.states[p] = st;
        }
    }
}

// COUNT = true is the instrumented measurement variant: it writes no records
// and accumulates per-ray work counters instead (stats[0..6]: primary rays,
// primary node visits, primary triangle tests, shadow rays, shadow node
// visits, shadow triangle tests, probe queries at hits).
template <bool COUNT>
__global__ void __launch_bounds__(128) k_trace_shade(DevScene s, VolView v, Lights L,
                                                     const float4* __restrict__ dirs, int R,
                                                     const int32_t* __restrict__ active,
                                                     const int32_t* __restrict__ count,
                                                     float4* __restrict__ records,
                                                     unsigned long long* stats) {
    TraceCount cp, cs;
    uint32_t n_rays = 0, n_shadow = 0, n_query = 0;
    const int64_t total = (int64_t)(*count) * R;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
        int slot = (int)(idx / R);
        int i = (int)(idx - (int64_t)slot * R);
        int p = __ldg(active + slot);
        float3 o = probe_pos_phys(v, p);
        float4 d4 = __ldg(dirs + i);
        float3 d = f3(d4.x, d4.y, d4.z);
        RayPre r = ray_pre(o, d);
        Hit h = traverse<false, COUNT>(s, r, &cp);
        if (COUNT) n_rays++;
        float4 rec;
        if (h.orig < 0) {
            float c = dot(d, L.sky_up);
            rec = make_float4(L.sky_a.x + L.sky_b.x * c, L.sky_a.y + L.sky_b.y * c,
                              L.sky_a.z + L.sky_b.z * c, v.t_max);
        } else {
            const float4* T = s.tris + 3 * (int64_t)h.k;
            float4 p0 = __ldg(T), p1 = __ldg(T + 1), p2 = __ldg(T + 2);
            float3 ng = cross(f3(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z),
                              f3(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z));
            if (dot(d, ng) > 0.0f) {
                // back face: radiance 0, depth shortened by 80% (Sec. 4.1)
                rec = make_float4(0.0f, 0.0f, 0.0f, fminf(0.2f * h.t, v.t_max));
            } else {
                float3 n = (1.0f / length(ng)) * ng;
                float3 x = o + h.t * d;
                int2 at = __ldg(s.attr + h.orig);
                float4 rho = __ldg(s.albedo + at.x);
                float3 Le = f3(0.0f, 0.0f, 0.0f);
                if (at.y >= 0) {
                    float4 e = __ldg(s.emit + at.y);
                    Le = f3(e.x, e.y, e.z);
                }
                float3 direct = f3(0.0f, 0.0f, 0.0f);
                float3 tol = f3(-L.sun_dir.x, -L.sun_dir.y, -L.sun_dir.z);
                float cosl = dot(n, tol);
                if (L.sun_on && cosl > 0.0f) {
                    float off = 1e-4f * (1.0f + length(x));
                    RayPre sr = ray_pre(x + off * n, tol);
                    Hit sh = traverse<true, COUNT>(s, sr, &cs);
                    if (COUNT) n_shadow++;
                    if (sh.orig < 0) {
                        float k = cosl * 0.318309886183790672f;   // 1/pi
                        direct = f3(L.sun_irr.x * k, L.sun_irr.y * k, L.sun_irr.z * k);
                    }
                }
                float3 M = query_M(v, x, n, f3(-d.x, -d.y, -d.z));
                if (COUNT) n_query++;
                rec = make_float4(Le.x + rho.x * (direct.x + M.x), Le.y + rho.y * (direct.y + M.y),
                                  Le.z + rho.z * (direct.z + M.z), fminf(h.t, v.t_max));
            }
        }
        if (!COUNT) records[idx] = rec;
    }
    if (COUNT) {
        atomicAdd(stats + 0, (unsigned long long)n_rays);
        atomicAdd(stats + 1, (unsigned long long)cp.nodes);
        atomicAdd(stats + 2, (unsigned long long)cp.tris);
        atomicAdd(stats + 3, (unsigned long long)n_shadow);
        atomicAdd(stats + 4, (unsigned long long)cs.nodes);
        atomicAdd(stats + 5, (unsigned long long)cs.tris);
        atomicAdd(stats + 6, (unsigned long long)n_query);
    }
}

__global__ void k_trace_rays(DevScene s, const float* __restrict__ orig, const float* __restrict__ dir,
                             int64_t n, float* __restrict__ t_out, int32_t* __restrict__ tri_out,
                             int32_t* __restrict__ bf_out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        float3 o = f3(orig[3 * q], orig[3 * q + 1], orig[3 * q + 2]);
        float3 d = f3(dir[3 * q], dir[3 * q + 1], dir[3 * q + 2]);
        Hit h = traverse<false>(s, ray_pre(o, d));
        t_out[q] = h.t;
        tri_out[q] = h.orig;
        if (bf_out) {
            int b = 0;
            if (h.orig >= 0) {
                const float4* T = s.tris + 3 * (int64_t)h.k;
                float4 p0 = __ldg(T), p1 = __ldg(T + 1), p2 = __ldg(T + 2);
                float3 ng = cross(f3(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z),
                                  f3(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z));
                b = dot(d, ng) > 0.0f;
            }
            bf_out[q] = b;
        }
    }
}

__global__ void k_gbuffer(DevScene s, float3 cpos, float3 fwd, float3 right, float3 up, float tan_half,
                          float aspect, int w, int h, float* __restrict__ out_pos,
                          float* __restrict__ out_nrm) {
    int64_t n = (int64_t)w * h;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        int y = (int)(q / w), x = (int)(q - (int64_t)y * w);
        float sx = ((x + 0.5f) / w * 2.0f - 1.0f) * tan_half * aspect;
        float sy = (1.0f - (y + 0.5f) / h * 2.0f) * tan_half;
        float3 d = fwd + sx * right + sy * up;
        d = (1.0f / length(d)) * d;
        Hit hh = traverse<false>(s, ray_pre(cpos, d));
        float3 p = f3(0.0f, 0.0f, 0.0f), nn = f3(0.0f, 0.0f, 0.0f);
        if (hh.orig >= 0) {
            const float4* T = s.tris + 3 * (int64_t)hh.k;
            float4 p0 = __ldg(T), p1 = __ldg(T + 1), p2 = __ldg(T + 2);
            float3 ng = cross(f3(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z),
                              f3(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z));
            nn = (1.0f / length(ng)) * ng;
            p = cpos + hh.t * d;
        }
        out_pos[3 * q] = p.x; out_pos[3 * q + 1] = p.y; out_pos[3 * q + 2] = p.z;
        out_nrm[3 * q] = nn.x; out_nrm[3 * q + 1] = nn.y; out_nrm[3 * q + 2] = nn.z;
    }
}

cudaError_t launch_classify(const DevScene& s, const VolView& v, const float4* dirs, int R,
                            const int32_t* list, const int32_t* count, int grid, cudaStream_t st) {
    k_classify<<<grid, 256, 0, st>>>(s, v, dirs, R, list, count);
    return cudaGetLastError();
}

cudaError_t launch_trace_shade(const DevScene& s, const VolView& v, const Lights& L, const float4* dirs,
                               int R, const int32_t* active, const int32_t* count, float4* records,
                               int grid, cudaStream_t st) {
    k_trace_shade<false><<<grid, 128, 0, st>>>(s, v, L, dirs, R, active, count, records, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_trace_shade_count(const DevScene& s, const VolView& v, const Lights& L,
                                     const float4* dirs, int R, const int32_t* active,
                                     const int32_t* count, unsigned long long* stats, int grid,
                                     cudaStream_t st) {
    k_trace_shade<true><<<grid, 128, 0, st>>>(s, v, L, dirs, R, active, count, nullptr, stats);
    return cudaGetLastError();
}

cudaError_t launch_trace_rays(const DevScene& s, const float* orig, const float* dir, int64_t n,
                              float* t, int32_t* tri, int32_t* backface, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + 127) / 128;
    int grid = (int)(blocks < 65535 ? blocks : 65535);
    k_trace_rays<<<grid, 128, 0, st>>>(s, orig, dir, n, t, tri, backface);
    return cudaGetLastError();
}

cudaError_t launch_gbuffer(const DevScene& s, float3 pos, float3 fwd, float3 right, float3 up,
                           float tan_half, float aspect, int w, int h, float* out_pos, float* out_nrm,
                           cudaStream_t st) {
    int64_t n = (int64_t)w * h;
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + 127) / 128;
    int grid = (int)(blocks < 65535 ? blocks : 65535);
    k_gbuffer<<<grid, 128, 0, st>>>(s, pos, fwd, right, up, tan_half, aspect, w, h, out_pos, out_nrm);
    return cudaGetLastError();
}

}  // namespace ddgi
