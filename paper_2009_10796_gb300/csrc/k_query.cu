// Shading-point query (Sec. 2.2, 4.1, 4.2) and probe-list compaction.
#include "probe_math.cuh"

namespace ddgi {

// One thread per point; positions and normals are [n][3] floats read with
// unit-stride scalar loads (coalesced per warp).  STAGE_OUT: a block's
// outputs are staged in shared memory and written as one contiguous run
// (16-byte stores when the run is aligned), so each warp writes whole lines,
// for page-locked host memory written across the host link; otherwise each
// thread stores its own three floats (device memory).
// The specialised form runs five CTAs per SM (48 registers, a short spill),
// which measured 1 us faster on the 1080p query than four; the general form
// keeps four.
constexpr int kQueryThreads = 256;
template <bool STAGE_OUT, bool FAST>
__global__ void __launch_bounds__(kQueryThreads, FAST ? 5 : 4) k_query(VolView v, const float* __restrict__ pos,
                                                         const float* __restrict__ nrm, int64_t n, float3 cam,
                                                         float* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    __shared__ __align__(16) float s_out[3 * kQueryThreads];
    for (int64_t q0 = (int64_t)blockIdx.x * kQueryThreads; q0 < n; q0 += (int64_t)gridDim.x * kQueryThreads) {
        const int64_t q = q0 + threadIdx.x;
        float3 E = f3(0.0f, 0.0f, 0.0f);
        if (q < n) {
            float3 x = f3(__ldg(pos + 3 * q), __ldg(pos + 3 * q + 1), __ldg(pos + 3 * q + 2));
            float3 nn = f3(__ldg(nrm + 3 * q), __ldg(nrm + 3 * q + 1), __ldg(nrm + 3 * q + 2));
            if (nn.x != 0.0f || nn.y != 0.0f || nn.z != 0.0f) {
                float3 wo = cam - x;
                float l = length(wo);
                wo = l < 1e-6f ? nn : (1.0f / l) * wo;
                float3 M = query_M<FAST>(v, x, nn, wo);
                const float pi = 3.14159265358979323846f;
                E = f3(pi * M.x, pi * M.y, pi * M.z);
            }
        }
        if (!STAGE_OUT) {
            if (q < n) {
                out[3 * q] = E.x;
                out[3 * q + 1] = E.y;
                out[3 * q + 2] = E.z;
            }
            continue;
        }
        s_out[3 * threadIdx.x] = E.x;
        s_out[3 * threadIdx.x + 1] = E.y;
        s_out[3 * threadIdx.x + 2] = E.z;
        __syncthreads();
        const int nf = 3 * (int)min((int64_t)kQueryThreads, n - q0);   // floats of this block's run
        float* dst = out + 3 * q0;
        if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
            for (int i = threadIdx.x; i < nf / 4; i += kQueryThreads)
                reinterpret_cast<float4*>(dst)[i] = reinterpret_cast<const float4*>(s_out)[i];
            for (int i = (nf / 4) * 4 + threadIdx.x; i < nf; i += kQueryThreads) dst[i] = s_out[i];
        } else {
            for (int i = threadIdx.x; i < nf; i += kQueryThreads) dst[i] = s_out[i];
        }
        __syncthreads();
    }
}

// Second-order glossy lookup (Sec. 4.4): one thread per reflection-ray hit;
// dirs are the unit directions the hits were reached along.  Output is the
// prefiltered radiance M read in the mirror direction (no factor pi).
template <bool FAST>
__global__ void __launch_bounds__(256) k_query_glossy(VolView v, const float* __restrict__ pos,
                                                      const float* __restrict__ nrm, const float* __restrict__ dirs,
                                                      int64_t n, float* __restrict__ out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        float3 x = f3(__ldg(pos + 3 * q), __ldg(pos + 3 * q + 1), __ldg(pos + 3 * q + 2));
        float3 nn = f3(__ldg(nrm + 3 * q), __ldg(nrm + 3 * q + 1), __ldg(nrm + 3 * q + 2));
        float3 d = f3(__ldg(dirs + 3 * q), __ldg(dirs + 3 * q + 1), __ldg(dirs + 3 * q + 2));
        float3 M = f3(0.0f, 0.0f, 0.0f);
        if (nn.x != 0.0f || nn.y != 0.0f || nn.z != 0.0f) {
            float dn = dot(d, nn);
            float3 r = d - (2.0f * dn) * nn;
            float lr = length(r);
            if (lr > 0.0f) r = (1.0f / lr) * r;
            M = query_M_look<FAST>(v, x, nn, f3(-d.x, -d.y, -d.z), r);
        }
        out[3 * q] = M.x;
        out[3 * q + 1] = M.y;
        out[3 * q + 2] = M.z;
    }
}

// Compacts probe indices whose state matches `which` (0: UNINIT, 1: active =
// traced and blended, 2: newly = Newly Vigilant or Newly Awake) into list[],
// count[0] += matches.  Warp-
// aggregated atomics: one atomic per warp.  List order is not deterministic;
// consumers carry the probe index with each entry.
__global__ void k_build_list(const uint8_t* __restrict__ states, int begin, int end, int which, int32_t* list,
                             int32_t* count) {
    const int lane = threadIdx.x & 31;
    for (int base = begin + blockIdx.x * blockDim.x; base < end; base += gridDim.x * blockDim.x) {
        int p = base + threadIdx.x;
        bool pred = false;
        if (p < end) {
            uint8_t s = states[p];
            pred = which == 0 ? s == DDGI_STATE_UNINIT : (which == 2 ? state_newly(s) : state_active(s));
        }
        unsigned mask = __ballot_sync(0xffffffffu, pred);
        if (mask == 0) continue;
        int leader = __ffs(mask) - 1;
        int off = 0;
        if (lane == leader) off = atomicAdd(count, __popc(mask));
        off = __shfl_sync(0xffffffffu, off, leader);
        if (pred) list[off + __popc(mask & ((1u << lane) - 1u))] = p;
    }
}

// Dynamic-object wake-up (Sec. 6.3): probes [begin, end); a Sleeping probe
// inside a box (already extended by one cell plus the self-shadow bias)
// becomes Newly Awake, an Awake probe inside none goes back to Sleeping.
__global__ void __launch_bounds__(256) k_wake(VolView v, const float* __restrict__ boxes, int n_boxes, int begin,
                                              int end) {
    extern __shared__ float sbox[];   // n_boxes x 6
    for (int k = threadIdx.x; k < 6 * n_boxes; k += blockDim.x) sbox[k] = boxes[k];
    __syncthreads();
    for (int p = begin + blockIdx.x * blockDim.x + threadIdx.x; p < end; p += gridDim.x * blockDim.x) {
        const uint8_t s = v.states[p];
        if (s != DDGI_STATE_SLEEPING && s != DDGI_STATE_AWAKE) continue;
        const float3 x = probe_pos_phys(v, p);
        bool inside = false;
        for (int b = 0; b < n_boxes && !inside; ++b) {
            const float* bx = sbox + 6 * b;
            inside = x.x >= bx[0] && x.y >= bx[1] && x.z >= bx[2] && x.x <= bx[3] && x.y <= bx[4] && x.z <= bx[5];
        }
        if (s == DDGI_STATE_SLEEPING && inside) v.states[p] = DDGI_STATE_NEWLY_AWAKE;
        else if (s == DDGI_STATE_AWAKE && !inside) v.states[p] = DDGI_STATE_SLEEPING;
    }
}

cudaError_t launch_wake(const VolView& v, const float* boxes, int n_boxes, int begin, int end, cudaStream_t st) {
    if (end <= begin) return cudaSuccess;
    int blocks = (end - begin + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_wake<<<blocks, 256, sizeof(float) * 6 * (size_t)n_boxes, st>>>(v, boxes, n_boxes, begin, end);
    return cudaGetLastError();
}

// Cascade query (Sec. 7.3): one thread per point, volumes densest first.
__global__ void __launch_bounds__(256) k_query_cascade(VolSet vs, const float* __restrict__ pos,
                                                       const float* __restrict__ nrm, int64_t n, float3 cam,
                                                       float* __restrict__ out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        float3 x = f3(__ldg(pos + 3 * q), __ldg(pos + 3 * q + 1), __ldg(pos + 3 * q + 2));
        float3 nn = f3(__ldg(nrm + 3 * q), __ldg(nrm + 3 * q + 1), __ldg(nrm + 3 * q + 2));
        float3 E = f3(0.0f, 0.0f, 0.0f);
        if (nn.x != 0.0f || nn.y != 0.0f || nn.z != 0.0f) {
            float3 wo = cam - x;
            float l = length(wo);
            wo = l < 1e-6f ? nn : (1.0f / l) * wo;
            float3 M = cascade_M(vs.table, vs.n, x, nn, wo);
            const float pi = 3.14159265358979323846f;
            E = f3(pi * M.x, pi * M.y, pi * M.z);
        }
        out[3 * q] = E.x;
        out[3 * q + 1] = E.y;
        out[3 * q + 2] = E.z;
    }
}

// List build over every volume of a set: global index g runs over the
// volumes' probes in order; entries are (volume << 24) | probe.
__global__ void k_build_list_multi(VolSet vs, int total, int which, int32_t* list, int32_t* count) {
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < total; base += gridDim.x * blockDim.x) {
        int g = base + threadIdx.x;
        bool pred = false;
        int entry = 0;
        if (g < total) {
            int k = 0, off = 0;
            while (k + 1 < vs.n && g >= off + vs.table[k].n_probes) {
                off += vs.table[k].n_probes;
                ++k;
            }
            int p = g - off;
            uint8_t s = vs.table[k].states[p];
            pred = which == 0 ? s == DDGI_STATE_UNINIT : state_active(s);
            entry = (k << kEntryShift) | p;
        }
        unsigned mask = __ballot_sync(0xffffffffu, pred);
        if (mask == 0) continue;
        int leader = __ffs(mask) - 1;
        int o = 0;
        if (lane == leader) o = atomicAdd(count, __popc(mask));
        o = __shfl_sync(0xffffffffu, o, leader);
        if (pred) list[o + __popc(mask & ((1u << lane) - 1u))] = entry;
    }
}

// Tracking-window reset (Sec. 7.2): every probe of a leapfrogged plane gets
// zero texels and state UNINIT.  The blocks share each plane's probes; a
// block zeroes one probe's tiles with consecutive 4-byte stores (every atlas
// format encodes 0 as zero bits).
__global__ void k_reset_planes(VolSet vs, const int4* __restrict__ planes, const int32_t* __restrict__ count) {
    const int n_planes = *count;
    for (int k = 0; k < n_planes; ++k) {
        const int4 pl = planes[k];          // (volume, axis, physical plane, 0)
        const VolView& v = vs.table[pl.x];
        const int cnt[3] = {v.counts.x, v.counts.y, v.counts.z};
        const int a = pl.y, b = (a + 1) % 3, c = (a + 2) % 3;
        const int n_probes = cnt[b] * cnt[c];
        const int irr_words = v.irr_tile * (v.irr_format == DDGI_IRR_FP32 ? 4 : (v.irr_format == DDGI_IRR_FP16 ? 2 : 1));
        const int dist_words = v.dist_tile * (v.dist_format == DDGI_DIST_FP32 ? 2 : 1);
        for (int q = blockIdx.x; q < n_probes; q += gridDim.x) {
            int ijk[3];
            ijk[a] = pl.z;
            ijk[b] = q % cnt[b];
            ijk[c] = q / cnt[b];
            const int p = ijk[0] + cnt[0] * (ijk[1] + cnt[1] * ijk[2]);
            if (threadIdx.x == 0) v.states[p] = DDGI_STATE_UNINIT;
            uint32_t* ti = reinterpret_cast<uint32_t*>(v.irr) + (int64_t)p * irr_words;
            uint32_t* td = reinterpret_cast<uint32_t*>(v.dist) + (int64_t)p * dist_words;
            for (int i = threadIdx.x; i < irr_words; i += blockDim.x) ti[i] = 0u;
            for (int i = threadIdx.x; i < dist_words; i += blockDim.x) td[i] = 0u;
        }
    }
}

cudaError_t launch_query_cascade(const VolSet& vs, const float* pos, const float* nrm, int64_t n, float3 camera,
                                 float* out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    int grid = (int)(blocks < 1048576 ? blocks : 1048576);
    k_query_cascade<<<grid, 256, 0, st>>>(vs, pos, nrm, n, camera, out);
    return cudaGetLastError();
}

cudaError_t launch_build_list_multi(const VolSet& vs, int total, int which, int32_t* list, int32_t* count,
                                    cudaStream_t st) {
    int blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_build_list_multi<<<blocks, 256, 0, st>>>(vs, total, which, list, count);
    return cudaGetLastError();
}

cudaError_t launch_reset_planes(const VolSet& vs, const int4* planes, const int32_t* count, int max_planes,
                                cudaStream_t st) {
    if (max_planes <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    k_reset_planes<<<2 * sms, 256, 0, st>>>(vs, planes, count);
    return cudaGetLastError();
}

cudaError_t launch_query(const VolView& v, const float* pos, const float* nrm, int64_t n, float3 camera,
                         float* out, cudaStream_t st, bool out_host) {
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + kQueryThreads - 1) / kQueryThreads;
    int grid = (int)(blocks < 1048576 ? blocks : 1048576);
    const bool fast = query_fast_view(v);
    if (out_host && fast) return launch_pdl(k_query<true, true>, grid, kQueryThreads, 0, st, v, pos, nrm, n, camera, out);
    if (out_host) return launch_pdl(k_query<true, false>, grid, kQueryThreads, 0, st, v, pos, nrm, n, camera, out);
    if (fast) return launch_pdl(k_query<false, true>, grid, kQueryThreads, 0, st, v, pos, nrm, n, camera, out);
    return launch_pdl(k_query<false, false>, grid, kQueryThreads, 0, st, v, pos, nrm, n, camera, out);
}

cudaError_t launch_query_glossy(const VolView& v, const float* pos, const float* nrm, const float* dirs, int64_t n,
                                float* out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    int grid = (int)(blocks < 1048576 ? blocks : 1048576);
    if (query_fast_view(v))
        k_query_glossy<true><<<grid, 256, 0, st>>>(v, pos, nrm, dirs, n, out);
    else
        k_query_glossy<false><<<grid, 256, 0, st>>>(v, pos, nrm, dirs, n, out);
    return cudaGetLastError();
}

cudaError_t launch_build_list(const uint8_t* states, int P, int which, int32_t* list, int32_t* count,
                              cudaStream_t st) {
    return launch_build_list_range(states, 0, P, which, list, count, st);
}

cudaError_t launch_build_list_range(const uint8_t* states, int begin, int end, int which, int32_t* list,
                                    int32_t* count, cudaStream_t st) {
    int blocks = (end - begin + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_build_list<<<blocks, 256, 0, st>>>(states, begin, end, which, list, count);
    return cudaGetLastError();
}

}  // namespace ddgi
