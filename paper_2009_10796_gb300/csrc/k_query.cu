// Shading-point query (Sec. 2.2, 4.1, 4.2) and probe-list compaction.
#include "probe_math.cuh"

namespace ddgi {

// One thread per point; positions, normals and outputs are [n][3] floats, read
// and written with unit-stride scalar accesses (coalesced per warp).
__global__ void __launch_bounds__(256) k_query(VolView v, const float* __restrict__ pos,
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
            float3 M = query_M(v, x, nn, wo);
            const float pi = 3.14159265358979323846f;
            E = f3(pi * M.x, pi * M.y, pi * M.z);
        }
        out[3 * q] = E.x;
        out[3 * q + 1] = E.y;
        out[3 * q + 2] = E.z;
    }
}

// Compacts probe indices whose state matches `which` (0: UNINIT, 1: active =
// NEWLY_VIGILANT or VIGILANT) into list[], count[0] += matches.  Warp-
// aggregated atomics: one atomic per warp.  List order is not deterministic;
// consumers carry the probe index with each entry.
__global__ void k_build_list(const uint8_t* __restrict__ states, int P, int which, int32_t* list,
                             int32_t* count) {
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < P; base += gridDim.x * blockDim.x) {
        int p = base + threadIdx.x;
        bool pred = false;
        if (p < P) {
            uint8_t s = states[p];
            pred = which == 0 ? s == DDGI_STATE_UNINIT : state_active(s);
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

cudaError_t launch_query(const VolView& v, const float* pos, const float* nrm, int64_t n, float3 camera,
                         float* out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    int grid = (int)(blocks < 1048576 ? blocks : 1048576);
    k_query<<<grid, 256, 0, st>>>(v, pos, nrm, n, camera, out);
    return cudaGetLastError();
}

cudaError_t launch_build_list(const uint8_t* states, int P, int which, int32_t* list, int32_t* count,
                              cudaStream_t st) {
    int blocks = (P + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_build_list<<<blocks, 256, 0, st>>>(states, P, which, list, count);
    return cudaGetLastError();
}

}  // namespace ddgi
