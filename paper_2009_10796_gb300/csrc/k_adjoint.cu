// Adjoint of the differentiable forward: n frames of the update from a zero
// atlas with hysteresis 0 (every probe tracing), then the query.  Parameters
// are the emitters' radiance and the objects' albedo; geometry is fixed, so
// hits, distances and the query's backface / Chebyshev / trilinear weights
// are constants.  Reverse order:
//   k_query_adjoint   dE at query points -> texel gradients of the last atlas
//   k_border_fold     border-texel gradients -> the interior texels they copy
//   k_blend_adjoint   texel gradients -> per-ray radiance gradients:
//                     dL_i = sum_t W[t][i] / s_t * de_t * de/dm (gamma chain)
//   k_shade_adjoint   rays re-traced: dL_i -> emitter radiance (front hits),
//                     albedo (direct + previous-frame term), and through the
//                     previous-frame query at the hit -> that atlas's texels
// Gradients accumulate with float atomics (order-dependent rounding only).
#include "traverse.cuh"

namespace ddgi {

// Reverse of query_M: M_c = A_c^2, A_c = sum_p w_p a_pc / sum_p w_p,
// a_pc = b_pc^(gamma/2), b the bilinear sample of probe p's tile in
// direction n.  Scatters dM into g_irr (float [P][tile][3]).
__device__ void query_M_adjoint(const VolView& v, float3 x, float3 n, float3 wo, float3 dM, float* g_irr) {
    const LocalPoint q = local_point(v, x, n, wo);
    float g[3] = {(q.hi.x + q.lb.x) / v.spacing.x, (q.hi.y + q.lb.y) / v.spacing.y,
                  (q.hi.z + q.lb.z) / v.spacing.z};
    int cnt[3] = {v.counts.x, v.counts.y, v.counts.z};
    int base[3];
    float fr[3];
    for (int a = 0; a < 3; ++a) {
        float b = floorf(g[a]);
        b = fminf(fmaxf(b, 0.0f), (float)(cnt[a] - 2));
        base[a] = (int)b;
        fr[a] = fminf(fmaxf(g[a] - b, 0.0f), 1.0f);
    }
    float w8[8];
    int p8[8];
    float3 b8[8];
    float sumw = 0.0f;
    float3 acc = f3(0.0f, 0.0f, 0.0f);
    Footprint fp = footprint(oct_encode(n), v.irr_n);
    for (int c = 0; c < 8; ++c) {
        int o0 = c & 1, o1 = (c >> 1) & 1, o2 = (c >> 2) & 1;
        int p = probe_phys(v, base[0] + o0, base[1] + o1, base[2] + o2);
        p8[c] = p;
        w8[c] = 0.0f;
        if (!state_active(v.states[p])) continue;
        float3 a = local_to_probe(v, q, base[0] + o0, base[1] + o1, base[2] + o2);
        if (v.offsets) {   // the probe's own (moved) position; the cage stays on the grid
            const float4 po = v.offsets[p];
            a = f3(a.x - po.x, a.y - po.y, a.z - po.z);
        }
        float wt = (o0 ? fr[0] : 1.0f - fr[0]) * (o1 ? fr[1] : 1.0f - fr[1]) * (o2 ? fr[2] : 1.0f - fr[2]);
        float3 dp = f3(-(a.x + q.lo.x), -(a.y + q.lo.y), -(a.z + q.lo.z));   // probe - x
        float ldp = length(dp);
        float cw = ldp > 0.0f ? dot(n, dp) / ldp : 1.0f;
        float hb = (1.0f + cw) * 0.5f;
        float wb = hb * hb + 0.2f;
        float3 pv = a + q.lb;                                                // biased point - probe
        float r = length(pv);
        float wc = 1.0f;
        if (r > 0.0f) {
            float2 mom = sample_dist(v, p, (1.0f / r) * pv);
            if (r > mom.x) {
                float var = fmaxf(mom.y - mom.x * mom.x, 0.0f);
                float dr = r - mom.x;
                wc = var / (var + dr * dr);
            }
        }
        float w = wt * wb * fmaxf(wc, 1e-6f);
        w8[c] = w;
        float3 e = sample_irr(v, p, n);
        b8[c] = e;
        acc.x += w * gamma_decode_half(e.x, v.half_gamma);
        acc.y += w * gamma_decode_half(e.y, v.half_gamma);
        acc.z += w * gamma_decode_half(e.z, v.half_gamma);
        sumw += w;
    }
    if (!(sumw > 0.0f)) return;
    float inv = 1.0f / sumw;
    float A[3] = {acc.x * inv, acc.y * inv, acc.z * inv};
    float dMv[3] = {dM.x, dM.y, dM.z};
    float bw[4] = {(1.0f - fp.tx) * (1.0f - fp.ty), fp.tx * (1.0f - fp.ty), (1.0f - fp.tx) * fp.ty, fp.tx * fp.ty};
    int bx[4] = {fp.x0, fp.x0 + 1, fp.x0, fp.x0 + 1}, by[4] = {fp.y0, fp.y0, fp.y0 + 1, fp.y0 + 1};
    const int N = v.irr_n + 2;
    for (int c = 0; c < 8; ++c) {
        if (!(w8[c] > 0.0f)) continue;
        float bb[3] = {b8[c].x, b8[c].y, b8[c].z};
        for (int ch = 0; ch < 3; ++ch) {
            if (!(bb[ch] > 0.0f)) continue;
            float d = dMv[ch] * 2.0f * A[ch] * w8[c] * inv * v.half_gamma * powf(bb[ch], v.half_gamma - 1.0f);
            for (int j = 0; j < 4; ++j)
                atomicAdd(g_irr + ((int64_t)p8[c] * v.irr_tile + by[j] * N + bx[j]) * 3 + ch, d * bw[j]);
        }
    }
}

__global__ void k_query_adjoint(VolView v, const float* __restrict__ pos, const float* __restrict__ nrm, int64_t n,
                                float3 cam, const float* __restrict__ dE, float* g_irr) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        float3 x = f3(pos[3 * q], pos[3 * q + 1], pos[3 * q + 2]);
        float3 nn = f3(nrm[3 * q], nrm[3 * q + 1], nrm[3 * q + 2]);
        if (nn.x == 0.0f && nn.y == 0.0f && nn.z == 0.0f) continue;
        float3 wo = cam - x;
        float l = length(wo);
        wo = l < 1e-6f ? nn : (1.0f / l) * wo;
        const float pi = 3.14159265358979323846f;
        query_M_adjoint(v, x, nn, wo, f3(pi * dE[3 * q], pi * dE[3 * q + 1], pi * dE[3 * q + 2]), g_irr);
    }
}

// One block per probe: each interior texel gathers the gradients of the
// border texels that copy it, then the border gradients are cleared.
__global__ void k_border_fold(float* g_irr, int n) {
    const int N = n + 2;
    float* t = g_irr + (int64_t)blockIdx.x * N * N * 3;
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
        int x = 1 + q % n, y = 1 + q / n;
        float add[3] = {0.0f, 0.0f, 0.0f};
        auto gather = [&](int bx, int by) {
            for (int c = 0; c < 3; ++c) add[c] += t[(by * N + bx) * 3 + c];
        };
        if (x == 1) gather(0, n + 1 - y);
        if (x == n) gather(n + 1, n + 1 - y);
        if (y == 1) gather(n + 1 - x, 0);
        if (y == n) gather(n + 1 - x, n + 1);
        if (x == n && y == n) gather(0, 0);
        if (x == 1 && y == n) gather(n + 1, 0);
        if (x == n && y == 1) gather(0, n + 1);
        if (x == 1 && y == 1) gather(n + 1, n + 1);
        for (int c = 0; c < 3; ++c) t[(y * N + x) * 3 + c] += add[c];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < N * N; q += blockDim.x) {
        int x = q % N, y = q / N;
        if (x == 0 || y == 0 || x == N - 1 || y == N - 1)
            for (int c = 0; c < 3; ++c) t[q * 3 + c] = 0.0f;
    }
}

// Thread per (probe, ray): dL = sum_t W[t][i] inv_s[t] g[t] * de/dm, with the
// texel value e of the atlas this frame wrote (e = m^(1/gamma)).
__global__ void k_blend_adjoint(VolView v_after, const float* __restrict__ w_irr, const float* __restrict__ inv_s,
                                const float* __restrict__ g_irr, int P, int R, float4* __restrict__ gL) {
    const int ni = v_after.irr_n, N = ni + 2, ti = ni * ni;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)P * R;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int p = (int)(idx / R), i = (int)(idx - (int64_t)p * R);
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
        for (int t = 0; t < ti; ++t) {
            float is = __ldg(inv_s + t);
            if (!(is >= 0.0f)) continue;
            float w = __ldg(w_irr + (int64_t)t * R + i) * is;
            if (w == 0.0f) continue;
            int x = 1 + t % ni, y = 1 + t / ni;
            const float* gg = g_irr + ((int64_t)p * v_after.irr_tile + y * N + x) * 3;
            float3 e = load_irr<true>(v_after, p, x, y);
            float ee[3] = {e.x, e.y, e.z};
            float gd[3];
            for (int c = 0; c < 3; ++c) {
                // de/dm = (1/gamma) e^(1 - gamma); at e = 0 only gamma = 1 has a derivative
                float d = ee[c] > 0.0f ? v_after.inv_gamma * powf(ee[c], 1.0f - v_after.gamma)
                                       : (v_after.gamma == 1.0f ? 1.0f : 0.0f);
                gd[c] = __ldg(gg + c) * d;
            }
            a0 = fmaf(w, gd[0], a0);
            a1 = fmaf(w, gd[1], a1);
            a2 = fmaf(w, gd[2], a2);
        }
        gL[idx] = make_float4(a0, a1, a2, 0.0f);
    }
}

// Thread per (probe, ray) of frame f, re-traced against the scene.  v_before
// is the atlas the frame's hit shading sampled (the previous frame's).
__global__ void k_shade_adjoint(DevScene s, VolView v_before, Lights L, const float4* __restrict__ dirs, int P,
                                int R, const float4* __restrict__ gL, float* d_emit, float* d_albedo,
                                float* g_prev, int with_prev) {
    const int64_t total = (int64_t)P * R;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const float3 tol = f3(-L.sun_dir.x, -L.sun_dir.y, -L.sun_dir.z);
    const RayPre r_sun = ray_pre(f3(0.0f, 0.0f, 0.0f), tol);
    int2 stack[kStackSize4];
    WwLane<kStackSize4, int2> w;
    w.stack = stack;
    // warp-uniform loop: 32 rays per warp through the warp-cooperative 4-wide
    // walk (rays without a gradient take part without tracing), then their
    // shadow rays the same way
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
        const int64_t idx = base + lane;
        const float4 g4 = idx < total ? gL[idx] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const bool valid = g4.x != 0.0f || g4.y != 0.0f || g4.z != 0.0f;
        const int64_t id = valid ? idx : 0;
        int p = (int)(id / R), i = (int)(id - (int64_t)p * R);
        float3 o = probe_pos_phys(v_before, p);
        float4 d4 = __ldg(dirs + i);
        float3 d = f3(d4.x, d4.y, d4.z);
        const RayPre r = ray_pre_packed(o, d, __ldg(dirs + R + 2 * i), __ldg(dirs + R + 2 * i + 1));
        ww_start(s, w, valid);
        do {
            ww4_round<false>(s, r, w);
        } while (__ballot_sync(0xffffffffu, w.node != kDone) != 0);
        const Hit h = w.h;
        bool front = false;
        float3 n = f3(0.0f, 0.0f, 1.0f), x = o;
        float cosl = 0.0f;
        if (valid && h.orig >= 0) {
            const float4* T = s.tris + 3 * (int64_t)h.k;
            float4 p0 = __ldg(T), p1 = __ldg(T + 1), p2 = __ldg(T + 2);
            float3 ng = cross(f3(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z), f3(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z));
            front = !(dot(d, ng) > 0.0f);   // back faces carry no radiance
            n = (1.0f / length(ng)) * ng;
            x = o + h.t * d;
            cosl = dot(n, tol);
        }
        const bool shadow = front && L.sun_on && cosl > 0.0f;
        RayPre sr = r_sun;
        if (shadow) ray_set_origin(sr, x + (1e-4f * (1.0f + length(x))) * n);
        ww_start(s, w, shadow);
        do {
            ww4_round<true>(s, sr, w);
        } while (__ballot_sync(0xffffffffu, w.node != kDone) != 0);
        const bool lit = shadow && w.h.orig < 0;
        if (!front) continue;
        int2 at = __ldg(s.attr + h.orig);
        if (at.y >= 0) {
            atomicAdd(d_emit + 3 * at.y + 0, g4.x);
            atomicAdd(d_emit + 3 * at.y + 1, g4.y);
            atomicAdd(d_emit + 3 * at.y + 2, g4.z);
        }
        float3 direct = f3(0.0f, 0.0f, 0.0f);
        if (lit) {
            float kk = cosl * 0.318309886183790672f;
            direct = f3(L.sun_irr.x * kk, L.sun_irr.y * kk, L.sun_irr.z * kk);
        }
        float3 wo = f3(-d.x, -d.y, -d.z);
        float3 M = query_M(v_before, x, n, wo);
        atomicAdd(d_albedo + 3 * at.x + 0, g4.x * (direct.x + M.x));
        atomicAdd(d_albedo + 3 * at.x + 1, g4.y * (direct.y + M.y));
        atomicAdd(d_albedo + 3 * at.x + 2, g4.z * (direct.z + M.z));
        if (with_prev) {
            float4 rho = __ldg(s.albedo + at.x);
            query_M_adjoint(v_before, x, n, wo, f3(g4.x * rho.x, g4.y * rho.y, g4.z * rho.z), g_prev);
        }
    }
}

// Copies per-object albedo [O][3] and per-emitter radiance [E][3] (device)
// into the scene's tables, keeping each object's flags.
__global__ void k_set_materials(float4* albedo, int n_obj, const float* __restrict__ alb, float4* emit, int n_em,
                                const float* __restrict__ em) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_obj + n_em; k += gridDim.x * blockDim.x) {
        if (k < n_obj) {
            if (alb) {
                float4 a = albedo[k];
                albedo[k] = make_float4(alb[3 * k], alb[3 * k + 1], alb[3 * k + 2], a.w);
            }
        } else if (em) {
            int e = k - n_obj;
            emit[e] = make_float4(em[3 * e], em[3 * e + 1], em[3 * e + 2], 0.0f);
        }
    }
}

static int grid_for(int64_t n, int block) {
    int64_t b = (n + block - 1) / block;
    return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

cudaError_t launch_query_adjoint(const VolView& v, const float* pos, const float* nrm, int64_t n, float3 cam,
                                 const float* dE, float* g_irr, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_query_adjoint<<<grid_for(n, 128), 128, 0, st>>>(v, pos, nrm, n, cam, dE, g_irr);
    return cudaGetLastError();
}

cudaError_t launch_border_fold(float* g_irr, int P, int n, cudaStream_t st) {
    k_border_fold<<<P, 64, 0, st>>>(g_irr, n);
    return cudaGetLastError();
}

cudaError_t launch_blend_adjoint(const VolView& v_after, const float* w_irr, const float* inv_s, const float* g_irr,
                                 int P, int R, float4* gL, cudaStream_t st) {
    k_blend_adjoint<<<grid_for((int64_t)P * R, 128), 128, 0, st>>>(v_after, w_irr, inv_s, g_irr, P, R, gL);
    return cudaGetLastError();
}

cudaError_t launch_shade_adjoint(const DevScene& s, const VolView& v_before, const Lights& L, const float4* dirs,
                                 int P, int R, const float4* gL, float* d_emit, float* d_albedo, float* g_prev,
                                 int with_prev, cudaStream_t st) {
    k_shade_adjoint<<<grid_for((int64_t)P * R, 128), 128, 0, st>>>(s, v_before, L, dirs, P, R, gL, d_emit,
                                                                   d_albedo, g_prev, with_prev);
    return cudaGetLastError();
}

cudaError_t launch_set_materials(float4* albedo, int n_obj, const float* alb, float4* emit, int n_em, const float* em,
                                 cudaStream_t st) {
    k_set_materials<<<grid_for(n_obj + n_em, 128), 128, 0, st>>>(albedo, n_obj, alb, emit, n_em, em);
    return cudaGetLastError();
}

}  // namespace ddgi
