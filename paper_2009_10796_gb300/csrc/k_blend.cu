// Per-frame ray pattern and the probe blend (Sec. 2.3 Eq. 1, Sec. 4.2, 4.3, 7.1).
//
// k_frame_setup computes, once per frame and shared by
// every probe, the ray directions w_i = R_t sf(i, R) and the texel weight
// matrices
//   W_irr[t][i]  = max(0, n_t . w_i)              (cosine weight)
//   W_dist[t][i] = max(0, n_t . w_i)^p            (power-cosine weight)
// with 1 / sum_i W per texel, in double precision, rounded once to float.
//
// The plain FP32 blend is a product of the texel weight matrices with each
// probe's ray records.  k_blend_tiled computes it register-tiled: a CTA owns
// a group of PG active probes whose records sit in shared memory as four
// channel planes (r, g, b, distance); the weight matrices stream through
// shared memory in chunks of kTileKC rays; each thread accumulates a 4-texel
// x 4-probe tile of distance moments (sum w d and sum w d^2, two FMAs per
// ray and texel) or a 4-texel x 2-probe tile of irradiance, so every
// shared-memory load feeds 8 to 16 FMAs.  k_blend_simt
// (one thread per (texel, probe) pair) covers the shapes the tiled kernel
// does not fit.  Both sum each texel's rays in ray order with the same
// operations, so they give the same bits.  The epilogue normalises, gamma-encodes,
// applies the per-texel hysteresis thresholds, lerps with the old texel and
// writes the texel plus the border texels that copy it (the octahedral
// border copy of Sec. 7.1 fused into the blend).  The probe's state advances
// Newly Vigilant -> Vigilant after its texels are written.
#include <algorithm>

#include "blend_epilogue.cuh"
#include "traverse.cuh"

namespace ddgi {

namespace {

// All three components of sf(i, n) at once (one sincos, one square root).
__device__ void sf_dir(int i, int n, double v[3]) {
    const double inv_phi = 0.61803398874989484820;
    double a = (double)i * inv_phi;
    double phi = 6.283185307179586477 * (a - floor(a));
    double z = 1.0 - (2.0 * i + 1.0) / (double)n;
    double r = sqrt(fmax(0.0, 1.0 - z * z));
    double sp, cp;
    sincos(phi, &sp, &cp);
    v[0] = cp * r;
    v[1] = sp * r;
    v[2] = z;
}

__device__ __forceinline__ void rotate_dir(const FrameRot& rot, const double sv[3], double out[3]) {
    for (int a = 0; a < 3; ++a) out[a] = rot.m[3 * a] * sv[0] + rot.m[3 * a + 1] * sv[1] + rot.m[3 * a + 2] * sv[2];
}

// The float ray direction and its packed traversal constants in a
// direction buffer of 3R float4 (directions, then two constants per ray).
__device__ __forceinline__ void store_frame_dir(float4* dirs, int R, int i, const double w[3]) {
    const float3 d = f3((float)w[0], (float)w[1], (float)w[2]);
    dirs[i] = make_float4(d.x, d.y, d.z, 0.0f);
    float4 a, b;
    dir_pre_pack(d, a, b);
    dirs[R + 2 * i] = a;
    dirs[R + 2 * i + 1] = b;
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

// c^p for c >= 0: repeated squaring when p is a small whole number (the
// usual power-cosine exponent), pow otherwise.
__device__ double cos_pow(double c, double p) {
    if (p >= 0.0 && p <= 1024.0 && p == floor(p)) {
        unsigned e = (unsigned)p;
        double r = 1.0, b = c;
        while (e) {
            if (e & 1u) r *= b;
            b *= b;
            e >>= 1;
        }
        return r;
    }
    return pow(c, p);
}

// The unrotated pattern sf(i, R) in double precision, once per volume.
__global__ void k_sf_table(int R, double* sf64) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < R) sf_dir(i, R, sf64 + 3 * i);
}

// One launch of the whole frame setup.  Block b < irr_n^2 handles
// irradiance texel b, the next dist_n^2 blocks the distance texels, rays
// strided over the block: each rotates the pattern itself from the sf table
// (the same double operations as the direction blocks, so the same
// directions), writes its weight row and 1 / row sum.  The remaining blocks
// write the frame's float directions and ray constants, and the first of
// them clears n_zero counters.  No block waits on another; a launch may
// cover a sub-range of the blocks (first_block).
template <bool ROT_DEV>
__global__ void __launch_bounds__(256) k_frame_setup(FrameRot rot_arg, const FrameRot* rot_dev, int R, int irr_n,
                                                     int dist_n, double cos_power,
                                                     const double* __restrict__ sf64, float4* dirs, float* w_irr,
                                                     float* inv_s_irr, float* w_dist, float* inv_s_dist,
                                                     int32_t* zero, int n_zero, int first_block) {
    pdl_wait();
    pdl_trigger();
    __shared__ double red[256];
    __shared__ double s_nt[3];
    const FrameRot rot = ROT_DEV ? *rot_dev : rot_arg;
    const int ti = irr_n * irr_n, nwb = ti + dist_n * dist_n;
    const int blk = (int)blockIdx.x + first_block;   // a launch may cover a sub-range of the blocks
    if (blk >= nwb) {
        if (blk == nwb && (int)threadIdx.x < n_zero) zero[threadIdx.x] = 0;
        const int i = (blk - nwb) * blockDim.x + threadIdx.x;
        if (i < R) {
            const double sv[3] = {sf64[3 * i], sf64[3 * i + 1], sf64[3 * i + 2]};
            double w[3];
            rotate_dir(rot, sv, w);
            store_frame_dir(dirs, R, i, w);
        }
        return;
    }
    const int b = blk;
    const bool is_irr = b < ti;
    const int t = is_irr ? b : b - ti;
    if (threadIdx.x == 0) texel_dir(t, is_irr ? irr_n : dist_n, s_nt);
    __syncthreads();
    const double nt[3] = {s_nt[0], s_nt[1], s_nt[2]};
    double acc = 0.0;
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
        const double sv[3] = {sf64[3 * i], sf64[3 * i + 1], sf64[3 * i + 2]};
        double w[3];
        rotate_dir(rot, sv, w);
        double c = fmax(0.0, nt[0] * w[0] + nt[1] * w[1] + nt[2] * w[2]);
        double wt = is_irr ? c : cos_pow(c, cos_power);
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

// Groups of `group` <= kProbes probes per CTA (fewer than kProbes when the
// group's records would not fit in shared memory at large R).
template <bool MULTI, int kProbes>
__global__ void __launch_bounds__(256) k_blend_simt(VolSet vs, BlendParams bp, int group,
                                                    const float* __restrict__ w_irr,
                                                    const float* __restrict__ inv_s_irr,
                                                    const float* __restrict__ w_dist,
                                                    const float* __restrict__ inv_s_dist,
                                                    const float4* __restrict__ records,
                                                    const int32_t* __restrict__ active,
                                                    const int32_t* __restrict__ count,
                                                    uint32_t* status) {
    extern __shared__ float4 srec[];   // group x (R + 1) records
    __shared__ int s_probe[kProbes];
    __shared__ int s_newly[kProbes];
    const int R = bp.R;
    const int stride = R + 1;
    const int n_act = *count;
    const VolView& v0 = vol_of<MULTI>(vs, 0);   // cascades share R and tile sizes
    const int ni = v0.irr_n, nd = v0.dist_n;
    const int ti = ni * ni, td = nd * nd;
    for (int g0 = blockIdx.x * group; g0 < n_act; g0 += gridDim.x * group) {
        const int np = min(group, n_act - g0);
        if (threadIdx.x < np) {
            int e = active[g0 + threadIdx.x];
            s_probe[threadIdx.x] = e;
            s_newly[threadIdx.x] =
                state_newly(vol_of<MULTI>(vs, e >> kEntryShift).states[e & kEntryMask]);
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
                m1 = fmaf(w, d, m1);
                m2 = fmaf(w, d * d, m2);
            }
            const int e = s_probe[pp];
            blend_dist_texel(vol_of<MULTI>(vs, e >> kEntryShift), bp, e & kEntryMask, t, m1, m2,
                             __ldg(inv_s_dist + t), s_newly[pp] != 0, status);
        }
        __syncthreads();
        if (threadIdx.x < np && s_newly[threadIdx.x]) {
            const int e = s_probe[threadIdx.x];
            {
                uint8_t* sp = vol_of<MULTI>(vs, e >> kEntryShift).states + (e & kEntryMask);
                *sp = state_advanced(*sp);
            }
        }
        __syncthreads();
    }
}

// Weight chunks of 32 rays in one buffer (the chunk's copy overlaps the
// other resident CTA's summing) measured 55.4 us on the city blend, against
// 58.3 us for chunks of 16 rays in two buffers (each chunk's copy in flight
// while the previous one is summed) and 59.4-65 us for 8-, 16- and 24-ray
// chunks in rings of one to four buffers: the chunk loop pays for its
// per-chunk barriers more than for the copies' latency.
constexpr int kTileKC = 32;   // rays per staged weight chunk
constexpr int kTileNS = 1;    // weight chunk buffers (kTileNS - 1 chunks in flight ahead)
constexpr int kTileWS = kTileKC + 4;   // weight row stride in floats: 16-byte rows, conflict-free columns
static_assert((kTileWS / 4) % 2 == 1, "eight rows at distinct 16-byte bank groups");
constexpr int kTileMaxThreads = 320;   // with 2 CTAs per SM: up to 102 registers per thread
constexpr int kRecBatch = 8;           // record loads in flight per thread while staging

// Threads, shared memory and feasibility of k_blend_tiled for a tile shape.
// Distance units fill whole warps first, so no warp runs both tile kinds.
struct TiledShape {
    int nqi, nqd;           // texel rows per register tile: ceil(texels / 4)
    int dist_units, dist_threads, irr_units, threads;
    size_t smem;
};

static TiledShape tiled_shape(int PG, int R, int irr_n, int dist_n) {
    TiledShape t;
    t.nqi = (irr_n * irr_n + 3) / 4;
    t.nqd = (dist_n * dist_n + 3) / 4;
    t.dist_units = t.nqd * (PG / 4);
    t.dist_threads = (t.dist_units + 31) / 32 * 32;
    t.irr_units = t.nqi * (PG / 2);
    t.threads = t.dist_threads + (t.irr_units + 31) / 32 * 32;
    t.smem = sizeof(float) * ((size_t)4 * PG * R + (size_t)kTileNS * 4 * (t.nqd + t.nqi) * kTileWS);
    // the epilogue reuses the same shared memory for the weighted sums and
    // the frame's inverse weight sums
    const size_t sums = sizeof(float) * ((size_t)PG * (2 * dist_n * dist_n + 3 * irr_n * irr_n) +
                                         dist_n * dist_n + irr_n * irr_n);
    if (sums > t.smem) t.smem = sums;
    return t;
}

// 16-byte asynchronous global -> shared copy (zero-filled when !valid).
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// every group but the kTileNS - 1 most recent complete
__device__ __forceinline__ void cp_async_wait_ahead() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kTileNS - 1) : "memory");
}

// Each CTA takes an equal share of the active probes (at most PG per pass;
// the grid is one wave of resident CTAs); blockDim = TiledShape::threads.
// Requires R % 4 == 0.  Thread u < dist_units owns distance texels
// tq + a * nqd (a < 4) of probes 4 pq .. 4 pq + 3; thread dist_threads + u'
// (u' < irr_units) owns irradiance texels tq + a * nqi of probes 2 pq,
// 2 pq + 1.  Striding the texels by nqd (not 4) puts a warp's weight rows on
// distinct banks.  The record planes are probe-interleaved ([ray][probe]),
// so one shared load gives a ray's value for all of a thread's probes and
// the probes pair up in packed FP32 FMAs (the same fused multiply-add per
// texel, probe and ray, in ray order, as the scalar kernel).  Weight chunks
// arrive by asynchronous copies into a ring of kTileNS buffers (with one
// buffer, the copy overlaps the other resident CTA's summing); the blend
// epilogue runs over the sums in shared memory.
template <bool MULTI, int PG>
__global__ void __launch_bounds__(kTileMaxThreads, 2) k_blend_tiled(VolSet vs, BlendParams bp,
                                                                    const float* __restrict__ w_irr,
                                                                    const float* __restrict__ inv_s_irr,
                                                                    const float* __restrict__ w_dist,
                                                                    const float* __restrict__ inv_s_dist,
                                                                    const float4* __restrict__ records,
                                                                    const int32_t* __restrict__ active,
                                                                    const int32_t* __restrict__ count,
                                                                    uint32_t* status) {
    static_assert(PG % 4 == 0, "probe groups come in quads");
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) float sm[];
    __shared__ int s_probe[PG];
    __shared__ int s_newly[PG];
    const int R = bp.R;
    const VolView& v0 = vol_of<MULTI>(vs, 0);   // cascades share R and tile sizes
    const int ni = v0.irr_n, nd = v0.dist_n;
    const int ti = ni * ni, td = nd * nd;
    const int nqi = (ti + 3) / 4, nqd = (td + 3) / 4;
    const int wrows = 4 * (nqd + nqi);          // distance rows, then irradiance rows
    float* pr = sm;                              // [R][PG] planes: radiance r, g, b and distance
    float* pgc = pr + PG * R;
    float* pbc = pgc + PG * R;
    float* pdc = pbc + PG * R;
    float* wbuf = pdc + PG * R;                  // 2 x [wrows][kTileWS] weight chunks
    const int dist_units = nqd * (PG / 4), irr_units = nqi * (PG / 2);
    const int dist_threads = (dist_units + 31) / 32 * 32;
    const int u = threadIdx.x;
    const bool is_dist = u < dist_units;
    const bool is_irr = u >= dist_threads && u - dist_threads < irr_units;
    const int ui = is_dist ? u : u - dist_threads;
    const int tq = is_dist ? ui % nqd : (is_irr ? ui % nqi : 0);
    const int pq = is_dist ? ui / nqd : (is_irr ? ui / nqi : 0);
    const int n_chunks = (R + kTileKC - 1) / kTileKC;
    const int n_act = *count;

    auto issue_chunk = [&](int c) {
        float* wb = wbuf + (c % kTileNS) * wrows * kTileWS;
        const int c0 = c * kTileKC;
        for (int k = threadIdx.x; k < wrows * (kTileKC / 4); k += blockDim.x) {
            int row = k / (kTileKC / 4), j = 4 * (k - row * (kTileKC / 4));
            bool dist_row = row < 4 * nqd;
            int t = dist_row ? row : row - 4 * nqd;
            bool ok = c0 + j < R && t < (dist_row ? td : ti);
            const float* src = (dist_row ? w_dist : w_irr) + (ok ? (int64_t)t * R + c0 + j : 0);
            cp_async16(wb + row * kTileWS + j, src, ok);
        }
        cp_async_commit();
    };

    const int per = min(PG, max(1, (n_act + (int)gridDim.x - 1) / (int)gridDim.x));
    for (int g0 = blockIdx.x * per; g0 < n_act; g0 += gridDim.x * per) {
        const int np = min(per, n_act - g0);
        const bool live = is_dist ? 4 * pq < np : 2 * pq < np;   // some of the thread's probes hold records
        for (int c = 0; c < kTileNS - 1; ++c) {   // the first chunks overlap the record staging below
            if (c < n_chunks) issue_chunk(c);
            else cp_async_commit();
        }
        if (threadIdx.x < np) {
            int e = active[g0 + threadIdx.x];
            s_probe[threadIdx.x] = e;
            const VolView& v = vol_of<MULTI>(vs, e >> kEntryShift);
            s_newly[threadIdx.x] = state_newly(v.states[e & kEntryMask]);
            // the probe's old tiles into L2 while the group is summed (the
            // epilogue then reads them from L2)
            prefetch_tiles_l2(v, e & kEntryMask);
        }
        // records -> planes, kRecBatch independent loads in flight per thread.
        // Item k is (ray pair, probe, ray within the pair): two threads read a
        // probe's 32 contiguous bytes, a warp writes 32 consecutive plane floats.
        for (int k0 = threadIdx.x; k0 < PG * R; k0 += kRecBatch * blockDim.x) {
            float4 rec[kRecBatch];
#pragma unroll
            for (int b = 0; b < kRecBatch; ++b) {
                const int k = k0 + b * blockDim.x;
                const int q = k >> 1, pp = q % PG, ray = 2 * (q / PG) + (k & 1);
                rec[b] = (k < PG * R && pp < np) ? records[(int64_t)(g0 + pp) * R + ray]
                                                 : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
#pragma unroll
            for (int b = 0; b < kRecBatch; ++b) {
                const int k = k0 + b * blockDim.x;
                if (k < PG * R) {
                    const int q = k >> 1, o = (2 * (q / PG) + (k & 1)) * PG + q % PG;
                    pr[o] = rec[b].x;
                    pgc[o] = rec[b].y;
                    pbc[o] = rec[b].z;
                    pdc[o] = rec[b].w;
                }
            }
        }
        // distance tile: sum w d of probes (4 pq, 4 pq + 1) at acc[2 a], of
        // (4 pq + 2, 4 pq + 3) at acc[2 a + 1], sum w d^2 at acc[8 + ...];
        // irradiance tile: r, g, b of probes (2 pq, 2 pq + 1) at acc[{0, 4, 8} + a]
        uint64_t acc[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k] = 0ull;
        for (int c = 0; c < n_chunks; ++c) {
            if (c + kTileNS - 1 < n_chunks) issue_chunk(c + kTileNS - 1);
            else cp_async_commit();
            cp_async_wait_ahead();
            __syncthreads();   // chunk c (and, at c = 0, the planes) visible to all
            const float* wb = wbuf + (c % kTileNS) * wrows * kTileWS;
            const int c0 = c * kTileKC, kc = min(kTileKC, R - c0);
            if (is_dist && live) {
#pragma unroll
                for (int j = 0; j < kTileKC; j += 4) {
                    if (j >= kc) break;
                    float4 w[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
                        w[a] = *reinterpret_cast<const float4*>(wb + (tq + a * nqd) * kTileWS + j);
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii) {
                        const float4 dq = *reinterpret_cast<const float4*>(pdc + (c0 + j + ii) * PG + 4 * pq);
                        const uint64_t d01 = f2_pack(dq.x, dq.y), d23 = f2_pack(dq.z, dq.w);
                        const uint64_t q01 = f2_mul(d01, d01), q23 = f2_mul(d23, d23);
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            const float wv = ii == 0 ? w[a].x : ii == 1 ? w[a].y : ii == 2 ? w[a].z : w[a].w;
                            const uint64_t w2 = f2_pack(wv, wv);
                            acc[2 * a] = f2_fma(w2, d01, acc[2 * a]);
                            acc[2 * a + 1] = f2_fma(w2, d23, acc[2 * a + 1]);
                            acc[8 + 2 * a] = f2_fma(w2, q01, acc[8 + 2 * a]);
                            acc[8 + 2 * a + 1] = f2_fma(w2, q23, acc[8 + 2 * a + 1]);
                        }
                    }
                }
            } else if (is_irr && live) {
                const float* wsi = wb + 4 * nqd * kTileWS;
#pragma unroll
                for (int j = 0; j < kTileKC; j += 4) {
                    if (j >= kc) break;
                    float4 w[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
                        w[a] = *reinterpret_cast<const float4*>(wsi + (tq + a * nqi) * kTileWS + j);
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii) {
                        const int o = (c0 + j + ii) * PG + 2 * pq;
                        const float2 lr = *reinterpret_cast<const float2*>(pr + o);
                        const float2 lg = *reinterpret_cast<const float2*>(pgc + o);
                        const float2 lb = *reinterpret_cast<const float2*>(pbc + o);
                        const uint64_t r2 = f2_pack(lr.x, lr.y), g2 = f2_pack(lg.x, lg.y), b2 = f2_pack(lb.x, lb.y);
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            const float wv = ii == 0 ? w[a].x : ii == 1 ? w[a].y : ii == 2 ? w[a].z : w[a].w;
                            const uint64_t w2 = f2_pack(wv, wv);
                            acc[a] = f2_fma(w2, r2, acc[a]);
                            acc[4 + a] = f2_fma(w2, g2, acc[4 + a]);
                            acc[8 + a] = f2_fma(w2, b2, acc[8 + a]);
                        }
                    }
                }
            }
            __syncthreads();   // this chunk's buffer is refilled two chunks later
        }
        // the sums go to shared memory (records and weights are consumed), then
        // every thread blends texels in a short rolled loop, consecutive threads
        // on consecutive texels of one probe: the blend code is fetched once per
        // loop, not once per unrolled output
        float* sum_d = sm;                    // [PG][td] x (m1, m2)
        float* sum_i = sm + 2 * PG * td;      // [PG][ti] x (r, g, b)
        if (is_dist && live) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int t = tq + a * nqd;
                float m1[4], m2[4];
                f2_unpack(acc[2 * a], m1[0], m1[1]);
                f2_unpack(acc[2 * a + 1], m1[2], m1[3]);
                f2_unpack(acc[8 + 2 * a], m2[0], m2[1]);
                f2_unpack(acc[8 + 2 * a + 1], m2[2], m2[3]);
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (t < td) {
                        const int o = (4 * pq + b) * td + t;
                        sum_d[2 * o] = m1[b];
                        sum_d[2 * o + 1] = m2[b];
                    }
            }
        } else if (is_irr && live) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int t = tq + a * nqi;
                float cr[2], cg[2], cb[2];
                f2_unpack(acc[a], cr[0], cr[1]);
                f2_unpack(acc[4 + a], cg[0], cg[1]);
                f2_unpack(acc[8 + a], cb[0], cb[1]);
#pragma unroll
                for (int b = 0; b < 2; ++b)
                    if (t < ti) {
                        const int o = (2 * pq + b) * ti + t;
                        sum_i[3 * o] = cr[b];
                        sum_i[3 * o + 1] = cg[b];
                        sum_i[3 * o + 2] = cb[b];
                    }
            }
        }
        float* inv_d = sum_i + 3 * PG * ti;   // [td], then [ti]
        float* inv_i = inv_d + td;
        for (int k = threadIdx.x; k < td; k += blockDim.x) inv_d[k] = __ldg(inv_s_dist + k);
        for (int k = threadIdx.x; k < ti; k += blockDim.x) inv_i[k] = __ldg(inv_s_irr + k);
        __syncthreads();
        // texels in batches per thread: every load of a batch (old texel,
        // sums, inverse sum) first, then the blends and stores, so a thread
        // has several independent texels in flight; the items of a batch are
        // distinct texels and touch disjoint memory
        constexpr int kBD = 4, kBI = 2;
        for (int o0 = threadIdx.x; o0 < np * td; o0 += kBD * blockDim.x) {
            float2 old[kBD];
            float m1[kBD], m2[kBD], inv[kBD];
            int pp[kBD], xs[kBD], ys[kBD];
#pragma unroll
            for (int u = 0; u < kBD; ++u) {
                const int o = min(o0 + u * (int)blockDim.x, np * td - 1);
                pp[u] = (int)fast_div((uint32_t)o, bp.div_td);
                const int t = o - pp[u] * td;
                const int y = (int)fast_div((uint32_t)t, bp.div_nd);
                xs[u] = 1 + t - y * nd;
                ys[u] = 1 + y;
                const int e = s_probe[pp[u]];
                old[u] = load_dist<false>(vol_of<MULTI>(vs, e >> kEntryShift), e & kEntryMask, xs[u], ys[u]);
                m1[u] = sum_d[2 * o];
                m2[u] = sum_d[2 * o + 1];
                inv[u] = inv_d[t];
            }
#pragma unroll
            for (int u = 0; u < kBD; ++u) {
                if (o0 + u * (int)blockDim.x >= np * td) break;
                const int e = s_probe[pp[u]];
                store_dist_with_borders(vol_of<MULTI>(vs, e >> kEntryShift), e & kEntryMask, xs[u], ys[u],
                                        blend_dist_value(bp, old[u], m1[u], m2[u], inv[u], s_newly[pp[u]] != 0,
                                                         status));
            }
        }
        for (int o0 = threadIdx.x; o0 < np * ti; o0 += kBI * blockDim.x) {
            float3 old[kBI], sum[kBI];
            float inv[kBI];
            int pp[kBI], xs[kBI], ys[kBI];
#pragma unroll
            for (int u = 0; u < kBI; ++u) {
                const int o = min(o0 + u * (int)blockDim.x, np * ti - 1);
                pp[u] = (int)fast_div((uint32_t)o, bp.div_ti);
                const int t = o - pp[u] * ti;
                const int y = (int)fast_div((uint32_t)t, bp.div_ni);
                xs[u] = 1 + t - y * ni;
                ys[u] = 1 + y;
                const int e = s_probe[pp[u]];
                old[u] = load_irr<false>(vol_of<MULTI>(vs, e >> kEntryShift), e & kEntryMask, xs[u], ys[u]);
                sum[u] = f3(sum_i[3 * o], sum_i[3 * o + 1], sum_i[3 * o + 2]);
                inv[u] = inv_i[t];
            }
#pragma unroll
            for (int u = 0; u < kBI; ++u) {
                if (o0 + u * (int)blockDim.x >= np * ti) break;
                const int e = s_probe[pp[u]];
                const VolView& v = vol_of<MULTI>(vs, e >> kEntryShift);
                store_irr_with_borders(v, e & kEntryMask, xs[u], ys[u],
                                       blend_irr_value(v, bp, old[u], sum[u].x, sum[u].y, sum[u].z, inv[u],
                                                       s_newly[pp[u]] != 0, status));
            }
        }
        __syncthreads();
        if (threadIdx.x < np && s_newly[threadIdx.x]) {
            const int e = s_probe[threadIdx.x];
            {
                uint8_t* sp = vol_of<MULTI>(vs, e >> kEntryShift).states + (e & kEntryMask);
                *sp = state_advanced(*sp);
            }
        }
        __syncthreads();
    }
}

// Optional converge pass for new probes (Sec. 6.3).  k_converge_accum adds
// one batch's weighted sums, per list slot q and texel t,
//   acc_irr[q][t] += sum_i W_irr[t][i] (r, g, b)_i,  acc_dist[q][t] += sum_i W_dist[t][i] (d, d^2)_i,
// and den[t] += sum_i W[t][i] (the same for every probe; written by the
// block of slot 0); init starts the sums.  Block per slot, thread per texel
// (irradiance texels first), the slot's R records staged in shared memory.
__global__ void __launch_bounds__(1024) k_converge_accum(int R, int ti, int td, const float* __restrict__ w_irr,
                                                        const float* __restrict__ w_dist,
                                                        const float4* __restrict__ records,
                                                        const int32_t* __restrict__ count, float4* acc_irr,
                                                        float2* acc_dist, float* den, int init) {
    extern __shared__ float4 s_rec[];
    const int n = *count;
    const int t = threadIdx.x;
    for (int q = blockIdx.x; q < n; q += gridDim.x) {
        __syncthreads();
        for (int i = t; i < R; i += blockDim.x) s_rec[i] = records[(int64_t)q * R + i];
        __syncthreads();
        if (t < ti) {
            const float* w = w_irr + (int64_t)t * R;
            float r = 0.0f, g = 0.0f, b = 0.0f, sw = 0.0f;
            for (int i = 0; i < R; ++i) {
                const float wi = __ldg(w + i);
                const float4 rec = s_rec[i];
                r = fmaf(wi, rec.x, r);
                g = fmaf(wi, rec.y, g);
                b = fmaf(wi, rec.z, b);
                sw += wi;
            }
            float4& a = acc_irr[(int64_t)q * ti + t];
            a = init ? make_float4(r, g, b, 0.0f) : make_float4(a.x + r, a.y + g, a.z + b, 0.0f);
            if (q == 0) den[t] = init ? sw : den[t] + sw;
        } else if (t < ti + td) {
            const int u = t - ti;
            const float* w = w_dist + (int64_t)u * R;
            float m1 = 0.0f, m2 = 0.0f, sw = 0.0f;
            for (int i = 0; i < R; ++i) {
                const float wi = __ldg(w + i);
                const float d = s_rec[i].w;
                m1 = fmaf(wi, d, m1);
                m2 = fmaf(wi, d * d, m2);
                sw += wi;
            }
            float2& a = acc_dist[(int64_t)q * td + u];
            a = init ? make_float2(m1, m2) : make_float2(a.x + m1, a.y + m2);
            if (q == 0) den[t] = init ? sw : den[t] + sw;
        }
    }
}

// The converge pass's texels: encoded ratio of sums (hysteresis 0), border
// copies, then Newly Vigilant / Newly Awake -> Vigilant / Awake.  A texel no
// ray reached (den = 0) keeps its value.
__global__ void __launch_bounds__(1024) k_converge_finish(VolView v, const int32_t* __restrict__ list,
                                                         const int32_t* __restrict__ count,
                                                         const float4* __restrict__ acc_irr,
                                                         const float2* __restrict__ acc_dist,
                                                         const float* __restrict__ den, uint32_t* status) {
    const int n = *count;
    const int ti = v.irr_n * v.irr_n, td = v.dist_n * v.dist_n;
    const int t = threadIdx.x;
    for (int q = blockIdx.x; q < n; q += gridDim.x) {
        const int p = list[q];
        if (t < ti) {
            const float sw = den[t];
            if (sw > 0.0f) {
                const float4 a = acc_irr[(int64_t)q * ti + t];
                const float inv = 1.0f / sw;
                const float3 e = f3(powf(a.x * inv, v.inv_gamma), powf(a.y * inv, v.inv_gamma),
                                    powf(a.z * inv, v.inv_gamma));
                if (!(isfinite(e.x) && isfinite(e.y) && isfinite(e.z))) atomicOr(status, 1u);
                const int x = 1 + t % v.irr_n, y = 1 + t / v.irr_n;
                store_irr(v, p, x, y, e);
                for_border_copies(x, y, v.irr_n, [&](int bx, int by) { store_irr(v, p, bx, by, e); });
            }
        } else if (t < ti + td) {
            const int u = t - ti;
            const float sw = den[t];
            if (sw > 0.0f) {
                const float2 a = acc_dist[(int64_t)q * td + u];
                const float inv = 1.0f / sw;
                const float2 e = make_float2(a.x * inv, a.y * inv);
                if (!(isfinite(e.x) && isfinite(e.y))) atomicOr(status, 1u);
                const int x = 1 + u % v.dist_n, y = 1 + u / v.dist_n;
                store_dist(v, p, x, y, e);
                for_border_copies(x, y, v.dist_n, [&](int bx, int by) { store_dist(v, p, bx, by, e); });
            }
        }
        if (t == 0) v.states[p] = state_advanced(v.states[p]);
    }
}

cudaError_t launch_converge_accum(int R, int irr_n, int dist_n, const float* w_irr, const float* w_dist,
                                  const float4* records, const int32_t* count, float4* acc_irr, float2* acc_dist,
                                  float* den, bool init, int grid, cudaStream_t st) {
    const int ti = irr_n * irr_n, td = dist_n * dist_n;
    const int threads = (ti + td + 31) / 32 * 32;
    if (threads > 1024) return cudaErrorInvalidValue;
    k_converge_accum<<<grid, threads, sizeof(float4) * (size_t)R, st>>>(R, ti, td, w_irr, w_dist, records, count,
                                                                         acc_irr, acc_dist, den, init ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_converge_finish(const VolView& v, const int32_t* list, const int32_t* count,
                                   const float4* acc_irr, const float2* acc_dist, const float* den, uint32_t* status,
                                   int grid, cudaStream_t st) {
    const int threads = (v.irr_n * v.irr_n + v.dist_n * v.dist_n + 31) / 32 * 32;
    if (threads > 1024) return cudaErrorInvalidValue;
    k_converge_finish<<<grid, threads, 0, st>>>(v, list, count, acc_irr, acc_dist, den, status);
    return cudaGetLastError();
}

cudaError_t launch_frame_dirs(const FrameRot& rot, int R, int irr_n, int dist_n, const double* sf64, float4* dirs,
                              cudaStream_t st) {
    // the direction blocks of k_frame_setup alone
    k_frame_setup<false><<<(R + 255) / 256, 256, 0, st>>>(rot, nullptr, R, irr_n, dist_n, 0.0, sf64, dirs, nullptr,
                                                           nullptr, nullptr, nullptr, nullptr, 0,
                                                           irr_n * irr_n + dist_n * dist_n);
    return cudaGetLastError();
}

cudaError_t launch_sf_table(int R, double* sf64, cudaStream_t st) {
    k_sf_table<<<(R + 127) / 128, 128, 0, st>>>(R, sf64);
    return cudaGetLastError();
}

static int frame_setup_grid(int R, int irr_n, int dist_n) { return irr_n * irr_n + dist_n * dist_n + (R + 255) / 256; }

cudaError_t launch_frame_setup(const FrameRot& rot, int R, int irr_n, int dist_n, float cos_power,
                               const double* sf64, float4* dirs, float* w_irr, float* inv_s_irr, float* w_dist,
                               float* inv_s_dist, int32_t* zero, int n_zero, cudaStream_t st) {
    k_frame_setup<false><<<frame_setup_grid(R, irr_n, dist_n), 256, 0, st>>>(
        rot, nullptr, R, irr_n, dist_n, (double)cos_power, sf64, dirs, w_irr, inv_s_irr, w_dist, inv_s_dist, zero,
        n_zero, 0);
    return cudaGetLastError();
}

cudaError_t launch_frame_setup_split(const FrameRot& rot, int R, int irr_n, int dist_n, float cos_power,
                                     const double* sf64, float4* dirs, float* w_irr, float* inv_s_irr,
                                     float* w_dist, float* inv_s_dist, int32_t* zero, int n_zero,
                                     cudaStream_t st_dirs, cudaStream_t st_weights) {
    const int nwb = irr_n * irr_n + dist_n * dist_n;
    k_frame_setup<false><<<nwb, 256, 0, st_weights>>>(rot, nullptr, R, irr_n, dist_n, (double)cos_power, sf64, dirs,
                                                      w_irr, inv_s_irr, w_dist, inv_s_dist, zero, n_zero, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the directions in blocks of 64 rays, so the FP64 rotations of the
    // frame's rays spread over several SMs' double-precision units
    if (n_zero > 64) return cudaErrorInvalidValue;
    return launch_pdl(k_frame_setup<false>, (R + 63) / 64, 64, 0, st_dirs, rot, nullptr, R, irr_n, dist_n,
                      (double)cos_power, sf64, dirs, w_irr, inv_s_irr, w_dist, inv_s_dist, zero, n_zero, nwb);
}

cudaError_t launch_frame_setup_dev(const FrameRot* rot_dev, int R, int irr_n, int dist_n, float cos_power,
                                   const double* sf64, float4* dirs, float* w_irr, float* inv_s_irr, float* w_dist,
                                   float* inv_s_dist, int32_t* zero, int n_zero, cudaStream_t st) {
    k_frame_setup<true><<<frame_setup_grid(R, irr_n, dist_n), 256, 0, st>>>(
        FrameRot{}, rot_dev, R, irr_n, dist_n, (double)cos_power, sf64, dirs, w_irr, inv_s_irr, w_dist, inv_s_dist,
        zero, n_zero, 0);
    return cudaGetLastError();
}

// Sets the kernel's dynamic shared-memory cap to the device's opt-in maximum
// less its static shared memory, once per device (host-side attribute; must
// not run under stream capture).
template <typename K>
static cudaError_t allow_max_smem(K kernel, DeviceOnce& once) {
    return once_per_device(once, [&]() {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa.sharedSizeBytes);
        return e;
    });
}

// The current device's opt-in shared memory per block (48 KB if it cannot
// be read).
static int smem_optin() {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        optin = 48 * 1024;
    return optin;
}

// Opts both blend kernels of one instantiation into the maximum dynamic
// shared memory, once per device.
template <bool MULTI, int PGS>
static cudaError_t opt_in_blend() {
    static DeviceOnce tiled, rows;
    cudaError_t e = allow_max_smem(k_blend_tiled<MULTI, PGS>, tiled);
    if (e == cudaSuccess) e = allow_max_smem(k_blend_simt<MULTI, PGS>, rows);
    return e;
}

template <int PG>
static bool tiled_fits(const BlendParams& bp, int irr_n, int dist_n) {
    const TiledShape ts = tiled_shape(PG, bp.R, irr_n, dist_n);
    return bp.R % 4 == 0 && ts.threads <= kTileMaxThreads && ts.smem + 1024 <= (size_t)smem_optin();
}

template <bool MULTI, int PG>
static cudaError_t launch_tiled(const VolSet& vs, const BlendParams& bp, int irr_n, int dist_n, const float* w_irr,
                                const float* inv_s_irr, const float* w_dist, const float* inv_s_dist,
                                const float4* records, const int32_t* active, const int32_t* count,
                                uint32_t* status, int grid, cudaStream_t st) {
    cudaError_t e = opt_in_blend<MULTI, PG>();
    if (e != cudaSuccess) return e;
    const TiledShape ts = tiled_shape(PG, bp.R, irr_n, dist_n);
    // one wave of resident CTAs; the kernel splits the active probes evenly
    int occ = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_blend_tiled<MULTI, PG>, ts.threads, ts.smem)) !=
        cudaSuccess)
        return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    grid = sms * (occ > 0 ? occ : 1);
    BlendParams bpt = bp;
    bpt.div_ti = make_fast_div((uint32_t)(irr_n * irr_n));
    bpt.div_td = make_fast_div((uint32_t)(dist_n * dist_n));
    bpt.div_ni = make_fast_div((uint32_t)irr_n);
    bpt.div_nd = make_fast_div((uint32_t)dist_n);
    k_blend_tiled<MULTI, PG><<<grid, ts.threads, ts.smem, st>>>(vs, bpt, w_irr, inv_s_irr, w_dist, inv_s_dist,
                                                                records, active, count, status);
    return cudaGetLastError();
}

// The tiled kernel with PGS probes per CTA, or with fewer when its tiles do
// not fit (larger texel counts need more threads per probe group); the row
// kernel when no group size fits.  The grid is scaled to keep the probes
// per launch wave.
template <bool MULTI, int PGS>
static cudaError_t blend_simt(const VolSet& vs, const BlendParams& bp, int irr_n, int dist_n, const float* w_irr,
                              const float* inv_s_irr, const float* w_dist, const float* inv_s_dist,
                              const float4* records, const int32_t* active, const int32_t* count,
                              uint32_t* status, int grid, cudaStream_t st) {
    if (PGS >= 16 && tiled_fits<16>(bp, irr_n, dist_n))
        return launch_tiled<MULTI, 16>(vs, bp, irr_n, dist_n, w_irr, inv_s_irr, w_dist, inv_s_dist, records, active,
                                       count, status, grid, st);
    if (PGS >= 8 && tiled_fits<8>(bp, irr_n, dist_n))
        return launch_tiled<MULTI, 8>(vs, bp, irr_n, dist_n, w_irr, inv_s_irr, w_dist, inv_s_dist, records, active,
                                      count, status, grid * (PGS / 8), st);
    if (tiled_fits<4>(bp, irr_n, dist_n))
        return launch_tiled<MULTI, 4>(vs, bp, irr_n, dist_n, w_irr, inv_s_irr, w_dist, inv_s_dist, records, active,
                                      count, status, grid * (PGS / 4), st);
    cudaError_t e = opt_in_blend<MULTI, PGS>();
    if (e != cudaSuccess) return e;
    // as many probes per CTA as fit (R <= 1024 leaves room for at least 13)
    const size_t per_probe = (size_t)(bp.R + 1) * sizeof(float4);
    const int group = (int)std::min<size_t>(PGS, ((size_t)smem_optin() - 1024) / per_probe);
    if (group < 1) return cudaErrorInvalidValue;
    k_blend_simt<MULTI, PGS><<<grid, 256, (size_t)group * per_probe, st>>>(vs, bp, group, w_irr, inv_s_irr, w_dist,
                                                                            inv_s_dist, records, active, count,
                                                                            status);
    return cudaGetLastError();
}

cudaError_t launch_blend(const VolView& v, const BlendParams& bp, const float* w_irr, const float* inv_s_irr,
                         const float* w_dist, const float* inv_s_dist, const float4* records,
                         const int32_t* active, const int32_t* count, uint32_t* status, int grid,
                         cudaStream_t st) {
    return blend_simt<false, 16>(single_set(v), bp, v.irr_n, v.dist_n, w_irr, inv_s_irr, w_dist, inv_s_dist,
                                records, active, count, status, grid, st);
}

cudaError_t launch_blend_set(const VolSet& vs, bool multi, const BlendParams& bp, int irr_n, int dist_n,
                             const float* w_irr,
                             const float* inv_s_irr, const float* w_dist, const float* inv_s_dist,
                             const float4* records, const int32_t* active, const int32_t* count,
                             uint32_t* status, int grid, int probes_per_cta, cudaStream_t st) {
#define DDGI_BLEND_CASE(M, P)                                                                                 \
    if (multi == M && probes_per_cta == P)                                                                   \
        return blend_simt<M, P>(vs, bp, irr_n, dist_n, w_irr, inv_s_irr, w_dist, inv_s_dist, records, active,   \
                                count, status, grid, st);
    DDGI_BLEND_CASE(false, 4)
    DDGI_BLEND_CASE(false, 8)
    DDGI_BLEND_CASE(false, 16)
    DDGI_BLEND_CASE(true, 4)
    DDGI_BLEND_CASE(true, 8)
    DDGI_BLEND_CASE(true, 16)
#undef DDGI_BLEND_CASE
    return cudaErrorInvalidValue;
}

// Sets the shared-memory opt-in of every SIMT blend instantiation (outside
// any stream capture).
cudaError_t prepare_blend_kernels(int) {
    cudaError_t e = opt_in_blend<false, 4>();
    if (e == cudaSuccess) e = opt_in_blend<false, 8>();
    if (e == cudaSuccess) e = opt_in_blend<false, 16>();
    if (e == cudaSuccess) e = opt_in_blend<true, 4>();
    if (e == cudaSuccess) e = opt_in_blend<true, 8>();
    if (e == cudaSuccess) e = opt_in_blend<true, 16>();
    return e;
}

}  // namespace ddgi
