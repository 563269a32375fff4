// Device math of the probe data structure: octahedral map, bilinear texel
// filtering of bordered tiles, probe addressing and the biased 8-probe query.
// Used by the query kernel and by hit shading in the update (the previous
// frame's probes give the indirect term).
#pragma once

#include <cuda_fp16.h>

#include "ddgi_internal.h"
#include "pdl.cuh"

namespace ddgi {

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float length(float3 a) { return sqrtf(dot(a, a)); }
__device__ __forceinline__ float sgnnz(float x) { return x >= 0.0f ? 1.0f : -1.0f; }

// Octahedral encode (Cigolle et al. 2014): v / |v|_1, lower hemisphere folded.
__device__ __forceinline__ float2 oct_encode(float3 v) {
    float l1 = fabsf(v.x) + fabsf(v.y) + fabsf(v.z);
    float px = v.x / l1, py = v.y / l1;
    if (v.z < 0.0f) {
        float qx = (1.0f - fabsf(py)) * sgnnz(px);
        float qy = (1.0f - fabsf(px)) * sgnnz(py);
        px = qx;
        py = qy;
    }
    return make_float2(px, py);
}

// The same map with the hardware reciprocal (__fdividef, about 2 ulp) for
// the per-probe lookups of the query, where IEEE division dominated.
__device__ __forceinline__ float2 oct_encode_fast(float3 v) {
    float inv = __fdividef(1.0f, fabsf(v.x) + fabsf(v.y) + fabsf(v.z));
    float px = v.x * inv, py = v.y * inv;
    if (v.z < 0.0f) {
        float qx = (1.0f - fabsf(py)) * sgnnz(px);
        float qy = (1.0f - fabsf(px)) * sgnnz(py);
        px = qx;
        py = qy;
    }
    return make_float2(px, py);
}

// Probe grid addressing: logical (i,j,k) of the window is stored at
// ((i+shift) mod count, ...); the tracking window moves `shift`, which a
// VolView holds reduced to [0, count).
__device__ __forceinline__ int wrap(int a, int m) { int r = a % m; return r < 0 ? r + m : r; }
// (a + s) mod m and (a - s) mod m for a, s in [0, m)
__device__ __forceinline__ int wrap_add(int a, int s, int m) { int r = a + s; return r >= m ? r - m : r; }
__device__ __forceinline__ int wrap_sub(int a, int s, int m) { int r = a - s; return r < 0 ? r + m : r; }

// Logical (i, j, k) inside the grid -> physical probe index.
__device__ __forceinline__ int probe_phys(const VolView& v, int i, int j, int k) {
    int a = wrap_add(i, v.shift.x, v.counts.x);
    int b = wrap_add(j, v.shift.y, v.counts.y);
    int c = wrap_add(k, v.shift.z, v.counts.z);
    return a + v.counts.x * (b + v.counts.y * c);
}

__device__ __forceinline__ float3 probe_pos_logical(const VolView& v, int i, int j, int k) {
    return f3(v.origin.x + (float)i * v.spacing.x, v.origin.y + (float)j * v.spacing.y,
              v.origin.z + (float)k * v.spacing.z);
}

// World position of physical probe p: its grid point plus its offset (Sec. 5).
__device__ __forceinline__ float3 probe_pos_phys(const VolView& v, int p) {
    const int q = (int)fast_div((uint32_t)p, v.div_x);   // p / counts.x
    const int c = (int)fast_div((uint32_t)p, v.div_xy);  // p / (counts.x counts.y)
    const int a = p - q * v.counts.x;
    const int b = q - c * v.counts.y;
    float3 x = probe_pos_logical(v, wrap_sub(a, v.shift.x, v.counts.x), wrap_sub(b, v.shift.y, v.counts.y),
                                 wrap_sub(c, v.shift.z, v.counts.z));
    if (v.offsets) {
        const float4 o = v.offsets[p];
        x = f3(x.x + o.x, x.y + o.y, x.z + o.z);
    }
    return x;
}

// Traced, blended and used by the query: vigilant probes and sleeping probes
// woken by a dynamic object (Sec. 6.3).
__device__ __forceinline__ bool state_active(uint8_t s) {
    return s == DDGI_STATE_NEWLY_VIGILANT || s == DDGI_STATE_VIGILANT || s == DDGI_STATE_NEWLY_AWAKE ||
           s == DDGI_STATE_AWAKE;
}
// First update after becoming active: blended with hysteresis 0.
__device__ __forceinline__ bool state_newly(uint8_t s) {
    return s == DDGI_STATE_NEWLY_VIGILANT || s == DDGI_STATE_NEWLY_AWAKE;
}
// The state after a probe's update.
__device__ __forceinline__ uint8_t state_advanced(uint8_t s) {
    return s == DDGI_STATE_NEWLY_VIGILANT ? (uint8_t)DDGI_STATE_VIGILANT
                                          : (s == DDGI_STATE_NEWLY_AWAKE ? (uint8_t)DDGI_STATE_AWAKE : s);
}

// Bilinear footprint in a bordered tile of n interior texels: the octahedral
// coordinate [-1,1] spans texel positions [1, n+1]; texel k has its centre at k+0.5.
// Two floats in one 64-bit register pair, for the packed FP32 pair
// arithmetic of sm_100 and later (sub / mul / fma .rn.f32x2: each half
// rounded exactly as the scalar instruction would).
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// a * b + c, each half one fused multiply-add (as fmaf)
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

struct Footprint {
    int x0, y0;
    float tx, ty;
};

__device__ __forceinline__ Footprint footprint(float2 u, int n) {
    float sx = 1.0f + (u.x + 1.0f) * 0.5f * (float)n - 0.5f;
    float sy = 1.0f + (u.y + 1.0f) * 0.5f * (float)n - 0.5f;
    float fx = floorf(sx), fy = floorf(sy);
    int x0 = (int)fx, y0 = (int)fy;
    x0 = min(max(x0, 0), n);
    y0 = min(max(y0, 0), n);
    Footprint f;
    f.x0 = x0;
    f.y0 = y0;
    f.tx = sx - (float)x0;
    f.ty = sy - (float)y0;
    return f;
}

// ---- texel storage formats -------------------------------------------------
// Irradiance FP32: 4 floats per texel (rgb + an unused 0), one 16-byte load.
// FP16: 4 halves (rgb + pad).
// RGB9E5: one 32-bit word, 9-bit mantissas with a shared 5-bit exponent
// (bias 15), as in the OpenGL EXT_texture_shared_exponent specification.

__device__ __forceinline__ float3 rgb9e5_decode(uint32_t w) {
    int e = (int)(w >> 27) - 15 - 9;
    float s = ldexpf(1.0f, e);
    return f3((float)(w & 511u) * s, (float)((w >> 9) & 511u) * s, (float)((w >> 18) & 511u) * s);
}

__device__ __forceinline__ uint32_t rgb9e5_encode(float3 c) {
    const float kMax = 65408.0f;   // (511/512) * 2^16
    float r = fminf(fmaxf(c.x, 0.0f), kMax);
    float g = fminf(fmaxf(c.y, 0.0f), kMax);
    float b = fminf(fmaxf(c.z, 0.0f), kMax);
    float mx = fmaxf(r, fmaxf(g, b));
    if (!(mx > 0.0f)) return 0u;
    // exponent such that mx / 2^(e-15-9) < 512, e >= 0
    int ex;
    frexpf(mx, &ex);                       // mx = m * 2^ex, m in [0.5, 1)
    int e = max(-16, ex - 1) + 1 + 15;     // shared exponent (biased)
    if (e < 0) e = 0;
    float s = ldexpf(1.0f, -(e - 15 - 9));
    int mmax = (int)floorf(mx * s + 0.5f);
    if (mmax == 512) { e += 1; s *= 0.5f; }
    if (e > 31) e = 31;
    uint32_t ir = (uint32_t)min(511, (int)floorf(r * s + 0.5f));
    uint32_t ig = (uint32_t)min(511, (int)floorf(g * s + 0.5f));
    uint32_t ib = (uint32_t)min(511, (int)floorf(b * s + 0.5f));
    return ir | (ig << 9) | (ib << 18) | ((uint32_t)e << 27);
}

// NC = true reads through the non-coherent (read-only) path: only for
// kernels that do not write the atlas.
template <bool NC>
__device__ __forceinline__ float ld(const float* p) { if (NC) return __ldg(p); else return *p; }
template <bool NC>
__device__ __forceinline__ uint32_t ld(const uint32_t* p) { if (NC) return __ldg(p); else return *p; }
template <bool NC>
__device__ __forceinline__ uint2 ld(const uint2* p) { if (NC) return __ldg(p); else return *p; }
template <bool NC>
__device__ __forceinline__ float2 ld(const float2* p) { if (NC) return __ldg(p); else return *p; }
template <bool NC>
__device__ __forceinline__ float4 ld(const float4* p) { if (NC) return __ldg(p); else return *p; }

template <bool NC = true>
__device__ __forceinline__ float3 load_irr(const VolView& v, int p, int x, int y) {
    int64_t t = (int64_t)p * v.irr_tile + (int64_t)y * (v.irr_n + 2) + x;
    if (v.irr_format == DDGI_IRR_FP32) {
        const float4 a = ld<NC>((const float4*)v.irr + t);
        return f3(a.x, a.y, a.z);
    } else if (v.irr_format == DDGI_IRR_FP16) {
        uint2 w = ld<NC>((const uint2*)v.irr + t);
        __half2 h0 = *reinterpret_cast<__half2*>(&w.x);
        __half2 h1 = *reinterpret_cast<__half2*>(&w.y);
        float2 a = __half22float2(h0);
        return f3(a.x, a.y, __low2float(h1));
    } else {
        return rgb9e5_decode(ld<NC>((const uint32_t*)v.irr + t));
    }
}

__device__ __forceinline__ void store_irr(const VolView& v, int p, int x, int y, float3 c) {
    int64_t t = (int64_t)p * v.irr_tile + (int64_t)y * (v.irr_n + 2) + x;
    if (v.irr_format == DDGI_IRR_FP32) {
        ((float4*)v.irr)[t] = make_float4(c.x, c.y, c.z, 0.0f);
    } else if (v.irr_format == DDGI_IRR_FP16) {
        __half2 h0 = __floats2half2_rn(c.x, c.y);
        __half2 h1 = __floats2half2_rn(c.z, 0.0f);
        uint2 w;
        w.x = *reinterpret_cast<uint32_t*>(&h0);
        w.y = *reinterpret_cast<uint32_t*>(&h1);
        ((uint2*)v.irr)[t] = w;
    } else {
        ((uint32_t*)v.irr)[t] = rgb9e5_encode(c);
    }
}

template <bool NC = true>
__device__ __forceinline__ float2 load_dist(const VolView& v, int p, int x, int y) {
    int64_t t = (int64_t)p * v.dist_tile + (int64_t)y * (v.dist_n + 2) + x;
    if (v.dist_format == DDGI_DIST_FP32) {
        return ld<NC>((const float2*)v.dist + t);
    } else {
        uint32_t w = ld<NC>((const uint32_t*)v.dist + t);
        return __half22float2(*reinterpret_cast<__half2*>(&w));
    }
}

__device__ __forceinline__ void store_dist(const VolView& v, int p, int x, int y, float2 m) {
    int64_t t = (int64_t)p * v.dist_tile + (int64_t)y * (v.dist_n + 2) + x;
    if (v.dist_format == DDGI_DIST_FP32) {
        ((float2*)v.dist)[t] = m;
    } else {
        __half2 h = __floats2half2_rn(m.x, m.y);
        ((uint32_t*)v.dist)[t] = *reinterpret_cast<uint32_t*>(&h);
    }
}

// Bilinear samples at a footprint: one storage-format dispatch per sample,
// then the four taps (rows y0, y0 + 1 of the bordered tile).
struct Bilerp {
    float w00, w10, w01, w11;
};

__device__ __forceinline__ Bilerp bilerp_weights(const Footprint& f) {
    Bilerp b;
    b.w00 = (1.0f - f.tx) * (1.0f - f.ty);
    b.w10 = f.tx * (1.0f - f.ty);
    b.w01 = (1.0f - f.tx) * f.ty;
    b.w11 = f.tx * f.ty;
    return b;
}

__device__ __forceinline__ float3 bilerp3(const Bilerp& w, float3 a, float3 b, float3 c, float3 d) {
    return f3(w.w00 * a.x + w.w10 * b.x + w.w01 * c.x + w.w11 * d.x,
              w.w00 * a.y + w.w10 * b.y + w.w01 * c.y + w.w11 * d.y,
              w.w00 * a.z + w.w10 * b.z + w.w01 * c.z + w.w11 * d.z);
}

// Irradiance at a footprint whose bilinear weights are already known (the
// query reads every cage probe at the same footprint).
__device__ __forceinline__ float3 sample_irr_at(const VolView& v, int p, const Footprint& f, const Bilerp& w) {
    const int row = v.irr_n + 2;
    const int64_t t = (int64_t)p * v.irr_tile + (int64_t)f.y0 * row + f.x0;
    if (v.irr_format == DDGI_IRR_FP32) {
        const float4* a = (const float4*)v.irr + t;
        const float4 q00 = __ldg(a), q10 = __ldg(a + 1), q01 = __ldg(a + row), q11 = __ldg(a + row + 1);
        return bilerp3(w, f3(q00.x, q00.y, q00.z), f3(q10.x, q10.y, q10.z), f3(q01.x, q01.y, q01.z),
                       f3(q11.x, q11.y, q11.z));
    }
    return bilerp3(w, load_irr(v, p, f.x0, f.y0), load_irr(v, p, f.x0 + 1, f.y0), load_irr(v, p, f.x0, f.y0 + 1),
                   load_irr(v, p, f.x0 + 1, f.y0 + 1));
}

__device__ __forceinline__ float3 sample_irr_at(const VolView& v, int p, const Footprint& f) {
    return sample_irr_at(v, p, f, bilerp_weights(f));
}

__device__ __forceinline__ float2 sample_dist_at(const VolView& v, int p, const Footprint& f) {
    const int row = v.dist_n + 2;
    float2 a, b, c, d;
    if (v.dist_format == DDGI_DIST_FP32) {
        const float2* q = (const float2*)v.dist + (int64_t)p * v.dist_tile + (int64_t)f.y0 * row + f.x0;
        a = __ldg(q);
        b = __ldg(q + 1);
        c = __ldg(q + row);
        d = __ldg(q + row + 1);
    } else {
        a = load_dist(v, p, f.x0, f.y0);
        b = load_dist(v, p, f.x0 + 1, f.y0);
        c = load_dist(v, p, f.x0, f.y0 + 1);
        d = load_dist(v, p, f.x0 + 1, f.y0 + 1);
    }
    float w00 = (1.0f - f.tx) * (1.0f - f.ty), w10 = f.tx * (1.0f - f.ty);
    float w01 = (1.0f - f.tx) * f.ty, w11 = f.tx * f.ty;
    return make_float2(w00 * a.x + w10 * b.x + w01 * c.x + w11 * d.x,
                       w00 * a.y + w10 * b.y + w01 * c.y + w11 * d.y);
}

// FP32-only form of sample_dist_at (the same loads and arithmetic).
__device__ __forceinline__ float2 sample_dist_fp32(const VolView& v, int p, const Footprint& f) {
    const int row = v.dist_n + 2;
    const float2* q = (const float2*)v.dist + (int64_t)p * v.dist_tile + (int64_t)f.y0 * row + f.x0;
    const float2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + row), d = __ldg(q + row + 1);
    float w00 = (1.0f - f.tx) * (1.0f - f.ty), w10 = f.tx * (1.0f - f.ty);
    float w01 = (1.0f - f.tx) * f.ty, w11 = f.tx * f.ty;
    return make_float2(w00 * a.x + w10 * b.x + w01 * c.x + w11 * d.x,
                       w00 * a.y + w10 * b.y + w01 * c.y + w11 * d.y);
}

__device__ __forceinline__ float3 sample_irr(const VolView& v, int p, float3 dir) {
    return sample_irr_at(v, p, footprint(oct_encode(dir), v.irr_n));
}

__device__ __forceinline__ float2 sample_dist(const VolView& v, int p, float3 dir) {
    return sample_dist_at(v, p, footprint(oct_encode(dir), v.dist_n));
}

// x^(gamma/2) on the gamma-encoded value; gamma = 5 uses x^2 sqrt(x).
__device__ __forceinline__ float gamma_decode_half(float e, float half_gamma) {
    e = fmaxf(e, 0.0f);
    if (half_gamma == 2.5f) return e * e * sqrtf(e);
    if (half_gamma == 0.5f) return sqrtf(e);
    return powf(e, half_gamma);
}

// The same with sqrt(x) as x * rsqrt(x) (hardware reciprocal square root,
// about 2 ulp), for the query's 8 probes x 3 channels.
__device__ __forceinline__ float gamma_decode_half_fast(float e, float half_gamma) {
    e = fmaxf(e, 0.0f);
    const float sq = e > 0.0f ? e * rsqrtf(e) : 0.0f;
    if (half_gamma == 2.5f) return e * e * sq;
    if (half_gamma == 0.5f) return sq;
    return powf(e, half_gamma);
}


// a - b for FP32 a, b as the unevaluated sum hi + lo, exactly (Knuth's
// TwoSum applied to a and -b, round-to-nearest); the intrinsics keep each
// step as written.
__device__ __forceinline__ void two_diff(float a, float b, float& hi, float& lo) {
    hi = __fsub_rn(a, b);
    const float bb = __fsub_rn(hi, a);
    lo = __fadd_rn(__fsub_rn(a, __fsub_rn(hi, bb)), __fsub_rn(-b, bb));
}

// A query point in the volume's own frame: x - origin = hi + lo exactly, and
// lb = lo + the self-shadow bias vector (Sec. 4.1), so the biased point is
// origin + hi + lb.  Probe-to-point vectors formed from these carry rounding
// errors relative to their own length, not to |x|: far from the world
// origin, 2^-24 |x| approaches the standard deviation the Chebyshev test
// divides by, and the weight then follows the rounding of x instead of x.
struct LocalPoint {
    float3 hi, lo, lb;
};

__device__ __forceinline__ LocalPoint local_point(const VolView& v, float3 x, float3 n, float3 wo) {
    const float k = 0.75f * v.min_spacing * v.bias;
    LocalPoint q;
    two_diff(x.x, v.origin.x, q.hi.x, q.lo.x);
    two_diff(x.y, v.origin.y, q.hi.y, q.lo.y);
    two_diff(x.z, v.origin.z, q.hi.z, q.lo.z);
    q.lb = f3(q.lo.x + (0.2f * n.x + 0.8f * wo.x) * k, q.lo.y + (0.2f * n.y + 0.8f * wo.y) * k,
              q.lo.z + (0.2f * n.z + 0.8f * wo.z) * k);
    return q;
}

// x - x_p for the grid point (i, j, k) of the cage: the high part of the
// difference (one rounding, relative to |x - x_p|); add q.lo for the
// unbiased point, q.lb for the biased one.
__device__ __forceinline__ float3 local_to_probe(const VolView& v, const LocalPoint& q, int i, int j, int k) {
    return f3(q.hi.x - (float)i * v.spacing.x, q.hi.y - (float)j * v.spacing.y, q.hi.z - (float)k * v.spacing.z);
}

// x^2.5 of a red / green pair of gamma-encoded values (gamma 5): e^2 times
// e * rsqrt(e), the squares and products as packed FP32 pairs.  The floor
// 1e-30 stands in for the zero test of gamma_decode_half_fast: below it both
// give 0 in FP32 (x^2.5 < 1e-75), above it they are the same operations.
__device__ __forceinline__ uint64_t gamma_decode_g5_pair(float er, float eg) {
    er = fmaxf(er, 1e-30f);
    eg = fmaxf(eg, 1e-30f);
    const uint64_t E = f2_pack(er, eg);
    const uint64_t S = f2_mul(E, f2_pack(rsqrtf(er), rsqrtf(eg)));
    return f2_mul(f2_mul(E, E), S);
}

// The specialised query of query_M_look<true> (FP32 atlases, gamma 5, no
// probe offsets; query_fast_view): the same operations in the same order,
// except the decode's zero test (gamma_decode_g5_pair), with the eight cage
// corners unrolled, so each corner's probe index, grid offset and
// trilinear factor are registers rather than per-probe selects, and the red
// and green channels of the irradiance taps and their decode carried as
// packed FP32 pairs (the blue channel scalar).
__device__ __forceinline__ float3 query_M_look_fast(const VolView& v, float3 x, float3 n, float3 wo, float3 look) {
    const LocalPoint q = local_point(v, x, n, wo);
    const float g[3] = {(q.hi.x + q.lb.x) / v.spacing.x, (q.hi.y + q.lb.y) / v.spacing.y,
                        (q.hi.z + q.lb.z) / v.spacing.z};
    const int cnt[3] = {v.counts.x, v.counts.y, v.counts.z};
    int base[3];
    float fr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float b = floorf(g[a]);
        b = fminf(fmaxf(b, 0.0f), (float)(cnt[a] - 2));
        base[a] = (int)b;
        fr[a] = fminf(fmaxf(g[a] - b, 0.0f), 1.0f);
    }
    const Footprint fn = footprint(oct_encode(look), v.irr_n);
    const Bilerp wn = bilerp_weights(fn);
    const uint64_t W00 = f2_pack(wn.w00, wn.w00), W10 = f2_pack(wn.w10, wn.w10);
    const uint64_t W01 = f2_pack(wn.w01, wn.w01), W11 = f2_pack(wn.w11, wn.w11);
    const int irow = v.irr_n + 2;
    const int64_t itap = (int64_t)fn.y0 * irow + fn.x0;
    // per axis, the cage's two planes: physical index, x - x_p (high part)
    // and trilinear factor
    const int px[2] = {wrap_add(base[0], v.shift.x, cnt[0]), wrap_add(base[0] + 1, v.shift.x, cnt[0])};
    const int py[2] = {wrap_add(base[1], v.shift.y, cnt[1]), wrap_add(base[1] + 1, v.shift.y, cnt[1])};
    const int pz[2] = {wrap_add(base[2], v.shift.z, cnt[2]), wrap_add(base[2] + 1, v.shift.z, cnt[2])};
    const float ax[2] = {q.hi.x - (float)base[0] * v.spacing.x, q.hi.x - (float)(base[0] + 1) * v.spacing.x};
    const float ay[2] = {q.hi.y - (float)base[1] * v.spacing.y, q.hi.y - (float)(base[1] + 1) * v.spacing.y};
    const float az[2] = {q.hi.z - (float)base[2] * v.spacing.z, q.hi.z - (float)(base[2] + 1) * v.spacing.z};
    const float tx[2] = {1.0f - fr[0], fr[0]}, ty[2] = {1.0f - fr[1], fr[1]}, tz[2] = {1.0f - fr[2], fr[2]};
    int pc[8];
    unsigned act = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        pc[c] = px[c & 1] + cnt[0] * (py[(c >> 1) & 1] + cnt[1] * pz[c >> 2]);
        act |= state_active(v.states[pc[c]]) ? 1u << c : 0u;
    }
    float sumw = 0.0f;
    float3 acc = f3(0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        if (!(act & (1u << c))) continue;
        const int o0 = c & 1, o1 = (c >> 1) & 1, o2 = c >> 2;
        const float3 a = f3(ax[o0], ay[o1], az[o2]);
        const float wt = tx[o0] * ty[o1] * tz[o2];
        const float3 dp = f3(-(a.x + q.lo.x), -(a.y + q.lo.y), -(a.z + q.lo.z));   // probe - x
        const float dd = dot(dp, dp);
        const float cw = dd > 0.0f ? dot(n, dp) * rsqrtf(dd) : 1.0f;
        const float hb = (1.0f + cw) * 0.5f;
        const float wb = hb * hb + 0.2f;
        const float3 pv = a + q.lb;                                                // biased point - probe
        const float rr = dot(pv, pv);
        float wc = 1.0f;
        if (rr > 0.0f) {
            const float ir = rsqrtf(rr);
            const float r = rr * ir;
            const float2 mom = sample_dist_fp32(v, pc[c], footprint(oct_encode_fast(ir * pv), v.dist_n));
            if (r > mom.x) {
                const float var = fmaxf(mom.y - mom.x * mom.x, 0.0f);
                const float dr = r - mom.x;
                wc = __fdividef(var, var + dr * dr);
            }
        }
        const float w = wt * wb * fmaxf(wc, 1e-6f);
        const float4* ia = (const float4*)v.irr + ((int64_t)pc[c] * v.irr_tile + itap);
        const float4 q00 = __ldg(ia), q10 = __ldg(ia + 1), q01 = __ldg(ia + irow), q11 = __ldg(ia + irow + 1);
        uint64_t rg = f2_mul(W00, f2_pack(q00.x, q00.y));
        rg = f2_fma(W10, f2_pack(q10.x, q10.y), rg);
        rg = f2_fma(W01, f2_pack(q01.x, q01.y), rg);
        rg = f2_fma(W11, f2_pack(q11.x, q11.y), rg);
        const float eb = wn.w00 * q00.z + wn.w10 * q10.z + wn.w01 * q01.z + wn.w11 * q11.z;
        float er, eg;
        f2_unpack(rg, er, eg);
        float dr_, dg_;
        f2_unpack(gamma_decode_g5_pair(er, eg), dr_, dg_);
        const float ebc = fmaxf(eb, 1e-30f);
        acc.x += w * dr_;
        acc.y += w * dg_;
        acc.z += w * (ebc * ebc * (ebc * rsqrtf(ebc)));
        sumw += w;
    }
    if (!(sumw > 0.0f)) return f3(0.0f, 0.0f, 0.0f);
    const float inv = 1.0f / sumw;
    const float3 m = inv * acc;
    return f3(m.x * m.x, m.y * m.y, m.z * m.z);
}

// Cosine-weighted mean radiance M at x with normal n, the self-shadow bias
// using w_o (Sec. 4.1 equation), the 8-probe cage (Sec. 2.2): trilinear,
// backface ((1 + n.w_p)/2)^2 + 0.2, Chebyshev visibility, weight floor
// 1e-6 * w_t * w_b, gamma decode (Sec. 4.2) normalised before squaring.
// Per-probe normalisations, the Chebyshev ratio and the square roots of the
// decode use the hardware reciprocal and reciprocal square root.
// `look` is the direction the irradiance tiles are read in: n for the
// irradiance query, the mirror direction for a second-order glossy lookup
// (Sec. 4.4); the bias and the backface weights use n either way.
// FAST: the view is known to hold FP32 atlases, gamma 5 and no probe
// offsets (query_fast_view); query_M_look_fast serves it.
template <bool FAST = false>
__device__ __forceinline__ float3 query_M_look(const VolView& v, float3 x, float3 n, float3 wo, float3 look) {
    if constexpr (FAST) return query_M_look_fast(v, x, n, wo, look);
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
    float sumw = 0.0f;
    float3 acc = f3(0.0f, 0.0f, 0.0f);
    const Footprint fn = footprint(oct_encode(look), v.irr_n);   // irradiance lookup, the same for every probe
    const Bilerp wn = bilerp_weights(fn);
    // physical indices of the cage's two planes per axis
    const int px0 = wrap_add(base[0], v.shift.x, cnt[0]), px1 = wrap_add(base[0] + 1, v.shift.x, cnt[0]);
    const int py0 = wrap_add(base[1], v.shift.y, cnt[1]), py1 = wrap_add(base[1] + 1, v.shift.y, cnt[1]);
    const int pz0 = wrap_add(base[2], v.shift.z, cnt[2]), pz1 = wrap_add(base[2] + 1, v.shift.z, cnt[2]);
    // the eight states first, as independent loads, so the probe loop below
    // does not wait on one state load per probe
    unsigned act = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int p = (c & 1 ? px1 : px0) + cnt[0] * ((c & 2 ? py1 : py0) + cnt[1] * (c & 4 ? pz1 : pz0));
        act |= state_active(v.states[p]) ? 1u << c : 0u;
    }
#pragma unroll 1
    for (; act != 0; act &= act - 1) {   // active probes in ascending c
        const int c = __ffs(act) - 1;
        int o0 = c & 1, o1 = (c >> 1) & 1, o2 = (c >> 2) & 1;
        int p = (o0 ? px1 : px0) + cnt[0] * ((o1 ? py1 : py0) + cnt[1] * (o2 ? pz1 : pz0));
        float3 a = local_to_probe(v, q, base[0] + o0, base[1] + o1, base[2] + o2);
        if (v.offsets) {   // the probe's own (moved) position; the cage stays on the grid
            const float4 po = __ldg(v.offsets + p);
            a = f3(a.x - po.x, a.y - po.y, a.z - po.z);
        }
        float wt = (o0 ? fr[0] : 1.0f - fr[0]) * (o1 ? fr[1] : 1.0f - fr[1]) * (o2 ? fr[2] : 1.0f - fr[2]);
        float3 dp = f3(-(a.x + q.lo.x), -(a.y + q.lo.y), -(a.z + q.lo.z));   // probe - x
        float dd = dot(dp, dp);
        float cw = dd > 0.0f ? dot(n, dp) * rsqrtf(dd) : 1.0f;
        float hb = (1.0f + cw) * 0.5f;
        float wb = hb * hb + 0.2f;
        float3 pv = a + q.lb;                                                // biased point - probe
        float rr = dot(pv, pv);
        float wc = 1.0f;
        if (rr > 0.0f) {
            float ir = rsqrtf(rr);
            float r = rr * ir;
            const Footprint fd = footprint(oct_encode_fast(ir * pv), v.dist_n);
            float2 mom = sample_dist_at(v, p, fd);
            if (r > mom.x) {
                float var = fmaxf(mom.y - mom.x * mom.x, 0.0f);
                float dr = r - mom.x;
                wc = __fdividef(var, var + dr * dr);
            }
        }
        float w = wt * wb * fmaxf(wc, 1e-6f);
        float3 e = sample_irr_at(v, p, fn, wn);
        acc.x += w * gamma_decode_half_fast(e.x, v.half_gamma);
        acc.y += w * gamma_decode_half_fast(e.y, v.half_gamma);
        acc.z += w * gamma_decode_half_fast(e.z, v.half_gamma);
        sumw += w;
    }
    if (!(sumw > 0.0f)) return f3(0.0f, 0.0f, 0.0f);
    float inv = 1.0f / sumw;
    float3 a = inv * acc;
    return f3(a.x * a.x, a.y * a.y, a.z * a.z);
}

template <bool FAST = false>
__device__ __forceinline__ float3 query_M(const VolView& v, float3 x, float3 n, float3 wo) {
    return query_M_look<FAST>(v, x, n, wo, n);
}

// Cascade value M at x (Sec. 7.3): volumes densest first; each volume's
// weight is the product over axes of its linear fall-off over the last cell
// of its blend box; accumulation stops once the weights reach 1; the sum is
// normalised by the weights taken (0 when no volume covers x).
__device__ __forceinline__ float volume_weight(const VolView& v, float3 x) {
    float wx = fminf(fmaxf(fminf(x.x - v.blend_lo.x, v.blend_hi.x - x.x) / v.spacing.x, 0.0f), 1.0f);
    float wy = fminf(fmaxf(fminf(x.y - v.blend_lo.y, v.blend_hi.y - x.y) / v.spacing.y, 0.0f), 1.0f);
    float wz = fminf(fmaxf(fminf(x.z - v.blend_lo.z, v.blend_hi.z - x.z) / v.spacing.z, 0.0f), 1.0f);
    return wx * wy * wz;
}

template <bool FAST = false>
__device__ __forceinline__ float3 cascade_M(const VolView* vols, int n, float3 x, float3 nrm, float3 wo) {
    float sum = 0.0f;
    float3 acc = f3(0.0f, 0.0f, 0.0f);
    for (int k = 0; k < n; ++k) {
        const VolView& v = vols[k];
        float take = fminf(volume_weight(v, x), 1.0f - sum);
        if (!(take > 0.0f)) continue;
        float3 M = query_M<FAST>(v, x, nrm, wo);
        acc = acc + take * M;
        sum += take;
        if (sum >= 1.0f) break;
    }
    if (!(sum > 0.0f)) return f3(0.0f, 0.0f, 0.0f);
    return (1.0f / sum) * acc;
}

}  // namespace ddgi
