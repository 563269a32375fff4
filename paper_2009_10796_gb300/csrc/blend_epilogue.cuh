// Blend epilogue shared by the SIMT and tensor-core blends (Sec. 2.3 Eq. 1,
// Sec. 4.2 gamma encoding, Sec. 4.3 per-texel thresholds, Sec. 7.1 border copy).
#pragma once

#include "probe_math.cuh"

namespace ddgi {

// Border texels that copy interior texel (x, y) of a bordered tile (tile
// coordinates, interior spans 1..n): the mirrored neighbour across each seam
// edge it touches and, for the four interior corners, the opposite outer corner.
template <typename F>
__device__ __forceinline__ void for_border_copies(int x, int y, int n, F&& f) {
    if (x == 1) f(0, n + 1 - y);
    if (x == n) f(n + 1, n + 1 - y);
    if (y == 1) f(n + 1 - x, 0);
    if (y == n) f(n + 1 - x, n + 1);
    if (x == n && y == n) f(0, 0);
    if (x == 1 && y == n) f(n + 1, 0);
    if (x == n && y == 1) f(0, n + 1);
    if (x == 1 && y == 1) f(n + 1, n + 1);
}

// The new value of one irradiance texel from its weighted sums and its old
// value: normalise, gamma-encode, per-texel hysteresis thresholds, lerp.
// inv < 0 marks a texel no ray reaches: it keeps its old value.
__device__ __forceinline__ float3 blend_irr_value(const VolView& v, const BlendParams& bp, float3 old, float ar,
                                                  float ag, float ab, float inv, bool newly, uint32_t* status) {
    float3 e = old;
    if (inv >= 0.0f) {
        float3 en = f3(powf(ar * inv, v.inv_gamma), powf(ag * inv, v.inv_gamma), powf(ab * inv, v.inv_gamma));
        float delta = fmaxf(fabsf(en.x - old.x), fmaxf(fabsf(en.y - old.y), fabsf(en.z - old.z)));
        float a = newly ? 0.0f : bp.hyst_irr;
        if (delta > bp.thr_low) a = fmaxf(0.0f, a - bp.thr_step);
        if (delta > bp.thr_high) a = 0.0f;
        e = f3((1.0f - a) * en.x + a * old.x, (1.0f - a) * en.y + a * old.y, (1.0f - a) * en.z + a * old.z);
        if (!(isfinite(e.x) && isfinite(e.y) && isfinite(e.z))) atomicOr(status, 1u);
    }
    return e;
}

// blend_irr_value with the gamma encode by the hardware exp2 / log2
// (__powf, about 2 ulp for exponents below 1), for the tensor-core blend's
// epilogue where the accurate powf dominated; radiance sums are >= 0.
__device__ __forceinline__ float3 blend_irr_value_fast(const VolView& v, const BlendParams& bp, float3 old, float ar,
                                                       float ag, float ab, float inv, bool newly, uint32_t* status) {
    float3 e = old;
    if (inv >= 0.0f) {
        float3 en = f3(__powf(ar * inv, v.inv_gamma), __powf(ag * inv, v.inv_gamma), __powf(ab * inv, v.inv_gamma));
        float delta = fmaxf(fabsf(en.x - old.x), fmaxf(fabsf(en.y - old.y), fabsf(en.z - old.z)));
        float a = newly ? 0.0f : bp.hyst_irr;
        if (delta > bp.thr_low) a = fmaxf(0.0f, a - bp.thr_step);
        if (delta > bp.thr_high) a = 0.0f;
        e = f3((1.0f - a) * en.x + a * old.x, (1.0f - a) * en.y + a * old.y, (1.0f - a) * en.z + a * old.z);
        if (!(isfinite(e.x) && isfinite(e.y) && isfinite(e.z))) atomicOr(status, 1u);
    }
    return e;
}

// The same for a distance texel: normalised moments lerped with the old ones.
__device__ __forceinline__ float2 blend_dist_value(const BlendParams& bp, float2 old, float m1, float m2, float inv,
                                                   bool newly, uint32_t* status) {
    float2 e = old;
    if (inv >= 0.0f) {
        float a = newly ? 0.0f : bp.hyst_vis;
        e = make_float2((1.0f - a) * (m1 * inv) + a * old.x, (1.0f - a) * (m2 * inv) + a * old.y);
        if (!(isfinite(e.x) && isfinite(e.y))) atomicOr(status, 1u);
    }
    return e;
}

// Bytes of one stored texel (DDGI_IRR_* / DDGI_DIST_* formats).
__device__ __forceinline__ int irr_texel_bytes(int fmt) {
    return fmt == DDGI_IRR_FP32 ? 16 : (fmt == DDGI_IRR_FP16 ? 8 : 4);
}
__device__ __forceinline__ int dist_texel_bytes(int fmt) { return fmt == DDGI_DIST_FP32 ? 8 : 4; }

// Requests probe p's two bordered tiles into L2 (one prefetch per 128-byte
// line, the last byte's line included), for a blend that reads them later.
__device__ __forceinline__ void prefetch_tiles_l2(const VolView& v, int p) {
    const int64_t bi = (int64_t)v.irr_tile * irr_texel_bytes(v.irr_format);
    const int64_t bd = (int64_t)v.dist_tile * dist_texel_bytes(v.dist_format);
    const char* a = (const char*)v.irr + p * bi;
    const char* d = (const char*)v.dist + p * bd;
    for (int64_t o = 0; o < bi; o += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(a + o));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a + bi - 1));
    for (int64_t o = 0; o < bd; o += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(d + o));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(d + bd - 1));
}

// A texel and the border texels that copy it (Sec. 7.1).
__device__ __forceinline__ void store_irr_with_borders(const VolView& v, int p, int x, int y, float3 e) {
    store_irr(v, p, x, y, e);
    for_border_copies(x, y, v.irr_n, [&](int bx, int by) { store_irr(v, p, bx, by, e); });
}

__device__ __forceinline__ void store_dist_with_borders(const VolView& v, int p, int x, int y, float2 e) {
    store_dist(v, p, x, y, e);
    for_border_copies(x, y, v.dist_n, [&](int bx, int by) { store_dist(v, p, bx, by, e); });
}

// Epilogues shared by the SIMT and tensor-core blends: one (texel, probe)
// pair from its weighted sums and the texel's old value, the texel at tile
// coordinates (x, y) (interior 1..n).
__device__ __forceinline__ void blend_irr_texel_at(const VolView& v, const BlendParams& bp, int p, int x, int y,
                                                   float ar, float ag, float ab, float inv, bool newly,
                                                   uint32_t* status) {
    const float3 old = load_irr<false>(v, p, x, y);
    store_irr_with_borders(v, p, x, y, blend_irr_value(v, bp, old, ar, ag, ab, inv, newly, status));
}

__device__ __forceinline__ void blend_dist_texel_at(const VolView& v, const BlendParams& bp, int p, int x, int y,
                                                    float m1, float m2, float inv, bool newly, uint32_t* status) {
    const float2 old = load_dist<false>(v, p, x, y);
    store_dist_with_borders(v, p, x, y, blend_dist_value(bp, old, m1, m2, inv, newly, status));
}

// The same by interior texel index t (row-major over the n x n interior).
__device__ __forceinline__ void blend_irr_texel(const VolView& v, const BlendParams& bp, int p, int t,
                                                float ar, float ag, float ab, float inv, bool newly,
                                                uint32_t* status) {
    blend_irr_texel_at(v, bp, p, 1 + t % v.irr_n, 1 + t / v.irr_n, ar, ag, ab, inv, newly, status);
}

__device__ __forceinline__ void blend_dist_texel(const VolView& v, const BlendParams& bp, int p, int t,
                                                 float m1, float m2, float inv, bool newly,
                                                 uint32_t* status) {
    blend_dist_texel_at(v, bp, p, 1 + t % v.dist_n, 1 + t / v.dist_n, m1, m2, inv, newly, status);
}

}  // namespace ddgi
