// Ray traversal of the scene's hierarchy in its two forms: the 4-wide
// nodes that the probe-ray passes walk warp-cooperatively (the while-while
// scheme of Aila and Laine, HPG 2009, over four child boxes per node), and
// the binary nodes that the one-ray-per-thread paths (G-buffer, raw ray
// queries, allocation-free update, adjoint) walk.  Triangles are tested with
// the watertight ray/triangle test of Woop, Benthin and Wald ("Watertight
// Ray/Triangle Intersection", JCGT 2013).  The edge
// functions are evaluated with explicitly rounded products and differences
// (no fused multiply-add), so a shared edge gives bitwise-negated values in
// its two triangles and rays cannot slip between them.  Box tests are made
// conservative by widening the exit distance by a few ulps (Ize, "Robust
// BVH Ray Traversal", JCGT 2013).
#pragma once

#include <cfloat>
#include <type_traits>

#include "probe_math.cuh"

namespace ddgi {

constexpr int kStackSize = 64;

struct RayPre {
    float3 o, d, idir;
    int kx, ky, kz;
    float Sx, Sy, Sz;
    int oct;    // bit a set: axis a runs toward -inf (its near slab plane is the box's hi)
};

__device__ __forceinline__ void ray_set_origin(RayPre& r, float3 o) { r.o = o; }

__device__ __forceinline__ float comp(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ __forceinline__ RayPre ray_pre(float3 o, float3 d) {
    RayPre r;
    r.o = o;
    r.d = d;
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    float dz = comp(d, kz);
    if (dz < 0.0f) { int t = kx; kx = ky; ky = t; }
    r.kx = kx;
    r.ky = ky;
    r.kz = kz;
    r.Sx = comp(d, kx) / dz;
    r.Sy = comp(d, ky) / dz;
    r.Sz = 1.0f / dz;
    const float eps = 1e-20f;
    r.idir = f3(1.0f / (fabsf(d.x) > eps ? d.x : copysignf(eps, d.x)),
                1.0f / (fabsf(d.y) > eps ? d.y : copysignf(eps, d.y)),
                1.0f / (fabsf(d.z) > eps ? d.z : copysignf(eps, d.z)));
    r.oct = (signbit(r.idir.x) ? 1 : 0) | (signbit(r.idir.y) ? 2 : 0) | (signbit(r.idir.z) ? 4 : 0);
    ray_set_origin(r, o);
    return r;
}

// The direction-only fields of RayPre packed into two float4 (idir, Sx;
// Sy, Sz, kx | ky << 2 | kz << 4, oct), so rays sharing a direction (the
// per-frame probe ray directions) take them from a table instead of six
// divisions per ray.  ray_pre_packed(o, d, a, b) equals ray_pre(o, d)
// field by field when (a, b) = dir_pre_pack(d).
__device__ __forceinline__ void dir_pre_pack(float3 d, float4& a, float4& b) {
    const RayPre r = ray_pre(f3(0.0f, 0.0f, 0.0f), d);
    a = make_float4(r.idir.x, r.idir.y, r.idir.z, r.Sx);
    b = make_float4(r.Sy, r.Sz, __int_as_float(r.kx | (r.ky << 2) | (r.kz << 4)), __int_as_float(r.oct));
}

__device__ __forceinline__ RayPre ray_pre_packed(float3 o, float3 d, float4 a, float4 b) {
    RayPre r;
    r.d = d;
    r.idir = f3(a.x, a.y, a.z);
    r.Sx = a.w;
    r.Sy = b.x;
    r.Sz = b.y;
    const int k = __float_as_int(b.z);
    r.kx = k & 3;
    r.ky = (k >> 2) & 3;
    r.kz = (k >> 4) & 3;
    r.oct = __float_as_int(b.w);
    ray_set_origin(r, o);
    return r;
}

// Three-input minimum / maximum (one PTX instruction on sm_100 and later).
__device__ __forceinline__ float fmin3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float fmax3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Returns t of a hit in (0, inf) or -1.
__device__ __forceinline__ float tri_hit(const RayPre& r, float4 p0, float4 p1, float4 p2) {
    float3 A = f3(p0.x - r.o.x, p0.y - r.o.y, p0.z - r.o.z);
    float3 B = f3(p1.x - r.o.x, p1.y - r.o.y, p1.z - r.o.z);
    float3 C = f3(p2.x - r.o.x, p2.y - r.o.y, p2.z - r.o.z);
    float Akz = comp(A, r.kz), Bkz = comp(B, r.kz), Ckz = comp(C, r.kz);
    float Ax = __fsub_rn(comp(A, r.kx), __fmul_rn(r.Sx, Akz));
    float Ay = __fsub_rn(comp(A, r.ky), __fmul_rn(r.Sy, Akz));
    float Bx = __fsub_rn(comp(B, r.kx), __fmul_rn(r.Sx, Bkz));
    float By = __fsub_rn(comp(B, r.ky), __fmul_rn(r.Sy, Bkz));
    float Cx = __fsub_rn(comp(C, r.kx), __fmul_rn(r.Sx, Ckz));
    float Cy = __fsub_rn(comp(C, r.ky), __fmul_rn(r.Sy, Ckz));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        // exact edge case: re-evaluate the edge functions in double precision
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return -1.0f;
    float det = U + V + W;
    if (det == 0.0f) return -1.0f;
    float T = U * (r.Sz * Akz) + V * (r.Sz * Bkz) + W * (r.Sz * Ckz);
    float t = T / det;
    return t > 0.0f ? t : -1.0f;
}

struct Hit {
    float t;
    int32_t orig;   // original triangle index, -1 = miss
    int32_t k;      // BVH-order triangle index
};

// Slab test of one child box; returns entry distance or +inf when missed.
__device__ __forceinline__ float box_enter(const RayPre& r, float lx, float hx, float ly, float hy,
                                           float lz, float hz, float tmax) {
    float t0x = (lx - r.o.x) * r.idir.x, t1x = (hx - r.o.x) * r.idir.x;
    float t0y = (ly - r.o.y) * r.idir.y, t1y = (hy - r.o.y) * r.idir.y;
    float t0z = (lz - r.o.z) * r.idir.z, t1z = (hz - r.o.z) * r.idir.z;
    float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), 0.0f));
    float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fminf(fmaxf(t0z, t1z), tmax));
    return tn <= tf * 1.0000005f ? tn : INFINITY;
}

// Slab test with the near and far planes already chosen by the ray's octant
// (nx = the box's lo.x when the ray runs toward +x, its hi.x otherwise, and
// so on): the same entry distance as box_enter, since per axis the near-plane
// distance is exactly the smaller of the two, without the per-axis min/max.
__device__ __forceinline__ float box_enter_oct(const RayPre& r, float nx, float fx, float ny, float fy, float nz,
                                               float fz, float tmax) {
    float tn = fmax3f((nx - r.o.x) * r.idir.x, (ny - r.o.y) * r.idir.y, fmaxf((nz - r.o.z) * r.idir.z, 0.0f));
    float tf = fmin3f((fx - r.o.x) * r.idir.x, (fy - r.o.y) * r.idir.y, fminf((fz - r.o.z) * r.idir.z, tmax));
    return tn <= tf * 1.0000005f ? tn : INFINITY;
}

// box_enter_oct for the four children of a 4-wide node at once: the slab
// distances of children (0, 1) and (2, 3) in packed pairs, the same IEEE
// operations lane by lane, so each k_c equals box_enter_oct's result.
__device__ __forceinline__ void box4_enter_oct(const RayPre& r, float4 nx, float4 fx, float4 ny, float4 fy, float4 nz,
                                               float4 fz, float tmax, float& k0, float& k1, float& k2, float& k3) {
    float tnx[4], tfx[4], tny[4], tfy[4], tnz[4], tfz[4];
    // the doubled operands are built per visit: holding them across the walk
    // cost more in registers (spills) than the moves cost here
    const uint64_t o2x = f2_pack(r.o.x, r.o.x), o2y = f2_pack(r.o.y, r.o.y), o2z = f2_pack(r.o.z, r.o.z);
    const uint64_t i2x = f2_pack(r.idir.x, r.idir.x), i2y = f2_pack(r.idir.y, r.idir.y),
                   i2z = f2_pack(r.idir.z, r.idir.z);
    f2_unpack(f2_mul(f2_sub(f2_pack(nx.x, nx.y), o2x), i2x), tnx[0], tnx[1]);
    f2_unpack(f2_mul(f2_sub(f2_pack(nx.z, nx.w), o2x), i2x), tnx[2], tnx[3]);
    f2_unpack(f2_mul(f2_sub(f2_pack(fx.x, fx.y), o2x), i2x), tfx[0], tfx[1]);
    f2_unpack(f2_mul(f2_sub(f2_pack(fx.z, fx.w), o2x), i2x), tfx[2], tfx[3]);
    f2_unpack(f2_mul(f2_sub(f2_pack(ny.x, ny.y), o2y), i2y), tny[0], tny[1]);
    f2_unpack(f2_mul(f2_sub(f2_pack(ny.z, ny.w), o2y), i2y), tny[2], tny[3]);
    f2_unpack(f2_mul(f2_sub(f2_pack(fy.x, fy.y), o2y), i2y), tfy[0], tfy[1]);
    f2_unpack(f2_mul(f2_sub(f2_pack(fy.z, fy.w), o2y), i2y), tfy[2], tfy[3]);
    f2_unpack(f2_mul(f2_sub(f2_pack(nz.x, nz.y), o2z), i2z), tnz[0], tnz[1]);
    f2_unpack(f2_mul(f2_sub(f2_pack(nz.z, nz.w), o2z), i2z), tnz[2], tnz[3]);
    f2_unpack(f2_mul(f2_sub(f2_pack(fz.x, fz.y), o2z), i2z), tfz[0], tfz[1]);
    f2_unpack(f2_mul(f2_sub(f2_pack(fz.z, fz.w), o2z), i2z), tfz[2], tfz[3]);
    float tn[4], tf[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        tn[c] = fmax3f(tnx[c], tny[c], fmaxf(tnz[c], 0.0f));
        tf[c] = fmin3f(tfx[c], tfy[c], fminf(tfz[c], tmax));
    }
    const uint64_t widen = f2_pack(1.0000005f, 1.0000005f);
    float w[4];
    f2_unpack(f2_mul(f2_pack(tf[0], tf[1]), widen), w[0], w[1]);
    f2_unpack(f2_mul(f2_pack(tf[2], tf[3]), widen), w[2], w[3]);
    k0 = tn[0] <= w[0] ? tn[0] : INFINITY;
    k1 = tn[1] <= w[1] ? tn[1] : INFINITY;
    k2 = tn[2] <= w[2] ? tn[2] : INFINITY;
    k3 = tn[3] <= w[3] ? tn[3] : INFINITY;
}

// Work counters of the measurement builds of the 4-wide walk.
struct TraceCount {
    uint32_t nodes = 0;   // 4-wide node visits (four child-box tests each)
    uint32_t tris = 0;    // triangle tests
};

// Traversal stack entries: a node or leaf reference alone (int; any-hit
// walks), or the reference with the entry distance of its box (int2;
// closest-hit walks).  A popped int2 entry whose box starts beyond the
// closest hit found since it was pushed is dropped without a visit: no
// triangle in that box can be closer.  An entry at exactly the hit distance
// is kept (the tie rule may still prefer a triangle in it).
template <typename E>
struct StackOps;
template <>
struct StackOps<int> {
    static __device__ __forceinline__ int make(int ref, float) { return ref; }
    static __device__ __forceinline__ bool live(int, float) { return true; }
    static __device__ __forceinline__ int ref(int e) { return e; }
};
template <>
struct StackOps<int2> {
    static __device__ __forceinline__ int2 make(int ref, float k) { return make_int2(ref, __float_as_int(k)); }
    static __device__ __forceinline__ bool live(int2 e, float t) { return __int_as_float(e.y) <= t; }
    static __device__ __forceinline__ int ref(int2 e) { return e.x; }
};

// Closest hit (ANY = false) or any hit among shadow casters (ANY = true)
// over the binary hierarchy, one ray per thread.
template <bool ANY>
__device__ __forceinline__ Hit traverse(const DevScene& s, const RayPre& r) {
    Hit h;
    h.t = INFINITY;
    h.orig = -1;
    h.k = -1;
    if (s.n_nodes == 0) return h;
    using E = typename std::conditional<ANY, int, int2>::type;
    E stack[kStackSize];
    int sp = 0;
    int node = 0;
    while (true) {
        const float4* N = s.nodes + 4 * (int64_t)node;
        float4 a = __ldg(N), b = __ldg(N + 1), z = __ldg(N + 2);
        int4 m = __ldg(reinterpret_cast<const int4*>(N + 3));
        float e0 = box_enter(r, a.x, a.y, a.z, a.w, z.x, z.y, h.t);
        float e1 = box_enter(r, b.x, b.y, b.z, b.w, z.z, z.w, h.t);
        bool h0 = e0 != INFINITY, h1 = e1 != INFINITY;
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            int child = c == 0 ? m.x : m.y;
            bool hitc = c == 0 ? h0 : h1;
            if (!hitc || child >= 0) continue;
            int first = ~child, cnt = c == 0 ? m.z : m.w;
            for (int k = first; k < first + cnt; ++k) {
                const float4* T = s.tris + 3 * (int64_t)k;
                float4 p0 = __ldg(T), p1 = __ldg(T + 1), p2 = __ldg(T + 2);
                if (ANY && !(__float_as_int(p1.w) & 1)) continue;
                float t = tri_hit(r, p0, p1, p2);
                if (t < 0.0f) continue;
                int orig = __float_as_int(p0.w);
                if (ANY) {
                    h.t = t;
                    h.orig = orig;
                    h.k = k;
                    return h;
                }
                if (t < h.t || (t == h.t && orig < h.orig)) {
                    h.t = t;
                    h.orig = orig;
                    h.k = k;
                }
            }
            if (c == 0) h0 = false; else h1 = false;
        }
        if (h0 && h1) {
            bool first0 = e0 <= e1;
            int nearc = first0 ? m.x : m.y, farc = first0 ? m.y : m.x;
            if (sp < kStackSize) stack[sp++] = StackOps<E>::make(farc, first0 ? e1 : e0);
            node = nearc;
        } else if (h0) {
            node = m.x;
        } else if (h1) {
            node = m.y;
        } else {
            // the next live entry (entries whose box starts beyond the
            // closest hit found since they were pushed are dropped)
            bool more = false;
            while (sp > 0) {
                const E e = stack[--sp];
                if (StackOps<E>::live(e, h.t)) {
                    node = StackOps<E>::ref(e);
                    more = true;
                    break;
                }
            }
            if (!more) break;
        }
    }
    return h;
}

// Warp-cooperative traversal with postponed leaves ("while-while", Aila and
// Laine, "Understanding the Efficiency of Ray Traversal on GPUs", HPG 2009).
// A lane that reaches a leaf parks it and keeps descending internal nodes
// until every lane of the warp holds a leaf; the parked leaves are then
// tested together, so the triangle loop runs with most lanes busy instead
// of once per node visit for whichever lane happened to reach a leaf.  The
// closest hit (smallest t, ties to the smaller original index) does not
// depend on the visiting order because box culling is conservative, so the
// result equals traverse<false>'s; for ANY, occlusion is the same.  The walk
// runs over the 4-wide form (ww4_round); every lane of the warp takes part
// (inactive lanes start with valid = false).
// Stack entries are node indices (>= 0) or leaf codes
// ~((first << kLeafBits) | (count - 1)) (1..kMaxLeafTris triangles).
constexpr int kNoLeaf = 0;              // "no parked leaf" (leaf codes are < 0)
constexpr int kDone = kRefDone;         // empty-stack sentinel, below every leaf code

__device__ __forceinline__ int leaf_code(int child, int cnt) { return ~(((~child) << kLeafBits) | (cnt - 1)); }

// Per-lane state of the warp-cooperative walk.  The stack array lives
// apart from the scalar fields (a pointer to the caller's local array), so
// the fields stay in registers while only the array goes to local memory.
template <int N = kStackSize, typename E = int>
struct WwLane {
    E* stack;   // N entries
    int sp;
    int node;   // next internal node, a leaf code taken from the stack, or kDone
    int leaf;   // parked leaf code or kNoLeaf
    Hit h;
};

template <int N, typename E>
__device__ __forceinline__ void ww_start(const DevScene& s, WwLane<N, E>& w, bool valid) {
    w.sp = 0;
    w.node = (valid && s.n_nodes > 0) ? 0 : kDone;
    w.leaf = kNoLeaf;
    w.h.t = INFINITY;
    w.h.orig = -1;
    w.h.k = -1;
}

// The next live stack entry (entries whose box starts beyond the current
// hit are dropped), or kDone.
template <int N, typename E>
__device__ __forceinline__ int ww_pop(WwLane<N, E>& w) {
    while (w.sp > 0) {
        const E e = w.stack[--w.sp];
        if (StackOps<E>::live(e, w.h.t)) return StackOps<E>::ref(e);
    }
    return kDone;
}

template <bool ANY, int N, bool COUNT = false, typename E = int>
__device__ __forceinline__ void ww_leaves(const DevScene& s, const RayPre& r, WwLane<N, E>& w,
                                          TraceCount* tc = nullptr);

// Leaf phase of a round: test the parked leaf and the leaves popped right
// after it.  COUNT adds triangle tests to *tc (measurement builds only).
template <bool ANY, int N, bool COUNT, typename E>
__device__ __forceinline__ void ww_leaves(const DevScene& s, const RayPre& r, WwLane<N, E>& w, TraceCount* tc) {
    while (w.leaf != kNoLeaf) {
        int code = ~w.leaf;
        int first = code >> kLeafBits, cnt = (code & ((1 << kLeafBits) - 1)) + 1;
        for (int k = first; k < first + cnt; ++k) {
            const float4* T = s.tris + 3 * (int64_t)k;
            float4 p0 = __ldg(T), p1 = __ldg(T + 1), p2 = __ldg(T + 2);
            if (ANY && !(__float_as_int(p1.w) & 1)) continue;
            if (COUNT) tc->tris++;
            float t = tri_hit(r, p0, p1, p2);
            if (t < 0.0f) continue;
            int orig = __float_as_int(p0.w);
            if (ANY) {
                w.h.t = t;
                w.h.orig = orig;
                w.h.k = k;
                break;
            }
            if (t < w.h.t || (t == w.h.t && orig < w.h.orig)) {
                w.h.t = t;
                w.h.orig = orig;
                w.h.k = k;
            }
        }
        if (ANY && w.h.orig >= 0) {
            w.node = kDone;
            w.leaf = kNoLeaf;
            break;
        }
        w.leaf = kNoLeaf;
        if (w.node < 0 && w.node != kDone) {
            w.leaf = w.node;
            w.node = ww_pop(w);
        }
    }
}

// Compare-exchange of (entry distance, reference) pairs, ascending.
__device__ __forceinline__ void cx(float& ka, int& va, float& kb, int& vb) {
    const bool sw = kb < ka;
    const float k = sw ? kb : ka;
    const int v = sw ? vb : va;
    kb = sw ? ka : kb;
    vb = sw ? va : vb;
    ka = k;
    va = v;
}

// The same round over the 4-wide hierarchy: a node tests its four child
// boxes, descends into the nearest hit child and pushes the other hits
// farthest first (for shadow rays too: near occluders are found first, and
// any hit ends them).  Leaves found among the children are parked or pushed
// as leaf codes exactly as in the binary walk.
template <bool ANY, bool COUNT = false, typename E = int>
__device__ __forceinline__ void ww4_round(const DevScene& s, const RayPre& r, WwLane<kStackSize4, E>& w,
                                          TraceCount* tc = nullptr) {
    while (true) {
        if (w.node >= 0) {
            if (COUNT) tc->nodes++;
            const float4* N = s.nodes4 + 8 * (int64_t)w.node;
            // near / far planes per axis by the ray's octant: lo and hi swap for
            // an axis the ray runs down
            const int ax = r.oct & 1, ay = (r.oct >> 1) & 1, az = (r.oct >> 2) & 1;
            const float4 nx = __ldg(N + ax), fx = __ldg(N + (ax ^ 1));
            const float4 ny = __ldg(N + 2 + ay), fy = __ldg(N + 2 + (ay ^ 1));
            const float4 nz = __ldg(N + 4 + az), fz = __ldg(N + 4 + (az ^ 1));
            const int4 ref = __ldg(reinterpret_cast<const int4*>(N + 6));
            float k0, k1, k2, k3;
            box4_enter_oct(r, nx, fx, ny, fy, nz, fz, w.h.t, k0, k1, k2, k3);
            int v0 = ref.x, v1 = ref.y, v2 = ref.z, v3 = ref.w;
            cx(k0, v0, k1, v1);
            cx(k2, v2, k3, v3);
            cx(k0, v0, k2, v2);
            cx(k1, v1, k3, v3);
            cx(k1, v1, k2, v2);
            // no bound test: scene creation checks that the hierarchy keeps the
            // stack within kStackSize4 (wide_stack_bound)
            if (k3 != INFINITY) w.stack[w.sp++] = StackOps<E>::make(v3, k3);
            if (k2 != INFINITY) w.stack[w.sp++] = StackOps<E>::make(v2, k2);
            if (k1 != INFINITY) w.stack[w.sp++] = StackOps<E>::make(v1, k1);
            w.node = k0 != INFINITY ? v0 : ww_pop(w);
            if (w.node < 0 && w.node != kDone && w.leaf == kNoLeaf) {
                w.leaf = w.node;
                w.node = ww_pop(w);
            }
        }
        if (__ballot_sync(0xffffffffu, w.node >= 0 && w.leaf == kNoLeaf) == 0) break;
    }
    ww_leaves<ANY, kStackSize4, COUNT, E>(s, r, w, tc);
}

}  // namespace ddgi
