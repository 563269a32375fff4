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

template <bool MULTI>
__global__ void __launch_bounds__(256) k_classify(DevScene s, VolSet vs, const float4* __restrict__ dirs,
                                                  int R, const int32_t* __restrict__ perm,
                                                  const int32_t* __restrict__ list,
                                                  const int32_t* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int n = *count;
    int2 stack[kStackSize4];
    WwLane<kStackSize4, int2> w;
    w.stack = stack;
    for (int q = warp; q < n; q += nwarps) {
        int e = list[q];
        const VolView& v = vol_of<MULTI>(vs, e >> kEntryShift);
        int p = e & kEntryMask;
        float3 o = probe_pos_phys(v, p);
        int bf = 0;
        float dmin = INFINITY;
        // the warp's lanes take 32 rays at a time through the warp-cooperative
        // 4-wide walk (lanes past R take part without a ray)
        for (int j0 = 0; j0 < R; j0 += 32) {
            const int j = j0 + lane;
            const bool valid = j < R;
            const int i = valid ? (perm ? __ldg(perm + j) : j) : 0;
            const float4 d4 = __ldg(dirs + i);
            const float3 d = f3(d4.x, d4.y, d4.z);
            const RayPre r = ray_pre_packed(o, d, __ldg(dirs + R + 2 * i), __ldg(dirs + R + 2 * i + 1));
            ww_start(s, w, valid);
            do {
                ww4_round<false>(s, r, w);
            } while (__ballot_sync(0xffffffffu, w.node != kDone) != 0);
            const Hit& h = w.h;
            if (valid && h.orig >= 0) {
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

// Classification in 32-ray batches: one work item per (list entry, batch),
// so the R rays of the few probes a frame classifies (the planes a tracking
// window scrolls in) spread over all warps instead of R / 32 sequential
// batches in one warp each.  A batch adds its backface count and maxes its
// nearest front-face distance (as 0x7f800000 - bits, so a zeroed word
// stands for +inf) into the entry's scratch, then counts itself done; the
// warp that completes an entry's last batch sets the state as k_classify
// does and zeroes the scratch for the next classification.  Counts and
// minima do not depend on the order the batches run in, so the states are
// k_classify's.  scratch: one zeroed int4 per list entry.
template <bool MULTI>
__global__ void __launch_bounds__(256) k_classify_split(DevScene s, VolSet vs, const float4* __restrict__ dirs,
                                                        int R, const int32_t* __restrict__ perm,
                                                        const int32_t* __restrict__ list,
                                                        const int32_t* __restrict__ count, int4* scratch) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nb = (R + 31) / 32;
    const int64_t items = (int64_t)(*count) * nb;
    int2 stack[kStackSize4];
    WwLane<kStackSize4, int2> w;
    w.stack = stack;
    for (int64_t it = warp; it < items; it += nwarps) {
        const int q = (int)(it / nb), b = (int)(it - (int64_t)q * nb);
        const int e = list[q];
        const VolView& v = vol_of<MULTI>(vs, e >> kEntryShift);
        const int p = e & kEntryMask;
        const float3 o = probe_pos_phys(v, p);
        const int j = 32 * b + lane;
        const bool valid = j < R;
        const int i = valid ? (perm ? __ldg(perm + j) : j) : 0;
        const float4 d4 = __ldg(dirs + i);
        const float3 d = f3(d4.x, d4.y, d4.z);
        const RayPre r = ray_pre_packed(o, d, __ldg(dirs + R + 2 * i), __ldg(dirs + R + 2 * i + 1));
        ww_start(s, w, valid);
        do {
            ww4_round<false>(s, r, w);
        } while (__ballot_sync(0xffffffffu, w.node != kDone) != 0);
        const Hit& h = w.h;
        bool back = false;
        float dmin = INFINITY;
        if (valid && h.orig >= 0) {
            const float4* T = s.tris + 3 * (int64_t)h.k;
            float4 p0 = __ldg(T), p1 = __ldg(T + 1), p2 = __ldg(T + 2);
            float3 ng = cross(f3(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z), f3(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z));
            if (dot(d, ng) > 0.0f) back = true;
            else dmin = h.t;
        }
        const int bf = __popc(__ballot_sync(0xffffffffu, back));
        for (int off = 16; off > 0; off >>= 1) dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, off));
        if (lane == 0) {
            int4* sc = scratch + q;
            if (bf) atomicAdd(&sc->x, bf);
            atomicMax(&sc->y, 0x7f800000 - __float_as_int(dmin));
            __threadfence();   // this batch's sums before its done count
            if (atomicAdd(&sc->z, 1) == nb - 1) {
                __threadfence();
                const int bft = atomicAdd(&sc->x, 0);
                const float dm = __int_as_float(0x7f800000 - atomicAdd(&sc->y, 0));
                uint8_t st;
                if (4 * bft > R) st = DDGI_STATE_OFF;
                else if (dm < v.min_spacing) st = DDGI_STATE_NEWLY_VIGILANT;
                else st = DDGI_STATE_SLEEPING;
                v.states[p] = st;
                *sc = make_int4(0, 0, 0, 0);   // no other batch of this entry is left
            }
        }
    }
}

// Fused trace + shade, one thread per probe ray (the allocation-free
// update's path: it needs no shadow or hit lists); rays and shadow rays go
// through the warp-cooperative 4-wide walk.
__global__ void __launch_bounds__(128) k_trace_shade(DevScene s, VolView v, Lights L,
                                                     const float4* __restrict__ dirs, int R,
                                                     const int32_t* __restrict__ active,
                                                     const int32_t* __restrict__ count,
                                                     float4* __restrict__ records) {
    const int64_t total = (int64_t)(*count) * R;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const float3 tol = f3(-L.sun_dir.x, -L.sun_dir.y, -L.sun_dir.z);
    const RayPre r_sun = ray_pre(f3(0.0f, 0.0f, 0.0f), tol);
    int2 stack[kStackSize4];
    WwLane<kStackSize4, int2> w;
    w.stack = stack;
    // warp-uniform loop: each warp takes 32 consecutive rays through the
    // warp-cooperative 4-wide walk, then their shadow rays the same way
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
        const int64_t idx = base + lane;
        const bool valid = idx < total;
        const int64_t id = valid ? idx : 0;
        int slot = (int)(id / R);
        int i = (int)(id - (int64_t)slot * R);
        int p = __ldg(active + slot);
        float3 o = probe_pos_phys(v, p);
        float4 d4 = __ldg(dirs + i);
        float3 d = f3(d4.x, d4.y, d4.z);
        const RayPre r = ray_pre_packed(o, d, __ldg(dirs + R + 2 * i), __ldg(dirs + R + 2 * i + 1));
        ww_start(s, w, valid);
        do {
            ww4_round<false>(s, r, w);
        } while (__ballot_sync(0xffffffffu, w.node != kDone) != 0);
        const Hit h = w.h;
        // the shadow ray of a sunlit front hit
        float3 n = f3(0.0f, 0.0f, 1.0f), x = o;
        float cosl = 0.0f;
        bool front = false;
        float3 ng = f3(0.0f, 0.0f, 1.0f);
        if (valid && h.orig >= 0) {
            const float4* T = s.tris + 3 * (int64_t)h.k;
            float4 p0 = __ldg(T), p1 = __ldg(T + 1), p2 = __ldg(T + 2);
            ng = cross(f3(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z), f3(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z));
            front = !(dot(d, ng) > 0.0f);
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
        if (!valid) continue;
        float4 rec;
        if (h.orig < 0) {
            float c = dot(d, L.sky_up);
            rec = make_float4(L.sky_a.x + L.sky_b.x * c, L.sky_a.y + L.sky_b.y * c,
                              L.sky_a.z + L.sky_b.z * c, v.t_max);
        } else if (!front) {
            // back face: radiance 0, depth shortened by 80% (Sec. 4.1)
            rec = make_float4(0.0f, 0.0f, 0.0f, fminf(0.2f * h.t, v.t_max));
        } else {
            int2 at = __ldg(s.attr + h.orig);
            float4 rho = __ldg(s.albedo + at.x);
            float3 Le = f3(0.0f, 0.0f, 0.0f);
            if (at.y >= 0) {
                float4 e = __ldg(s.emit + at.y);
                Le = f3(e.x, e.y, e.z);
            }
            float3 direct = f3(0.0f, 0.0f, 0.0f);
            if (lit) {
                float k = cosl * 0.318309886183790672f;   // 1/pi
                direct = f3(L.sun_irr.x * k, L.sun_irr.y * k, L.sun_irr.z * k);
            }
            float3 M = query_M(v, x, n, f3(-d.x, -d.y, -d.z));
            rec = make_float4(Le.x + rho.x * (direct.x + M.x), Le.y + rho.y * (direct.y + M.y),
                              Le.z + rho.z * (direct.z + M.z), fminf(h.t, v.t_max));
        }
        records[idx] = rec;
    }
}

// ---------------------------------------------------------------------------
// Wavefront form of trace + shade: three coherent passes over the same rays.
//   k_trace_primary  closest hit of every ray over the 4-wide hierarchy;
//                    writes the final record of misses (sky) and back faces,
//                    stores (t, BVH triangle index, 0, 0) for front hits and
//                    appends them to the hit list, and those facing the sun
//                    to the shadow-ray list
//   k_trace_shadow   any-hit shadow rays over that list; sets the visibility
//   k_shade          shading and the previous-frame query at each front hit;
//                    writes the final (r, g, b, d) record over the hit record
// Each pass keeps its lanes on one kind of work, where the fused kernel ran
// traversal, shadow rays and queries divergently in the same warp.  The
// arithmetic of every value is the fused kernel's, in the same order.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void hit_frame(const DevScene& s, int k, float3& ng) {
    const float4* T = s.tris + 3 * (int64_t)k;
    float4 p0 = __ldg(T), p1 = __ldg(T + 1), p2 = __ldg(T + 2);
    ng = cross(f3(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z), f3(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z));
}

// Persistent passes: each warp walks its lanes' rays in while-while rounds
// and, once kRefillLanes lanes have finished, hands the idle lanes the next
// work items from a global counter with one warp-aggregated atomic (Aila and
// Laine 2009, persistent threads).  kRefillLanes = 32 (refill only when the
// whole warp is idle) measured fastest on the city workload: 4, 8 and 16
// cost more in lost ray coherence than they won back in busy lanes.
constexpr int kRefillLanes = 32;

// Hands idle lanes the next work items; returns the lane's item or -1.
// Probe slot of work item (or record) idx = slot * R + ray.
__device__ __forceinline__ int ray_slot(int64_t idx, int R, FastDiv dR) {
    return idx <= INT32_MAX ? (int)fast_div((uint32_t)idx, dR) : (int)(idx / R);
}

__device__ __forceinline__ int64_t refill(unsigned long long* next, int64_t total, bool idle_lane,
                                          bool& exhausted) {
    const unsigned idle = __ballot_sync(0xffffffffu, idle_lane);
    if (exhausted || !(idle == 0xffffffffu || __popc(idle) >= kRefillLanes)) return -1;
    const int lane = threadIdx.x & 31;
    const int n = __popc(idle), leader = __ffs(idle) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(next, (unsigned long long)n);
    base = __shfl_sync(0xffffffffu, base, leader);
    if ((int64_t)base + n >= total) exhausted = true;
    if (!idle_lane) return -1;
    int64_t w = (int64_t)base + __popc(idle & ((1u << lane) - 1u));
    return w < total ? w : -1;
}

// COUNT: measurement build that adds its 4-wide node visits and triangle
// tests to stats[1], stats[2] (otherwise identical).
template <bool MULTI, bool COUNT = false>
__global__ void __launch_bounds__(256, 5) k_trace_primary(DevScene s, VolSet vs, Lights L,
                                                       const float4* __restrict__ dirs, int R, FastDiv dR,
                                                       const int32_t* __restrict__ perm,
                                                       const int32_t* __restrict__ active,
                                                       const int32_t* __restrict__ count,
                                                       float4* __restrict__ hits,
                                                       int32_t* __restrict__ shadow_list,
                                                       int32_t* __restrict__ hit_list,
                                                       int32_t* shadow_count,
                                                       unsigned long long* next,
                                                       unsigned long long* stats = nullptr) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int64_t total = (int64_t)(*count) * R;
    TraceCount tc;
    const float3 tol = f3(-L.sun_dir.x, -L.sun_dir.y, -L.sun_dir.z);
    int64_t rec = -1;   // record index of the lane's ray, -1 when idle
    int entry = 0;      // its probe's list entry
    bool exhausted = false;
    RayPre r = ray_pre(f3(0.0f, 0.0f, 0.0f), f3(0.0f, 0.0f, 1.0f));   // the lane's ray (r.d its direction)
    int2 stack[kStackSize4];
    WwLane<kStackSize4, int2> w;
    w.stack = stack;
    ww_start(s, w, false);
    while (true) {
        int64_t item = refill(next, total, rec < 0, exhausted);
        if (item >= 0) {
            // work item -> (probe slot, ray): consecutive items take a compact
            // cone of directions; the record keeps its canonical ray index
            int slot = ray_slot(item, R, dR);
            int j = (int)(item - (int64_t)slot * R);
            int i = perm ? __ldg(perm + j) : j;
            rec = (int64_t)slot * R + i;
            entry = __ldg(active + slot);
            float3 o = probe_pos_phys(vol_of<MULTI>(vs, entry >> kEntryShift), entry & kEntryMask);
            const float4 d4 = __ldg(dirs + i);
            r = ray_pre_packed(o, f3(d4.x, d4.y, d4.z), __ldg(dirs + R + 2 * i), __ldg(dirs + R + 2 * i + 1));
            ww_start(s, w, true);
        }
        if (__ballot_sync(0xffffffffu, rec >= 0) == 0) break;
        ww4_round<false, COUNT>(s, r, w, &tc);
        bool need = false, front = false;
        int64_t done = -1;
        if (rec >= 0 && w.node == kDone) {
            // misses and back faces get their final record here; front hits
            // keep (t, triangle) for the shading pass
            const Hit& h = w.h;
            const float t_max = vol_of<MULTI>(vs, entry >> kEntryShift).t_max;
            float4 out;
            if (h.orig < 0) {
                float c = dot(r.d, L.sky_up);
                out = make_float4(L.sky_a.x + L.sky_b.x * c, L.sky_a.y + L.sky_b.y * c, L.sky_a.z + L.sky_b.z * c,
                                  t_max);
            } else {
                float3 ng;
                hit_frame(s, h.k, ng);
                if (dot(r.d, ng) > 0.0f) {
                    out = make_float4(0.0f, 0.0f, 0.0f, fminf(0.2f * h.t, t_max));
                } else {
                    front = true;
                    if (L.sun_on) {
                        float3 n = (1.0f / length(ng)) * ng;
                        need = dot(n, tol) > 0.0f;
                    }
                    out = make_float4(h.t, __int_as_float(h.k), 0.0f, 0.0f);
                }
            }
            hits[rec] = out;
            done = rec;
            rec = -1;
        }
        unsigned mask = __ballot_sync(0xffffffffu, need);
        if (mask) {
            int leader = __ffs(mask) - 1;
            int off = 0;
            if (lane == leader) off = atomicAdd(shadow_count, __popc(mask));
            off = __shfl_sync(0xffffffffu, off, leader);
            if (need) shadow_list[off + __popc(mask & ((1u << lane) - 1u))] = (int32_t)done;
        }
        mask = __ballot_sync(0xffffffffu, front);
        if (mask) {
            int leader = __ffs(mask) - 1;
            int off = 0;
            if (lane == leader) off = atomicAdd(shadow_count + 1, __popc(mask));
            off = __shfl_sync(0xffffffffu, off, leader);
            if (front) hit_list[off + __popc(mask & ((1u << lane) - 1u))] = (int32_t)done;
        }
    }
    if (COUNT) {
        atomicAdd(stats + 1, (unsigned long long)tc.nodes);
        atomicAdd(stats + 2, (unsigned long long)tc.tris);
    }
}

// COUNT: adds 4-wide node visits and triangle tests to stats[4], stats[5].
template <bool MULTI, bool COUNT = false>
__global__ void __launch_bounds__(256) k_trace_shadow(DevScene s, VolSet vs, Lights L,
                                                      const float4* __restrict__ dirs, int R, FastDiv dR,
                                                      const int32_t* __restrict__ active,
                                                      float4* __restrict__ hits,
                                                      const int32_t* __restrict__ shadow_list,
                                                      const int32_t* __restrict__ shadow_count,
                                                      unsigned long long* next,
                                                      unsigned long long* stats = nullptr) {
    pdl_wait();
    pdl_trigger();
    const int64_t total = *shadow_count;
    TraceCount tc;
    const float3 tol = f3(-L.sun_dir.x, -L.sun_dir.y, -L.sun_dir.z);
    int64_t rec = -1;
    bool exhausted = false;
    const RayPre r_sun = ray_pre(f3(0.0f, 0.0f, 0.0f), tol);   // every shadow ray runs towards the sun
    RayPre r = r_sun;
    int stack[kStackSize4];   // any-hit walk: plain references (no hit distance to prune by)
    WwLane<kStackSize4> w;
    w.stack = stack;
    ww_start(s, w, false);
    while (true) {
        int64_t item = refill(next, total, rec < 0, exhausted);
        if (item >= 0) {
            rec = __ldg(shadow_list + item);
            int slot = ray_slot(rec, R, dR);
            int i = (int)(rec - (int64_t)slot * R);
            int e = __ldg(active + slot);
            float3 o = probe_pos_phys(vol_of<MULTI>(vs, e >> kEntryShift), e & kEntryMask);
            float4 d4 = __ldg(dirs + i);
            float3 d = f3(d4.x, d4.y, d4.z);
            float4 hr = hits[rec];
            float3 ng;
            hit_frame(s, __float_as_int(hr.y), ng);
            float3 nn = (1.0f / length(ng)) * ng;
            float3 x = o + hr.x * d;
            float off = 1e-4f * (1.0f + length(x));
            r = r_sun;
            ray_set_origin(r, x + off * nn);
            ww_start(s, w, true);
        }
        if (__ballot_sync(0xffffffffu, rec >= 0) == 0) break;
        ww4_round<true, COUNT>(s, r, w, &tc);
        if (rec >= 0 && w.node == kDone) {
            if (w.h.orig < 0) reinterpret_cast<float*>(hits)[4 * rec + 2] = 1.0f;
            rec = -1;
        }
    }
    if (COUNT) {
        atomicAdd(stats + 4, (unsigned long long)tc.nodes);
        atomicAdd(stats + 5, (unsigned long long)tc.tris);
    }
}

// Shading of the front hits (Sec. 2.3 ray radiance, multi-bounce through the
// previous frame's probes), one thread per entry of the compacted hit list.
template <bool MULTI, bool FAST>
__global__ void __launch_bounds__(256, 4) k_shade(DevScene s, VolSet vs, Lights L, const float4* __restrict__ dirs,
                                               int R, FastDiv dR, const int32_t* __restrict__ active,
                                               const int32_t* __restrict__ hit_list,
                                               const int32_t* __restrict__ hit_count, float4* records) {
    pdl_wait();
    pdl_trigger();
    const int n_hits = *hit_count;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_hits; q += gridDim.x * blockDim.x) {
        const int64_t idx = __ldg(hit_list + q);
        const int slot = ray_slot(idx, R, dR);
        const int i = (int)(idx - (int64_t)slot * R);
        float4 d4 = __ldg(dirs + i);
        float3 d = f3(d4.x, d4.y, d4.z);
        float4 hr = records[idx];
        int k = __float_as_int(hr.y);
        const int e = __ldg(active + slot);
        const VolView& v = vol_of<MULTI>(vs, e >> kEntryShift);
        float3 ng;
        hit_frame(s, k, ng);
        float t = hr.x;
        float3 o = probe_pos_phys(v, e & kEntryMask);
        float3 n = (1.0f / length(ng)) * ng;
        float3 x = o + t * d;
        // the sun's cosine term (zero when the shadow ray was blocked) and the
        // triangle's material index now; the previous frame's probes at the
        // hit (the volume itself, or the whole cascade) next, with little
        // else held across that query; the material terms after it
        const float3 tol = f3(-L.sun_dir.x, -L.sun_dir.y, -L.sun_dir.z);
        const float kk = hr.z != 0.0f ? dot(n, tol) * 0.318309886183790672f : 0.0f;   // 1/pi
        const int orig = __float_as_int(__ldg(&s.tris[3 * (int64_t)k].w));
        float3 M = MULTI ? cascade_M<FAST>(vs.table, vs.n, x, n, f3(-d.x, -d.y, -d.z))
                         : query_M<FAST>(v, x, n, f3(-d.x, -d.y, -d.z));
        int2 at = __ldg(s.attr + orig);
        float4 rho = __ldg(s.albedo + at.x);
        float3 Le = f3(0.0f, 0.0f, 0.0f);
        if (at.y >= 0) {
            float4 em = __ldg(s.emit + at.y);
            Le = f3(em.x, em.y, em.z);
        }
        const float3 direct = f3(L.sun_irr.x * kk, L.sun_irr.y * kk, L.sun_irr.z * kk);
        records[idx] = make_float4(Le.x + rho.x * (direct.x + M.x), Le.y + rho.y * (direct.y + M.y),
                                   Le.z + rho.z * (direct.z + M.z), fminf(t, v.t_max));
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

// One iteration of the probe position optimizer (Sec. 5 and its listing),
// one warp per UNINIT probe: the lanes trace the iteration's rays from the
// probe's current position and reduce, as (t bits << 32 | ray) keys, the
// closest backface, the closest front face and the farthest front face
// (ties: smaller ray index for closest, larger for farthest); lane 0 moves
// the offset:
//   more than 25% backfaces: along t * w of the closest backface, by the
//     largest scale keeping every component within +-limit (less 1 mm),
//     only when that scale exceeds 1 (the move goes through the backface);
//   otherwise, unless the farthest front face lies within 60 degrees of the
//     closest: min(0.2, t) along the farthest front face, clamped to +-limit.
__global__ void __launch_bounds__(256) k_optimize(DevScene s, VolView v, const float4* __restrict__ dirs, int R,
                                                  const int32_t* __restrict__ list,
                                                  const int32_t* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int n = *count;
    const DevScene& sc = s;
    int2 stack[kStackSize4];
    WwLane<kStackSize4, int2> w;
    w.stack = stack;
    for (int q = warp; q < n; q += nwarps) {
        const int p = list[q];
        const float3 o = probe_pos_phys(v, p);
        int bf = 0;
        unsigned long long cb = ~0ull, cf = ~0ull, ff = 0ull;
        // 32 rays at a time through the warp-cooperative 4-wide walk (lanes
        // past R take part without a ray)
        for (int i0 = 0; i0 < R; i0 += 32) {
            const int i = i0 + lane;
            const bool valid = i < R;
            const int ii = valid ? i : 0;
            const float4 d4 = __ldg(dirs + ii);
            const float3 d = f3(d4.x, d4.y, d4.z);
            const RayPre r = ray_pre_packed(o, d, __ldg(dirs + R + 2 * ii), __ldg(dirs + R + 2 * ii + 1));
            ww_start(sc, w, valid);
            do {
                ww4_round<false>(sc, r, w);
            } while (__ballot_sync(0xffffffffu, w.node != kDone) != 0);
            const Hit h = w.h;
            if (!valid || h.orig < 0) continue;
            const float4* T = s.tris + 3 * (int64_t)h.k;
            float4 p0 = __ldg(T), p1 = __ldg(T + 1), p2 = __ldg(T + 2);
            float3 ng = cross(f3(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z), f3(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z));
            const unsigned long long key = ((unsigned long long)__float_as_uint(h.t) << 32) | (unsigned)i;
            if (dot(d, ng) > 0.0f) {
                bf++;
                cb = key < cb ? key : cb;
            } else {
                cf = key < cf ? key : cf;
                ff = key > ff ? key : ff;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            bf += __shfl_xor_sync(0xffffffffu, bf, off);
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, cb, off);
            const unsigned long long b = __shfl_xor_sync(0xffffffffu, cf, off);
            const unsigned long long c = __shfl_xor_sync(0xffffffffu, ff, off);
            cb = a < cb ? a : cb;
            cf = b < cf ? b : cf;
            ff = c > ff ? c : ff;
        }
        if (lane != 0) continue;
        const float4 c4 = v.offsets[p];
        float3 cur = f3(c4.x, c4.y, c4.z);
        const float3 lim = f3(v.offset_limit * v.spacing.x, v.offset_limit * v.spacing.y,
                              v.offset_limit * v.spacing.z);
        if (4 * bf > R) {
            const float4 w = __ldg(dirs + (int)(cb & 0xffffffffu));
            const float tb = __uint_as_float((unsigned)(cb >> 32));
            const float3 vec = f3(tb * w.x, tb * w.y, tb * w.z);
            const float sx = fmaxf((lim.x - cur.x) / vec.x, (-lim.x - cur.x) / vec.x);
            const float sy = fmaxf((lim.y - cur.y) / vec.y, (-lim.y - cur.y) / vec.y);
            const float sz = fmaxf((lim.z - cur.z) / vec.z, (-lim.z - cur.z) / vec.z);
            const float scale = fminf(fminf(sx, sy), sz) - 1e-3f;
            if (scale > 1.0f) cur = f3(cur.x + vec.x * scale, cur.y + vec.y * scale, cur.z + vec.z * scale);
        } else if (ff != 0ull && cf != ~0ull) {
            const float4 wf = __ldg(dirs + (int)(ff & 0xffffffffu));
            const float4 wc = __ldg(dirs + (int)(cf & 0xffffffffu));
            if (!(wf.x * wc.x + wf.y * wc.y + wf.z * wc.z > 0.5f)) {
                const float step = fminf(0.2f, __uint_as_float((unsigned)(ff >> 32)));
                cur = f3(fminf(fmaxf(cur.x + step * wf.x, -lim.x), lim.x),
                         fminf(fmaxf(cur.y + step * wf.y, -lim.y), lim.y),
                         fminf(fmaxf(cur.z + step * wf.z, -lim.z), lim.z));
            }
        }
        v.offsets[p] = make_float4(cur.x, cur.y, cur.z, 0.0f);
    }
}

cudaError_t launch_optimize(const DevScene& s, const VolView& v, const float4* dirs, int R, const int32_t* list,
                            const int32_t* count, int grid, cudaStream_t st) {
    k_optimize<<<grid, 256, 0, st>>>(s, v, dirs, R, list, count);
    return cudaGetLastError();
}

cudaError_t launch_classify(const DevScene& s, const VolView& v, const float4* dirs, int R, const int32_t* perm,
                            const int32_t* list, const int32_t* count, int4* scratch, int grid, cudaStream_t st) {
    if (scratch)
        k_classify_split<false><<<grid, 256, 0, st>>>(s, single_set(v), dirs, R, perm, list, count, scratch);
    else
        k_classify<false><<<grid, 256, 0, st>>>(s, single_set(v), dirs, R, perm, list, count);
    return cudaGetLastError();
}

cudaError_t launch_classify_multi(const DevScene& s, const VolSet& vs, const float4* dirs, int R,
                                  const int32_t* perm, const int32_t* list, const int32_t* count, int4* scratch,
                                  int grid, cudaStream_t st) {
    if (scratch)
        k_classify_split<true><<<grid, 256, 0, st>>>(s, vs, dirs, R, perm, list, count, scratch);
    else
        k_classify<true><<<grid, 256, 0, st>>>(s, vs, dirs, R, perm, list, count);
    return cudaGetLastError();
}

cudaError_t launch_trace_shade(const DevScene& s, const VolView& v, const Lights& L, const float4* dirs,
                               int R, const int32_t* active, const int32_t* count, float4* records,
                               int grid, cudaStream_t st) {
    k_trace_shade<<<grid, 128, 0, st>>>(s, v, L, dirs, R, active, count, records);
    return cudaGetLastError();
}

template <bool MULTI>
static cudaError_t trace_wavefront(const DevScene& s, const VolSet& vs, const Lights& L, const float4* dirs, int R,
                                   const int32_t* perm, const int32_t* active, const int32_t* count,
                                   float4* records, int32_t* shadow_list, int32_t* hit_list, int32_t* shadow_count,
                                   int grid, cudaStream_t st, cudaEvent_t* marks, bool fast_query) {
    // shadow_count (zeroed by the caller): [0] shadow rays, [1] front hits,
    // [2..3] and [4..5] the 64-bit work counters of the two persistent passes
    unsigned long long* next = reinterpret_cast<unsigned long long*>(shadow_count + 2);
    unsigned long long* next_shadow = reinterpret_cast<unsigned long long*>(shadow_count + 4);
    cudaError_t e = cudaSuccess;
    if (marks && (e = cudaEventRecord(marks[0], st)) != cudaSuccess) return e;
    const FastDiv dR = make_fast_div((uint32_t)R);
    if ((e = launch_pdl(k_trace_primary<MULTI>, grid, 256, 0, st, s, vs, L, dirs, R, dR, perm, active, count, records,
                        shadow_list, hit_list, shadow_count, next, nullptr)) != cudaSuccess)
        return e;
    if (marks && (e = cudaEventRecord(marks[1], st)) != cudaSuccess) return e;
    if ((e = launch_pdl(k_trace_shadow<MULTI>, grid, 256, 0, st, s, vs, L, dirs, R, dR, active, records, shadow_list,
                        shadow_count, next_shadow, nullptr)) != cudaSuccess)
        return e;
    if (marks && (e = cudaEventRecord(marks[2], st)) != cudaSuccess) return e;
    e = fast_query ? launch_pdl(k_shade<MULTI, true>, grid, 256, 0, st, s, vs, L, dirs, R, dR, active, hit_list,
                                shadow_count + 1, records)
                   : launch_pdl(k_shade<MULTI, false>, grid, 256, 0, st, s, vs, L, dirs, R, dR, active, hit_list,
                                shadow_count + 1, records);
    if (e != cudaSuccess) return e;
    if (marks && (e = cudaEventRecord(marks[3], st)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t launch_trace_count(const DevScene& s, const VolView& v, const Lights& L, const float4* dirs, int R,
                               const int32_t* perm, const int32_t* active, const int32_t* count, float4* records,
                               int32_t* shadow_list, int32_t* hit_list, int32_t* shadow_count,
                               unsigned long long* stats, int grid, cudaStream_t st) {
    const VolSet vs = single_set(v);
    unsigned long long* next = reinterpret_cast<unsigned long long*>(shadow_count + 2);
    unsigned long long* next_shadow = reinterpret_cast<unsigned long long*>(shadow_count + 4);
    cudaError_t e = cudaMemsetAsync(shadow_count, 0, 6 * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    const FastDiv dR = make_fast_div((uint32_t)R);
    k_trace_primary<false, true><<<grid, 256, 0, st>>>(s, vs, L, dirs, R, dR, perm, active, count, records,
                                                        shadow_list, hit_list, shadow_count, next, stats);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_trace_shadow<false, true><<<grid, 256, 0, st>>>(s, vs, L, dirs, R, dR, active, records, shadow_list,
                                                       shadow_count, next_shadow, stats);
    return cudaGetLastError();
}

cudaError_t launch_trace_wavefront(const DevScene& s, const VolView& v, const Lights& L, const float4* dirs,
                                   int R, const int32_t* perm, const int32_t* active, const int32_t* count,
                                   float4* records, int32_t* shadow_list, int32_t* hit_list, int32_t* shadow_count,
                                   int grid, cudaStream_t st, cudaEvent_t* marks) {
    return trace_wavefront<false>(s, single_set(v), L, dirs, R, perm, active, count, records, shadow_list, hit_list,
                                  shadow_count, grid, st, marks, query_fast_view(v));
}

cudaError_t launch_trace_wavefront_multi(const DevScene& s, const VolSet& vs, const Lights& L,
                                         const float4* dirs, int R, const int32_t* perm, const int32_t* active,
                                         const int32_t* count, float4* records, int32_t* shadow_list,
                                         int32_t* hit_list, int32_t* shadow_count, int grid, cudaStream_t st,
                                         bool fast_query) {
    return trace_wavefront<true>(s, vs, L, dirs, R, perm, active, count, records, shadow_list, hit_list,
                                 shadow_count, grid, st, nullptr, fast_query);
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
