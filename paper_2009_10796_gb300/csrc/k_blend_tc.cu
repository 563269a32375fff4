// Tensor-core probe blend on sm_103a (tcgen05 MMA, TMEM accumulators).
//
// With one ray pattern per frame shared by every probe, the blend of Sec. 2.3
// (Eq. 1) is a dense contraction per frame:
//   irradiance  D_irr[t][(c,p)]  = sum_i W_irr[t][i]  * L[p][i][c]     c in {r, g, b}
//   distance    D_dist[t][(c,p)] = sum_i W_dist[t][i] * X[p][i][c]     c in {d_hi, d2_hi, d_lo, d2_lo}
// texels t on the MMA's M side (one 128-row tile of irradiance texels, two of
// distance texels), probes and channels on N, rays on K.
//
// Work split.  One persistent CTA of 288 threads per SM takes an equal,
// contiguous share of the active list and blends it in rounds of up to PG
// probes; each round walks the rays in chunks of KC.  The warps specialise:
//   * the control warp (warp 8, its lane 0) copies each chunk's pre-packed
//     weight tiles (k_pack_weights: the MMA A operands, L2 resident, shared
//     by all probes) into a ring of stages (3 for X3, 5 otherwise) with 1D
//     bulk copies issued ring depth - 1 chunks ahead, completion counted on
//     the stage's mbarrier; per chunk it waits for the weights and for the
//     chunk's B tile, issues the MMAs into TMEM from descriptors built once
//     per chunk, and commits them to the stage's second mbarrier, which
//     frees the weight stage and the B tile;
//   * the eight converter warps, one thread per (probe slot, ray pair):
//     each fetches its 32 bytes of ray records with its own asynchronous
//     copies NR - 1 chunks ahead, converts them into B operands (channel-
//     major rows, hi / lo splits) of a double-buffered B tile once the MMAs
//     that last read that tile are done, and arrives on the tile's mbarrier.
// The round's epilogue copies the old atlas tiles of its probes into shared
// memory; the converter warps move the accumulators from TMEM into a
// staging array (warp w: TMEM lanes 32 (w % 4) .. + 31, the columns of
// probes 16 (w / 4) .. + 15); then every thread finishes texels as the SIMT
// blend does (normalise, gamma, per-texel hysteresis, lerp, border copies,
// Sec. 4.2, 4.3, 7.1) in the staged tiles, which go back to the atlases with
// coalesced 16-byte stores.  mbarrier parities follow from a chunk counter
// that runs across rounds.
//
// Precision modes.
//   TF32: irradiance with TF32 operands; the distance moments keep FP32
//         accuracy with d and d^2 split into a TF32 high part and the FP32
//         remainder on the B side; TF32 weights, normalised by the sum of
//         the same rounded weights (so mu2 - mu^2 stays the variance of one
//         weighted distribution).
//   BF16: irradiance with BF16 operands; distance as TF32.
//   X3:   every contraction FP32-accurate: weights and values both split
//         into TF32 high and low parts, the three products hi.hi + hi.lo +
//         lo.hi accumulated in FP32 (the lo.lo term is below 2^-22 of the
//         product); normalised by the sum of hi + lo.
//
// Operand layout: K-major, no swizzle: 8-row x 16-byte core matrices, the K
// core matrices of a row group adjacent (LBO = 128 B), row groups SBO apart.
//
// Every wait on an mbarrier is bounded; when one gives up the kernel sets bit
// 2 of the status word, drains what it issued (bounded again), frees its TMEM
// and returns.
#include <cuda_bf16.h>

#include "blend_epilogue.cuh"

namespace ddgi {

namespace {

constexpr int PG = 32;                       // probes per round at most (MMA N columns per channel)
constexpr int KC = 16;                       // rays per chunk
constexpr int kMaxNS = 5;                    // weight ring stages, at most
constexpr int NCW = 8;                       // converter warps
constexpr int NCT = NCW * 32;                // converter threads: one per (probe slot, ray pair) of a chunk
constexpr int NT = NCT + 32;                 // plus the control warp (weight copies, MMAs)
constexpr int NR = 4;                        // raw record ring depth (per-thread asynchronous copies)
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t COL_IRR = 0, COL_DIST0 = 192, COL_DIST1 = 320;
constexpr uint32_t kWaitLimit = 1u << 22;
static_assert(NCT == PG * KC / 2, "one converter thread per (probe slot, ray pair)");

enum : int { kTF32 = 0, kBF16 = 1, kX3 = 2 };

// Shared-memory layout and operand shapes of one precision mode: the weight
// ring (ns stages of one packed chunk), the raw record ring (NR stages, probe
// rows padded so a warp's 16-byte reads of consecutive probes hit distinct
// banks), two B tiles.
template <int MODE>
struct Tc {
    static constexpr uint32_t es_irr = MODE == kBF16 ? 2u : 4u;          // irradiance operand element size
    static constexpr uint32_t irr_hi_bytes = 128 * KC * es_irr;
    static constexpr uint32_t irr_bytes = MODE == kX3 ? 2 * irr_hi_bytes : irr_hi_bytes;
    static constexpr uint32_t dist_hi_bytes = 256 * KC * 4;
    static constexpr uint32_t off_irr_lo = irr_hi_bytes;
    static constexpr uint32_t off_dist_hi = irr_bytes;
    static constexpr uint32_t off_dist_lo = irr_bytes + dist_hi_bytes;
    static constexpr uint32_t a_bytes = irr_bytes + (MODE == kX3 ? 2u : 1u) * dist_hi_bytes;   // one packed chunk
    static constexpr int ns = MODE == kX3 ? 3 : 5;                       // weight ring depth
    static constexpr uint32_t raw_stride = KC * 16 + 16;                 // probes 68 words apart
    static constexpr uint32_t raw_bytes = PG * raw_stride;
    static constexpr int irr_rows = MODE == kX3 ? 6 * PG : 3 * PG;      // irradiance B rows (MMA N)
    static constexpr uint32_t b_irr_bytes = irr_rows * KC * es_irr;
    static constexpr uint32_t b_dist_bytes = 4 * PG * KC * 4;
    static constexpr uint32_t b_bytes = b_irr_bytes + b_dist_bytes;
    static constexpr uint32_t off_raw = ns * a_bytes;
    static constexpr uint32_t off_b = off_raw + NR * raw_bytes;
    static constexpr uint32_t smem_bytes = off_b + 2 * b_bytes;
    static constexpr uint32_t sbo_irr = KC * es_irr * 8;
    static constexpr uint32_t sbo4 = KC * 4 * 8;
    static constexpr int ksteps_irr = MODE == kBF16 ? KC / 16 : KC / 8;
    static constexpr int ksteps_dist = KC / 8;
    static_assert(a_bytes % 1024 == 0 && off_b % 16 == 0 && b_bytes % 16 == 0, "operand alignment");
    static_assert(smem_bytes <= 227 * 1024, "fits the shared-memory opt-in");
    static_assert(COL_IRR + irr_rows <= COL_DIST0 && COL_DIST1 + 4 * PG <= TMEM_COLS, "TMEM columns");
};

__device__ __forceinline__ uint32_t canon(uint32_t row, uint32_t kbyte, uint32_t sbo) {
    return (row >> 3) * sbo + (kbyte >> 4) * 128u + (row & 7u) * 16u + (kbyte & 15u);
}

__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor: FP32 accumulate, K-major A and B, a/b format code
// (kind::f16: 1 = BF16; kind::tf32: 2 = TF32), N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the completion of the phase with this parity, a bounded number
// of polls; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (BF16) {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* out) {
    uint32_t r[16];
    // the wait sits in the same statement: the registers are valid only after it
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) out[j] = __uint_as_float(r[j]);
}

// Per-thread asynchronous global -> shared copies (16 or 4 bytes; 16-byte
// copies of invalid sources zero-fill and read nothing).
__device__ __forceinline__ void cpa16(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cpa4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ float comp4(float4 v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : v.z); }

}  // namespace

// Weight tiles of one frame in the MMA operand layout, one block of
// Tc<MODE>::a_bytes per chunk of KC rays: irradiance rows (128) high part
// (TF32 truncated, or BF16 rounded), [X3: the TF32 remainder], distance rows
// (256) TF32 high part, [X3: remainder].  Rows past the texel count and rays
// past R are zero.  inv_* are 1 / (sum of the weights as the MMAs see them)
// per texel, -1 when no ray reaches the texel.  Blocks [0,128) pack
// irradiance rows, [128,384) distance rows.
template <int MODE>
__global__ void __launch_bounds__(128) k_pack_weights(const float* __restrict__ w_irr,
                                                      const float* __restrict__ w_dist, int R, int ti, int td,
                                                      int nchunks, uint8_t* __restrict__ pack,
                                                      float* __restrict__ inv_irr, float* __restrict__ inv_dist) {
    using C = Tc<MODE>;
    __shared__ double red[128];
    const int b = blockIdx.x;
    const bool is_irr = b < 128;
    const int row = is_irr ? b : b - 128;
    const int valid = is_irr ? ti : td;
    const int KP = nchunks * KC;
    double acc = 0.0;
    for (int k = threadIdx.x; k < KP; k += blockDim.x) {
        float w = 0.0f;
        if (row < valid && k < R) w = is_irr ? w_irr[(int64_t)row * R + k] : w_dist[(int64_t)row * R + k];
        const int c = k / KC, kk = k - c * KC;
        uint8_t* chunk = pack + (size_t)c * C::a_bytes;
        if (is_irr && MODE == kBF16) {
            const __nv_bfloat16 h = __float2bfloat16_rn(w);
            acc += (double)__bfloat162float(h);
            *reinterpret_cast<__nv_bfloat16*>(chunk + canon(row, kk * 2, C::sbo_irr)) = h;
            continue;
        }
        const float hi = tf32_trunc(w);
        const float lo = tf32_trunc(w - hi);
        const uint32_t off_hi = is_irr ? canon(row, kk * 4, C::sbo_irr) : C::off_dist_hi + canon(row, kk * 4, C::sbo4);
        *reinterpret_cast<float*>(chunk + off_hi) = hi;
        acc += (double)hi;
        if (MODE == kX3) {
            const uint32_t off_lo =
                is_irr ? C::off_irr_lo + canon(row, kk * 4, C::sbo_irr) : C::off_dist_lo + canon(row, kk * 4, C::sbo4);
            *reinterpret_cast<float*>(chunk + off_lo) = lo;
            acc += (double)lo;
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0 && row < valid) {
        float inv = red[0] > 0.0 ? (float)(1.0 / red[0]) : -1.0f;
        if (is_irr) inv_irr[row] = inv;
        else inv_dist[row] = inv;
    }
}

template <int MODE, bool MULTI>
__global__ void __launch_bounds__(NT, 1) k_blend_tc(VolSet vs, BlendParams bp, const uint8_t* __restrict__ pack,
                                                    int nchunks, const float* __restrict__ inv_irr,
                                                    const float* __restrict__ inv_dist,
                                                    const float4* __restrict__ records,
                                                    const int32_t* __restrict__ active,
                                                    const int32_t* __restrict__ count, uint32_t* status) {
    using C = Tc<MODE>;
    constexpr int NS = C::ns;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t afull[kMaxNS];     // a weight chunk landed
    __shared__ __align__(8) uint64_t mma_bar[kMaxNS];   // a chunk's MMAs are done: its weight stage and B tile are free
    __shared__ __align__(8) uint64_t bfull[2];          // the converters filled a B tile
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    __shared__ int s_probe[PG];
    __shared__ int s_newly[PG];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool control = warp == NCW;
    const int R = bp.R;
    const VolView& v0 = vol_of<MULTI>(vs, 0);   // cascades share R, tile sizes, formats and gamma
    const int ni = v0.irr_n, nd = v0.dist_n;
    const int ti = ni * ni, td = nd * nd;
    const bool two_dist_tiles = td > 128;
    // epilogue layout (the whole dynamic shared memory, free by then): the
    // summed accumulators S [texel][channel * PG + probe] (rows padded by one
    // float), then the round's old tiles T, irradiance then distance
    constexpr int SI = 3 * PG + 1, SD = 2 * PG + 1;
    const uint32_t s_bytes = ((uint32_t)(ti * SI + td * SD) * 4u + 15u) & ~15u;
    const uint32_t tile_i = (uint32_t)(v0.irr_tile * irr_texel_bytes(v0.irr_format));
    const uint32_t tile_d = (uint32_t)(v0.dist_tile * dist_texel_bytes(v0.dist_format));
    const int pgr = min(PG, (int)((C::smem_bytes - s_bytes) / (tile_i + tile_d)));   // probes per round

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&afull[s], 1);
            mbar_init(&mma_bar[s], 1);
        }
        mbar_init(&bfull[0], NCT);
        mbar_init(&bfull[1], NCT);
        s_abort = pgr < 1;   // tiles too large for the epilogue (the launcher rejects them first)
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t sbase = smem_u32(smem);

    const int n_act = *count;
    const int per = (n_act + (int)gridDim.x - 1) / (int)gridDim.x;
    const int lo = (int)blockIdx.x * per, hi = min(n_act, lo + per);

    // global chunk index g across rounds: weight stage g % NS, raw stage
    // g % NR, B tile g & 1, mbarrier parities from the use counts; the
    // control lane keeps what it issued for the drain after an abort
    uint32_t gc = 0;
    int64_t a_issued = -1, a_waited = -1, committed = -1;
    bool abort = false;
    const int cp = tid % PG, cpair = tid / PG;   // converter: probe slot, ray pair (rays 2 cpair, 2 cpair + 1)

    auto issue_a = [&](int c, uint32_t g) {   // control lane: weight chunk c
        const int s = (int)(g % NS);
        mbar_expect_tx(&afull[s], C::a_bytes);
        bulk_g2s(sbase + (uint32_t)s * C::a_bytes, pack + (size_t)c * C::a_bytes, C::a_bytes, &afull[s]);
        a_issued = (int64_t)g;
    };
    auto issue_raw = [&](int c, int g0, int np, uint32_t g) {   // converter: its 32 bytes of chunk c
        if (c < nchunks && cp < np) {
            const int k = c * KC + 2 * cpair;
            uint8_t* dst = smem + C::off_raw + (g % NR) * C::raw_bytes + cp * C::raw_stride + cpair * 32;
            const float4* src = records + (int64_t)(g0 + cp) * R + k;
            cpa16(dst, k < R ? (const void*)src : (const void*)records, k < R);
            cpa16(dst + 16, k + 1 < R ? (const void*)(src + 1) : (const void*)records, k + 1 < R);
        }
        cpa_commit();   // one group per chunk (empty past the round's chunks)
    };

    for (int g0 = lo; g0 < hi && !s_abort; g0 += max(pgr, 1)) {
        const int np = min(pgr, hi - g0);
        if (tid < PG) {
            const int e = tid < np ? active[g0 + tid] : 0;
            s_probe[tid] = e;
            s_newly[tid] = tid < np && state_newly(vol_of<MULTI>(vs, e >> kEntryShift).states[e & kEntryMask]);
        }
        __syncthreads();
        if (control) {
            // weight copies NS - 1 chunks ahead; per chunk: wait for its
            // weights and its B tile, issue the MMAs, commit
            if (lane == 0) {
                for (int c = 0; c < min(NS - 1, nchunks); ++c) issue_a(c, gc + c);
                for (int c = 0; c < nchunks; ++c) {
                    const uint32_t g = gc + c;
                    const int s = (int)(g % NS), b = (int)(g & 1u);
                    bool ok = mbar_wait(&afull[s], (g / NS) & 1u);
                    if (ok) a_waited = (int64_t)g;
                    ok = ok && mbar_wait(&bfull[b], (g >> 1) & 1u);
                    if (!ok) {
                        abort = true;
                        break;
                    }
                    tc_fence_after();
                    // descriptors of the stage's and the B tile's bases; an
                    // operand at byte offset o adds o >> 4 to the address field
                    const uint64_t dA = smem_desc(sbase + (uint32_t)s * C::a_bytes, 128, C::sbo_irr);
                    const uint64_t dA4 = smem_desc(sbase + (uint32_t)s * C::a_bytes, 128, C::sbo4);
                    const uint64_t dB = smem_desc(sbase + C::off_b + (uint32_t)b * C::b_bytes, 128, C::sbo_irr);
                    const uint64_t dB4 = smem_desc(sbase + C::off_b + (uint32_t)b * C::b_bytes, 128, C::sbo4);
                    constexpr uint32_t id_irr = make_idesc(MODE == kBF16 ? 1u : 2u, 128, C::irr_rows);
                    constexpr uint32_t id_irr_lo = make_idesc(2u, 128, 3 * PG);
                    constexpr uint32_t id_dist = make_idesc(2u, 128, 4 * PG);
                    constexpr uint32_t id_dist_lo = make_idesc(2u, 128, 2 * PG);
                    const uint32_t first = c > 0 ? 1u : 0u;
#pragma unroll
                    for (int k = 0; k < C::ksteps_irr; ++k) {
                        const uint64_t bdesc = dB + (uint64_t)(k * 256 >> 4);
                        mma<MODE == kBF16>(tmem + COL_IRR, dA + (uint64_t)(k * 256 >> 4), bdesc, id_irr,
                                           k > 0 ? 1u : first);
                        if (MODE == kX3)
                            mma<false>(tmem + COL_IRR, dA + (uint64_t)((C::off_irr_lo + k * 256) >> 4), bdesc,
                                       id_irr_lo, 1u);
                    }
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        if (m == 1 && !two_dist_tiles) break;
#pragma unroll
                        for (int k = 0; k < C::ksteps_dist; ++k) {
                            const uint64_t bdesc = dB4 + (uint64_t)((C::b_irr_bytes + k * 256) >> 4);
                            const uint32_t col = m ? COL_DIST1 : COL_DIST0;
                            mma<false>(tmem + col, dA4 + (uint64_t)((C::off_dist_hi + m * 8192 + k * 256) >> 4), bdesc,
                                       id_dist, k > 0 ? 1u : first);
                            if (MODE == kX3)
                                mma<false>(tmem + col, dA4 + (uint64_t)((C::off_dist_lo + m * 8192 + k * 256) >> 4),
                                           bdesc, id_dist_lo, 1u);
                        }
                    }
                    mma_commit(&mma_bar[s]);
                    committed = (int64_t)g;
                    // chunk c + NS - 1 into the stage of chunk c - 1 once its MMAs are done
                    if (c + NS - 1 < nchunks) {
                        if (c >= 1 && !mbar_wait(&mma_bar[(g - 1) % NS], ((g - 1) / NS) & 1u)) {
                            abort = true;
                            break;
                        }
                        issue_a(c + NS - 1, g + NS - 1);
                    }
                }
            }
        } else {
            // converters: own records of chunk c (asynchronous copies NR - 1
            // chunks ahead) -> B tile, once that tile's MMAs two chunks back are done
            for (int c = 0; c < NR - 1; ++c) issue_raw(c, g0, np, gc + c);
            for (int c = 0; c < nchunks; ++c) {
                const uint32_t g = gc + c;
                const int b = (int)(g & 1u);
                cpa_wait<NR - 2>();
                if (c >= 2 && !mbar_wait(&mma_bar[(g - 2) % NS], ((g - 2) / NS) & 1u)) {
                    abort = true;
                    break;
                }
                float4 r0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), r1 = r0;
                if (cp < np) {
                    const uint8_t* raw = smem + C::off_raw + (g % NR) * C::raw_bytes + cp * C::raw_stride + cpair * 32;
                    r0 = *reinterpret_cast<const float4*>(raw);
                    r1 = *reinterpret_cast<const float4*>(raw + 16);
                }
                uint8_t* B = smem + C::off_b + (uint32_t)b * C::b_bytes;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float x0 = comp4(r0, ch), x1 = comp4(r1, ch);
                    if (MODE == kBF16) {
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
                        *reinterpret_cast<__nv_bfloat162*>(B + canon(ch * PG + cp, 4 * cpair, C::sbo_irr)) = h2;
                    } else if (MODE == kX3) {
                        const float2 h = make_float2(tf32_trunc(x0), tf32_trunc(x1));
                        *reinterpret_cast<float2*>(B + canon(ch * PG + cp, 8 * cpair, C::sbo_irr)) = h;
                        *reinterpret_cast<float2*>(B + canon((3 + ch) * PG + cp, 8 * cpair, C::sbo_irr)) =
                            make_float2(x0 - h.x, x1 - h.y);
                    } else {
                        *reinterpret_cast<float2*>(B + canon(ch * PG + cp, 8 * cpair, C::sbo_irr)) =
                            make_float2(x0, x1);
                    }
                }
                {
                    const float d0 = r0.w, d1 = r1.w, q0 = d0 * d0, q1 = d1 * d1;
                    const float dh0 = tf32_trunc(d0), dh1 = tf32_trunc(d1), qh0 = tf32_trunc(q0), qh1 = tf32_trunc(q1);
                    uint8_t* Bd = B + C::b_irr_bytes;
                    *reinterpret_cast<float2*>(Bd + canon(cp, 8 * cpair, C::sbo4)) = make_float2(dh0, dh1);
                    *reinterpret_cast<float2*>(Bd + canon(PG + cp, 8 * cpair, C::sbo4)) = make_float2(qh0, qh1);
                    *reinterpret_cast<float2*>(Bd + canon(2 * PG + cp, 8 * cpair, C::sbo4)) =
                        make_float2(d0 - dh0, d1 - dh1);
                    *reinterpret_cast<float2*>(Bd + canon(3 * PG + cp, 8 * cpair, C::sbo4)) =
                        make_float2(q0 - qh0, q1 - qh1);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&bfull[b]);
                issue_raw(c + NR - 1, g0, np, g + NR - 1);
            }
            cpa_wait<0>();   // no copy lands after this thread moves on
        }
        if (abort) s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        // the last chunk's commit covers every MMA of the round
        if (!mbar_wait(&mma_bar[(gc + nchunks - 1) % NS], ((gc + nchunks - 1) / NS) & 1u)) s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        tc_fence_after();

        // epilogue: the round's old tiles -> T (asynchronous copies, whole
        // tiles); the accumulators, split parts added, -> S (converter warps:
        // warp w reads TMEM lanes 32 (w % 4) .. + 31, the columns of probes
        // 16 (w / 4) .. + 15); new texels and their border copies written in
        // T in place; T -> the atlases with coalesced 16-byte stores
        float* S = reinterpret_cast<float*>(smem);
        float* Sd = S + ti * SI;
        uint8_t* Ti = smem + s_bytes;
        uint8_t* Td = Ti + np * tile_i;
        const bool g16 = (tile_i % 16u) == 0 && (tile_d % 16u) == 0;
        {
            const int gran = g16 ? 16 : 4;
            const int ui = (int)tile_i / gran, ud = (int)tile_d / gran;
            for (int k = tid; k < np * (ui + ud); k += NT) {
                const int pp = k / (ui + ud), u = k - pp * (ui + ud);
                const int e = s_probe[pp];
                const VolView& v = vol_of<MULTI>(vs, e >> kEntryShift);
                const int64_t pb = e & kEntryMask;
                const uint8_t* src = u < ui ? (const uint8_t*)v.irr + pb * tile_i + gran * u
                                            : (const uint8_t*)v.dist + pb * tile_d + gran * (u - ui);
                uint8_t* dst = u < ui ? Ti + pp * tile_i + gran * u : Td + pp * tile_d + gran * (u - ui);
                if (g16) cpa16(dst, src, true);
                else cpa4(dst, src);
            }
            cpa_commit();
        }
        if (!control) {
            const int quarter = warp & 3, half = warp >> 2;
            const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
            const int row = quarter * 32 + lane;
            if (quarter * 32 < ti) {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    float a[16];
                    tmem_ld16(tmem + lane_base + COL_IRR + ch * PG + 16 * half, a);
                    if constexpr (MODE == kX3) {
                        float l[16];
                        tmem_ld16(tmem + lane_base + COL_IRR + (3 + ch) * PG + 16 * half, l);
#pragma unroll
                        for (int j = 0; j < 16; ++j) a[j] += l[j];
                    }
                    if (row < ti)
#pragma unroll
                        for (int j = 0; j < 16; ++j) S[row * SI + ch * PG + 16 * half + j] = a[j];
                }
            }
#pragma unroll 1
            for (int m = 0; m < 2; ++m) {
                if (m * 128 + quarter * 32 >= td) continue;
                float d[4][16];
#pragma unroll
                for (int gi = 0; gi < 4; ++gi)
                    tmem_ld16(tmem + lane_base + (m ? COL_DIST1 : COL_DIST0) + gi * PG + 16 * half, d[gi]);
                const int t = m * 128 + row;
                if (t < td)
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        Sd[t * SD + 16 * half + j] = d[0][j] + d[2][j];        // sum w d   (hi + lo parts)
                        Sd[t * SD + PG + 16 * half + j] = d[1][j] + d[3][j];   // sum w d^2
                    }
            }
        }
        cpa_wait<0>();
        __syncthreads();
        {
            VolView vt = v0;   // the round's tiles in T, probe index = round slot
            vt.irr = Ti;
            vt.dist = Td;
            if (v0.irr_format == DDGI_IRR_FP32 && v0.dist_format == DDGI_DIST_FP32) {
                // FP32 atlases (the default): typed shared-memory tiles
                float4* Ti4 = reinterpret_cast<float4*>(Ti);
                float2* Td2 = reinterpret_cast<float2*>(Td);
                const int wi = ni + 2, wd = nd + 2;
                for (int q = tid; q < np * ti; q += NT) {
                    const int pp = (int)fast_div((uint32_t)q, bp.div_ti), t = q - pp * ti;
                    const int yy = (int)fast_div((uint32_t)t, bp.div_ni), x = 1 + t - yy * ni, y = 1 + yy;
                    float4* tile = Ti4 + pp * v0.irr_tile;
                    const float4 o = tile[y * wi + x];
                    const float* a = S + t * SI + pp;
                    const float3 e = blend_irr_value_fast(v0, bp, f3(o.x, o.y, o.z), a[0], a[PG], a[2 * PG],
                                                          __ldg(inv_irr + t), s_newly[pp] != 0, status);
                    const float4 e4 = make_float4(e.x, e.y, e.z, 0.0f);
                    tile[y * wi + x] = e4;
                    for_border_copies(x, y, ni, [&](int bx, int by) { tile[by * wi + bx] = e4; });
                }
                for (int q = tid; q < np * td; q += NT) {
                    const int pp = (int)fast_div((uint32_t)q, bp.div_td), t = q - pp * td;
                    const int yy = (int)fast_div((uint32_t)t, bp.div_nd), x = 1 + t - yy * nd, y = 1 + yy;
                    float2* tile = Td2 + pp * v0.dist_tile;
                    const float* a = Sd + t * SD + pp;
                    const float2 e = blend_dist_value(bp, tile[y * wd + x], a[0], a[PG], __ldg(inv_dist + t),
                                                      s_newly[pp] != 0, status);
                    tile[y * wd + x] = e;
                    for_border_copies(x, y, nd, [&](int bx, int by) { tile[by * wd + bx] = e; });
                }
            } else {
                // batches of independent items per thread: all their shared-memory
                // loads first, then the blends and stores
                constexpr int kUI = 2, kUD = 4;
                for (int q0 = tid; q0 < np * ti; q0 += kUI * NT) {
                    float3 old[kUI], sum[kUI];
                    int pi[kUI], xi[kUI], yi[kUI], tt[kUI];
    #pragma unroll
                    for (int u = 0; u < kUI; ++u) {
                        const int q = min(q0 + u * NT, np * ti - 1);
                        pi[u] = (int)fast_div((uint32_t)q, bp.div_ti);
                        tt[u] = q - pi[u] * ti;
                        const int yy = (int)fast_div((uint32_t)tt[u], bp.div_ni);
                        xi[u] = 1 + tt[u] - yy * ni;
                        yi[u] = 1 + yy;
                        const float* a = S + tt[u] * SI + pi[u];
                        sum[u] = f3(a[0], a[PG], a[2 * PG]);
                        old[u] = load_irr<false>(vt, pi[u], xi[u], yi[u]);
                    }
    #pragma unroll
                    for (int u = 0; u < kUI; ++u)
                        if (q0 + u * NT < np * ti)
                            store_irr_with_borders(vt, pi[u], xi[u], yi[u],
                                                   blend_irr_value_fast(vt, bp, old[u], sum[u].x, sum[u].y, sum[u].z,
                                                                        __ldg(inv_irr + tt[u]), s_newly[pi[u]] != 0,
                                                                        status));
                }
                for (int q0 = tid; q0 < np * td; q0 += kUD * NT) {
                    float2 old[kUD], mom[kUD];
                    int pi[kUD], xi[kUD], yi[kUD], tt[kUD];
    #pragma unroll
                    for (int u = 0; u < kUD; ++u) {
                        const int q = min(q0 + u * NT, np * td - 1);
                        pi[u] = (int)fast_div((uint32_t)q, bp.div_td);
                        tt[u] = q - pi[u] * td;
                        const int yy = (int)fast_div((uint32_t)tt[u], bp.div_nd);
                        xi[u] = 1 + tt[u] - yy * nd;
                        yi[u] = 1 + yy;
                        const float* a = Sd + tt[u] * SD + pi[u];
                        mom[u] = make_float2(a[0], a[PG]);
                        old[u] = load_dist<false>(vt, pi[u], xi[u], yi[u]);
                    }
    #pragma unroll
                    for (int u = 0; u < kUD; ++u)
                        if (q0 + u * NT < np * td)
                            store_dist_with_borders(vt, pi[u], xi[u], yi[u],
                                                    blend_dist_value(bp, old[u], mom[u].x, mom[u].y,
                                                                     __ldg(inv_dist + tt[u]), s_newly[pi[u]] != 0,
                                                                     status));
                }
            }
            }
        __syncthreads();
        {
            const int gran = g16 ? 16 : 4;
            const int ui = (int)tile_i / gran, ud = (int)tile_d / gran;
            for (int k = tid; k < np * (ui + ud); k += NT) {
                const int pp = k / (ui + ud), u = k - pp * (ui + ud);
                const int e = s_probe[pp];
                const VolView& v = vol_of<MULTI>(vs, e >> kEntryShift);
                const int64_t pb = e & kEntryMask;
                uint8_t* dst = u < ui ? (uint8_t*)v.irr + pb * tile_i + gran * u
                                      : (uint8_t*)v.dist + pb * tile_d + gran * (u - ui);
                const uint8_t* src = u < ui ? Ti + pp * tile_i + gran * u : Td + pp * tile_d + gran * (u - ui);
                if (g16) *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
                else *reinterpret_cast<uint32_t*>(dst) = *reinterpret_cast<const uint32_t*>(src);
            }
        }
        if (tid < np && s_newly[tid]) {
            const int e = s_probe[tid];
            uint8_t* sp = vol_of<MULTI>(vs, e >> kEntryShift).states + (e & kEntryMask);
            *sp = state_advanced(*sp);
        }
        // the next round's weight copies (async proxy) overwrite what these accesses used
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        gc += (uint32_t)nchunks;
        __syncthreads();
    }
    if (s_abort && control && lane == 0 && pgr >= 1) {
        // a wait gave up: report, then drain (bounded) the copies and MMAs this CTA issued
        atomicOr(status, 2u);
        for (int64_t g = a_waited + 1; g <= a_issued; ++g) mbar_wait(&afull[g % NS], (uint32_t)(g / NS) & 1u);
        if (committed >= 0) mbar_wait(&mma_bar[committed % NS], (uint32_t)(committed / NS) & 1u);
    }
    if (pgr < 1 && tid == 0) atomicOr(status, 2u);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

int tc_blend_chunks(int R) { return (R + KC - 1) / KC; }
size_t tc_pack_bytes(int R) { return (size_t)tc_blend_chunks(R) * Tc<kX3>::a_bytes; }
bool tc_blend_supported(int irr_n, int dist_n) { return irr_n * irr_n <= 128 && dist_n * dist_n <= 256; }

// Tensor-core mode of a blend precision (DDGI_BLEND_*).
static int tc_mode(int precision) {
    return precision == DDGI_BLEND_BF16 ? kBF16 : (precision == DDGI_BLEND_TF32X3 ? kX3 : kTF32);
}

cudaError_t launch_pack_weights(const float* w_irr, const float* w_dist, int R, int irr_n, int dist_n, int precision,
                                uint8_t* pack, float* inv_irr, float* inv_dist, cudaStream_t st) {
    const int ti = irr_n * irr_n, td = dist_n * dist_n, nch = tc_blend_chunks(R);
    switch (tc_mode(precision)) {
        case kBF16:
            k_pack_weights<kBF16><<<384, 128, 0, st>>>(w_irr, w_dist, R, ti, td, nch, pack, inv_irr, inv_dist);
            break;
        case kX3:
            k_pack_weights<kX3><<<384, 128, 0, st>>>(w_irr, w_dist, R, ti, td, nch, pack, inv_irr, inv_dist);
            break;
        default:
            k_pack_weights<kTF32><<<384, 128, 0, st>>>(w_irr, w_dist, R, ti, td, nch, pack, inv_irr, inv_dist);
    }
    return cudaGetLastError();
}

template <int MODE, bool MULTI>
static cudaError_t blend_tc(const VolSet& vs, const BlendParams& bp_in, int irr_n, int dist_n, const uint8_t* pack,
                            const float* inv_irr,
                            const float* inv_dist, const float4* records, const int32_t* active, const int32_t* count,
                            uint32_t* status, int grid, cudaStream_t st) {
    static DeviceOnce configured;
    cudaError_t e = once_per_device(configured, [] {
        return cudaFuncSetAttribute(k_blend_tc<MODE, MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Tc<MODE>::smem_bytes);
    });
    if (e != cudaSuccess) return e;
    BlendParams bp = bp_in;   // the epilogue's divisors: texel counts and tile widths
    bp.div_ti = make_fast_div((uint32_t)(irr_n * irr_n));
    bp.div_td = make_fast_div((uint32_t)(dist_n * dist_n));
    bp.div_ni = make_fast_div((uint32_t)irr_n);
    bp.div_nd = make_fast_div((uint32_t)dist_n);
    k_blend_tc<MODE, MULTI><<<grid, NT, Tc<MODE>::smem_bytes, st>>>(vs, bp, pack, tc_blend_chunks(bp.R), inv_irr,
                                                                     inv_dist, records, active, count, status);
    return cudaGetLastError();
}

cudaError_t launch_blend_tc_set(const VolSet& vs, bool multi, const BlendParams& bp, int precision, int irr_n,
                                int dist_n, const uint8_t* pack, const float* inv_irr, const float* inv_dist,
                                const float4* records, const int32_t* active, const int32_t* count, uint32_t* status,
                                int grid, cudaStream_t st) {
#define DDGI_TC_CASE(M, MU)                                                                                          \
    if (tc_mode(precision) == M && multi == MU)                                                                     \
        return blend_tc<M, MU>(vs, bp, irr_n, dist_n, pack, inv_irr, inv_dist, records, active, count, status, grid,  \
                               st);
    DDGI_TC_CASE(kTF32, false)
    DDGI_TC_CASE(kTF32, true)
    DDGI_TC_CASE(kBF16, false)
    DDGI_TC_CASE(kBF16, true)
    DDGI_TC_CASE(kX3, false)
    DDGI_TC_CASE(kX3, true)
#undef DDGI_TC_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_blend_tc(const VolView& v, const BlendParams& bp, int precision, const uint8_t* pack,
                            const float* inv_irr, const float* inv_dist, const float4* records, const int32_t* active,
                            const int32_t* count, uint32_t* status, int grid, cudaStream_t st) {
    return launch_blend_tc_set(single_set(v), false, bp, precision, v.irr_n, v.dist_n, pack, inv_irr, inv_dist,
                               records, active, count, status, grid, st);
}

// Shared-memory opt-in of every tensor-core blend instantiation (outside any stream capture).
cudaError_t prepare_blend_tc_kernels() {
    cudaError_t e = cudaSuccess;
#define DDGI_TC_OPT(M, MU)                                                                                           \
    if (e == cudaSuccess)                                                                                          \
        e = cudaFuncSetAttribute(k_blend_tc<M, MU>, cudaFuncAttributeMaxDynamicSharedMemorySize,                   \
                                 (int)Tc<M>::smem_bytes);
    DDGI_TC_OPT(kTF32, false)
    DDGI_TC_OPT(kTF32, true)
    DDGI_TC_OPT(kBF16, false)
    DDGI_TC_OPT(kBF16, true)
    DDGI_TC_OPT(kX3, false)
    DDGI_TC_OPT(kX3, true)
#undef DDGI_TC_OPT
    return e;
}

}  // namespace ddgi
