// Tensor-core probe blend on sm_103a (tcgen05 MMA, TMEM accumulators).
//
// With one ray pattern per frame shared by every probe, the blend of Sec. 2.3
// (Eq. 1) is a dense contraction per frame:
//   irradiance  D_irr[t][(p,c)]  = sum_i W_irr[t][i]  * L[p][i][c]     c in {r, g, b}
//   distance    D_dist[t][(p,c)] = sum_i W_dist[t][i] * X[p][i][c]     c in {d_hi, d_lo, d2_hi, d2_lo}
// A persistent CTA (one per SM, 256 threads) takes groups of 32 active probes
// and walks the rays in chunks of 32:
//   * the weight tiles of the chunk (pre-packed by k_pack_weights in the
//     operand layout) arrive by two bulk TMA copies, completion counted on an
//     mbarrier;
//   * the threads stage the chunk's ray records as the B operands;
//   * one thread issues the MMAs (irradiance M=128 N=96; distance two M=128
//     tiles, N=128) accumulating in TMEM and commits them to a second mbarrier
//     that frees the stage (two stages, so staging overlaps the MMAs).
// The accumulators are read back with tcgen05.ld into shared memory and the
// epilogue of the SIMT blend finishes each texel (normalise, gamma, per-texel
// hysteresis, lerp, border copy).
//
// Precision.  Irradiance runs in TF32 or BF16 (one pass).  The distance
// moments keep FP32 accuracy: d and d^2 enter as hi + lo TF32 pairs (the hi part
// truncated to TF32, the lo part the exact FP32 remainder) and accumulate in
// FP32; the weights are TF32, and both moments are normalised by the sum of the
// same rounded weights, so mu2 - mu^2 remains the variance of one weighted
// distribution.
//
// Operand layout: K-major, no swizzle: 8-row x 16-byte core matrices, K chunks
// of a row group adjacent (LBO = 128 B), row groups after all of a tile's K
// chunks (SBO = 32 * element size * 8 B).
//
// Every wait on an mbarrier is bounded; when one gives up the kernel sets bit
// 2 of the status word, drains what it issued (bounded again), frees its TMEM
// and returns.
#include <cuda_bf16.h>

#include "blend_epilogue.cuh"

namespace ddgi {

namespace {

constexpr int PG = 32;                       // probes per group
constexpr int KC = 32;                       // rays per chunk
constexpr int NT = 256;                      // threads per CTA: staging, TMEM readback, epilogue
constexpr int IRR_N = 3 * PG;                // 96 accumulator columns
constexpr int DIST_N = 4 * PG;               // 128 accumulator columns
constexpr uint32_t COL_IRR = 0, COL_DIST0 = 128, COL_DIST1 = 256, TMEM_COLS = 512;

constexpr uint32_t A_IRR_MAX = 128 * KC * 4;          // 16 KB (BF16 uses half)
constexpr uint32_t A_DIST_BYTES = 256 * KC * 4;       // 32 KB
constexpr uint32_t OFF_A_IRR = 0;
constexpr uint32_t OFF_A_DIST = OFF_A_IRR + A_IRR_MAX;
constexpr uint32_t OFF_B_IRR = OFF_A_DIST + A_DIST_BYTES;
constexpr uint32_t OFF_B_DIST = OFF_B_IRR + IRR_N * KC * 4;
constexpr uint32_t STAGE_BYTES = OFF_B_DIST + DIST_N * KC * 4;   // 77,824 B
// accumulator rows in shared memory for the epilogue, padded by one float so
// a warp reading one column of consecutive rows hits distinct banks
constexpr int DIRR_STRIDE = IRR_N + 1;
constexpr int DDIST_STRIDE = DIST_N + 1;
// two stages plus slack: an operand read of up to 256 rows from the last
// tile, and the epilogue's accumulator copy (128 x 97 + 256 x 129 floats),
// both stay inside the allocation
constexpr uint32_t SMEM_BYTES = 2 * STAGE_BYTES + 32768;
constexpr uint32_t OFF_D_DIST = 128 * DIRR_STRIDE * 4;
static_assert(OFF_D_DIST + 256 * DDIST_STRIDE * 4 <= SMEM_BYTES, "epilogue copy fits");

constexpr uint32_t kWaitLimit = 1u << 22;

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

__device__ __forceinline__ float comp4(float4 v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : v.z); }

}  // namespace

// Weight tiles of one frame in the MMA operand layout, chunk after chunk:
// irradiance rows (128 per chunk) in TF32 (truncated) or BF16 (rounded),
// distance rows (256 per chunk) in TF32; rows past the texel count and rays
// past R are zero.  inv_* are 1 / (sum of the rounded weights) per texel, -1 when
// no ray reaches the texel.  Blocks [0,128) pack irradiance rows, [128,384) distance.
__global__ void __launch_bounds__(128) k_pack_weights(const float* __restrict__ w_irr,
                                                      const float* __restrict__ w_dist, int R, int ti, int td,
                                                      int nchunks, int irr_bf16, uint8_t* __restrict__ a_irr,
                                                      uint8_t* __restrict__ a_dist, float* __restrict__ inv_irr,
                                                      float* __restrict__ inv_dist) {
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
        int c = k / KC, kk = k - c * KC;
        if (is_irr && irr_bf16) {
            __nv_bfloat16 h = __float2bfloat16_rn(w);
            acc += (double)__bfloat162float(h);
            *reinterpret_cast<__nv_bfloat16*>(a_irr + (size_t)c * (128 * KC * 2) + canon(row, kk * 2, KC * 2 * 8)) = h;
        } else {
            float wt = tf32_trunc(w);
            acc += (double)wt;
            uint8_t* base = is_irr ? a_irr + (size_t)c * (128 * KC * 4) : a_dist + (size_t)c * (256 * KC * 4);
            *reinterpret_cast<float*>(base + canon(row, kk * 4, KC * 4 * 8)) = wt;
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

template <bool BF16, bool MULTI>
__global__ void __launch_bounds__(NT, 1) k_blend_tc(VolSet vs, BlendParams bp, const uint8_t* __restrict__ a_irr_pack,
                                                    const uint8_t* __restrict__ a_dist_pack, int nchunks,
                                                    const float* __restrict__ inv_irr,
                                                    const float* __restrict__ inv_dist,
                                                    const float4* __restrict__ records,
                                                    const int32_t* __restrict__ active,
                                                    const int32_t* __restrict__ count, uint32_t* status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full_bar[2];
    __shared__ __align__(8) uint64_t empty_bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_probe[PG];
    __shared__ int s_newly[PG];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = bp.R;
    const VolView& v0 = vol_of<MULTI>(vs, 0);   // cascades share R and tile sizes
    const int ti = v0.irr_n * v0.irr_n, td = v0.dist_n * v0.dist_n;
    constexpr uint32_t es_irr = BF16 ? 2u : 4u;
    constexpr uint32_t sbo_irr = KC * es_irr * 8;
    constexpr uint32_t sbo4 = KC * 4 * 8;
    constexpr uint32_t a_irr_bytes = 128 * KC * es_irr;
    constexpr uint32_t idesc_irr = make_idesc(BF16 ? 1u : 2u, 128, IRR_N);
    constexpr uint32_t idesc_dist = make_idesc(2u, 128, DIST_N);
    constexpr int ksteps_irr = BF16 ? KC / 16 : KC / 8;
    constexpr int ksteps_dist = KC / 8;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&full_bar[0], 1);
        mbar_init(&full_bar[1], 1);
        mbar_init(&empty_bar[0], 1);
        mbar_init(&empty_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t sbase = smem_u32(smem);

    uint32_t full_phase[2] = {0u, 0u}, empty_phase[2] = {0u, 0u};
    bool empty_pending[2] = {false, false};   // every thread: MMAs committed on this stage, not yet waited
    bool tma_pending[2] = {false, false};     // thread 0: bulk copies issued, not yet waited
    bool committed[2] = {false, false};       // thread 0: MMAs committed, completion not yet seen
    bool abort = false;
    const int n_act = *count;

    for (int g0 = blockIdx.x * PG; g0 < n_act; g0 += gridDim.x * PG) {
        const int np = min(PG, n_act - g0);
        if (tid < PG) {
            int e = tid < np ? active[g0 + tid] : 0;
            s_probe[tid] = e;
            s_newly[tid] = tid < np &&
                           state_newly(vol_of<MULTI>(vs, e >> kEntryShift).states[e & kEntryMask]);
        }
        for (int c = 0; c < nchunks; ++c) {
            const int s = c & 1;
            abort = __syncthreads_or(abort);
            if (abort) break;
            if (empty_pending[s]) {
                if (!mbar_wait(&empty_bar[s], empty_phase[s])) abort = true;
                else committed[s] = false;
                empty_phase[s] ^= 1u;
                empty_pending[s] = false;
            }
            abort = __syncthreads_or(abort);
            if (abort) break;
            uint8_t* stage = smem + s * STAGE_BYTES;
            const uint32_t sstage = sbase + s * STAGE_BYTES;
            if (tid == 0) {
                mbar_expect_tx(&full_bar[s], a_irr_bytes + A_DIST_BYTES);
                bulk_g2s(sstage + OFF_A_IRR, a_irr_pack + (size_t)c * a_irr_bytes, a_irr_bytes, &full_bar[s]);
                bulk_g2s(sstage + OFF_A_DIST, a_dist_pack + (size_t)c * A_DIST_BYTES, A_DIST_BYTES, &full_bar[s]);
                tma_pending[s] = true;
            }
            // ray records of the chunk -> B operands; a thread takes 4 rays of one probe
            for (int item = tid; item < PG * (KC / 4); item += NT) {
                const int pp = item % PG, q = item / PG;
                float4 rr[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    int k = c * KC + 4 * q + j;
                    rr[j] = (pp < np && k < R) ? __ldg(records + (int64_t)(g0 + pp) * R + k)
                                               : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    uint8_t* dst = stage + OFF_B_IRR + canon(3 * pp + ch, 4 * q * es_irr, sbo_irr);
                    if (BF16) {
                        __nv_bfloat162 lo = __floats2bfloat162_rn(comp4(rr[0], ch), comp4(rr[1], ch));
                        __nv_bfloat162 hi = __floats2bfloat162_rn(comp4(rr[2], ch), comp4(rr[3], ch));
                        uint2 w;
                        w.x = *reinterpret_cast<uint32_t*>(&lo);
                        w.y = *reinterpret_cast<uint32_t*>(&hi);
                        *reinterpret_cast<uint2*>(dst) = w;
                    } else {
                        *reinterpret_cast<float4*>(dst) =
                            make_float4(comp4(rr[0], ch), comp4(rr[1], ch), comp4(rr[2], ch), comp4(rr[3], ch));
                    }
                }
                float dh[4], dl[4], qh[4], ql[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float d = rr[j].w, d2 = d * d;
                    dh[j] = tf32_trunc(d);
                    dl[j] = d - dh[j];
                    qh[j] = tf32_trunc(d2);
                    ql[j] = d2 - qh[j];
                }
                *reinterpret_cast<float4*>(stage + OFF_B_DIST + canon(4 * pp + 0, 16 * q, sbo4)) =
                    make_float4(dh[0], dh[1], dh[2], dh[3]);
                *reinterpret_cast<float4*>(stage + OFF_B_DIST + canon(4 * pp + 1, 16 * q, sbo4)) =
                    make_float4(dl[0], dl[1], dl[2], dl[3]);
                *reinterpret_cast<float4*>(stage + OFF_B_DIST + canon(4 * pp + 2, 16 * q, sbo4)) =
                    make_float4(qh[0], qh[1], qh[2], qh[3]);
                *reinterpret_cast<float4*>(stage + OFF_B_DIST + canon(4 * pp + 3, 16 * q, sbo4)) =
                    make_float4(ql[0], ql[1], ql[2], ql[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                bool ok = mbar_wait(&full_bar[s], full_phase[s]);
                full_phase[s] ^= 1u;
                tma_pending[s] = false;
                if (!ok) {
                    abort = true;
                } else {
                    tc_fence_after();
#pragma unroll
                    for (int k = 0; k < ksteps_irr; ++k)
                        mma<BF16>(tmem + COL_IRR, smem_desc(sstage + OFF_A_IRR + k * 256, 128, sbo_irr),
                                  smem_desc(sstage + OFF_B_IRR + k * 256, 128, sbo_irr), idesc_irr,
                                  (c > 0 || k > 0) ? 1u : 0u);
#pragma unroll
                    for (int m = 0; m < 2; ++m)
#pragma unroll
                        for (int k = 0; k < ksteps_dist; ++k)
                            mma<false>(tmem + (m ? COL_DIST1 : COL_DIST0),
                                       smem_desc(sstage + OFF_A_DIST + m * 16384 + k * 256, 128, sbo4),
                                       smem_desc(sstage + OFF_B_DIST + k * 256, 128, sbo4), idesc_dist,
                                       (c > 0 || k > 0) ? 1u : 0u);
                    mma_commit(&empty_bar[s]);
                    committed[s] = true;
                }
            }
            empty_pending[s] = true;
        }
        abort = __syncthreads_or(abort);
        if (abort) break;
        // all MMAs of the group complete before the accumulators are read
        for (int s = 0; s < 2; ++s) {
            if (empty_pending[s]) {
                if (!mbar_wait(&empty_bar[s], empty_phase[s])) abort = true;
                else committed[s] = false;
                empty_phase[s] ^= 1u;
                empty_pending[s] = false;
            }
        }
        abort = __syncthreads_or(abort);
        if (abort) break;
        tc_fence_after();
        // accumulators -> shared memory (stage buffers are free now); warp w
        // reads TMEM lanes 32 (w % 4) .. + 31, the two warps of a lane quarter
        // splitting the columns
        float* Dirr = reinterpret_cast<float*>(smem);
        float* Ddist = reinterpret_cast<float*>(smem + OFF_D_DIST);
        const int quarter = warp & 3, half = warp >> 2;
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        const int row = quarter * 32 + lane;
        if (quarter * 32 < ti) {
            for (int cb = half * (IRR_N / 2); cb < (half + 1) * (IRR_N / 2); cb += 16) {
                float r16[16];
                tmem_ld16(tmem + lane_base + COL_IRR + cb, r16);
                if (row < ti)
#pragma unroll
                    for (int j = 0; j < 16; ++j) Dirr[row * DIRR_STRIDE + cb + j] = r16[j];
            }
        }
        for (int m = 0; m < 2; ++m) {
            if (m * 128 + quarter * 32 >= td) continue;
            const int drow = m * 128 + row;
            for (int cb = half * (DIST_N / 2); cb < (half + 1) * (DIST_N / 2); cb += 16) {
                float r16[16];
                tmem_ld16(tmem + lane_base + (m ? COL_DIST1 : COL_DIST0) + cb, r16);
                if (drow < td)
#pragma unroll
                    for (int j = 0; j < 16; ++j) Ddist[drow * DDIST_STRIDE + cb + j] = r16[j];
            }
        }
        tc_fence_before();
        __syncthreads();
        // epilogue: consecutive threads on consecutive texels of one probe,
        // two texels in flight per thread
#pragma unroll 2
        for (int q = tid; q < ti * np; q += NT) {
            const int pp = q / ti, t = q - pp * ti;
            const float* a = Dirr + t * DIRR_STRIDE + 3 * pp;
            const int e = s_probe[pp];
            blend_irr_texel(vol_of<MULTI>(vs, e >> kEntryShift), bp, e & kEntryMask, t, a[0], a[1], a[2],
                            __ldg(inv_irr + t), s_newly[pp] != 0, status);
        }
#pragma unroll 2
        for (int q = tid; q < td * np; q += NT) {
            const int pp = q / td, t = q - pp * td;
            const float* a = Ddist + t * DDIST_STRIDE + 4 * pp;
            const int e = s_probe[pp];
            blend_dist_texel(vol_of<MULTI>(vs, e >> kEntryShift), bp, e & kEntryMask, t, a[0] + a[1], a[2] + a[3],
                             __ldg(inv_dist + t), s_newly[pp] != 0, status);
        }
        // the next group's bulk copies (async proxy) overwrite what these reads used
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid < np && s_newly[tid]) {
            const int e = s_probe[tid];
            {
                uint8_t* sp = vol_of<MULTI>(vs, e >> kEntryShift).states + (e & kEntryMask);
                *sp = state_advanced(*sp);
            }
        }
        __syncthreads();
    }
    if (abort) {
        // a wait gave up: report, then drain (bounded) what this CTA issued
        if (tid == 0) {
            atomicOr(status, 2u);
            for (int s = 0; s < 2; ++s) {
                if (tma_pending[s]) mbar_wait(&full_bar[s], full_phase[s]);
                if (committed[s]) mbar_wait(&empty_bar[s], empty_phase[s]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

int tc_blend_chunks(int R) { return (R + KC - 1) / KC; }
size_t tc_pack_irr_bytes(int R) { return (size_t)tc_blend_chunks(R) * A_IRR_MAX; }
size_t tc_pack_dist_bytes(int R) { return (size_t)tc_blend_chunks(R) * A_DIST_BYTES; }
bool tc_blend_supported(int irr_n, int dist_n) { return irr_n * irr_n <= 128 && dist_n * dist_n <= 256; }

cudaError_t launch_pack_weights(const float* w_irr, const float* w_dist, int R, int irr_n, int dist_n, int irr_bf16,
                                uint8_t* a_irr, uint8_t* a_dist, float* inv_irr, float* inv_dist, cudaStream_t st) {
    k_pack_weights<<<384, 128, 0, st>>>(w_irr, w_dist, R, irr_n * irr_n, dist_n * dist_n, tc_blend_chunks(R),
                                        irr_bf16, a_irr, a_dist, inv_irr, inv_dist);
    return cudaGetLastError();
}

template <bool BF16, bool MULTI>
static cudaError_t blend_tc(const VolSet& vs, const BlendParams& bp, const uint8_t* a_irr, const uint8_t* a_dist,
                            const float* inv_irr, const float* inv_dist, const float4* records,
                            const int32_t* active, const int32_t* count, uint32_t* status, int grid,
                            cudaStream_t st) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_blend_tc<BF16, MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SMEM_BYTES);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_blend_tc<BF16, MULTI><<<grid, NT, SMEM_BYTES, st>>>(vs, bp, a_irr, a_dist, tc_blend_chunks(bp.R), inv_irr,
                                                          inv_dist, records, active, count, status);
    return cudaGetLastError();
}

cudaError_t launch_blend_tc_set(const VolSet& vs, bool multi, const BlendParams& bp, int bf16,
                                const uint8_t* a_irr, const uint8_t* a_dist, const float* inv_irr,
                                const float* inv_dist, const float4* records, const int32_t* active,
                                const int32_t* count, uint32_t* status, int grid, cudaStream_t st) {
    if (bf16 && multi)
        return blend_tc<true, true>(vs, bp, a_irr, a_dist, inv_irr, inv_dist, records, active, count, status, grid, st);
    if (bf16)
        return blend_tc<true, false>(vs, bp, a_irr, a_dist, inv_irr, inv_dist, records, active, count, status, grid, st);
    if (multi)
        return blend_tc<false, true>(vs, bp, a_irr, a_dist, inv_irr, inv_dist, records, active, count, status, grid, st);
    return blend_tc<false, false>(vs, bp, a_irr, a_dist, inv_irr, inv_dist, records, active, count, status, grid, st);
}

cudaError_t launch_blend_tc(const VolView& v, const BlendParams& bp, int bf16, const uint8_t* a_irr,
                            const uint8_t* a_dist, const float* inv_irr, const float* inv_dist,
                            const float4* records, const int32_t* active, const int32_t* count, uint32_t* status,
                            int grid, cudaStream_t st) {
    return launch_blend_tc_set(single_set(v), false, bp, bf16, a_irr, a_dist, inv_irr, inv_dist, records, active,
                               count, status, grid, st);
}

// Shared-memory opt-in of every tensor-core blend instantiation (outside any stream capture).
cudaError_t prepare_blend_tc_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_blend_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_blend_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_blend_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_blend_tc<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    return e;
}

}  // namespace ddgi
