// Measurement kernel for the traversal's cache roofline: the rate at which
// the SMs read a buffer that sits in L2.  Loads bypass L1 (ld.global.cg), so
// every 16-byte load is an L2 request; a caller sizes the buffer below the
// L2 capacity, reads it once to make it resident, then times the call.
#include <string>

#include "ddgi_internal.h"

namespace ddgi {
namespace {

constexpr int kL2Threads = 512;
constexpr int kL2BlocksPerSm = 4;   // 2048 resident threads per SM
constexpr uint32_t kSinkValue = 0x2545F491u;

// Every pass reads all n16 16-byte words once, four independent loads in
// flight per thread; the XOR of the words keeps the loads live and is
// written out only when it equals kSinkValue.
__global__ void __launch_bounds__(kL2Threads) k_l2_read(const uint4* __restrict__ buf, uint64_t n16, int passes,
                                                        uint32_t* sink) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint32_t acc = 0;
    for (int p = 0; p < passes; ++p) {
        uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n16; i += 4 * stride) {
            const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
            const uint4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
            acc ^= (a.x ^ a.y ^ a.z ^ a.w) ^ (b.x ^ b.y ^ b.z ^ b.w) ^ (c.x ^ c.y ^ c.z ^ c.w) ^
                   (d.x ^ d.y ^ d.z ^ d.w);
        }
        for (; i < n16; i += stride) {
            const uint4 a = __ldcg(buf + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    if (acc == kSinkValue) atomicAdd(sink, 1u);
}

}  // namespace
}  // namespace ddgi

using namespace ddgi;

extern "C" ddgi_status ddgi_measure_l2_read(const void* buf_dev, size_t bytes, int32_t passes, uint32_t* sink_dev,
                                            ddgi_stream stream) {
    if (!buf_dev || !sink_dev) return set_error(DDGI_ERR_INVALID_ARG, "NULL argument");
    if (((uintptr_t)buf_dev & 15u) || ((uintptr_t)sink_dev & 3u))
        return set_error(DDGI_ERR_INVALID_ARG, "buffer must be 16-byte aligned, sink 4-byte aligned");
    if (bytes == 0 || (bytes & 15u)) return set_error(DDGI_ERR_INVALID_ARG, "bytes must be a positive multiple of 16");
    if (passes < 1) return set_error(DDGI_ERR_INVALID_ARG, "passes must be at least 1");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_error(DDGI_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
    k_l2_read<<<sms * kL2BlocksPerSm, kL2Threads, 0, (cudaStream_t)stream>>>(
        static_cast<const uint4*>(buf_dev), (uint64_t)(bytes / 16), passes, sink_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(DDGI_ERR_CUDA, std::string("k_l2_read: ") + cudaGetErrorString(e));
    return DDGI_OK;
}
