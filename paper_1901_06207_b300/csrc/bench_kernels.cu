// Roof measurement: random-address RED.OR into an L2-sized buffer.
#include "cbaa_bench.h"
#include "cbaa_internal.cuh"

namespace {

__global__ void __launch_bounds__(256) k_red_probe(uint32_t *__restrict__ buf, uint32_t mask, uint64_t n_ops,
                                                   uint32_t seed) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_ops; i += stride) {
        const uint32_t h = cbaa::mix32((uint32_t)i ^ cbaa::mix32((uint32_t)(i >> 32) ^ seed));
        const uint32_t b = cbaa::mix32(h);
        asm volatile("red.global.or.b32 [%0], %1;" ::"l"(buf + (h & mask)), "r"(1u << (b & 31u)) : "memory");
    }
}

}  // namespace

extern "C" int cbaa_bench_red_or(uint32_t *dev_buf, size_t words, size_t n_ops, uint32_t seed, void *stream) {
    if (!dev_buf || words == 0 || (words & (words - 1)) || words > (1ull << 32) ||
        (reinterpret_cast<uintptr_t>(dev_buf) & 15u))
        return CBAA_ERR_INVALID_ARG;
    if (n_ops == 0) return CBAA_OK;
    const unsigned blocks = (unsigned)cbaa::num_sms() * 8;
    k_red_probe<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(dev_buf, (uint32_t)(words - 1), n_ops,
                                                                           seed);
    return cbaa::cuda_status(cudaGetLastError());
}
