// mk_calib.cu -- integer logic-op issue-rate calibration (Sec. 8's uint32
// XOR/AND/OR ceiling, measured here as three-input LOP3 throughput).
//
// Each thread runs MK_CALIB_CHAINS independent dependency chains of
// lop3.b32 (inline PTX, so the compiler can neither merge nor drop them);
// the chains are long enough to hide the instruction latency, so the kernel
// measures the logic-op issue ceiling of the SMs.  One launch performs
// blocks * threads * iters * MK_CALIB_OPS_PER_ITER logic ops.
#include <cuda_runtime.h>

#include <cstdint>

#include "mk.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) lop3_ceiling_kernel(uint32_t *sink, uint32_t iters, uint32_t seed) {
    uint32_t a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed * (2u * c + 1u) ^ (threadIdx.x + 977u * c);
    uint32_t b = seed ^ 0x9E3779B9u ^ blockIdx.x, d = ~seed ^ threadIdx.x;
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                asm("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[c]) : "r"(b), "r"(d));
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) x ^= a[c];
    if (x == 0x12345678u) sink[blockIdx.x] = x;   // keeps the chains live
}

}  // namespace

extern "C" uint64_t mk_calibrate_ops_per_launch(int32_t blocks, int32_t threads, uint32_t iters) {
    return (uint64_t)blocks * (uint64_t)threads * (uint64_t)iters * (uint64_t)(kChains * kUnroll);
}

extern "C" int mk_calibrate_lop3(uint32_t *d_sink, int32_t blocks, int32_t threads, uint32_t iters,
                                 uint32_t seed, void *stream) {
    if (!d_sink || blocks < 1 || threads < 32 || threads > 256 || (threads & 31)) return MK_E_ARG;
    lop3_ceiling_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(d_sink, iters, seed);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}
