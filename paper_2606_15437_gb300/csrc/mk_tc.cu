// mk_tc.cu -- the pair-ranking MLP's first layer on the 5th-generation
// tensor cores (tcgen05): h1 = relu(x W1 + b1) for pairs of truth vectors,
// x = [a xor b, a and b] (0/1 features, exact in BF16), W1 in BF16, FP32
// accumulation in tensor memory.
//
// One CTA (4 warps) computes 128 pairs x 256 hidden units: the accumulator
// is 256 TMEM columns (FP32, lane = pair).  The feature dimension is walked
// in blocks of 64 (one 128-byte BF16 row per pair and per hidden unit);
// each block is one pipeline stage in shared memory, in the 128-byte
// swizzled K-major layout the MMA descriptors name:
//   A (128 x 64): built on chip -- every thread copies its pair's two words
//     of each truth vector (cp.async), combines them (xor / and) and writes
//     the 64 features as BF16 0/1, 16 bytes at a time, swizzled;
//   B (256 x 64): the W1^T rows, copied 16 bytes at a time (cp.async) into
//     the same swizzled layout.
// Four stages; loads run two blocks ahead.  Thread 0 issues the four
// K=16 MMAs of a block (tcgen05.mma.cta_group::1.kind::f16, M=128, N=256)
// and commits them to the stage's mbarrier; a stage is refilled only after
// that barrier completes.  The epilogue reads the accumulator with
// tcgen05.ld (32 lanes x 32 columns per warp and step), adds the bias,
// applies the ReLU and stores h1.
//
// Every wait on an mbarrier is bounded: a thread that gives up sets
// MK_ST_TIMEOUT, the CTA agrees on it (__syncthreads_or), skips the rest,
// lets its copies drain and frees its tensor memory before returning.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "mk.h"

namespace mkd {

constexpr int TC_M = 128;                 // pairs per CTA (TMEM lanes)
constexpr int TC_N = 256;                 // hidden units (TMEM columns, FP32)
constexpr int TC_KB = 64;                 // features per stage (128 bytes of BF16)
constexpr int TC_STAGES = 4;
constexpr int TC_AHEAD = 2;               // blocks loaded ahead of the one computed
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_A_BYTES = TC_M * TC_KB * 2;   // 16 KB
constexpr uint32_t TC_B_BYTES = TC_N * TC_KB * 2;   // 32 KB
constexpr uint32_t TC_RAW_BYTES = TC_M * 16;        // 2 words of each vector per pair
constexpr uint32_t TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES + TC_RAW_BYTES;
// layout: [1024-byte alignment slack][stages][mbarriers + TMEM address]
constexpr uint32_t TC_SMEM_BYTES = 1024 + TC_STAGES * TC_STAGE_BYTES + 128;
constexpr uint32_t TC_WAIT_SPINS = 1u << 24;         // x ~100 ns: about 2 s

static_assert(TC_A_BYTES % 1024 == 0 && TC_B_BYTES % 1024 == 0 && TC_STAGE_BYTES % 1024 == 0,
              "swizzle atoms of every tile start on 1024-byte boundaries");

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the completion of the given phase; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < TC_WAIT_SPINS; ++i) {
        if (mbar_test(bar, parity)) return true;
        __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128
// bytes, 8-row swizzle atoms 1024 bytes apart (stride byte offset), the
// leading byte offset unused for this layout (encoded as 1), descriptor
// version 1 (bits 46-48), swizzle mode 2 = 128 bytes (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 0/1 bits -> BF16 (1.0 = 0x3F80) pairs packed in a word: bits 2i, 2i+1 of x.
__device__ __forceinline__ uint32_t bf16_pair(uint32_t x, int i) {
    return ((x >> (2 * i)) & 1u ? 0x3F80u : 0u) | ((x >> (2 * i + 1)) & 1u ? 0x3F800000u : 0u);
}

struct TcArgs {
    const uint32_t *vec;       // truth vectors, vwords words each
    int32_t vwords;            // features = 64 * vwords
    const int32_t *pa, *pb;
    int32_t batch;
    const __nv_bfloat16 *w1t;  // [TC_N][features]
    const float *b1;
    float *h1;                 // [batch][TC_N]
    int32_t *status;
};

__global__ void __launch_bounds__(TC_THREADS, 1) mlp_l1_tc_kernel(TcArgs a) {
    extern __shared__ uint8_t tc_smem_raw[];
    // 1024-byte aligned base for the swizzled tiles
    const uint32_t raw0 = smem_addr(tc_smem_raw);
    const uint32_t pad = (1024u - (raw0 & 1023u)) & 1023u;
    uint8_t *base = tc_smem_raw + pad;
    const uint32_t sbase = raw0 + pad;
    uint64_t *bars = (uint64_t *)(base + TC_STAGES * TC_STAGE_BYTES);   // [TC_STAGES] + done
    uint32_t *s_tmem = (uint32_t *)(bars + TC_STAGES + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p0 = blockIdx.x * TC_M;
    const int features = a.vwords * 64, half = a.vwords * 32;
    const int nkb = features / TC_KB;

    if (tid == 0) {
        for (int s = 0; s <= TC_STAGES; ++s) mbar_init(smem_addr(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                     "r"(TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;

    // this thread's pair (rows past the batch read pair 0 and are never stored)
    const int my_p = p0 + tid;
    const int ia = my_p < a.batch ? a.pa[my_p] : 0, ib = my_p < a.batch ? a.pb[my_p] : 0;
    const uint32_t *va = a.vec + (size_t)ia * a.vwords, *vb = a.vec + (size_t)ib * a.vwords;

    auto stage_a = [&](int s) { return sbase + (uint32_t)s * TC_STAGE_BYTES; };
    auto stage_b = [&](int s) { return sbase + (uint32_t)s * TC_STAGE_BYTES + TC_A_BYTES; };
    auto stage_raw = [&](int s) { return base + (size_t)s * TC_STAGE_BYTES + TC_A_BYTES + TC_B_BYTES; };

    // loads of feature block kb into stage kb % TC_STAGES (one commit group)
    auto load_block = [&](int kb) {
        const int s = kb % TC_STAGES;
        const int f0 = kb * TC_KB;
        const int w0 = (f0 < half ? f0 : f0 - half) >> 5;       // even: 8-byte aligned
        const uint32_t raw = smem_addr(stage_raw(s) + (size_t)tid * 16);
        cp_async8(raw, va + w0);
        cp_async8(raw + 8, vb + w0);
        const uint32_t bs = stage_b(s);
#pragma unroll
        for (int i = 0; i < (TC_N * 8) / TC_THREADS; ++i) {
            const int q = tid + i * TC_THREADS;                  // 16-byte chunk of the tile
            const int n = q >> 3, c = q & 7;
            cp_async16(bs + (uint32_t)n * 128 + (uint32_t)((c ^ (n & 7)) << 4),
                       a.w1t + (size_t)n * features + f0 + c * 8);
        }
    };

    // one commit group per block (empty past the end), so that after the
    // commit of iteration kb the group of block kb is the (AHEAD+1)-th newest
    for (int kb = 0; kb < TC_AHEAD; ++kb) {
        if (kb < nkb) load_block(kb);
        cp_async_commit();
    }

    bool timed_out = false;
    for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % TC_STAGES;
        // the stage refilled now was last read by the MMAs of block kb+AHEAD-STAGES
        const int refill = kb + TC_AHEAD;
        if (refill < nkb) {
            const int prev = refill - TC_STAGES;
            if (prev >= 0 && !timed_out)
                timed_out = !mbar_wait(smem_addr(&bars[refill % TC_STAGES]), (uint32_t)((prev / TC_STAGES) & 1));
            if (!timed_out) load_block(refill);
        }
        cp_async_commit();
        cp_async_wait<TC_AHEAD>();                               // block kb's copies are complete
        // this thread's row of the A tile: 64 features as BF16, swizzled
        {
            const uint32_t *raw = (const uint32_t *)(stage_raw(s) + (size_t)tid * 16);
            const int f0 = kb * TC_KB;
            const uint32_t x0 = f0 < half ? raw[0] ^ raw[2] : raw[0] & raw[2];
            const uint32_t x1 = f0 < half ? raw[1] ^ raw[3] : raw[1] & raw[3];
            uint8_t *arow = base + (size_t)s * TC_STAGE_BYTES + (size_t)tid * 128;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const uint32_t x = (c < 4 ? x0 : x1) >> ((c & 3) * 8);
                uint4 v;
                v.x = bf16_pair(x, 0);
                v.y = bf16_pair(x, 1);
                v.z = bf16_pair(x, 2);
                v.w = bf16_pair(x, 3);
                *reinterpret_cast<uint4 *>(arow + ((c ^ (tid & 7)) << 4)) = v;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (__syncthreads_or(timed_out ? 1 : 0)) {
            timed_out = true;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ad = stage_a(s), bd = stage_b(s);
#pragma unroll
            for (int k = 0; k < TC_KB / 16; ++k)                // K = 16 per MMA: 32 bytes along the row
                tc_mma(tmem, sw128_desc(ad + k * 32), sw128_desc(bd + k * 32), (kb > 0 || k > 0) ? 1u : 0u);
            tc_commit(smem_addr(&bars[s]));
        }
    }
    cp_async_wait<0>();
    if (!timed_out) {
        if (tid == 0) tc_commit(smem_addr(&bars[TC_STAGES]));
        const bool ok = mbar_wait(smem_addr(&bars[TC_STAGES]), 0);
        timed_out = __syncthreads_or(ok ? 0 : 1) != 0;
    }
    if (timed_out) {
        if (tid == 0) atomicOr(a.status, (int)MK_ST_TIMEOUT);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int p = p0 + warp * 32 + lane;                      // TMEM lane = pair row
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < TC_N; c0 += 32) {
            uint32_t r[32];
            tc_ld32(trow + (uint32_t)c0, r);
            if (p < a.batch) {
                float *out = a.h1 + (size_t)p * TC_N + c0;
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    float4 v;
                    v.x = fmaxf(__uint_as_float(r[j]) + a.b1[c0 + j], 0.f);
                    v.y = fmaxf(__uint_as_float(r[j + 1]) + a.b1[c0 + j + 1], 0.f);
                    v.z = fmaxf(__uint_as_float(r[j + 2]) + a.b1[c0 + j + 2], 0.f);
                    v.w = fmaxf(__uint_as_float(r[j + 3]) + a.b1[c0 + j + 3], 0.f);
                    *reinterpret_cast<float4 *>(out + j) = v;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N));
}

}  // namespace mkd

namespace {
std::once_flag g_tc_attr;
}

extern "C" int mk_mlp_layer1_tc(const uint32_t *d_vec, int32_t features, const int32_t *d_pa, const int32_t *d_pb,
                                int32_t batch, const void *d_w1t, const float *d_b1, float *d_h1, int32_t *d_status,
                                void *stream) {
    using namespace mkd;
    // features % 128: vector rows of an even number of words (8-byte copies) and
    // feature blocks that never straddle the xor / and halves
    if (features <= 0 || features % 128 || batch < 0 || !d_status) return MK_E_ARG;
    if (batch == 0) return MK_OK;
    if (!d_vec || !d_pa || !d_pb || !d_w1t || !d_b1 || !d_h1) return MK_E_ARG;
    // 8- and 16-byte copies: truth-vector rows and W1^T rows must stay aligned
    if (((uintptr_t)d_vec & 7) || ((uintptr_t)d_w1t & 15) || ((uintptr_t)d_h1 & 15)) return MK_E_ARG;
    std::call_once(g_tc_attr, [] {
        cudaFuncSetAttribute(mlp_l1_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_BYTES);
    });
    TcArgs a;
    a.vec = d_vec;
    a.vwords = features / 64;
    a.pa = d_pa;
    a.pb = d_pb;
    a.batch = batch;
    a.w1t = (const __nv_bfloat16 *)d_w1t;
    a.b1 = d_b1;
    a.h1 = d_h1;
    a.status = d_status;
    mlp_l1_tc_kernel<<<(batch + TC_M - 1) / TC_M, TC_THREADS, TC_SMEM_BYTES, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}
