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
// lets its copies drain, waits (bounded) for the MMAs it already issued --
// one more tcgen05.commit covers all of them -- and only then frees its
// tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "mk.h"
#include "mk_attr.h"

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
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t spins = TC_WAIT_SPINS) {
    for (uint32_t i = 0; i < spins; ++i) {
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
    int mma_blocks = 0;                                          // thread 0: blocks of MMAs issued
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
            ++mma_blocks;
        }
    }
    cp_async_wait<0>();
    if (!timed_out) {
        if (tid == 0) tc_commit(smem_addr(&bars[TC_STAGES]));
        const bool ok = mbar_wait(smem_addr(&bars[TC_STAGES]), 0);
        timed_out = __syncthreads_or(ok ? 0 : 1) != 0;
    } else if (tid == 0 && mma_blocks > 0) {
        // MMAs issued before the abort still read shared memory and write
        // tensor memory: a last commit tracks all of them; wait for it
        tc_commit(smem_addr(&bars[TC_STAGES]));
        mbar_wait(smem_addr(&bars[TC_STAGES]), 0);
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

// --------------------------------------------------------------------------
// Warp-specialised version: 256 pairs per CTA (two M=128 accumulators, all
// 512 TMEM columns) share every W1 tile.  Three roles, decoupled by
// mbarriers (full / empty per ring slot):
//   - warps 0-3 produce the A tiles (a ring of WS_ASTAGES slots): each
//     thread owns two pair rows, prefetches their truth-vector words two
//     blocks ahead with plain loads, and writes the BF16 rows;
//   - lane 0 of warp 5 streams the W1 tiles into a ring of
//     WS_BSTAGES slots ahead of the MMAs, one bulk copy (cp.async.bulk, completion counted in
//     bytes on the slot's "full" mbarrier) per block, from a W1 image
//     pre-arranged in the swizzled tile layout (mlp_w1_tiles_kernel);
//   - lane 0 of warp 4 issues the MMAs of a block once both its slots are
//     full, then commits to both slots' "empty" barriers.
// Warp 4 allocates and frees the tensor memory.
constexpr int WS_MT = 2;                                   // M=128 tiles per CTA
constexpr int WS_PAIRS = WS_MT * TC_M;                      // 256 pairs
constexpr int WS_ASTAGES = 3;
constexpr int WS_BSTAGES = 3;
constexpr int WS_PRODUCERS = 128;
constexpr int WS_THREADS = WS_PRODUCERS + 64;             // + MMA warp + W1 loader warp
constexpr uint32_t WS_A_BYTES = WS_MT * TC_A_BYTES;         // 32 KB per A slot
constexpr uint32_t WS_B_OFF = WS_ASTAGES * WS_A_BYTES;      // B ring after the A ring
constexpr uint32_t WS_RING_BYTES = WS_B_OFF + WS_BSTAGES * TC_B_BYTES;
constexpr uint32_t WS_SMEM_BYTES = 1024 + WS_RING_BYTES + 128;
constexpr uint32_t WS_TMEM_COLS = WS_MT * TC_N;             // 512
static_assert(WS_A_BYTES % 1024 == 0 && WS_B_OFF % 1024 == 0, "tiles stay 1024-byte aligned");
static_assert(WS_SMEM_BYTES <= 232448, "fits the 227 KB opt-in shared memory");

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Bounded wait (at most `spins` tests) that also gives up when another
// role has aborted.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, volatile int *abort,
                                                   uint32_t spins) {
    for (uint32_t i = 0; i < spins; ++i) {
        if (mbar_test(bar, parity)) return true;
        if (*abort) return false;
        __nanosleep(32);
    }
    return false;
}

// W1 (FP32 [features][256] in the parameter buffer) -> BF16 tiles: block kb
// of 64 features is a 32 KB image of the swizzled K-major B tile, row n =
// hidden unit n (128 bytes), 16-byte chunk c at position c ^ (n & 7).
__global__ void mlp_w1_tiles_kernel(const float *w1, int32_t features, uint4 *tiles) {
    const size_t nchunks = (size_t)(features / TC_KB) * TC_N * 8;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nchunks; q += (size_t)gridDim.x * blockDim.x) {
        const int kb = (int)(q / (TC_N * 8)), rem = (int)(q % (TC_N * 8));
        const int n = rem >> 3, c = rem & 7;
        const int f = kb * TC_KB + c * 8;
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __nv_bfloat16 lo = __float2bfloat16(w1[(size_t)(f + 2 * i) * TC_N + n]);
            const __nv_bfloat16 hi = __float2bfloat16(w1[(size_t)(f + 2 * i + 1) * TC_N + n]);
            w[i] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        }
        tiles[(size_t)kb * (TC_B_BYTES / 16) + n * 8 + (c ^ (n & 7))] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

struct TcWsArgs {
    const uint32_t *vec;
    int32_t vwords;
    const int32_t *pa, *pb;
    int32_t batch;
    const uint8_t *w1tiles;    // [features/64][32 KB]
    const float *b1;
    float *h1;
    int32_t *status;
    uint32_t spins;            // limit of the role waits (the drains after an abort use TC_WAIT_SPINS)
};

__global__ void __launch_bounds__(WS_THREADS, 1) mlp_l1_tc_ws_kernel(TcWsArgs a) {
    extern __shared__ uint8_t tc_smem_raw[];
    const uint32_t raw0 = smem_addr(tc_smem_raw);
    const uint32_t pad = (1024u - (raw0 & 1023u)) & 1023u;
    uint8_t *base = tc_smem_raw + pad;
    const uint32_t sbase = raw0 + pad;
    // barriers: fullA[A], emptyA[A], fullB[B], emptyB[B], done
    uint64_t *bars = (uint64_t *)(base + WS_RING_BYTES);
    uint32_t *s_tmem = (uint32_t *)(bars + 2 * WS_ASTAGES + 2 * WS_BSTAGES + 1);
    volatile int *s_abort = (volatile int *)(s_tmem + 1);
    auto fullA = [&](int s) { return smem_addr(&bars[s]); };
    auto emptyA = [&](int s) { return smem_addr(&bars[WS_ASTAGES + s]); };
    auto fullB = [&](int s) { return smem_addr(&bars[2 * WS_ASTAGES + s]); };
    auto emptyB = [&](int s) { return smem_addr(&bars[2 * WS_ASTAGES + WS_BSTAGES + s]); };
    const uint32_t done = smem_addr(&bars[2 * WS_ASTAGES + 2 * WS_BSTAGES]);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int p0 = blockIdx.x * WS_PAIRS;
    const int features = a.vwords * 64, half = a.vwords * 32;
    const int nkb = features / TC_KB;

    if (tid == 0) {
        for (int s = 0; s < WS_ASTAGES; ++s) {
            mbar_init(fullA(s), WS_PRODUCERS);
            mbar_init(emptyA(s), 1);
        }
        for (int s = 0; s < WS_BSTAGES; ++s) {
            mbar_init(fullB(s), 1);
            mbar_init(emptyB(s), 1);
        }
        mbar_init(done, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                     "r"(WS_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;
    bool ok = true;
    int bulk_issued = 0;       // W1 loader: bulk copies issued
    int mma_blocks = 0;        // MMA issuer: blocks of MMAs issued
    bool done_committed = false;
    const uint32_t spins = a.spins;

    if (warp < 4) {
        // ---------------------------------------------------------- producers
        const uint32_t *va[WS_MT], *vb[WS_MT];
#pragma unroll
        for (int m = 0; m < WS_MT; ++m) {
            const int p = p0 + m * TC_M + tid;
            const int ia = p < a.batch ? a.pa[p] : 0, ib = p < a.batch ? a.pb[p] : 0;
            va[m] = a.vec + (size_t)ia * a.vwords;
            vb[m] = a.vec + (size_t)ib * a.vwords;
        }
        auto fetch = [&](int kb, uint2 (&wa)[WS_MT], uint2 (&wb)[WS_MT]) {
            const int f0 = kb * TC_KB;
            const int w0 = (f0 < half ? f0 : f0 - half) >> 5;
#pragma unroll
            for (int m = 0; m < WS_MT; ++m) {
                wa[m] = *reinterpret_cast<const uint2 *>(va[m] + w0);
                wb[m] = *reinterpret_cast<const uint2 *>(vb[m] + w0);
            }
        };
        // words of blocks kb (c*), kb+1 (n*) in registers; kb+2 requested now
        uint2 ca[WS_MT], cb[WS_MT], na[WS_MT], nb[WS_MT];
        fetch(0, ca, cb);
        if (nkb > 1) fetch(1, na, nb);
        for (int kb = 0; kb < nkb && ok; ++kb) {
            const int s = kb % WS_ASTAGES;
            uint2 fa[WS_MT], fb[WS_MT];
            if (kb + 2 < nkb) fetch(kb + 2, fa, fb);
            if (kb >= WS_ASTAGES)
                ok = mbar_wait_or_abort(emptyA(s), (uint32_t)(((kb - WS_ASTAGES) / WS_ASTAGES) & 1), s_abort, spins);
            if (!ok) break;
            const bool xr = kb * TC_KB < half;
#pragma unroll
            for (int m = 0; m < WS_MT; ++m) {
                const uint32_t x0 = xr ? ca[m].x ^ cb[m].x : ca[m].x & cb[m].x;
                const uint32_t x1 = xr ? ca[m].y ^ cb[m].y : ca[m].y & cb[m].y;
                uint8_t *arow = base + (size_t)s * WS_A_BYTES + (size_t)m * TC_A_BYTES + (size_t)tid * 128;
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
            mbar_arrive(fullA(s));
#pragma unroll
            for (int m = 0; m < WS_MT; ++m) {
                ca[m] = na[m];
                cb[m] = nb[m];
                na[m] = fa[m];
                nb[m] = fb[m];
            }
        }
        if (!ok) *s_abort = 1;
        if (ok) ok = mbar_wait_or_abort(done, 0, s_abort, spins);
        if (!ok) *s_abort = 1;
    } else if (tid == WS_PRODUCERS + 32) {
        // ---------------------------- W1 loader (its own warp: its polling
        // never delays the MMA issuer)
        for (int kb = 0; kb < nkb && ok; ++kb) {
            const int s = kb % WS_BSTAGES;
            if (kb >= WS_BSTAGES)
                ok = mbar_wait_or_abort(emptyB(s), (uint32_t)(((kb - WS_BSTAGES) / WS_BSTAGES) & 1), s_abort, spins);
            if (!ok) break;
            mbar_expect_tx(fullB(s), TC_B_BYTES);
            mbar_arrive(fullB(s));
            bulk_g2s(sbase + WS_B_OFF + (uint32_t)s * TC_B_BYTES, a.w1tiles + (size_t)kb * TC_B_BYTES, TC_B_BYTES,
                     fullB(s));
            ++bulk_issued;
        }
        if (!ok) *s_abort = 1;
    } else if (tid == WS_PRODUCERS) {
        // --------------------------------------------------------- MMA issuer
        for (int kb = 0; kb < nkb && ok; ++kb) {
            const int sa = kb % WS_ASTAGES, sb = kb % WS_BSTAGES;
            ok = mbar_wait_or_abort(fullB(sb), (uint32_t)((kb / WS_BSTAGES) & 1), s_abort, spins) &&
                 mbar_wait_or_abort(fullA(sa), (uint32_t)((kb / WS_ASTAGES) & 1), s_abort, spins);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t aa = sbase + (uint32_t)sa * WS_A_BYTES, bb = sbase + WS_B_OFF + (uint32_t)sb * TC_B_BYTES;
#pragma unroll
            for (int m = 0; m < WS_MT; ++m)
#pragma unroll
                for (int k = 0; k < TC_KB / 16; ++k)
                    tc_mma(tmem + (uint32_t)(m * TC_N), sw128_desc(aa + m * TC_A_BYTES + k * 32),
                           sw128_desc(bb + k * 32), (kb > 0 || k > 0) ? 1u : 0u);
            tc_commit(emptyA(sa));
            tc_commit(emptyB(sb));
            ++mma_blocks;
        }
        if (ok) {
            tc_commit(done);
            done_committed = true;
        } else {
            *s_abort = 1;
        }
    }
    __syncthreads();
    const bool aborted = *s_abort != 0;
    if (aborted) {
        // Nothing asynchronous may outlive the CTA's shared and tensor memory.
        if (tid == WS_PRODUCERS + 32) {
            atomicOr(a.status, (int)MK_ST_TIMEOUT);
            // the last copy issued into each ring slot completes that slot's
            // "full" phase (the earlier ones were consumed before the slot was
            // refilled): wait for those phases
            const int first = bulk_issued > WS_BSTAGES ? bulk_issued - WS_BSTAGES : 0;
            for (int kb = first; kb < bulk_issued; ++kb)
                mbar_wait(fullB(kb % WS_BSTAGES), (uint32_t)((kb / WS_BSTAGES) & 1));
        } else if (tid == WS_PRODUCERS && mma_blocks > 0) {
            // one commit after the last MMA tracks every MMA this thread
            // issued; "done" is committed at most once, so its phase 0 ends
            // when they all have completed
            if (!done_committed) tc_commit(done);
            mbar_wait(done, 0);
        }
    } else if (warp < 4) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int lane = tid & 31;
#pragma unroll 1
        for (int m = 0; m < WS_MT; ++m) {
            const int p = p0 + m * TC_M + warp * 32 + lane;      // TMEM lane = pair row of tile m
            const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(m * TC_N);
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
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(WS_TMEM_COLS));
}

}  // namespace mkd


extern "C" size_t mk_mlp_w1_tiles_bytes(int32_t features) {
    return features > 0 && features % 128 == 0 ? (size_t)(features / mkd::TC_KB) * mkd::TC_B_BYTES : 0;
}

extern "C" int mk_mlp_w1_tiles(const float *d_params, int32_t features, int32_t hidden, void *d_tiles, void *stream) {
    using namespace mkd;
    if (hidden != TC_N || features <= 0 || features % 128 || !d_params || !d_tiles || ((uintptr_t)d_tiles & 15))
        return MK_E_ARG;
    mlp_w1_tiles_kernel<<<1024, 256, 0, (cudaStream_t)stream>>>(d_params, features, (uint4 *)d_tiles);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

namespace {

int layer1_tc_ws(const uint32_t *d_vec, int32_t features, const int32_t *d_pa, const int32_t *d_pb, int32_t batch,
                 const void *d_w1_tiles, const float *d_b1, float *d_h1, int32_t *d_status, uint32_t spins,
                 void *stream) {
    using namespace mkd;
    if (features <= 0 || features % 128 || batch < 0 || !d_status) return MK_E_ARG;
    if (batch == 0) return MK_OK;
    if (!d_vec || !d_pa || !d_pb || !d_w1_tiles || !d_b1 || !d_h1) return MK_E_ARG;
    if (((uintptr_t)d_vec & 7) || ((uintptr_t)d_w1_tiles & 15) || ((uintptr_t)d_h1 & 15)) return MK_E_ARG;
    ensure_dynamic_smem((const void *)mlp_l1_tc_ws_kernel, WS_SMEM_BYTES);
    TcWsArgs a;
    a.vec = d_vec;
    a.vwords = features / 64;
    a.pa = d_pa;
    a.pb = d_pb;
    a.batch = batch;
    a.w1tiles = (const uint8_t *)d_w1_tiles;
    a.b1 = d_b1;
    a.h1 = d_h1;
    a.status = d_status;
    a.spins = spins;
    mlp_l1_tc_ws_kernel<<<(batch + WS_PAIRS - 1) / WS_PAIRS, WS_THREADS, WS_SMEM_BYTES, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

}  // namespace

extern "C" int mk_mlp_layer1_tc_ws(const uint32_t *d_vec, int32_t features, const int32_t *d_pa, const int32_t *d_pb,
                                   int32_t batch, const void *d_w1_tiles, const float *d_b1, float *d_h1,
                                   int32_t *d_status, void *stream) {
    return layer1_tc_ws(d_vec, features, d_pa, d_pb, batch, d_w1_tiles, d_b1, d_h1, d_status, mkd::TC_WAIT_SPINS,
                        stream);
}

extern "C" int mk_mlp_layer1_tc_ws_bounded(const uint32_t *d_vec, int32_t features, const int32_t *d_pa,
                                           const int32_t *d_pb, int32_t batch, const void *d_w1_tiles,
                                           const float *d_b1, float *d_h1, int32_t *d_status, uint32_t wait_spins,
                                           void *stream) {
    if (wait_spins == 0) return MK_E_ARG;
    return layer1_tc_ws(d_vec, features, d_pa, d_pb, batch, d_w1_tiles, d_b1, d_h1, d_status, wait_spins, stream);
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
    ensure_dynamic_smem((const void *)mlp_l1_tc_kernel, TC_SMEM_BYTES);
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
