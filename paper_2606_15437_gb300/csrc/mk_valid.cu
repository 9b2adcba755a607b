// mk_valid.cu -- frame correspondents (Sec. 10, Prop. "soundness over the
// searched universe", Table 9): which frames validate a formula, which
// frames satisfy a first-order condition, and how far the two sets differ.
//
// validity_kernel: the census's bit-sliced K frame words (32 frames per
// register word, n*n edge words from the thread's index) and its
// accumulator interpreter, but the output is per frame: a lane stays set
// while no valuation refutes it, and each (formula, frame word) writes
// one word of the formula's validity bitmap.  A CTA stops walking a
// formula's valuations as soon as every frame in it has been refuted
// (__syncthreads_and at each row-chunk boundary).
//
// condition_kernel: every library condition on the same frame words, each
// a first-order definition with its quantifiers unrolled into three-input
// logic ops over the edge words (transitivity: AND over w,v,u of
// ~E[wv] | ~E[vu] | E[wu], and so on).
//
// mismatch_kernel: for formula i and library entry j (one condition, or
// the conjunction of two), the number of frames on which the validity
// bitmap and the condition differ: popcount of a ^ (b1 & b2) over all
// words.  Recovery (an exact correspondent over the frames searched) is
// mismatch == 0.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "mk.h"
#include "mk_attr.h"
#include "mk_eval.cuh"

namespace mkd {

constexpr int VA_ROW_CAP = 128;
constexpr int VA_OPS_STRIDE = MK_MAX_CODE + 2;
constexpr int VA_BLOCK = 256;
constexpr int VA_U = 8;
constexpr int VA_MAX_TILE = 32;

struct ValidArgs {
    const mk_program *progs;
    int32_t nprog, tile, depth;
    uint64_t nwords;           // frame words of the layer (2^(n*n) / 32, rounded up)
    uint64_t nframes;
    uint32_t *bits;            // bits[p * ld + word]
    uint64_t ld;
    int32_t *status;
};

template <int N, int U, int BLOCK>
struct ValidSmem {
    static constexpr size_t code_bytes(int tile) { return ((size_t)tile * VA_OPS_STRIDE * 3 + 15) & ~(size_t)15; }
    static constexpr size_t meta_bytes(int tile) { return ((size_t)tile * 8 + 15) & ~(size_t)15; }
    static constexpr size_t row_bytes() { return (size_t)(VA_ROW_CAP + U) * RowShape<N>::WORDS * 4; }
    static constexpr size_t stack_bytes(int depth) { return (size_t)depth * U * N * BLOCK * 4; }
    static size_t total(int tile, int depth) {
        return code_bytes(tile) + meta_bytes(tile) + row_bytes() + stack_bytes(depth);
    }
};

template <int N, int U, int BLOCK>
__global__ void __launch_bounds__(BLOCK) validity_kernel(ValidArgs a) {
    using SM = ValidSmem<N, U, BLOCK>;
    constexpr int RW = RowShape<N>::WORDS;
    extern __shared__ __align__(16) uint8_t smem[];
    const int tile = a.tile;
    uint16_t *s_offs = (uint16_t *)smem;
    uint8_t *s_ops = smem + (size_t)tile * VA_OPS_STRIDE * 2;
    int *s_nin = (int *)(smem + SM::code_bytes(tile));
    int *s_k = s_nin + tile;
    uint32_t *s_rows = (uint32_t *)(smem + SM::code_bytes(tile) + SM::meta_bytes(tile));
    uint32_t *s_stack = (uint32_t *)((uint8_t *)s_rows + SM::row_bytes()) + threadIdx.x;

    const int p0 = blockIdx.y * tile;
    const int np = min(tile, a.nprog - p0);
    const bool report = blockIdx.x == 0;
    for (int i = threadIdx.x; i < np; i += BLOCK) {
        const mk_program &p = a.progs[p0 + i];
        int nin = -1;
        if (program_ok(p) && p.depth <= a.depth) {
            nin = p.n_instr;
            if (p.nvars * N > 24) {
                nin = -1;
                if (report) atomicOr(a.status, (int)MK_ST_LIMIT);
            }
        } else if (report) {
            atomicOr(a.status, (int)MK_ST_PROGRAM);
        }
        s_nin[i] = nin;
        s_k[i] = p.nvars;
        if (nin >= 0) decode_program<N, U, BLOCK>(p, s_ops + i * VA_OPS_STRIDE, s_offs + i * VA_OPS_STRIDE);
    }
    __syncthreads();

    const uint64_t word = (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
    uint32_t E[1][N * N];
    uint32_t valid = 0;
    if (word < a.nwords) {
        k_frame_word<N>(word, E[0]);
        const uint64_t base = word << 5;
        const uint64_t left = a.nframes - base;
        valid = left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
    } else {
#pragma unroll
        for (int e = 0; e < N * N; ++e) E[0][e] = 0;
    }
    int rows_c0 = -1;
    for (int fi = 0; fi < np; ++fi) {
        const int nin = s_nin[fi];
        if (nin < 0) continue;
        const uint32_t nval = 1u << (s_k[fi] * N);
        const uint8_t *ops = s_ops + fi * VA_OPS_STRIDE;
        const uint16_t *offs = s_offs + fi * VA_OPS_STRIDE;
        uint32_t rf = 0;                                    // lanes refuted so far
        for (uint32_t c0 = 0; c0 < nval; c0 += VA_ROW_CAP) {
            // uniform: every thread takes the same staging decisions; the
            // CTA leaves the formula once all its frames are refuted
            if (__syncthreads_and(rf == valid)) break;
            if (rows_c0 != (int)c0) {
                constexpr int W = RowShape<N>::WORDS;
                for (uint32_t i = threadIdx.x; i < VA_ROW_CAP * W; i += BLOCK)
                    s_rows[i] = atom_row_word<N>(c0 + i / W, (int)(i % W));
                __syncthreads();
                rows_c0 = (int)c0;
            }
            const uint32_t cn = min((uint32_t)VA_ROW_CAP, nval - c0);
            if (rf != valid) {
                for (uint32_t jj = 0; jj < cn; jj += U) {
                    uint32_t A[U][N];
                    run_program<N, U, 1, BLOCK, RW>(ops, offs, s_rows + jj * RW, E, s_stack, A);
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        uint32_t all = A[u][0];
#pragma unroll
                        for (int w = 1; w < N; ++w) all &= A[u][w];
                        if (jj + u < cn) rf |= ~all & valid;
                    }
                }
            }
        }
        if (word < a.nwords) a.bits[(size_t)(p0 + fi) * a.ld + word] = valid & ~rf;
    }
}

// Library conditions on a frame word (bit l <-> frame 32*word + l).
template <int N>
__device__ __forceinline__ uint32_t condition_word(int c, const uint32_t (&E)[N * N]) {
#define EE(w, v) E[(w) * N + (v)]
    uint32_t m = 0xFFFFFFFFu;
    switch (c) {
    case 0: break;
    case 1: m = 0; break;
    case 2:
        for (int w = 0; w < N; ++w) m &= EE(w, w);
        break;
    case 3:
        for (int w = 0; w < N; ++w) m &= ~EE(w, w);
        break;
    case 4:
        for (int w = 0; w < N; ++w) {
            uint32_t any = 0;
            for (int v = 0; v < N; ++v) any |= EE(w, v);
            m &= any;
        }
        break;
    case 5:
        for (int w = 0; w < N; ++w)
            for (int v = 0; v < N; ++v)
                for (int u = 0; u < N; ++u) m &= ~EE(w, v) | ~EE(v, u) | EE(w, u);
        break;
    case 6:
        for (int w = 0; w < N; ++w)
            for (int v = w + 1; v < N; ++v) m &= ~(EE(w, v) ^ EE(v, w));
        break;
    case 7:
        for (int w = 0; w < N; ++w)
            for (int v = 0; v < N; ++v)
                for (int u = 0; u < N; ++u) m &= ~EE(w, v) | ~EE(w, u) | EE(v, u);
        break;
    case 8: case 9:
        for (int w = 0; w < N; ++w)
            for (int v = 0; v < N; ++v)
                for (int u = v + 1; u < N; ++u) m &= ~(EE(w, v) & EE(w, u));
        if (c == 9)
            for (int w = 0; w < N; ++w) {
                uint32_t any = 0;
                for (int v = 0; v < N; ++v) any |= EE(w, v);
                m &= any;
            }
        break;
    case 10:
        for (int w = 0; w < N; ++w)
            for (int v = 0; v < N; ++v) {
                uint32_t via = 0;
                for (int u = 0; u < N; ++u) via |= EE(w, u) & EE(u, v);
                m &= ~EE(w, v) | via;
            }
        break;
    case 11:
        for (int w = 0; w < N; ++w)
            for (int v = 0; v < N; ++v)
                for (int u = v; u < N; ++u) {
                    uint32_t meet = 0;
                    for (int x = 0; x < N; ++x) meet |= EE(v, x) & EE(u, x);
                    m &= ~(EE(w, v) & EE(w, u)) | meet;
                }
        break;
    case 12:
        for (int w = 0; w < N; ++w)
            for (int v = w + 1; v < N; ++v) m &= ~(EE(w, v) & EE(v, w));
        break;
    case 13:
        for (int w = 0; w < N; ++w)
            for (int v = w; v < N; ++v) m &= ~(EE(w, v) & EE(v, w));
        break;
    case 14:
        for (int w = 0; w < N; ++w)
            for (int v = 0; v < N; ++v)
                for (int u = v + 1; u < N; ++u) m &= ~(EE(w, v) & EE(w, u)) | EE(v, u) | EE(u, v);
        break;
    case 15:
        for (int w = 0; w < N; ++w)
            for (int v = 0; v < N; ++v) m &= ~EE(w, v) | EE(v, v);
        break;
    case 16:
        for (int e = 0; e < N * N; ++e) m &= ~E[e];
        break;
    case 17:
        for (int w = 0; w < N; ++w)
            for (int v = 0; v < N; ++v)
                if (v != w) m &= ~EE(w, v);
        break;
    default: m = 0;
    }
#undef EE
    return m;
}

template <int N>
__global__ void condition_kernel(uint64_t nwords, uint64_t nframes, uint32_t *bits, uint64_t ld) {
    const uint64_t word = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (word >= nwords) return;
    uint32_t E[N * N];
    k_frame_word<N>(word, E);
    const uint64_t left = nframes - (word << 5);
    const uint32_t valid = left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
    for (int c = 0; c < MK_NUM_CONDITIONS; ++c) bits[(size_t)c * ld + word] = condition_word<N>(c, E) & valid;
}

// One CTA per formula row: the row is read once, every library entry is
// compared with it by one warp at a time.
__global__ void mismatch_kernel(const uint32_t *a, uint64_t lda, const uint32_t *b, int32_t nb, uint64_t ldb,
                                const int32_t *conj, int32_t nconj, uint64_t words, uint32_t *out) {
    const uint32_t *row = a + (size_t)blockIdx.x * lda;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = warp; j < nconj; j += nw) {
        const int c1 = conj[2 * j], c2 = conj[2 * j + 1];
        if (c1 < 0 || c1 >= nb || c2 < 0 || c2 >= nb) {        // not a library row
            if (lane == 0) out[(size_t)blockIdx.x * nconj + j] = 0xFFFFFFFFu;
            continue;
        }
        const uint32_t *b1 = b + (size_t)c1 * ldb, *b2 = b + (size_t)c2 * ldb;
        uint32_t d = 0;
        for (uint64_t w = lane; w < words; w += 32) d += __popc(row[w] ^ (b1[w] & b2[w]));
        d = __reduce_add_sync(0xFFFFFFFFu, d);
        if (lane == 0) out[(size_t)blockIdx.x * nconj + j] = d;
    }
}

}  // namespace mkd

namespace {

using namespace mkd;

template <typename K>
void va_smem(K kern, size_t bytes) {
    ensure_dynamic_smem((const void *)kern, bytes);
}

template <int N>
void launch_valid(ValidArgs a, cudaStream_t s) {
    using SM = ValidSmem<N, VA_U, VA_BLOCK>;
    auto kern = validity_kernel<N, VA_U, VA_BLOCK>;
    const size_t sm = SM::total(a.tile, a.depth);
    va_smem(kern, sm);
    dim3 grid((unsigned)((a.nwords + VA_BLOCK - 1) / VA_BLOCK), (unsigned)((a.nprog + a.tile - 1) / a.tile));
    kern<<<grid, VA_BLOCK, sm, s>>>(a);
}

}  // namespace

extern "C" uint64_t mk_frame_words(int32_t n) {
    if (n < 1 || n > MK_MAX_WORLDS_VALIDITY) return 0;
    return ((1ull << (n * n)) + 31) / 32;
}

extern "C" int mk_frame_validity(const mk_program *d_progs, int32_t nprog, int32_t n, int32_t max_depth,
                                 uint32_t *d_bits, uint64_t ld_words, int32_t *d_status, void *stream) {
    if (n < 1 || n > MK_MAX_WORLDS_VALIDITY || nprog < 0 || !d_status) return MK_E_ARG;
    if (max_depth < 0 || max_depth > MK_MAX_STACK) return MK_E_ARG;
    const uint64_t nw = mk_frame_words(n);
    if (ld_words < nw) return MK_E_ARG;
    if (nprog == 0) return MK_OK;
    if (!d_progs || !d_bits) return MK_E_ARG;
    ValidArgs a;
    std::memset(&a, 0, sizeof(a));
    a.progs = d_progs;
    a.nprog = nprog;
    a.depth = max_depth ? max_depth : MK_MAX_STACK;
    a.nwords = nw;
    a.nframes = 1ull << (n * n);
    a.bits = d_bits;
    a.ld = ld_words;
    a.status = d_status;
    // few frame words (n <= 3): one formula per CTA spreads the work
    a.tile = nw >= 4096 ? VA_MAX_TILE : 1;
    if ((nprog + a.tile - 1) / a.tile > 65535) return MK_E_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    switch (n) {
    case 1: launch_valid<1>(a, s); break;
    case 2: launch_valid<2>(a, s); break;
    case 3: launch_valid<3>(a, s); break;
    case 4: launch_valid<4>(a, s); break;
    case 5: launch_valid<5>(a, s); break;
    }
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

extern "C" int mk_frame_conditions(int32_t n, uint32_t *d_bits, uint64_t ld_words, void *stream) {
    if (n < 1 || n > MK_MAX_WORLDS_VALIDITY || !d_bits) return MK_E_ARG;
    const uint64_t nw = mk_frame_words(n);
    if (ld_words < nw) return MK_E_ARG;
    const unsigned grid = (unsigned)((nw + 255) / 256);
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t nf = 1ull << (n * n);
    switch (n) {
    case 1: condition_kernel<1><<<grid, 256, 0, s>>>(nw, nf, d_bits, ld_words); break;
    case 2: condition_kernel<2><<<grid, 256, 0, s>>>(nw, nf, d_bits, ld_words); break;
    case 3: condition_kernel<3><<<grid, 256, 0, s>>>(nw, nf, d_bits, ld_words); break;
    case 4: condition_kernel<4><<<grid, 256, 0, s>>>(nw, nf, d_bits, ld_words); break;
    case 5: condition_kernel<5><<<grid, 256, 0, s>>>(nw, nf, d_bits, ld_words); break;
    }
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

extern "C" int mk_bitmap_mismatch(const uint32_t *d_a, int32_t na, uint64_t lda, const uint32_t *d_b, int32_t nb,
                                  uint64_t ldb, const int32_t *d_conj, int32_t nconj, uint64_t words,
                                  uint32_t *d_out, void *stream) {
    if (na < 0 || nb < 0 || nconj < 0 || lda < words || ldb < words) return MK_E_ARG;
    if (na == 0 || nconj == 0) return MK_OK;
    if (!d_a || !d_b || !d_conj || !d_out) return MK_E_ARG;
    if (na > 0x7FFFFFFF) return MK_E_ARG;
    mismatch_kernel<<<(unsigned)na, 256, 0, (cudaStream_t)stream>>>(d_a, lda, d_b, nb, ldb, d_conj, nconj, words,
                                                                  d_out);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}
