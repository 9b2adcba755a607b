// mk_separate.cu -- distinguishing-pair search (Def. 2, Prop. 4).
//
// A pair (phi, psi) is separated on a pointed model iff their truth sets
// differ there, i.e. iff the biconditional phi <-> psi is refuted (Prop. 4).
// The kernel runs both programs on the same bit-sliced frame words (U words
// per thread, one valuation at a time), takes d[w] = t_phi[w] ^ t_psi[w]
// per world and keeps the least (frame, valuation, world) with a set bit,
// as one packed u64 key per pair that also carries n in its top bits; a
// global atomicMin merges CTAs.
//
// Sizes are launched in increasing n; the K frames of the largest sizes are
// launched in ascending chunks.  Before every launch a one-CTA kernel lists
// the pairs still without a split below the launch's first frame (ascending
// pair order, in the caller's workspace), and the launch's tiles are cut
// from that list only, so no CTA stages a finished pair; CTAs whose tile
// lies past the list's end exit at once.  A CTA stages its tile once and
// walks a strip of several frame-word groups, dropping a pair for the rest
// of the strip once the CTA has found its split, and at staging it also
// drops pairs whose key is already below the least key it could produce
// (another CTA of the same chunk got there first): work on a pair stops soon
// after its first split, without any wait.  Sampled sizes (7, 8) generate
// their relations on the device from the counter-based SplitMix64 stream,
// 32 samples per frame word.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "mk.h"
#include "mk_attr.h"
#include "mk_eval.cuh"

namespace mkd {

constexpr int SEP_ROW_CAP = 128;
constexpr int SEP_OPS_STRIDE = MK_MAX_CODE + 2;

struct SepArgs {
    const mk_program *phi;
    const mk_program *psi;
    int32_t npairs;
    int32_t tile;
    const uint32_t *samples;   // this size's sampled valuations (device)
    uint32_t S;
    int32_t sampled;           // 1: frames are sampled relations
    uint64_t rel_state;        // SplitMix64 state of the relation stream
    uint64_t word_lo, word_hi; // frame words of this launch
    uint64_t nframes;          // frames (K) or samples of this size
    uint64_t f_lo, f_hi;       // K-index filter (exhaustive sizes)
    int32_t full_range;
    int32_t groups;            // frame-word groups (BLOCK * U words each) per CTA
    int32_t depth;             // stack entries provided (the batch's largest program depth)
    const int32_t *nactive;    // pairs listed in active[] for this launch
    const int32_t *active;     // pair indices, ascending
    uint64_t *split;
    int32_t *status;
};

template <int N, int U, int BLOCK>
struct SepSmem {
    static constexpr size_t code_bytes(int tile) { return ((size_t)tile * SEP_OPS_STRIDE * 6 + 15) & ~(size_t)15; }
    // 4 int + u64 per pair, rounded up so the atom rows after it stay
    // 16-byte aligned (they are read with 16-byte loads)
    static constexpr size_t meta_bytes(int tile) { return ((size_t)tile * 24 + 15) & ~(size_t)15; }
    static constexpr size_t row_bytes() { return (size_t)SEP_ROW_CAP * RowShape<N>::WORDS * 4; }
    static constexpr size_t stack_bytes(int depth) { return (size_t)depth * U * N * BLOCK * 4; }
    static size_t total(int tile, int depth) {
        return code_bytes(tile) + meta_bytes(tile) + row_bytes() + stack_bytes(depth);
    }
};

// Edge words of 32 sampled relations s = base .. base+31 (lane l <- s).
template <int N>
__device__ __forceinline__ uint32_t sampled_frame_word(uint64_t state, uint64_t base, uint64_t nframes,
                                                       uint32_t (&E)[N * N]) {
#pragma unroll
    for (int e = 0; e < N * N; ++e) E[e] = 0;
    uint32_t valid = 0;
    for (int l = 0; l < 32; ++l) {
        const uint64_t s = base + (uint64_t)l;
        if (s >= nframes) break;
        valid |= 1u << l;
        const uint64_t d0 = sm_out(state, 9 * s);
        const uint64_t t = 26 + (((d0 >> 32) * 103ull) >> 32);
#pragma unroll
        for (int g = 0; g < (N * N + 7) / 8; ++g) {
            const uint64_t d = sm_out(state, 9 * s + 1 + (uint64_t)g);
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                if (g * 8 + b < N * N) E[g * 8 + b] |= (uint32_t)(((d >> (8 * b)) & 0xFFu) < t) << l;
            }
        }
    }
    return valid;
}

// Valid lanes of frame word `word` of this launch (frames that exist and,
// for a K-index window, lie inside it).
__device__ __forceinline__ uint32_t sep_valid_lanes(const SepArgs &a, uint64_t word) {
    const uint64_t base = word << 5;
    if (word >= a.word_hi || base >= a.nframes) return 0;
    const uint64_t left = a.nframes - base;
    uint32_t valid = left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
    if (!a.sampled && !a.full_range) {
        for (int l = 0; l < 32; ++l)
            if (base + l < a.f_lo || base + l >= a.f_hi) valid &= ~(1u << l);
    }
    return valid;
}

// log2 of the unit count (U a power of two <= 8)
template <int U>
constexpr int ulog2() { return U >= 8 ? 3 : U >= 4 ? 2 : U >= 2 ? 1 : 0; }

// Edge words of the U consecutive K frame words w0, w0+1, ... (w0 a multiple
// of U).  Frame f = 32*word + lane has edge bit e = bit e of f: bits 0-4 are
// the lane patterns, bits 5 .. 5+log2(U)-1 are the bits of the unit u (all
// ones or all zeros, known at compile time once u and e are), and every
// higher bit is the same for all U words.  Written per unit, the identical
// words collapse to one register and the constant ones into the logic ops.
template <int N, int U>
__device__ __forceinline__ void k_unit_words(uint64_t w0, uint32_t (&E)[U][N * N]) {
    constexpr int LU = ulog2<U>();
    const uint64_t base = w0 << 5;
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int e = 0; e < N * N; ++e)
            E[u][e] = e < 5 ? lane_pattern(e)
                    : e < 5 + LU ? (((u >> (e - 5)) & 1) ? 0xFFFFFFFFu : 0u)
                    : bit_word(base, e);
}

// SAMPLED: frames are sampled relations (edge words built per unit);
// otherwise K frames, U consecutive words per thread (k_unit_words).
template <int N, int U, int BLOCK, bool SAMPLED>
__global__ void __launch_bounds__(BLOCK) separate_kernel(SepArgs a) {
    using SM = SepSmem<N, U, BLOCK>;
    constexpr int RW = RowShape<N>::WORDS;
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_active;
    const int tile = a.tile;
    // this CTA's tile of the active-pair list (uniform: one load of the count)
    const int na_list = *a.nactive;
    const int t0 = blockIdx.y * tile;
    if (t0 >= na_list) return;
    const int np = min(tile, na_list - t0);
    uint16_t *s_offs_a = (uint16_t *)smem;
    uint16_t *s_offs_b = s_offs_a + (size_t)tile * SEP_OPS_STRIDE;
    uint8_t *s_ops_a = (uint8_t *)(s_offs_b + (size_t)tile * SEP_OPS_STRIDE);
    uint8_t *s_ops_b = s_ops_a + (size_t)tile * SEP_OPS_STRIDE;
    int *s_na = (int *)(smem + SM::code_bytes(tile));
    int *s_pair = s_na + tile;
    int *s_k = s_pair + tile;
    int *s_pad = s_k + tile;
    unsigned long long *s_key = (unsigned long long *)(s_pad + tile);
    uint32_t *s_rows = (uint32_t *)(smem + SM::code_bytes(tile) + SM::meta_bytes(tile));
    uint32_t *s_stack = (uint32_t *)((uint8_t *)s_rows + SM::row_bytes()) + threadIdx.x;

    const uint64_t group_words = (uint64_t)BLOCK * U;   // frame words of one group (U per thread)
    const uint64_t cta_word0 = a.word_lo + (uint64_t)blockIdx.x * a.groups * group_words;
    if (cta_word0 >= a.word_hi) return;
    const unsigned long long floor_key = split_key(a.sampled, N, cta_word0 << 5, 0, 0);
    if (threadIdx.x == 0) s_active = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < np; i += BLOCK) {
        const int pi = a.active[t0 + i];
        const mk_program &pa = a.phi[pi], &pb = a.psi[pi];
        int ok = program_ok(pa) && program_ok(pb) && pa.depth <= a.depth && pb.depth <= a.depth;
        if (!ok && blockIdx.x == 0) atomicOr(a.status, (int)MK_ST_PROGRAM);
        const int k = pa.nvars > pb.nvars ? pa.nvars : pb.nvars;
        const bool exh = exhaustive_vals(k, N, a.S);
        const uint64_t nval = exh ? (1ull << (k * N)) : a.S;
        if (ok && (nval > (1ull << 21) || (exh && k * N > 21))) {
            ok = 0;
            if (blockIdx.x == 0) atomicOr(a.status, (int)MK_ST_LIMIT);
        }
        // a split already below this CTA's least key ends the pair here
        if (ok && ((volatile unsigned long long *)a.split)[pi] < floor_key) ok = 0;
        s_na[i] = ok ? pa.n_instr : -1;
        s_pair[i] = pi;
        s_k[i] = k;
        s_key[i] = ~0ull;
        if (ok) {
            atomicAdd(&s_active, 1);
            decode_program<N, U, BLOCK, false>(pa, s_ops_a + i * SEP_OPS_STRIDE, s_offs_a + i * SEP_OPS_STRIDE);
            decode_program<N, U, BLOCK, false>(pb, s_ops_b + i * SEP_OPS_STRIDE, s_offs_b + i * SEP_OPS_STRIDE);
        }
    }
    __syncthreads();
    if (s_active == 0) return;

    const int lane = threadIdx.x & 31;
    int rows_kind = -1;
    uint32_t rows_c0 = 0;
    for (int g = 0; g < a.groups; ++g) {
        const uint64_t gw0 = cta_word0 + (uint64_t)g * group_words;
        if (gw0 >= a.word_hi) break;                       // uniform
        uint32_t E[U][N * N];
        uint32_t valid[U];
        const uint64_t tw0 = gw0 + (uint64_t)threadIdx.x * U;
        if constexpr (SAMPLED) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                valid[u] = sep_valid_lanes(a, tw0 + u);
                if (valid[u]) {
                    sampled_frame_word<N>(a.rel_state, (tw0 + u) << 5, a.nframes, E[u]);
                } else {
#pragma unroll
                    for (int e = 0; e < N * N; ++e) E[u][e] = 0;
                }
            }
        } else {
            k_unit_words<N, U>(tw0, E);
#pragma unroll
            for (int u = 0; u < U; ++u) valid[u] = sep_valid_lanes(a, tw0 + u);
        }
        // pairs whose split this CTA found in an earlier group: read by every
        // thread before any thread can write s_key again, so the skips below
        // (and the barriers of row staging) are uniform across the CTA
        uint64_t found = 0;
        for (int fi = 0; fi < np; ++fi)
            if (s_key[fi] != ~0ull) found |= 1ull << fi;
        __syncthreads();
        for (int fi = 0; fi < np; ++fi) {
            if (s_na[fi] < 0 || ((found >> fi) & 1ull)) continue;   // finished pair, or split found here
            const int k = s_k[fi];
            const bool exh = exhaustive_vals(k, N, a.S);
            const uint32_t nval = exh ? (1u << (k * N)) : a.S;
            const uint8_t *oa = s_ops_a + fi * SEP_OPS_STRIDE, *ob = s_ops_b + fi * SEP_OPS_STRIDE;
            const uint16_t *fa = s_offs_a + fi * SEP_OPS_STRIDE, *fb = s_offs_b + fi * SEP_OPS_STRIDE;
            int best_o = U * 32, best_w = 0;     // o = u * 32 + lane: ascending frames
            uint32_t best_j = 0;
            for (uint32_t c0 = 0; c0 < nval; c0 += SEP_ROW_CAP) {
                const uint32_t cn = min((uint32_t)SEP_ROW_CAP, nval - c0);
                if (rows_kind != (exh ? 0 : 1) || rows_c0 != c0) {
                    __syncthreads();
                    constexpr int W = RowShape<N>::WORDS;
                    const uint32_t rows = exh ? (uint32_t)SEP_ROW_CAP : min((uint32_t)SEP_ROW_CAP, a.S - c0);
                    for (uint32_t i = threadIdx.x; i < rows * W; i += BLOCK) {
                        const uint32_t j = c0 + i / W;
                        s_rows[i] = atom_row_word<N>(exh ? j : a.samples[j], (int)(i % W));
                    }
                    __syncthreads();
                    rows_kind = exh ? 0 : 1;
                    rows_c0 = c0;
                }
                for (uint32_t jj = 0; jj < cn && best_o > 0; ++jj) {
                    uint32_t A[U][N], B[U][N];
                    run_program<N, U, U, BLOCK, 0, false>(oa, fa, s_rows + jj * RW, E, s_stack, A);
                    run_program<N, U, U, BLOCK, 0, false>(ob, fb, s_rows + jj * RW, E, s_stack, B);
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        uint32_t any = 0;
#pragma unroll
                        for (int w = 0; w < N; ++w) any |= A[u][w] ^ B[u][w];
                        any &= valid[u];
                        if (any) {
                            const int o = u * 32 + __ffs(any) - 1;
                            if (o < best_o) {
                                const int l = o - u * 32;
                                best_o = o;
                                best_j = c0 + jj;
                                int bw = 0;
#pragma unroll
                                for (int w = N - 1; w >= 0; --w)
                                    if (((A[u][w] ^ B[u][w]) >> l) & 1u) bw = w;
                                best_w = bw;
                            }
                        }
                    }
                }
            }
            const uint32_t hit = __ballot_sync(0xFFFFFFFFu, best_o < U * 32);
            if (hit) {
                // threads hold ascending frame words, so the lowest hit lane wins
                const int src_lane = __ffs(hit) - 1;
                uint64_t my = 0;
                if (lane == src_lane) {
                    const uint64_t f = ((gw0 + (uint64_t)threadIdx.x * U) << 5) + (uint64_t)best_o;
                    my = split_key(a.sampled, N, f, best_j, (uint64_t)best_w);
                }
                const uint64_t key = __shfl_sync(0xFFFFFFFFu, my, src_lane);
                if (lane == 0) atomicMin(&s_key[fi], (unsigned long long)key);
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < np; i += BLOCK)
        if (s_key[i] != ~0ull) atomicMin((unsigned long long *)&a.split[s_pair[i]], s_key[i]);
}

// The pairs of split[] whose key is not below floor_key (no split found
// before the next launch's first frame), in ascending order: one CTA of
// SEP_LIST_THREADS threads, a ballot-and-scan compaction per 1,024 pairs.
constexpr int SEP_LIST_THREADS = 1024;
__global__ void __launch_bounds__(SEP_LIST_THREADS) active_pairs_kernel(const uint64_t *split, int npairs,
                                                                        uint64_t floor_key, int32_t *nactive,
                                                                        int32_t *active) {
    __shared__ int s_warp[SEP_LIST_THREADS / 32];
    __shared__ int s_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int b = 0; b < npairs; b += SEP_LIST_THREADS) {
        const int i = b + threadIdx.x;
        const bool act = i < npairs && split[i] >= floor_key;
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, act);
        if (lane == 0) s_warp[warp] = __popc(m);
        __syncthreads();
        if (warp == 0) {
            const int v = s_warp[lane];
            int inc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                if (lane >= o) inc += t;
            }
            s_warp[lane] = inc - v;                         // exclusive offset of each warp
        }
        __syncthreads();
        if (act) active[s_base + s_warp[warp] + __popc(m & ((1u << lane) - 1u))] = i;
        __syncthreads();
        if (threadIdx.x == SEP_LIST_THREADS - 1) s_base += s_warp[warp] + __popc(m);
        __syncthreads();
    }
    if (threadIdx.x == 0) *nactive = s_base;
}

__global__ void init_split_kernel(uint64_t *split, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) split[i] = ~0ull;
}

}  // namespace mkd

namespace {

using namespace mkd;

constexpr int SEP_BLOCK = 256;

// Frame words per thread: K frames share their edge words across units
// (k_unit_words), sampled relations need a full set per unit.
template <int N, bool SAMPLED>
constexpr int sep_units() { return SAMPLED ? (N <= 6 ? 2 : 1) : 4; }

// CTAs per launch below which a strip holds a single group: four waves of
// two CTAs on 152 SMs, so that even a single active tile fills the GPU.
constexpr uint64_t SEP_MIN_CTAS = 1216;
constexpr uint64_t SEP_MAX_GROUPS = 8;

template <int N, bool SAMPLED>
void launch_sep(SepArgs a, cudaStream_t s) {
    constexpr int U = sep_units<N, SAMPLED>();
    const uint64_t words = a.word_hi > a.word_lo ? a.word_hi - a.word_lo : 0;
    if (words == 0 || a.npairs == 0) return;
    const uint64_t per_group = (uint64_t)SEP_BLOCK * U;
    const uint64_t groups = (words + per_group - 1) / per_group;
    uint64_t g = groups / SEP_MIN_CTAS;
    g = g < 1 ? 1 : (g > SEP_MAX_GROUPS ? SEP_MAX_GROUPS : g);
    a.groups = (int32_t)g;
    dim3 grid((unsigned)((groups + g - 1) / g), (unsigned)((a.npairs + a.tile - 1) / a.tile));
    const size_t sm = SepSmem<N, U, SEP_BLOCK>::total(a.tile, a.depth);
    auto kern = separate_kernel<N, U, SEP_BLOCK, SAMPLED>;
    ensure_dynamic_smem((const void *)kern, sm);
    // the pairs without a split below this launch's first frame
    const uint64_t floor_key = split_key(a.sampled, N, a.word_lo << 5, 0, 0);
    active_pairs_kernel<<<1, SEP_LIST_THREADS, 0, s>>>(a.split, a.npairs, floor_key, (int32_t *)a.nactive,
                                                       (int32_t *)a.active);
    kern<<<grid, SEP_BLOCK, sm, s>>>(a);
}

void launch_sep_n(int n, const SepArgs &a, cudaStream_t s) {
    if (a.sampled) {
        switch (n) {
        case 1: launch_sep<1, true>(a, s); break;
        case 2: launch_sep<2, true>(a, s); break;
        case 3: launch_sep<3, true>(a, s); break;
        case 4: launch_sep<4, true>(a, s); break;
        case 5: launch_sep<5, true>(a, s); break;
        case 6: launch_sep<6, true>(a, s); break;
        case 7: launch_sep<7, true>(a, s); break;
        case 8: launch_sep<8, true>(a, s); break;
        }
    } else {
        switch (n) {
        case 1: launch_sep<1, false>(a, s); break;
        case 2: launch_sep<2, false>(a, s); break;
        case 3: launch_sep<3, false>(a, s); break;
        case 4: launch_sep<4, false>(a, s); break;
        case 5: launch_sep<5, false>(a, s); break;
        case 6: launch_sep<6, false>(a, s); break;
        }
    }
}

int check_sep(const mk_separate_cfg *cfg, int32_t npairs) {
    if (!cfg || npairs < 0) return MK_E_ARG;
    if (cfg->n_exh_max > MK_MAX_WORLDS_EXH || cfg->n_exh_min > cfg->n_exh_max) return MK_E_ARG;
    if (cfg->n_exh_max && cfg->n_exh_min < 1) return MK_E_ARG;
    if (cfg->n_smp_max) {
        if (cfg->n_smp_min < 1 || cfg->n_smp_min > cfg->n_smp_max || cfg->n_smp_max > MK_MAX_WORLDS_SAMPLED)
            return MK_E_ARG;
        if (cfg->n_exh_max && cfg->n_smp_min <= cfg->n_exh_max) return MK_E_ARG;
        if (cfg->frames_per_n >= (1ull << 36)) return MK_E_ARG;
    }
    if ((cfg->samples == 0) != (cfg->d_samples == nullptr)) return MK_E_ARG;
    if (cfg->frame_lo > cfg->frame_hi) return MK_E_ARG;
    const mk_tune &t = cfg->tune;
    if (t.block && t.block != SEP_BLOCK) return MK_E_ARG;
    if (t.tile > 64) return MK_E_ARG;
    if (cfg->max_depth > MK_MAX_STACK) return MK_E_ARG;
    return MK_OK;
}

}  // namespace

// Workspace: the active-pair count (16 bytes) and the active-pair list.
extern "C" size_t mk_separate_workspace_size(const mk_separate_cfg *cfg, int32_t npairs) {
    (void)cfg;
    if (npairs <= 0) return 0;
    return ((size_t)npairs * 4 + 16 + 255) & ~(size_t)255;
}

extern "C" uint64_t mk_sample_relation(uint64_t seed, int32_t n, uint64_t s) {
    if (n < 1 || n > MK_MAX_WORLDS_SAMPLED) return 0;
    return sample_relation(sm_stream(seed, 2, (uint64_t)n), n, s);
}

namespace {

// Walks the launches of a search in order: every size, and within a size
// its chunks of frame words.  With a non-null stream pointer it launches
// them; it returns the number of kernel launches either way.
int64_t separate_walk(const mk_separate_cfg *cfg, SepArgs &a, const cudaStream_t *s) {
    const uint64_t chunk_words = 1ull << 22;   // exhaustive sizes: 2^27 frames per launch
    const uint64_t sampled_words = 1ull << 18; // sampled sizes: 2^23 relations per launch
    int64_t launches = 1;                       // the split keys' initialisation
    if (cfg->n_exh_max) {
        for (int n = cfg->n_exh_min; n <= cfg->n_exh_max; ++n) {
            const uint64_t kf = 1ull << (n * n);
            const uint64_t hi = cfg->frame_hi < kf ? cfg->frame_hi : kf;
            a.samples = cfg->samples ? cfg->d_samples + (size_t)n * cfg->samples : nullptr;
            a.sampled = 0;
            a.nframes = kf;
            a.f_lo = cfg->frame_lo;
            a.f_hi = cfg->frame_hi;
            a.full_range = (cfg->frame_lo == 0 && cfg->frame_hi >= kf) ? 1 : 0;
            // the first word rounded down to a multiple of 8 (so every thread's
            // first word is a multiple of its unit count); the frames below
            // frame_lo are masked off as the window demands
            const uint64_t w0 = (cfg->frame_lo / 32) & ~(uint64_t)7;
            const uint64_t w1 = cfg->frame_lo >= hi ? w0 : (hi + 31) / 32;
            for (uint64_t w = w0; w < w1; w += chunk_words) {
                a.word_lo = w;
                a.word_hi = w + chunk_words < w1 ? w + chunk_words : w1;
                if (s) launch_sep_n(n, a, *s);
                launches += 2;                  // the active-pair list, then the search
            }
        }
    }
    if (cfg->n_smp_max) {
        for (int n = cfg->n_smp_min; n <= cfg->n_smp_max; ++n) {
            a.samples = cfg->samples ? cfg->d_samples + (size_t)n * cfg->samples : nullptr;
            a.sampled = 1;
            a.rel_state = sm_stream(cfg->seed, 2, (uint64_t)n);
            a.nframes = cfg->frames_per_n;
            a.full_range = 1;
            const uint64_t w1 = (cfg->frames_per_n + 31) / 32;
            for (uint64_t w = 0; w < w1; w += sampled_words) {
                a.word_lo = w;
                a.word_hi = w + sampled_words < w1 ? w + sampled_words : w1;
                if (s) launch_sep_n(n, a, *s);
                launches += 2;
            }
        }
    }
    return launches;
}

}  // namespace

extern "C" int64_t mk_separate_launches(const mk_separate_cfg *cfg, int32_t npairs) {
    if (check_sep(cfg, npairs) != MK_OK) return -1;
    if (npairs == 0) return 0;
    SepArgs a;
    std::memset(&a, 0, sizeof(a));
    return separate_walk(cfg, a, nullptr);
}

extern "C" int mk_separate(const mk_program *d_phi, const mk_program *d_psi, int32_t npairs,
                           const mk_separate_cfg *cfg, uint64_t *d_split, int32_t *d_status,
                           void *d_workspace, size_t ws_bytes, void *stream) {
    int rc = check_sep(cfg, npairs);
    if (rc != MK_OK) return rc;
    if (npairs > 0 && (!d_phi || !d_psi || !d_split)) return MK_E_ARG;
    if (!d_status) return MK_E_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (npairs == 0) return MK_OK;
    if (ws_bytes < mk_separate_workspace_size(cfg, npairs)) return MK_E_WORKSPACE;
    if (!d_workspace || ((uintptr_t)d_workspace & 15)) return MK_E_ARG;
    init_split_kernel<<<(npairs + 255) / 256, 256, 0, s>>>(d_split, npairs);

    SepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.phi = d_phi;
    a.psi = d_psi;
    a.npairs = npairs;
    a.tile = cfg->tune.tile ? cfg->tune.tile : 16;
    a.depth = cfg->max_depth ? cfg->max_depth : MK_MAX_STACK;
    a.S = cfg->samples;
    a.split = d_split;
    a.status = d_status;
    a.nactive = (const int32_t *)d_workspace;
    a.active = (const int32_t *)((uint8_t *)d_workspace + 16);
    separate_walk(cfg, a, &s);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

extern "C" int mk_split_cert(const mk_program *h_phi, const mk_program *h_psi, const char *phi,
                             const char *psi, uint64_t seed, uint32_t samples, const uint32_t *h_samples_n,
                             uint64_t key, mk_cert *out) {
    if (!h_phi || !h_psi || !phi || !psi || !out || key == ~0ull) return MK_E_ARG;
    const int sampled = (int)(key >> 63);
    const int n = (int)((key >> 60) & 7u) + 1;
    const uint64_t f = (key >> 24) & ((1ull << 36) - 1);
    const uint32_t j = (uint32_t)((key >> 3) & ((1u << 21) - 1));
    const int w = (int)(key & 7u);
    if (n < 1 || n > MK_MAX_WORLDS_SAMPLED || w >= n) return MK_E_ARG;
    const int k = h_phi->nvars > h_psi->nvars ? h_phi->nvars : h_psi->nvars;
    const bool exh = exhaustive_vals(k, n, samples);
    if (!exh && !h_samples_n) return MK_E_ARG;
    if (!sampled && n > MK_MAX_WORLDS_EXH) return MK_E_ARG;
    const uint64_t rel = sampled ? sample_relation(sm_stream(seed, 2, (uint64_t)n), n, f) : f;
    const uint32_t x = exh ? j : h_samples_n[j];
    const uint32_t full = (1u << n) - 1u;
    std::memset(out, 0, sizeof(*out));
    out->phi = phi;
    out->psi = psi;
    out->n = (uint8_t)n;
    out->cls = 0;
    out->world = (uint8_t)w;
    for (int v = 0; v < n; ++v) out->succ[v] = (uint32_t)((rel >> (v * n)) & full);
    for (int i = 0; i < k; ++i) out->val[i] = (x >> (i * n)) & full;
    return MK_OK;
}
