// mk_census.cu -- the census: Alg. 1 (fused corpus scan) over every
// selected (class, n) layer, redesigned for sm_103a.
//
// Unit of work ("tile"): a set of formulas of one layer (class, n) and a
// range of frame words.  A thread owns one frame word at a time (32
// consecutive frames, synthesised from its index: no frame is read from
// HBM) and keeps its n*n edge words in registers.  For each formula of the
// tile it walks the layer's valuations U at a time, interpreting the
// postfix program on an accumulator in registers (mk_eval.cuh); atom truth
// sets are read from shared-memory rows (one row per valuation, re-staged
// in chunks when a formula needs more rows than fit).  Refuted lanes are
// ~(AND_w t[w]) & valid; the count is a popcount, the first witness the
// lowest refuted lane at the first valuation that refutes it.  Reduction:
// warp (__reduce_add_sync, ballot + shuffle for the witness), CTA (shared
// atomics), then one global atomicAdd / atomicMin per CTA, tile and
// formula (Sec. 4's hierarchical reduction).
//
// Two launch shapes run the same tile routine:
//   - mk_census: one grid per layer, blockIdx.x = frame words, blockIdx.y =
//     formula tile (all formulas share the classes and n range);
//   - mk_census_uneven: one persistent grid that takes work items (tile x
//     layer x word range) from a host-built plan through an atomic cursor,
//     for batches where every formula has its own class and n_max.
//
// Classes: K frames are every index; T frames are enumerated by their
// compact index (diagonal forced on); S4 and S5 frames are first listed by a
// three-kernel filter over the T frames (count, scan, write; ascending K
// order) into the caller's workspace, then scanned from that list; K4
// frames (transitive, not necessarily reflexive) are listed the same way by
// a filter over the K frames.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "mk.h"
#include "mk_attr.h"
#include "mk_eval.cuh"

namespace mkd {

constexpr int SRC_K = 0, SRC_T = 1, SRC_LIST = 2;
constexpr int ROW_CAP = 128;                   // atom rows staged at a time
constexpr int OPS_STRIDE = MK_MAX_CODE + 2;   // decoded ops per program (END + prefetch pad)
constexpr int MAX_TILE = 64;
constexpr int VCHUNK = 32;                     // valuation-split granularity (whole units)

// Valuation groups of a CTA (see census_tile): a split layer's CTA with
// fewer frame words than BLOCK / 2 also shares its valuations among G groups
// of nwr threads (nwr = its words rounded up to a power of two).
__host__ __device__ inline int vgroups(uint64_t nw, int block, int units, int *nwr_out) {
    int nwr = block;
    while (nwr > 1 && (uint64_t)(nwr / 2) >= nw) nwr /= 2;
    if (nwr_out) *nwr_out = nwr;
    const int g = block / nwr, cap = ROW_CAP / units;
    return g < cap ? g : cap;
}

// The split kernel variant is built for the default tune only (U = 8,
// BLOCK = 256); layers of other tunes are never split.
template <int U, int BLOCK>
constexpr bool kSplitTune = U == 8 && BLOCK == 256;

// Chunk granularity of a split CTA: whole passes of its G groups, at least
// VCHUNK valuations, so each thread has several units to amortise its
// program staging.
__host__ __device__ inline uint64_t vgran(int G, int units) {
    const uint64_t g = (uint64_t)G * units;
    return g > (uint64_t)VCHUNK ? g : (uint64_t)VCHUNK;
}

// One tile: where its formulas, frames and outputs are.
struct TileCtx {
    const mk_program *progs;
    const mk_job *jobs;        // uneven batches: jobs and the plan's job list
    const uint32_t *jlist;     //   (NULL: formulas p0 .. p0+np-1 of progs)
    int32_t p0, np;
    mk_result *out;            // census: out + p*out_stride + out_off
    int32_t out_stride, out_off;   // uneven: out + job*6 + (n-1)
    int32_t src;
    const uint64_t *flist;     // SRC_LIST: K indices, ascending
    uint64_t nframes;          // frames in the source (by ordinal)
    uint64_t w0, w1;           // frame words of this tile
    uint64_t f_lo, f_hi;       // K-index filter
    int32_t full_range;        // 1: f_lo/f_hi do not cut this layer
    const uint32_t *samples;   // this layer's sampled valuations
    uint32_t S;
    int32_t depth;             // stack entries provided
    int32_t tile_cap;          // formulas the shared-memory layout holds
    int32_t report;            // 1: this CTA reports program errors
    int32_t *status;
};

// A split layer (valuations shared out over grid.z): kept apart from TileCtx
// so the unsplit kernels see exactly the context they always had.
struct SplitCtx {
    uint32_t vsplit, vpart;    // valuation chunks of the layer; this CTA's chunk
    uint32_t *rf_bits;         // OR of refuted lanes per (formula, word)
    uint64_t rf_w0, rf_words;  //   the layer's first word and its words per formula
};

// Shared memory of one CTA (tile <= MAX_TILE formulas, frames of <= NM worlds).
template <int NM, int U, int BLOCK>
struct TileSmem {
    static constexpr size_t code_bytes(int tile) { return ((size_t)tile * OPS_STRIDE * 3 + 15) & ~(size_t)15; }
    // 2 int + 3 u64 + ptr per formula, rounded up so the atom rows after it
    // stay 16-byte aligned (they are read with 16-byte loads)
    static constexpr size_t meta_bytes(int tile) { return ((size_t)tile * 40 + 15) & ~(size_t)15; }
    // ROW_CAP rows plus U rows of slack read (and masked) by a partial last step
    static constexpr size_t row_bytes() { return (size_t)(ROW_CAP + U) * RowShape<NM>::WORDS * 4; }
    static constexpr size_t stack_bytes(int depth) { return (size_t)depth * U * NM * BLOCK * 4; }
    static size_t total(int tile, int depth) {
        return code_bytes(tile) + meta_bytes(tile) + row_bytes() + stack_bytes(depth);
    }
};

// K index of lane l of a word.
template <int N>
__device__ __forceinline__ uint64_t lane_kindex(const TileCtx &t, uint64_t word, int l) {
    const uint64_t ord = (word << 5) + (uint64_t)l;
    if (t.src == SRC_K) return ord;
    if (t.src == SRC_T) return t_to_k(ord, N);
    return t.flist[ord];
}

template <int N>
__device__ __forceinline__ uint32_t build_word(const TileCtx &t, uint64_t word, uint32_t (&E)[N * N]) {
    const uint64_t base = word << 5;
    uint32_t valid = 0;
    if (base < t.nframes) {
        const uint64_t left = t.nframes - base;
        valid = left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
    }
    if (t.src == SRC_K) {
        k_frame_word<N>(word, E);
    } else if (t.src == SRC_T) {
        t_frame_word<N>(word, E);
    } else {
        const int cnt = __popc(valid);
        list_frame_word<N>(t.flist + base, cnt, E);
    }
    if (!t.full_range && valid) {
        for (int l = 0; l < 32; ++l) {
            if ((valid >> l) & 1u) {
                const uint64_t f = lane_kindex<N>(t, word, l);
                if (f < t.f_lo || f >= t.f_hi) valid &= ~(1u << l);
            }
        }
    }
    return valid;
}

// Stage atom rows [c0, c0 + rows) of one valuation kind (exhaustive: the
// valuation value is the index; sampled: samples[j]).
template <int N, int BLOCK>
__device__ __forceinline__ void stage_rows(uint32_t *s_rows, bool exh, const uint32_t *samples, uint32_t c0,
                                           uint32_t rows) {
    constexpr int W = RowShape<N>::WORDS;
    for (uint32_t i = threadIdx.x; i < rows * W; i += BLOCK) {
        const uint32_t j = c0 + i / W;
        const uint32_t val = exh ? j : samples[j];
        s_rows[i] = atom_row_word<N>(val, (int)(i % W));
    }
}

// The census of one tile on n = N worlds.  All threads of the CTA call it
// with the same t; smem is laid out by TileSmem<NM, U, BLOCK> with NM >= N.
template <int N, int NM, int U, int BLOCK, bool SPLIT = false>
__device__ __forceinline__ void census_tile(const TileCtx &t, uint8_t *smem, const SplitCtx &sp = SplitCtx()) {
    using SM = TileSmem<NM, U, BLOCK>;
    constexpr int RW = RowShape<N>::WORDS;
    const int np = t.np, cap = t.tile_cap;
    uint16_t *s_offs = (uint16_t *)smem;
    uint8_t *s_ops = smem + (size_t)cap * OPS_STRIDE * 2;
    int *s_nin = (int *)(smem + SM::code_bytes(cap));
    int *s_k = s_nin + cap;
    unsigned long long *s_cm = (unsigned long long *)(s_k + cap);
    unsigned long long *s_rf = s_cm + cap;
    unsigned long long *s_key = s_rf + cap;
    mk_result **s_out = (mk_result **)(s_key + cap);
    uint32_t *s_rows = (uint32_t *)(smem + SM::code_bytes(cap) + SM::meta_bytes(cap));
    uint32_t *s_stack = (uint32_t *)((uint8_t *)s_rows + SM::row_bytes()) + threadIdx.x;

    // stage the tile's programs (checked once per tile)
    for (int i = threadIdx.x; i < np; i += BLOCK) {
        const mk_program *pp;
        mk_result *o;
        if (t.jlist) {
            const uint32_t j = t.jlist[t.p0 + i];
            pp = t.progs + t.jobs[j].prog;
            o = t.out + (size_t)j * 6 + (N - 1);
        } else {
            pp = t.progs + (t.p0 + i);
            o = t.out + (size_t)(t.p0 + i) * t.out_stride + t.out_off;
        }
        const mk_program &p = *pp;
        int nin = -1;
        if (program_ok(p) && p.depth <= t.depth) {
            nin = p.n_instr;
            if (exhaustive_vals(p.nvars, N, t.S) && p.nvars * N > 24) {
                nin = -1;
                if (t.report) atomicOr(t.status, (int)MK_ST_LIMIT);
            }
        } else if (t.report) {
            atomicOr(t.status, (int)MK_ST_PROGRAM);
        }
        s_nin[i] = nin;
        s_k[i] = p.nvars;
        s_cm[i] = 0;
        s_rf[i] = 0;
        s_key[i] = ~0ull;
        s_out[i] = o;
        if (nin >= 0) decode_program<N, U, BLOCK>(p, s_ops + i * OPS_STRIDE, s_offs + i * OPS_STRIDE);
    }
    __syncthreads();
    int rows_kind = -1;          // staged rows: 0 exhaustive, 1 sampled
    uint32_t rows_c0 = 0;
    const int lane = threadIdx.x & 31;
    // A split layer's CTA with few frame words (a tiny window under many
    // valuations) also shares each staged block of valuations among its
    // threads: G groups of nwr threads (nwr = words rounded up to a power of
    // two), group g taking units g, g + G, ... of the block.  Threads with the
    // same word then OR their refuted lanes into the split bitmap and take
    // the CTA's least witness key by an atomic min.
    // (all of the split -- chunks, groups, the bitmap -- is a compile-time
    // variant, so the kernels of unsplit layers carry none of it)
    int nwr = BLOCK, G = 1;
    if constexpr (SPLIT) G = vgroups(t.w1 - t.w0, BLOCK, U, &nwr);
    const uint32_t sub = SPLIT ? (uint32_t)(threadIdx.x / nwr) : 0u;
    const uint64_t gran = vgran(G, U);

    for (uint64_t wg = t.w0; wg < t.w1; wg += BLOCK) {
        const uint64_t word = wg + (SPLIT ? (threadIdx.x & (nwr - 1)) : threadIdx.x);
        uint32_t E[1][N * N];
        uint32_t valid = 0;
        if (word < t.w1) valid = build_word<N>(t, word, E[0]);
        else {
#pragma unroll
            for (int e = 0; e < N * N; ++e) E[0][e] = 0;
        }
        for (int fi = 0; fi < np; ++fi) {
            const int nin = s_nin[fi];
            if (nin < 0) continue;
            const int k = s_k[fi];
            const bool exh = exhaustive_vals(k, N, t.S);
            const uint32_t nval = exh ? (1u << (k * N)) : t.S;
            // this CTA's chunk of the valuations, a multiple of its granule
            // (whole passes of its groups); rows are staged from its start
            uint32_t v_lo = 0, v_hi = nval;
            if constexpr (SPLIT) {
                const uint64_t per = ((nval + (uint64_t)sp.vsplit - 1) / sp.vsplit + gran - 1) / gran * gran;
                v_lo = (uint32_t)min((uint64_t)nval, (uint64_t)sp.vpart * per);
                v_hi = (uint32_t)min((uint64_t)nval, (uint64_t)v_lo + per);
                if (v_lo >= v_hi) continue;
            }
            const uint8_t *ops = s_ops + fi * OPS_STRIDE;
            const uint16_t *offs = s_offs + fi * OPS_STRIDE;
            uint32_t cnt = 0, rf = 0, best_j = 0;
            int best_l = 32, best_w = 0;
            for (uint32_t c0 = v_lo; c0 < v_hi; c0 += ROW_CAP) {
                const uint32_t cn = min((uint32_t)ROW_CAP, v_hi - c0);
                // uniform across the CTA: every thread takes the same decisions.
                // Exhaustive rows are staged ROW_CAP at a time, sampled ones up to S.
                if (rows_kind != (exh ? 0 : 1) || rows_c0 != c0) {
                    __syncthreads();
                    stage_rows<N, BLOCK>(s_rows, exh, t.samples, c0,
                                         exh ? (uint32_t)ROW_CAP : min((uint32_t)ROW_CAP, t.S - c0));
                    __syncthreads();
                    rows_kind = exh ? 0 : 1;
                    rows_c0 = c0;
                }
                // valid lanes per unit: all lanes of the frame word, except the
                // units past the chunk's end in its last step
                uint32_t vm[U];
#pragma unroll
                for (int u = 0; u < U; ++u) vm[u] = valid;
                for (uint32_t jj = SPLIT ? sub * U : 0u; jj < cn; jj += SPLIT ? (uint32_t)G * U : (uint32_t)U) {
                    if (jj + U > cn) {
#pragma unroll
                        for (int u = 0; u < U; ++u) vm[u] = (jj + u < cn) ? valid : 0u;
                    }
                    uint32_t A[U][N];
                    run_program<N, U, 1, BLOCK, RW>(ops, offs, s_rows + jj * RW, E, s_stack, A);
                    uint32_t bad[U], any = 0;
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        uint32_t all = A[u][0];
#pragma unroll
                        for (int w = 1; w < N; ++w) all &= A[u][w];
                        bad[u] = ~all & vm[u];
                        cnt += __popc(bad[u]);
                        any |= bad[u];
                    }
                    rf |= any;
                    // a lane below the best so far: its first refuting valuation is
                    // the first unit (in valuation order) that refutes it
                    uint32_t lowmask = (best_l < 32 ? (1u << best_l) : 0u) - 1u;
                    if (any & lowmask) {
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const uint32_t lower = bad[u] & lowmask;
                            if (lower) {
                                const int l = __ffs(lower) - 1;
                                best_l = l;
                                best_j = c0 + jj + u;
                                int bw = 0;
#pragma unroll
                                for (int w = N - 1; w >= 0; --w)
                                    if (!((A[u][w] >> l) & 1u)) bw = w;
                                best_w = bw;
                                lowmask = (1u << l) - 1u;
                            }
                        }
                    }
                }
            }
            // warp reduction: counts split in 16-bit halves so the sums fit
            const uint32_t c_hi = __reduce_add_sync(0xFFFFFFFFu, cnt >> 16);
            const uint32_t c_lo = __reduce_add_sync(0xFFFFFFFFu, cnt & 0xFFFFu);
            // frames refuted: a popcount, unless other CTAs hold other valuations
            // of the same frames; then the frame words are ORed and counted later
            uint32_t f_sum = 0;
            if constexpr (SPLIT) {
                if (rf) atomicOr(&sp.rf_bits[(size_t)(t.p0 + fi) * sp.rf_words + (word - sp.rf_w0)], rf);
            } else {
                f_sum = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)__popc(rf));
            }
            if (SPLIT && G > 1 && best_l < 32)
                atomicMin(&s_key[fi], (unsigned long long)((lane_kindex<N>(t, word, best_l) << 27) |
                                                           ((uint64_t)best_j << 3) | (uint64_t)best_w));
            const uint32_t hit = (SPLIT && G > 1) ? 0u : __ballot_sync(0xFFFFFFFFu, best_l < 32);
            uint64_t key = ~0ull;
            if (hit) {
                // lanes hold ascending frames, so the lowest hit lane has the least frame
                const int src_lane = __ffs(hit) - 1;
                uint64_t my = 0;
                if (lane == src_lane)
                    my = (lane_kindex<N>(t, word, best_l) << 27) | ((uint64_t)best_j << 3) | (uint64_t)best_w;
                key = __shfl_sync(0xFFFFFFFFu, my, src_lane);
            }
            if (lane == 0) {
                const uint64_t c = ((uint64_t)c_hi << 16) + c_lo;
                if (c) atomicAdd(&s_cm[fi], (unsigned long long)c);
                if (f_sum) atomicAdd(&s_rf[fi], (unsigned long long)f_sum);
                if (hit) atomicMin(&s_key[fi], (unsigned long long)key);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < np; i += BLOCK) {
        mk_result *o = s_out[i];
        if (s_cm[i]) atomicAdd((unsigned long long *)&o->cm_count, s_cm[i]);
        if (s_rf[i]) atomicAdd((unsigned long long *)&o->frames_refuted, s_rf[i]);
        if (s_key[i] != ~0ull) atomicMin((unsigned long long *)&o->witness_key, s_key[i]);
    }
    __syncthreads();
}

// ------------------------------------------------ per-layer grid launch

struct LayerArgs {
    TileCtx t;                 // w0/w1: the layer's word range; p0/np unused
    int32_t tile;
    const uint64_t *list_len;  // SRC_LIST: device count
    SplitCtx sp;               // split layers: vsplit > 1
    uint32_t *rf_done;         //   and their CTAs finished, per formula tile
};

// The end of a split layer's CTA: the last CTA of its formula tile to finish
// (counted on rf_done, the pattern of a threadfence reduction) counts the
// tile's ORed frame words into frames_refuted, then clears the words and the
// counter for the next split layer.  Nothing waits: the other CTAs just exit.
template <int BLOCK>
__device__ void split_layer_tail(const LayerArgs &a, const TileCtx &t, const SplitCtx &sp) {
    __shared__ int s_last;
    __shared__ unsigned long long s_sum;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned total = gridDim.x * gridDim.z;
        s_last = atomicAdd(&a.rf_done[blockIdx.y], 1u) == total - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int i = 0; i < t.np; ++i) {
        uint32_t *b = sp.rf_bits + (size_t)(t.p0 + i) * sp.rf_words;
        if (threadIdx.x == 0) s_sum = 0;
        __syncthreads();
        uint32_t sum = 0;
        for (uint64_t w = threadIdx.x; w < sp.rf_words; w += BLOCK) {
            sum += __popc(__ldcg(b + w));
            b[w] = 0;
        }
        sum = __reduce_add_sync(0xFFFFFFFFu, sum);
        if ((threadIdx.x & 31) == 0 && sum) atomicAdd(&s_sum, (unsigned long long)sum);
        __syncthreads();
        if (threadIdx.x == 0)
            t.out[(size_t)(t.p0 + i) * t.out_stride + t.out_off].frames_refuted = s_sum;
        __syncthreads();
    }
    if (threadIdx.x == 0) a.rf_done[blockIdx.y] = 0;
}

template <int N, int U, int BLOCK, bool SPLIT>
__global__ void __launch_bounds__(BLOCK) census_layer_kernel(LayerArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    TileCtx t = a.t;
    t.p0 = blockIdx.y * a.tile;
    t.np = min(a.tile, t.np - t.p0);
    t.w0 = a.t.w0 + (uint64_t)blockIdx.x * BLOCK;
    t.w1 = min(t.w0 + BLOCK, a.t.w1);
    t.report = blockIdx.x == 0 && (!SPLIT || blockIdx.z == 0);
    t.tile_cap = a.tile;
    if (t.src == SRC_LIST) {
        const uint64_t len = *a.list_len;
        t.nframes = len < t.nframes ? len : t.nframes;
    }
    if constexpr (SPLIT) {
        SplitCtx sp = a.sp;
        sp.vpart = blockIdx.z;
        census_tile<N, N, U, BLOCK, true>(t, smem, sp);
        split_layer_tail<BLOCK>(a, t, sp);
    } else {
        census_tile<N, N, U, BLOCK>(t, smem);
    }
}

// Clears the results and, when some layer splits its valuations, the frame
// bitmap and the per-tile CTA counters that follow it.
__global__ void init_results_kernel(mk_result *out, size_t n, uint32_t *clear, size_t nclear) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        out[i].cm_count = 0;
        out[i].frames_refuted = 0;
        out[i].witness_key = ~0ull;
    }
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nclear; i += stride) clear[i] = 0;
}

// ------------------------------------------------- persistent work queue

struct QueueArgs {
    const mk_program *progs;
    const mk_job *jobs;
    const uint32_t *jlist;
    const mk_work_item *items;
    uint32_t nitems;
    uint32_t *cursor;
    const uint64_t *lists[2][7];     // S4 / S5 lists by n
    const uint64_t *list_len[2][7];
    const uint32_t *samples;         // [(n_max+1) * S]
    uint32_t S;
    int32_t depth;
    int32_t tile_cap;
    mk_result *out;
    int32_t *status;
};

template <int NM, int U, int BLOCK>
__global__ void __launch_bounds__(BLOCK) census_queue_kernel(QueueArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.cursor, 1u);
        __syncthreads();
        const uint32_t it = s_item;
        __syncthreads();
        if (it >= a.nitems) return;
        const mk_work_item w = a.items[it];
        TileCtx t;
        t.progs = a.progs;
        t.jobs = a.jobs;
        t.jlist = a.jlist;
        t.p0 = (int32_t)w.lbeg;
        t.np = w.np;
        t.out = a.out;
        t.out_stride = 6;
        t.out_off = 0;
        const int n = w.n;
        if (w.cls == 0) {
            t.src = SRC_K;
            t.flist = nullptr;
            t.nframes = 1ull << (n * n);
        } else if (w.cls == 1) {
            t.src = SRC_T;
            t.flist = nullptr;
            t.nframes = 1ull << (n * n - n);
        } else {
            t.src = SRC_LIST;
            t.flist = a.lists[w.cls - 2][n];
            t.nframes = *a.list_len[w.cls - 2][n];
        }
        t.w0 = w.w0;
        t.w1 = w.w1;
        t.f_lo = 0;
        t.f_hi = ~0ull;
        t.full_range = 1;
        t.samples = a.S ? a.samples + (size_t)n * a.S : nullptr;
        t.S = a.S;
        t.depth = a.depth;
        t.tile_cap = a.tile_cap;
        t.report = 1;
        t.status = a.status;
        switch (n) {
        case 1: census_tile<1, NM, U, BLOCK>(t, smem); break;
        case 2: census_tile<2, NM, U, BLOCK>(t, smem); break;
        case 3: census_tile<3, NM, U, BLOCK>(t, smem); break;
        case 4: census_tile<4, NM, U, BLOCK>(t, smem); break;
        case 5: census_tile<5, NM, U, BLOCK>(t, smem); break;
        default:
            if constexpr (NM >= 6) census_tile<6, NM, U, BLOCK>(t, smem);
            break;
        }
    }
}

__global__ void reset_cursor_kernel(uint32_t *cursor) { *cursor = 0; }

// ----------------------------------------------- S4 / S5 / K4 frame lists

// List kinds: S4 and S5 filter the T frames (word = 32 compact indices) by
// transitivity (S5: and symmetry); K4 filters the K frames by transitivity.
constexpr int LIST_S4 = 0, LIST_S5 = 1, LIST_K4 = 2, NLISTS = 3;

template <int N>
__device__ __forceinline__ uint32_t class_word_mask(uint64_t word, uint64_t nframes, int kind) {
    uint32_t E[N * N];
    if (kind == LIST_K4) k_frame_word<N>(word, E);
    else t_frame_word<N>(word, E);
    const uint64_t base = word << 5;
    uint32_t valid = 0;
    if (base < nframes) {
        const uint64_t left = nframes - base;
        valid = left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
    }
    return valid & preorder_mask<N>(E, kind == LIST_S5);
}

template <int N>
__global__ void __launch_bounds__(256) list_count_kernel(uint32_t *blk, uint64_t word0, uint64_t nwords,
                                                         uint64_t nframes, int kind) {
    __shared__ uint32_t s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t m = i < nwords ? class_word_mask<N>(word0 + i, nframes, kind) : 0u;
    const uint32_t s = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)__popc(m));
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(&s_sum, s);
    __syncthreads();
    if (threadIdx.x == 0) blk[blockIdx.x] = s_sum;
}

// exclusive scan of blk[0..nblk) in place by one CTA of 1024 threads;
// *total = the sum
__global__ void __launch_bounds__(1024) list_scan_kernel(uint32_t *blk, uint32_t nblk, uint64_t *total) {
    __shared__ uint64_t s_part[1024];
    const uint32_t per = (nblk + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = threadIdx.x * per, hi = min(nblk, lo + per);
    uint64_t sum = 0;
    for (uint32_t i = lo; i < hi; ++i) sum += blk[i];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        uint64_t v = threadIdx.x >= (unsigned)off ? s_part[threadIdx.x - off] : 0;
        __syncthreads();
        s_part[threadIdx.x] += v;
        __syncthreads();
    }
    uint64_t run = s_part[threadIdx.x] - sum;   // exclusive prefix of this segment
    for (uint32_t i = lo; i < hi; ++i) {
        const uint32_t c = blk[i];
        blk[i] = (uint32_t)run;
        run += c;
    }
    if (threadIdx.x == blockDim.x - 1) *total = s_part[threadIdx.x];
}

template <int N>
__global__ void __launch_bounds__(256) list_write_kernel(const uint32_t *blk, uint64_t *list, uint64_t cap,
                                                         uint64_t word0, uint64_t nwords, uint64_t nframes,
                                                         int kind, int32_t *status) {
    __shared__ uint32_t s_warp[8];
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t word = word0 + i;
    const uint32_t m = i < nwords ? class_word_mask<N>(word, nframes, kind) : 0u;
    const uint32_t c = (uint32_t)__popc(m);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // inclusive warp prefix of c
    uint32_t x = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    uint64_t pos = (uint64_t)blk[blockIdx.x] + before + (x - c);
    for (int l = 0; l < 32; ++l) {
        if ((m >> l) & 1u) {
            const uint64_t ord = (word << 5) + (uint64_t)l;
            if (pos < cap) list[pos] = kind == LIST_K4 ? ord : t_to_k(ord, N);
            else atomicOr(status, (int)MK_ST_INTERNAL);
            ++pos;
        }
    }
}

}  // namespace mkd

// ================================================================== host

namespace {

using namespace mkd;

const uint64_t kPreorders[7] = {0, 1, 4, 29, 355, 6942, 209527};
const uint64_t kEquivalences[7] = {0, 1, 2, 5, 15, 52, 203};
const uint64_t kTransitive[7] = {0, 2, 13, 171, 3994, 154303, 9415189};   // OEIS A006905
constexpr uint32_t kAllClasses = MK_CLASS_K | MK_CLASS_T | MK_CLASS_S4 | MK_CLASS_S5 | MK_CLASS_K4;
constexpr int kNumClasses = 5;   // class index c <-> bit 1 << c: K, T, S4, S5, K4

int class_count(uint32_t classes) { return __builtin_popcount(classes & kAllClasses); }

// list kind of class index c >= 2
int list_kind(int c) { return c == 2 ? LIST_S4 : c == 3 ? LIST_S5 : LIST_K4; }
uint32_t list_class_bit(int kind) { return kind == LIST_S4 ? MK_CLASS_S4 : kind == LIST_S5 ? MK_CLASS_S5 : MK_CLASS_K4; }
uint64_t list_cap(int kind, int n) {
    return kind == LIST_S4 ? kPreorders[n] : kind == LIST_S5 ? kEquivalences[n] : kTransitive[n];
}

uint64_t t_frames(int n) { return 1ull << (n * n - n); }

uint64_t layer_frames(int cls, int n) {
    switch (cls) {
    case 0: return 1ull << (n * n);
    case 1: return t_frames(n);
    case 2: return kPreorders[n];
    case 3: return kEquivalences[n];
    default: return kTransitive[n];
    }
}

// Number of T frames (compact indices) whose K index is below x: t_to_k is
// monotone, so a binary search over compact indices.
uint64_t t_rank(uint64_t x, int n) {
    uint64_t lo = 0, hi = t_frames(n);
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (t_to_k(mid, n) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Frame words [w0, w1) a layer scans: K frames of the window by index, T
// frames of the window by compact index (a contiguous range, since t_to_k is
// monotone), S4/S5 lists whole (their lanes are filtered by K index).
void layer_words(const mk_census_cfg *cfg, int c, int n, uint64_t *w0, uint64_t *w1) {
    uint64_t lo, hi;
    if (c == 0) {
        const uint64_t kf = 1ull << (n * n);
        lo = cfg->frame_lo;
        hi = cfg->frame_hi < kf ? cfg->frame_hi : kf;
    } else if (c == 1) {
        lo = t_rank(cfg->frame_lo, n);
        hi = t_rank(cfg->frame_hi, n);
    } else {
        lo = 0;
        hi = layer_frames(c, n);
    }
    *w0 = lo / 32;
    *w1 = lo >= hi ? *w0 : (hi + 31) / 32;
}

// Valuation chunks of a layer.  A layer whose grid (frame words x formula
// tiles) is too small to keep the GPU busy -- few formulas on few frames
// with many valuations each, the underfilled shapes of Table 4 -- also
// splits the valuations over grid.z, up to kFillCtas CTAs: four waves of
// census_layer_kernel's two resident CTAs on each of a GB300's 152 SMs (so
// the last wave's tail costs at most a quarter).
constexpr uint64_t kFillCtas = 4ull * 2 * 152;
constexpr uint32_t kMaxVsplit = 4096;

uint32_t layer_vsplit(const mk_census_cfg *cfg, int n, uint64_t words, int32_t nprog) {
    const int block = cfg->tune.block ? cfg->tune.block : 256;
    const int units = cfg->tune.units ? cfg->tune.units : 8;
    if (words == 0 || nprog == 0 || cfg->vsplit == 1 || units != 8 || block != 256) return 1;
    if (cfg->vsplit > 1) return cfg->vsplit;
    const uint64_t tile = cfg->tune.tile ? cfg->tune.tile : 16;
    const uint64_t wpc = words < (uint64_t)block ? words : (uint64_t)block;   // words of a CTA
    const int G = vgroups(wpc, block, units, nullptr);
    const uint64_t ctas = ((words + block - 1) / block) * ((nprog + tile - 1) / tile);
    if (ctas >= kFillCtas) return 1;
    uint64_t v = (kFillCtas + ctas - 1) / ctas;
    if (v > kMaxVsplit) v = kMaxVsplit;
    if (cfg->max_vars) {
        // no more chunks than the batch's largest valuation set has granules
        uint64_t nval = 1;
        for (int k = 0; k <= cfg->max_vars && k <= MK_MAX_VARS; ++k) {
            const uint64_t m = exhaustive_vals(k, n, cfg->samples) ? (k * n < 64 ? 1ull << (k * n) : ~0ull)
                                                                   : cfg->samples;
            if (m > nval) nval = m;
        }
        const uint64_t gran = vgran(G, units);
        const uint64_t blocks = (nval + gran - 1) / gran;
        if (v > blocks) v = blocks;
    }
    return (uint32_t)(v > 1 ? v : 1);
}

struct ListPlan {
    size_t list_off[NLISTS][7];   // [S4, S5, K4][n]: byte offset of the list
    size_t len_off[NLISTS][7];    // device count
    size_t blk_off;          // scan scratch
    size_t cursor_off;       // queue cursor
    size_t total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// lists for the classes in `classes` (bits as MK_CLASS_*) at n in [n_min, n_max]
ListPlan plan_lists(uint32_t classes, int n_min, int n_max) {
    ListPlan p;
    std::memset(&p, 0, sizeof(p));
    size_t off = 0;
    uint64_t max_blk = 1;
    for (int c = 0; c < NLISTS; ++c) {
        if (!(classes & list_class_bit(c))) continue;
        for (int n = n_min; n <= n_max; ++n) {
            const uint64_t cap = list_cap(c, n);
            p.len_off[c][n] = off;
            off = align256(off + 8);
            p.list_off[c][n] = off;
            off = align256(off + cap * 8);
            const uint64_t scanned = c == LIST_K4 ? (1ull << (n * n)) : t_frames(n);
            const uint64_t nw = (scanned + 31) / 32;
            const uint64_t nb = (nw + 255) / 256;
            if (nb > max_blk) max_blk = nb;
        }
    }
    p.blk_off = off;
    off = align256(off + max_blk * 4);
    p.cursor_off = off;
    p.total = off;
    return p;
}

// Lists plus, after them, the frame-word bitmap that split layers OR their
// refuted lanes into (one region, reused layer after layer).
struct CensusPlan {
    ListPlan lists;
    size_t rf_off, rf_bytes;   // frame bitmap of the largest split layer
    size_t done_off;           // then one CTA counter per formula tile
    size_t clear_words;        // bitmap + counters, cleared at the start
    size_t total;
};

CensusPlan plan_census(const mk_census_cfg *cfg, int32_t nprog) {
    CensusPlan p;
    p.lists = plan_lists(cfg->classes, cfg->n_min, cfg->n_max);
    p.rf_off = align256(p.lists.total);
    p.rf_bytes = 0;
    for (int c = 0; c < kNumClasses; ++c) {
        if (!(cfg->classes & (1u << c))) continue;
        for (int n = cfg->n_min; n <= cfg->n_max; ++n) {
            uint64_t w0, w1;
            layer_words(cfg, c, n, &w0, &w1);
            if (layer_vsplit(cfg, n, w1 - w0, nprog) > 1) {
                const size_t b = (size_t)nprog * (w1 - w0) * 4;
                if (b > p.rf_bytes) p.rf_bytes = b;
            }
        }
    }
    const uint64_t tile = cfg->tune.tile ? cfg->tune.tile : 16;
    p.done_off = p.rf_off + p.rf_bytes;
    p.clear_words = 0;
    p.total = p.lists.total;
    if (p.rf_bytes) {
        const size_t done_bytes = (size_t)((nprog + tile - 1) / tile) * 4;
        p.clear_words = (p.rf_bytes + done_bytes) / 4;
        p.total = align256(p.done_off + done_bytes);
    }
    return p;
}

int check_cfg(const mk_census_cfg *cfg, int32_t nprog) {
    if (!cfg || nprog < 0) return MK_E_ARG;
    if ((cfg->classes & kAllClasses) == 0 || (cfg->classes & ~kAllClasses)) return MK_E_ARG;
    if (cfg->n_min < 1 || cfg->n_max > MK_MAX_WORLDS_EXH || cfg->n_min > cfg->n_max) return MK_E_ARG;
    if ((cfg->samples == 0) != (cfg->d_samples == nullptr)) return MK_E_ARG;
    if (cfg->frame_lo > cfg->frame_hi) return MK_E_ARG;
    if (cfg->vsplit > 4096) return MK_E_ARG;
    const mk_tune &t = cfg->tune;
    if (t.block && t.block != 128 && t.block != 256) return MK_E_ARG;
    if (t.tile > MAX_TILE) return MK_E_ARG;
    if (cfg->max_depth > MK_MAX_STACK) return MK_E_ARG;
    if (t.units && t.units != 2 && t.units != 4 && t.units != 8) return MK_E_ARG;
    return MK_OK;
}

// Dynamic shared memory above 48 KB needs a per-kernel attribute; it is
// raised when a kernel first needs more (so a call made once before a
// stream capture leaves nothing to set during the capture).

template <typename K>
void ensure_smem(K kern, size_t bytes) {
    ensure_dynamic_smem((const void *)kern, bytes);
}

template <int N, int U, int BLOCK>
void launch_layer_b(const LayerArgs &a, cudaStream_t s) {
    const uint64_t words = a.t.w1 > a.t.w0 ? a.t.w1 - a.t.w0 : 0;
    if (words == 0 || a.t.np == 0) return;
    dim3 grid((unsigned)((words + BLOCK - 1) / BLOCK), (unsigned)((a.t.np + a.tile - 1) / a.tile),
              a.sp.vsplit);
    const size_t sm = TileSmem<N, U, BLOCK>::total(a.tile, a.t.depth);
    // split layers (default tune only) take the split variant
    auto kern = census_layer_kernel<N, U, BLOCK, false>;
    if constexpr (kSplitTune<U, BLOCK>)
        if (a.sp.vsplit > 1) kern = census_layer_kernel<N, U, BLOCK, true>;
    ensure_smem(kern, sm);
    kern<<<grid, BLOCK, sm, s>>>(a);
}

template <int N, int U>
void launch_layer_u(const LayerArgs &a, int block, cudaStream_t s) {
    if (block == 128) launch_layer_b<N, U, 128>(a, s);
    else launch_layer_b<N, U, 256>(a, s);
}

template <int N>
void launch_layer(const LayerArgs &a, int block, int units, cudaStream_t s) {
    if (units == 2) launch_layer_u<N, 2>(a, block, s);
    else if (units == 8) launch_layer_u<N, 8>(a, block, s);
    else launch_layer_u<N, 4>(a, block, s);
}

void launch_layer_n(int n, const LayerArgs &a, int block, int units, cudaStream_t s) {
    switch (n) {
    case 1: launch_layer<1>(a, block, units, s); break;
    case 2: launch_layer<2>(a, block, units, s); break;
    case 3: launch_layer<3>(a, block, units, s); break;
    case 4: launch_layer<4>(a, block, units, s); break;
    case 5: launch_layer<5>(a, block, units, s); break;
    case 6: launch_layer<6>(a, block, units, s); break;
    }
}

// List of kind c at N worlds: S4/S5 filter the T frames, K4 the K frames,
// those in frame words [w0, w1) of the scanned enumeration (a census whose
// K-index window leaves out the rest lists only the window's words).
template <int N>
void launch_list(uint8_t *ws, const ListPlan &p, int c, int32_t *status, cudaStream_t s, uint64_t w0,
                 uint64_t w1) {
    const uint64_t nf = c == LIST_K4 ? (1ull << (N * N)) : t_frames(N);
    const uint64_t all = (nf + 31) / 32;
    if (w1 > all) w1 = all;
    if (w0 > w1) w0 = w1;
    const uint64_t nw = w1 - w0;
    const unsigned nb = (unsigned)((nw + 255) / 256 > 0 ? (nw + 255) / 256 : 1);
    uint32_t *blk = (uint32_t *)(ws + p.blk_off);
    uint64_t *len = (uint64_t *)(ws + p.len_off[c][N]);
    uint64_t *list = (uint64_t *)(ws + p.list_off[c][N]);
    const uint64_t cap = list_cap(c, N);
    list_count_kernel<N><<<nb, 256, 0, s>>>(blk, w0, nw, nf, c);
    list_scan_kernel<<<1, 1024, 0, s>>>(blk, nb, len);
    list_write_kernel<N><<<nb, 256, 0, s>>>(blk, list, cap, w0, nw, nf, c, status);
}

void launch_list_n(int n, uint8_t *ws, const ListPlan &p, int c, int32_t *status, cudaStream_t s,
                   uint64_t w0 = 0, uint64_t w1 = ~0ull) {
    switch (n) {
    case 1: launch_list<1>(ws, p, c, status, s, w0, w1); break;
    case 2: launch_list<2>(ws, p, c, status, s, w0, w1); break;
    case 3: launch_list<3>(ws, p, c, status, s, w0, w1); break;
    case 4: launch_list<4>(ws, p, c, status, s, w0, w1); break;
    case 5: launch_list<5>(ws, p, c, status, s, w0, w1); break;
    case 6: launch_list<6>(ws, p, c, status, s, w0, w1); break;
    }
}

void launch_init(mk_result *out, size_t n, cudaStream_t s, uint32_t *clear = nullptr, size_t nclear = 0) {
    const size_t m = n > nclear ? n : nclear;
    if (!m) return;
    const size_t blocks = (m + 255) / 256;
    init_results_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(out, n, clear, nclear);
}

}  // namespace

extern "C" uint64_t mk_class_frames(uint32_t cls, int32_t n) {
    if (n < 1 || n > MK_MAX_WORLDS_EXH) return 0;
    switch (cls) {
    case MK_CLASS_K: return 1ull << (n * n);
    case MK_CLASS_T: return t_frames(n);
    case MK_CLASS_S4: return kPreorders[n];
    case MK_CLASS_S5: return kEquivalences[n];
    case MK_CLASS_K4: return kTransitive[n];
    default: return 0;
    }
}

extern "C" int32_t mk_census_launches(const mk_census_cfg *cfg, int32_t nprog) {
    if (check_cfg(cfg, nprog) != MK_OK) return -1;
    const int nn = cfg->n_max - cfg->n_min + 1;
    int lists = 0;
    for (int c = 0; c < NLISTS; ++c) lists += (cfg->classes & list_class_bit(c)) ? 1 : 0;
    if (nprog == 0) return lists * nn * 3;
    int layers = 0;
    for (int c = 0; c < kNumClasses; ++c)
        if (cfg->classes & (1u << c))
            for (int n = cfg->n_min; n <= cfg->n_max; ++n) {
                uint64_t w0, w1;
                layer_words(cfg, c, n, &w0, &w1);
                if (w1 == w0) continue;
                ++layers;
            }
    return 1 + lists * nn * 3 + layers;
}

extern "C" size_t mk_census_workspace_size(const mk_census_cfg *cfg, int32_t nprog) {
    if (check_cfg(cfg, nprog) != MK_OK) return 0;
    return plan_census(cfg, nprog).total;
}

// The least workspace mk_census accepts: the frame lists alone.  With less
// than mk_census_workspace_size it runs every layer unsplit.
size_t mk_census_min_workspace(const mk_census_cfg *cfg, int32_t nprog) {
    if (check_cfg(cfg, nprog) != MK_OK) return 0;
    return plan_lists(cfg->classes, cfg->n_min, cfg->n_max).total;
}

extern "C" int mk_census(const mk_program *d_progs, int32_t nprog, const mk_census_cfg *cfg,
                         mk_result *d_out, int32_t *d_status, void *d_workspace, size_t ws_bytes,
                         void *stream) {
    int rc = check_cfg(cfg, nprog);
    if (rc != MK_OK) return rc;
    if (nprog > 0 && (!d_progs || !d_out)) return MK_E_ARG;
    if (!d_status) return MK_E_ARG;
    const CensusPlan cplan = plan_census(cfg, nprog);
    const ListPlan &plan = cplan.lists;
    if (!d_workspace || ws_bytes < plan.total) return MK_E_WORKSPACE;
    const bool may_split = ws_bytes >= cplan.total;
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t *ws = (uint8_t *)d_workspace;

    const int ncls = class_count(cfg->classes);
    const int nn = cfg->n_max - cfg->n_min + 1;
    launch_init(d_out, (size_t)nprog * ncls * nn, s, may_split ? (uint32_t *)(ws + cplan.rf_off) : nullptr,
                may_split ? cplan.clear_words : 0);

    const int block = cfg->tune.block ? cfg->tune.block : 256;
    const int tile = cfg->tune.tile ? cfg->tune.tile : 16;
    const int depth = cfg->max_depth ? cfg->max_depth : MK_MAX_STACK;
    const int units = cfg->tune.units ? cfg->tune.units : 8;

    // class lists for S4 / S5 / K4, over the words of the K-index window
    // (K4 scans K frames by index, S4/S5 T frames by compact index, which is
    // monotone in the K index)
    for (int c = 0; c < NLISTS; ++c) {
        if (!(cfg->classes & list_class_bit(c))) continue;
        for (int n = cfg->n_min; n <= cfg->n_max; ++n) {
            uint64_t w0, w1;
            layer_words(cfg, c == LIST_K4 ? 0 : 1, n, &w0, &w1);
            launch_list_n(n, ws, plan, c, d_status, s, w0, w1);
        }
    }

    int ci = 0;
    for (int c = 0; c < kNumClasses; ++c) {
        const uint32_t bit = 1u << c;
        if (!(cfg->classes & bit)) continue;
        for (int n = cfg->n_min; n <= cfg->n_max; ++n) {
            LayerArgs a;
            std::memset(&a, 0, sizeof(a));
            TileCtx &t = a.t;
            t.progs = d_progs;
            t.np = nprog;
            a.tile = tile;
            t.S = cfg->samples;
            t.samples = cfg->samples ? cfg->d_samples + (size_t)n * cfg->samples : nullptr;
            t.f_lo = cfg->frame_lo;
            t.f_hi = cfg->frame_hi;
            const uint64_t kframes = 1ull << (n * n);
            t.full_range = (cfg->frame_lo == 0 && cfg->frame_hi >= kframes) ? 1 : 0;
            t.out = d_out;
            t.out_stride = ncls * nn;
            t.out_off = ci * nn + (n - cfg->n_min);
            t.depth = depth;
            t.status = d_status;
            layer_words(cfg, c, n, &t.w0, &t.w1);
            if (c == 0) {
                t.src = SRC_K;
                t.nframes = kframes;
            } else if (c == 1) {
                t.src = SRC_T;
                t.nframes = t_frames(n);
            } else {
                const int li = list_kind(c);
                t.src = SRC_LIST;
                t.flist = (const uint64_t *)(ws + plan.list_off[li][n]);
                a.list_len = (const uint64_t *)(ws + plan.len_off[li][n]);
                t.nframes = list_cap(li, n);
            }
            if (t.w1 == t.w0) continue;
            a.sp.vsplit = may_split ? layer_vsplit(cfg, n, t.w1 - t.w0, nprog) : 1;
            if (a.sp.vsplit > 1) {
                a.sp.rf_bits = (uint32_t *)(ws + cplan.rf_off);
                a.sp.rf_w0 = t.w0;
                a.sp.rf_words = t.w1 - t.w0;
                a.rf_done = (uint32_t *)(ws + cplan.done_off);
            }
            launch_layer_n(n, a, block, units, s);
        }
        ++ci;
    }
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}

// ------------------------------------------------------ uneven batches

namespace {

struct PlanHeader {             // at offset 0 of every plan
    uint32_t magic, version;
    uint32_t nitems, nlist;
    uint32_t list_off, items_off;
    uint32_t njobs, reserved;
};
constexpr uint32_t kPlanMagic = 0x4E414C50u;   // "PLAN"

uint64_t valuations_of(int k, int n, uint32_t S) {
    return exhaustive_vals(k, n, S) ? (1ull << (k * n)) : S;
}

double program_ops(const mk_program &p, int n) {
    return (double)n * p.n_bool + (double)n * n * p.n_modal + n + 4.0 * p.n_instr;
}

int length_bucket(const mk_program &p) {
    return p.n_instr <= 8 ? 0 : p.n_instr <= 16 ? 1 : p.n_instr <= 32 ? 2 : 3;
}

}  // namespace

extern "C" int mk_plan_uneven(const mk_program *h_progs, int32_t nprog, const mk_job *h_jobs, int32_t njobs,
                              uint32_t samples, const uint16_t *tiles, const mk_tune *tune, void *h_plan,
                              size_t plan_bytes, mk_plan_info *info) {
    if (!h_progs || !h_jobs || !info || nprog < 0 || njobs < 0) return MK_E_ARG;
    const int block = tune && tune->block ? tune->block : 256;
    const int units = tune && tune->units ? tune->units : 8;
    if ((block != 128 && block != 256) || (units != 4 && units != 8)) return MK_E_ARG;
    uint16_t tl[4] = {16, 16, 16, 16};
    if (tiles)
        for (int i = 0; i < 4; ++i) {
            if (tiles[i] < 1 || tiles[i] > MAX_TILE) return MK_E_ARG;
            tl[i] = tiles[i];
        }
    int n_max = 1, depth = 1;
    for (int j = 0; j < njobs; ++j) {
        const mk_job &jb = h_jobs[j];
        if (jb.prog < 0 || jb.prog >= nprog || jb.cls > 3 || jb.n_max < 1 || jb.n_max > MK_MAX_WORLDS_EXH)
            return MK_E_ARG;
        if (jb.n_max > n_max) n_max = jb.n_max;
        const int d = h_progs[jb.prog].depth;
        if (d > depth) depth = d;
    }
    if (depth > MK_MAX_STACK) return MK_E_ARG;

    // job list and items: layer (c, n) -> jobs sorted by cost -> tiles -> word ranges
    struct Item { mk_work_item w; double cost; };
    std::vector<uint32_t> jlist;
    std::vector<Item> items;
    double total_ops = 0;
    for (int c = 0; c < 4; ++c) {
        for (int n = 1; n <= n_max; ++n) {
            std::vector<std::pair<double, uint32_t>> members;
            for (int j = 0; j < njobs; ++j) {
                const mk_job &jb = h_jobs[j];
                if (jb.cls != c || jb.n_max < n) continue;
                const mk_program &p = h_progs[jb.prog];
                const double cost = (double)valuations_of(p.nvars, n, samples) * program_ops(p, n);
                members.push_back({cost, (uint32_t)j});
            }
            if (members.empty()) continue;
            std::stable_sort(members.begin(), members.end(), [&](const auto &x, const auto &y) {
                const int bx = length_bucket(h_progs[h_jobs[x.second].prog]);
                const int by = length_bucket(h_progs[h_jobs[y.second].prog]);
                return bx != by ? bx > by : x.first > y.first;
            });
            const uint64_t words = (layer_frames(c, n) + 31) / 32;
            // items of a few thousand words, at least one CTA step each
            const uint64_t chunk = std::max<uint64_t>((uint64_t)block, std::min<uint64_t>(words, (uint64_t)block * 8));
            size_t i = 0;
            while (i < members.size()) {
                const int b = length_bucket(h_progs[h_jobs[members[i].second].prog]);
                size_t e = i;
                double tile_cost = 0;
                while (e < members.size() && e - i < tl[b] &&
                       length_bucket(h_progs[h_jobs[members[e].second].prog]) == b) {
                    tile_cost += members[e].first;
                    ++e;
                }
                const uint32_t lbeg = (uint32_t)jlist.size();
                for (size_t q = i; q < e; ++q) jlist.push_back(members[q].second);
                for (uint64_t w = 0; w < words; w += chunk) {
                    Item it;
                    it.w.lbeg = lbeg;
                    it.w.np = (uint16_t)(e - i);
                    it.w.n = (uint8_t)n;
                    it.w.cls = (uint8_t)c;
                    it.w.w0 = w;
                    it.w.w1 = std::min(words, w + chunk);
                    it.cost = tile_cost * (double)(it.w.w1 - it.w.w0);
                    items.push_back(it);
                }
                total_ops += tile_cost * (double)layer_frames(c, n) / 32.0;
                i = e;
            }
        }
    }
    // longest first, so the queue's tail is made of short items
    std::stable_sort(items.begin(), items.end(), [](const Item &a, const Item &b) { return a.cost > b.cost; });

    std::memset(info, 0, sizeof(*info));
    const size_t list_off = align256(sizeof(PlanHeader));
    const size_t items_off = align256(list_off + jlist.size() * 4);
    info->bytes = items_off + items.size() * sizeof(mk_work_item);
    info->nitems = (uint32_t)items.size();
    info->nlist = (uint32_t)jlist.size();
    info->list_off = (uint32_t)list_off;
    info->items_off = (uint32_t)items_off;
    info->n_max = (uint8_t)n_max;
    info->max_depth = (uint8_t)depth;
    info->block = (uint16_t)block;
    info->units = (uint16_t)units;
    info->tile_cap = (uint16_t)std::max(std::max(tl[0], tl[1]), std::max(tl[2], tl[3]));
    info->ops = total_ops;
    if (!h_plan) return MK_OK;
    if (plan_bytes < info->bytes) return MK_E_WORKSPACE;
    uint8_t *pb = (uint8_t *)h_plan;
    std::memset(pb, 0, info->bytes);
    PlanHeader h = {kPlanMagic, 1, info->nitems, info->nlist, info->list_off, info->items_off, (uint32_t)njobs, 0};
    std::memcpy(pb, &h, sizeof(h));
    if (!jlist.empty()) std::memcpy(pb + list_off, jlist.data(), jlist.size() * 4);
    for (size_t i = 0; i < items.size(); ++i) std::memcpy(pb + items_off + i * sizeof(mk_work_item), &items[i].w, sizeof(mk_work_item));
    return MK_OK;
}

extern "C" size_t mk_uneven_workspace_size(const mk_plan_info *info) {
    if (!info || info->n_max < 1 || info->n_max > MK_MAX_WORLDS_EXH) return 0;
    const ListPlan p = plan_lists(MK_CLASS_S4 | MK_CLASS_S5, 1, info->n_max);
    return p.total + 256;   // + the queue cursor
}

namespace {

template <int NM, int U, int BLOCK>
void launch_queue(const QueueArgs &a, int depth, cudaStream_t s) {
    const size_t sm = TileSmem<NM, U, BLOCK>::total(a.tile_cap, depth);
    auto kern = census_queue_kernel<NM, U, BLOCK>;
    ensure_smem(kern, sm);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, sm);
    if (per_sm < 1) per_sm = 1;
    kern<<<(unsigned)(sms * per_sm), BLOCK, sm, s>>>(a);
}

}  // namespace

extern "C" int mk_census_uneven(const mk_program *d_progs, const mk_job *d_jobs, int32_t njobs, const void *d_plan,
                                const mk_plan_info *info, uint32_t samples, const uint32_t *d_samples,
                                mk_result *d_out, int32_t *d_status, void *d_workspace, size_t ws_bytes,
                                void *stream) {
    if (!info || njobs < 0 || !d_status) return MK_E_ARG;
    if (njobs > 0 && (!d_progs || !d_jobs || !d_plan || !d_out)) return MK_E_ARG;
    if ((samples == 0) != (d_samples == nullptr)) return MK_E_ARG;
    if (info->n_max < 1 || info->n_max > MK_MAX_WORLDS_EXH || info->max_depth < 1 ||
        info->max_depth > MK_MAX_STACK || info->tile_cap < 1 || info->tile_cap > MAX_TILE)
        return MK_E_ARG;
    const size_t need = mk_uneven_workspace_size(info);
    if (!d_workspace || ws_bytes < need) return MK_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t *ws = (uint8_t *)d_workspace;
    const ListPlan lp = plan_lists(MK_CLASS_S4 | MK_CLASS_S5, 1, info->n_max);

    launch_init(d_out, (size_t)njobs * 6, s);
    if (njobs == 0 || info->nitems == 0) return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
    for (int c = 0; c < 2; ++c)
        for (int n = 1; n <= info->n_max; ++n) launch_list_n(n, ws, lp, c, d_status, s);
    uint32_t *cursor = (uint32_t *)(ws + lp.cursor_off);
    reset_cursor_kernel<<<1, 1, 0, s>>>(cursor);

    QueueArgs a;
    std::memset(&a, 0, sizeof(a));
    a.progs = d_progs;
    a.jobs = d_jobs;
    a.jlist = (const uint32_t *)((const uint8_t *)d_plan + info->list_off);
    a.items = (const mk_work_item *)((const uint8_t *)d_plan + info->items_off);
    a.nitems = info->nitems;
    a.cursor = cursor;
    for (int c = 0; c < 2; ++c)
        for (int n = 1; n <= info->n_max; ++n) {
            a.lists[c][n] = (const uint64_t *)(ws + lp.list_off[c][n]);
            a.list_len[c][n] = (const uint64_t *)(ws + lp.len_off[c][n]);
        }
    a.samples = d_samples;
    a.S = samples;
    a.depth = info->max_depth;
    a.tile_cap = info->tile_cap;
    a.out = d_out;
    a.status = d_status;
    const bool six = info->n_max > 5;
    const bool u8 = info->units != 4;
    const bool b256 = info->block != 128;
    if (six) {
        if (u8) b256 ? launch_queue<6, 8, 256>(a, a.depth, s) : launch_queue<6, 8, 128>(a, a.depth, s);
        else b256 ? launch_queue<6, 4, 256>(a, a.depth, s) : launch_queue<6, 4, 128>(a, a.depth, s);
    } else {
        if (u8) b256 ? launch_queue<5, 8, 256>(a, a.depth, s) : launch_queue<5, 8, 128>(a, a.depth, s);
        else b256 ? launch_queue<5, 4, 256>(a, a.depth, s) : launch_queue<5, 4, 128>(a, a.depth, s);
    }
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}
