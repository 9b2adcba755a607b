// mk_census.cu -- the census: Alg. 1 (fused corpus scan) over every
// selected (class, n) layer, redesigned for sm_103a.
//
// Per layer one grid launch: blockIdx.x picks BLOCK frame words, blockIdx.y
// a tile of formulas.  A thread owns one frame word (32 consecutive frames,
// synthesised from its index: no frame is read from HBM) and keeps its n*n
// edge words in registers.  For each formula of the tile it walks the
// layer's valuations U at a time, interpreting the postfix program on an
// accumulator in registers (mk_eval.cuh); atom truth sets are read from
// shared-memory rows staged once per CTA (one row per valuation, re-staged
// in chunks when a formula needs more rows than fit).  Refuted lanes are
// ~(AND_w t[w]) & valid; the count is a popcount, the first witness the
// lowest refuted lane at the first valuation that refutes it.  Reduction:
// warp (__reduce_add_sync, ballot + shuffle for the witness), CTA (shared
// atomics), then one global atomicAdd / atomicMin per CTA and formula
// (Sec. 4's hierarchical reduction).
//
// Classes: K frames are every index; T frames are enumerated by their
// compact index (diagonal forced on); S4 and S5 frames are first listed by a
// three-kernel filter over the T frames (count, scan, write; ascending K
// order) into the caller's workspace, then scanned from that list.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "mk.h"
#include "mk_eval.cuh"

namespace mkd {

constexpr int SRC_K = 0, SRC_T = 1, SRC_LIST = 2;
constexpr int ROW_CAP = 128;          // atom rows staged at a time
constexpr int OPS_STRIDE = MK_MAX_CODE + 2;   // decoded ops per program (END + prefetch pad)

struct LayerArgs {
    const mk_program *progs;
    int32_t nprog;
    int32_t tile;
    const uint32_t *samples;   // this layer's sampled valuations (device)
    uint32_t S;
    int32_t src;
    const uint64_t *list;      // SRC_LIST: K indices, ascending
    const uint64_t *list_len;  // SRC_LIST: device count
    uint64_t word_lo, word_hi; // frame words to scan
    uint64_t nframes;          // frames in the source (by ordinal)
    uint64_t f_lo, f_hi;       // K-index filter
    int32_t full_range;        // 1: f_lo/f_hi do not cut this layer
    mk_result *out;
    int32_t out_stride, out_off;
    int32_t depth;             // stack entries provided (programs deeper are rejected)
    int32_t *status;
};

// Shared memory of one census CTA.
template <int N, int U, int BLOCK>
struct CensusSmem {
    static constexpr size_t code_bytes(int tile) { return ((size_t)tile * OPS_STRIDE * 3 + 15) & ~(size_t)15; }
    static constexpr size_t meta_bytes(int tile) { return (size_t)tile * 32; }   // 2 int + 3 u64
    // ROW_CAP rows plus U rows of slack read (and masked) by a partial last step
    static constexpr size_t row_bytes() { return (size_t)(ROW_CAP + U) * RowShape<N>::WORDS * 4; }
    static constexpr size_t stack_bytes(int depth) { return (size_t)depth * U * N * BLOCK * 4; }
    static size_t total(int tile, int depth) {
        return code_bytes(tile) + meta_bytes(tile) + row_bytes() + stack_bytes(depth);
    }
};

// K index of lane l of a word, for each source.
template <int N>
__device__ __forceinline__ uint64_t lane_kindex(const LayerArgs &a, uint64_t word, int l) {
    const uint64_t ord = (word << 5) + (uint64_t)l;
    if (a.src == SRC_K) return ord;
    if (a.src == SRC_T) return t_to_k(ord, N);
    return a.list[ord];
}

template <int N>
__device__ __forceinline__ uint32_t build_word(const LayerArgs &a, uint64_t word, uint64_t nframes,
                                               uint32_t (&E)[N * N]) {
    const uint64_t base = word << 5;
    uint32_t valid = 0;
    if (base < nframes) {
        const uint64_t left = nframes - base;
        valid = left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
    }
    if (a.src == SRC_K) {
        k_frame_word<N>(word, E);
    } else if (a.src == SRC_T) {
        t_frame_word<N>(word, E);
    } else {
        const int cnt = __popc(valid);
        list_frame_word<N>(a.list + base, cnt, E);
    }
    if (!a.full_range && valid) {
        for (int l = 0; l < 32; ++l) {
            if ((valid >> l) & 1u) {
                const uint64_t f = lane_kindex<N>(a, word, l);
                if (f < a.f_lo || f >= a.f_hi) valid &= ~(1u << l);
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

template <int N, int U, int BLOCK>
__global__ void __launch_bounds__(BLOCK) census_layer_kernel(LayerArgs a) {
    using SM = CensusSmem<N, U, BLOCK>;
    constexpr int RW = RowShape<N>::WORDS;
    extern __shared__ __align__(16) uint8_t smem[];
    const int tile = a.tile;
    uint16_t *s_offs = (uint16_t *)smem;
    uint8_t *s_ops = smem + (size_t)tile * OPS_STRIDE * 2;
    int *s_nin = (int *)(smem + SM::code_bytes(tile));
    int *s_k = s_nin + tile;
    unsigned long long *s_cm = (unsigned long long *)(s_k + tile);
    unsigned long long *s_rf = s_cm + tile;
    unsigned long long *s_key = s_rf + tile;
    uint32_t *s_rows = (uint32_t *)(smem + SM::code_bytes(tile) + SM::meta_bytes(tile));
    uint32_t *s_stack = (uint32_t *)((uint8_t *)s_rows + SM::row_bytes()) + threadIdx.x;

    const int p0 = blockIdx.y * tile;
    const int np = min(tile, a.nprog - p0);

    // stage the tile's programs (checked once per CTA)
    for (int i = threadIdx.x; i < np; i += BLOCK) {
        const mk_program &p = a.progs[p0 + i];
        int nin = -1;
        if (program_ok(p) && p.depth <= a.depth) {
            nin = p.n_instr;
            if (exhaustive_vals(p.nvars, N, a.S) && p.nvars * N > 24) {
                nin = -1;
                if (blockIdx.x == 0) atomicOr(a.status, (int)MK_ST_LIMIT);
            }
        } else if (blockIdx.x == 0) {
            atomicOr(a.status, (int)MK_ST_PROGRAM);
        }
        s_nin[i] = nin;
        s_k[i] = p.nvars;
        s_cm[i] = 0;
        s_rf[i] = 0;
        s_key[i] = ~0ull;
        if (nin >= 0) decode_program<N, U, BLOCK>(p, s_ops + i * OPS_STRIDE, s_offs + i * OPS_STRIDE);
    }

    uint64_t nframes = a.nframes;
    if (a.src == SRC_LIST) {
        const uint64_t len = *a.list_len;
        nframes = len < nframes ? len : nframes;
    }
    const uint64_t word = a.word_lo + (uint64_t)blockIdx.x * BLOCK + threadIdx.x;
    uint32_t E[1][N * N];
    uint32_t valid = 0;
    if (word < a.word_hi) valid = build_word<N>(a, word, nframes, E[0]);
    else {
#pragma unroll
        for (int e = 0; e < N * N; ++e) E[0][e] = 0;
    }
    const int lane = threadIdx.x & 31;
    int rows_kind = -1;          // staged rows: 0 exhaustive, 1 sampled
    uint32_t rows_c0 = 0;
    __syncthreads();

    for (int fi = 0; fi < np; ++fi) {
        const int nin = s_nin[fi];
        if (nin < 0) continue;
        const int k = s_k[fi];
        const bool exh = exhaustive_vals(k, N, a.S);
        const uint32_t nval = exh ? (1u << (k * N)) : a.S;
        const uint8_t *ops = s_ops + fi * OPS_STRIDE;
        const uint16_t *offs = s_offs + fi * OPS_STRIDE;
        uint32_t cnt = 0, rf = 0, best_j = 0;
        int best_l = 32, best_w = 0;
        for (uint32_t c0 = 0; c0 < nval; c0 += ROW_CAP) {
            const uint32_t cn = min((uint32_t)ROW_CAP, nval - c0);
            // uniform across the CTA: every thread takes the same decisions.
            // Exhaustive rows are staged ROW_CAP at a time, sampled ones up to S.
            if (rows_kind != (exh ? 0 : 1) || rows_c0 != c0) {
                __syncthreads();
                stage_rows<N, BLOCK>(s_rows, exh, a.samples, c0,
                                     exh ? (uint32_t)ROW_CAP : min((uint32_t)ROW_CAP, a.S - c0));
                __syncthreads();
                rows_kind = exh ? 0 : 1;
                rows_c0 = c0;
            }
            // valid lanes per unit: all lanes of the frame word, except the
            // units past the chunk's end in its last step
            uint32_t vm[U];
#pragma unroll
            for (int u = 0; u < U; ++u) vm[u] = valid;
            for (uint32_t jj = 0; jj < cn; jj += U) {
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
        const uint32_t f_sum = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)__popc(rf));
        const uint32_t hit = __ballot_sync(0xFFFFFFFFu, best_l < 32);
        uint64_t key = ~0ull;
        if (hit) {
            // lanes hold ascending frames, so the lowest hit lane has the least frame
            const int src_lane = __ffs(hit) - 1;
            uint64_t my = 0;
            if (lane == src_lane)
                my = (lane_kindex<N>(a, word, best_l) << 27) | ((uint64_t)best_j << 3) | (uint64_t)best_w;
            key = __shfl_sync(0xFFFFFFFFu, my, src_lane);
        }
        if (lane == 0) {
            const uint64_t c = ((uint64_t)c_hi << 16) + c_lo;
            if (c) atomicAdd(&s_cm[fi], (unsigned long long)c);
            if (f_sum) atomicAdd(&s_rf[fi], (unsigned long long)f_sum);
            if (hit) atomicMin(&s_key[fi], (unsigned long long)key);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < np; i += BLOCK) {
        mk_result *o = a.out + (size_t)(p0 + i) * a.out_stride + a.out_off;
        if (s_cm[i]) atomicAdd((unsigned long long *)&o->cm_count, s_cm[i]);
        if (s_rf[i]) atomicAdd((unsigned long long *)&o->frames_refuted, s_rf[i]);
        if (s_key[i] != ~0ull) atomicMin((unsigned long long *)&o->witness_key, s_key[i]);
    }
}

__global__ void init_results_kernel(mk_result *out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        out[i].cm_count = 0;
        out[i].frames_refuted = 0;
        out[i].witness_key = ~0ull;
    }
}

// ---------------------------------------------------- S4 / S5 frame lists

template <int N>
__device__ __forceinline__ uint32_t class_word_mask(uint64_t word, uint64_t tframes, bool sym) {
    uint32_t E[N * N];
    t_frame_word<N>(word, E);
    const uint64_t base = word << 5;
    uint32_t valid = 0;
    if (base < tframes) {
        const uint64_t left = tframes - base;
        valid = left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
    }
    return valid & preorder_mask<N>(E, sym);
}

template <int N>
__global__ void __launch_bounds__(256) list_count_kernel(uint32_t *blk, uint64_t nwords, uint64_t tframes, int sym) {
    __shared__ uint32_t s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    const uint64_t word = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t m = word < nwords ? class_word_mask<N>(word, tframes, sym != 0) : 0u;
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
                                                         uint64_t nwords, uint64_t tframes, int sym,
                                                         int32_t *status) {
    __shared__ uint32_t s_warp[8];
    const uint64_t word = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t m = word < nwords ? class_word_mask<N>(word, tframes, sym != 0) : 0u;
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
            if (pos < cap) list[pos] = t_to_k((word << 5) + (uint64_t)l, N);
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

int class_count(uint32_t classes) { return __builtin_popcount(classes & 15u); }

uint64_t t_frames(int n) { return 1ull << (n * n - n); }

struct CensusPlan {
    size_t list_off[2][7];   // [S4, S5][n]: byte offset of the list
    size_t len_off[2][7];    // device count
    size_t blk_off;          // scan scratch
    size_t total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

CensusPlan plan_workspace(const mk_census_cfg *cfg) {
    CensusPlan p;
    std::memset(&p, 0, sizeof(p));
    size_t off = 0;
    uint64_t max_blk = 1;
    for (int c = 0; c < 2; ++c) {
        const uint32_t bit = c == 0 ? MK_CLASS_S4 : MK_CLASS_S5;
        if (!(cfg->classes & bit)) continue;
        for (int n = cfg->n_min; n <= cfg->n_max; ++n) {
            const uint64_t cap = c == 0 ? kPreorders[n] : kEquivalences[n];
            p.len_off[c][n] = off;
            off = align256(off + 8);
            p.list_off[c][n] = off;
            off = align256(off + cap * 8);
            const uint64_t nw = (t_frames(n) + 31) / 32;
            const uint64_t nb = (nw + 255) / 256;
            if (nb > max_blk) max_blk = nb;
        }
    }
    p.blk_off = off;
    off = align256(off + max_blk * 4);
    p.total = off;
    return p;
}

int check_cfg(const mk_census_cfg *cfg, int32_t nprog) {
    if (!cfg || nprog < 0) return MK_E_ARG;
    if ((cfg->classes & 15u) == 0 || (cfg->classes & ~15u)) return MK_E_ARG;
    if (cfg->n_min < 1 || cfg->n_max > MK_MAX_WORLDS_EXH || cfg->n_min > cfg->n_max) return MK_E_ARG;
    if ((cfg->samples == 0) != (cfg->d_samples == nullptr)) return MK_E_ARG;
    if (cfg->frame_lo > cfg->frame_hi) return MK_E_ARG;
    const mk_tune &t = cfg->tune;
    if (t.block && t.block != 128 && t.block != 256) return MK_E_ARG;
    if (t.tile > 64) return MK_E_ARG;
    if (cfg->max_depth > MK_MAX_STACK) return MK_E_ARG;
    if (t.units && t.units != 2 && t.units != 4 && t.units != 8) return MK_E_ARG;
    return MK_OK;
}

template <int N, int U, int BLOCK>
void launch_layer_b(const LayerArgs &a, cudaStream_t s) {
    const uint64_t words = a.word_hi > a.word_lo ? a.word_hi - a.word_lo : 0;
    if (words == 0 || a.nprog == 0) return;
    dim3 grid((unsigned)((words + BLOCK - 1) / BLOCK), (unsigned)((a.nprog + a.tile - 1) / a.tile));
    const size_t sm = CensusSmem<N, U, BLOCK>::total(a.tile, a.depth);
    auto kern = census_layer_kernel<N, U, BLOCK>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
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

template <int N>
void launch_list(uint8_t *ws, const CensusPlan &p, int c, int32_t *status, cudaStream_t s) {
    const uint64_t tf = t_frames(N);
    const uint64_t nw = (tf + 31) / 32;
    const unsigned nb = (unsigned)((nw + 255) / 256);
    uint32_t *blk = (uint32_t *)(ws + p.blk_off);
    uint64_t *len = (uint64_t *)(ws + p.len_off[c][N]);
    uint64_t *list = (uint64_t *)(ws + p.list_off[c][N]);
    const uint64_t cap = c == 0 ? kPreorders[N] : kEquivalences[N];
    list_count_kernel<N><<<nb, 256, 0, s>>>(blk, nw, tf, c);
    list_scan_kernel<<<1, 1024, 0, s>>>(blk, nb, len);
    list_write_kernel<N><<<nb, 256, 0, s>>>(blk, list, cap, nw, tf, c, status);
}

void launch_list_n(int n, uint8_t *ws, const CensusPlan &p, int c, int32_t *status, cudaStream_t s) {
    switch (n) {
    case 1: launch_list<1>(ws, p, c, status, s); break;
    case 2: launch_list<2>(ws, p, c, status, s); break;
    case 3: launch_list<3>(ws, p, c, status, s); break;
    case 4: launch_list<4>(ws, p, c, status, s); break;
    case 5: launch_list<5>(ws, p, c, status, s); break;
    case 6: launch_list<6>(ws, p, c, status, s); break;
    }
}

}  // namespace

extern "C" uint64_t mk_class_frames(uint32_t cls, int32_t n) {
    if (n < 1 || n > MK_MAX_WORLDS_EXH) return 0;
    switch (cls) {
    case MK_CLASS_K: return 1ull << (n * n);
    case MK_CLASS_T: return t_frames(n);
    case MK_CLASS_S4: return kPreorders[n];
    case MK_CLASS_S5: return kEquivalences[n];
    default: return 0;
    }
}

extern "C" int32_t mk_census_launches(const mk_census_cfg *cfg, int32_t nprog) {
    if (check_cfg(cfg, nprog) != MK_OK) return -1;
    const int nn = cfg->n_max - cfg->n_min + 1;
    const int lists = ((cfg->classes & MK_CLASS_S4) ? 1 : 0) + ((cfg->classes & MK_CLASS_S5) ? 1 : 0);
    if (nprog == 0) return lists * nn * 3;
    int layers = 0;
    for (int c = 0; c < 4; ++c)
        if (cfg->classes & (1u << c))
            for (int n = cfg->n_min; n <= cfg->n_max; ++n) {
                if (c == 0) {
                    const uint64_t kf = 1ull << (n * n);
                    const uint64_t hi = cfg->frame_hi < kf ? cfg->frame_hi : kf;
                    if (cfg->frame_lo >= hi) continue;
                }
                ++layers;
            }
    return 1 + lists * nn * 3 + layers;
}

extern "C" size_t mk_census_workspace_size(const mk_census_cfg *cfg, int32_t nprog) {
    if (check_cfg(cfg, nprog) != MK_OK) return 0;
    return plan_workspace(cfg).total;
}

extern "C" int mk_census(const mk_program *d_progs, int32_t nprog, const mk_census_cfg *cfg,
                         mk_result *d_out, int32_t *d_status, void *d_workspace, size_t ws_bytes,
                         void *stream) {
    int rc = check_cfg(cfg, nprog);
    if (rc != MK_OK) return rc;
    if (nprog > 0 && (!d_progs || !d_out)) return MK_E_ARG;
    if (!d_status) return MK_E_ARG;
    const CensusPlan plan = plan_workspace(cfg);
    if (!d_workspace || ws_bytes < plan.total) return MK_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t *ws = (uint8_t *)d_workspace;

    const int ncls = class_count(cfg->classes);
    const int nn = cfg->n_max - cfg->n_min + 1;
    const size_t nout = (size_t)nprog * ncls * nn;
    if (nout) init_results_kernel<<<(unsigned)((nout + 255) / 256 < 4096 ? (nout + 255) / 256 : 4096), 256, 0, s>>>(d_out, nout);

    const int block = cfg->tune.block ? cfg->tune.block : 256;
    const int tile = cfg->tune.tile ? cfg->tune.tile : 16;
    const int depth = cfg->max_depth ? cfg->max_depth : MK_MAX_STACK;
    const int units = cfg->tune.units ? cfg->tune.units : 8;

    // class lists for S4 / S5
    for (int c = 0; c < 2; ++c) {
        const uint32_t bit = c == 0 ? MK_CLASS_S4 : MK_CLASS_S5;
        if (!(cfg->classes & bit)) continue;
        for (int n = cfg->n_min; n <= cfg->n_max; ++n) launch_list_n(n, ws, plan, c, d_status, s);
    }

    int ci = 0;
    for (int c = 0; c < 4; ++c) {
        const uint32_t bit = 1u << c;
        if (!(cfg->classes & bit)) continue;
        for (int n = cfg->n_min; n <= cfg->n_max; ++n) {
            LayerArgs a;
            std::memset(&a, 0, sizeof(a));
            a.progs = d_progs;
            a.nprog = nprog;
            a.tile = tile;
            a.S = cfg->samples;
            a.samples = cfg->samples ? cfg->d_samples + (size_t)n * cfg->samples : nullptr;
            a.f_lo = cfg->frame_lo;
            a.f_hi = cfg->frame_hi;
            const uint64_t kframes = 1ull << (n * n);
            a.full_range = (cfg->frame_lo == 0 && cfg->frame_hi >= kframes) ? 1 : 0;
            a.out = d_out;
            a.out_stride = ncls * nn;
            a.out_off = ci * nn + (n - cfg->n_min);
            a.depth = depth;
            a.status = d_status;
            if (c == 0) {
                a.src = SRC_K;
                a.nframes = kframes;
                const uint64_t hi = cfg->frame_hi < kframes ? cfg->frame_hi : kframes;
                a.word_lo = cfg->frame_lo / 32;
                a.word_hi = cfg->frame_lo >= hi ? a.word_lo : (hi + 31) / 32;
            } else if (c == 1) {
                a.src = SRC_T;
                a.nframes = t_frames(n);
                a.word_lo = 0;
                a.word_hi = (a.nframes + 31) / 32;
            } else {
                const int li = c - 2;
                a.src = SRC_LIST;
                a.list = (const uint64_t *)(ws + plan.list_off[li][n]);
                a.list_len = (const uint64_t *)(ws + plan.len_off[li][n]);
                a.nframes = li == 0 ? kPreorders[n] : kEquivalences[n];
                a.word_lo = 0;
                a.word_hi = (a.nframes + 31) / 32;
            }
            launch_layer_n(n, a, block, units, s);
        }
        ++ci;
    }
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}
