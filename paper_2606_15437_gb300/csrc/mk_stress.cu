// mk_stress.cu -- separation over explicit relations on up to 16 worlds
// (Sec. 7: stress templates; Table 2: adversarial relation synthesis).
//
// Beyond six worlds the frames are no longer enumerated: a pair is checked
// on a list of relations (templates, or relations drawn by a generator).
// Relations are bit-sliced 32 to a "relation block" exactly like the frame
// words of the census (bit l of word (w, v) = R(w, v) of relation 32b+l),
// but n*n edge words per block no longer fit one thread at n = 16.  So the
// work of one block is split over n threads ("world-split" layout): thread
// j of a group holds row j of the block (its n edge words E[j][v]) and the
// truth word of world j of every subformula.  Boolean connectives stay one
// logic op per thread; a modal step needs the operand's truth words of all
// n worlds, which the group exchanges through shared memory:
//     every thread stores t[j]; __syncwarp; thread j reads t[0..n) with
//     16-byte loads and computes  box: AND_v (t[v] | ~E[j][v])
//                                 dia: OR_v  (t[v] &  E[j][v])
// i.e. still n logic ops per world and 32 relations, n*n per modal step,
// the same work as the census (Lemma 1).  Groups are packed floor(32/n) to
// a warp.  Every thread walks U relation blocks at once, so that each
// dispatched instruction carries U times the logic work.
//
// Valuations are uniform over a group (all 32 relations of a block share
// one), so atom p_i at world j under valuation x is the all-ones or
// all-zeros word of bit i*n + j of x: no atom rows are needed.  For each
// pair, each thread keeps its least (relation, valuation) with a split at
// its world, and the CTA merges (relation, valuation, world) keys with a
// shared atomicMin before one global atomicMin per pair.  Large valuation
// ranges (one-variable pairs at n up to 16) are cut over grid.z.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "mk.h"
#include "mk_attr.h"
#include "mk_eval.cuh"
#include "mk_relgen.cuh"

namespace mkd {

constexpr int ST_OPS_STRIDE = MK_MAX_CODE + 2;
constexpr int ST_BLOCK = 256;
constexpr int ST_MAX_TILE = 64;
constexpr int ST_KEY_X = 4, ST_KEY_S = 20;   // key = s << 20 | x << 4 | w

// World-split layout of n = N worlds, W worlds per thread: a group of
// T = ceil(N/W) threads holds one relation block; thread j holds worlds
// j*W .. j*W+W-1 (worlds >= N are padding: no edges, never reported).
template <int N, int W>
struct WS {
    static constexpr int T = (N + W - 1) / W;       // threads per group
    static constexpr int GW = 32 / T;               // groups per warp
    static constexpr int RN = (T * W + 3) & ~3;     // exchange row of a group (16-byte multiple)
    static constexpr int XW = (31 / T + 1) * RN;    // exchange words per warp and unit (idle lanes too)
};

// Units per dispatched instruction: UB relation blocks x V valuations.
// Constant pairs have one valuation, so their launch walks UB0 blocks;
// pairs with variables walk one block under V consecutive valuations
// (the edge registers of a block serve all V valuations).  W: worlds per
// thread: 2 from 7 worlds up (more lanes hold a world at 11 and 12, and
// the group exchange costs half as much per logic op).
template <int N>
constexpr int st_ub0() { return N <= 5 ? 8 : N <= 8 ? 6 : 4; }
template <int N>
constexpr int st_w1() { return N >= 7 ? 2 : 1; }
template <int N>
constexpr int st_v1() { return st_w1<N>() == 2 ? 8 : 16; }

struct StressArgs {
    const mk_program *phi;
    const mk_program *psi;
    int32_t npairs;
    int32_t tile;
    const uint32_t *words;
    uint64_t count;          // relations
    uint64_t nblocks;        // relation blocks
    uint64_t blk_lo;         // first relation block of this launch
    uint64_t index_base;
    uint32_t vchunk;         // valuations per grid.z slice
    int32_t with_vars;       // 0: this launch takes the constant pairs, 1: the others
    int32_t count_splits;
    uint64_t *key;
    uint32_t *nsplit;
    int32_t *status;
};

template <int N, int W, int U, int BLOCK>
struct StressSmem {
    static constexpr size_t code_bytes(int tile) { return ((size_t)tile * ST_OPS_STRIDE * 6 + 15) & ~(size_t)15; }
    // na, nb, k, count (4 x 4 B) + key (8 B) per pair, rounded to 16 bytes
    static constexpr size_t meta_bytes(int tile) { return ((size_t)tile * 24 + 15) & ~(size_t)15; }
    static constexpr size_t stack_bytes() { return (size_t)MK_MAX_STACK * U * W * BLOCK * 4; }
    static constexpr size_t xbuf_bytes() { return (size_t)(BLOCK / 32) * U * WS<N, W>::XW * 4; }
    static size_t total(int tile) { return code_bytes(tile) + meta_bytes(tile) + stack_bytes() + xbuf_bytes(); }
};

// Decode for the world-split interpreter: stack operands scaled to the
// thread's stack column (d -> d*U*W*BLOCK), variable operands to the bit
// offset of p_i in a valuation (i -> i*N).
// A PUSH followed by an op that does not read A is folded into that op
// (MK_DEC_PUSH flag and the stack entry in bits 6-7), as in decode_program.
template <int N, int SW, int BLOCK>
__device__ __forceinline__ void decode_ws(const mk_program &p, uint8_t *ops, uint16_t *offs) {
    int j = 0;
    uint32_t push = 0;
    for (int i = 0; i < p.n_instr; ++i) {
        const int op = p.code[i] & 31, arg = p.code[i] >> 5;
        if (op == MK_OP_PUSH && !push && i + 1 < p.n_instr && fresh_op(p.code[i + 1] & 31)) {
            push = MK_DEC_PUSH | ((uint32_t)arg << 6);
            continue;
        }
        ops[j] = (uint8_t)(op | push);
        push = 0;
        const bool stack_op = op >= MK_OP_PUSH && op <= MK_OP_IFF_S;
        offs[j] = (uint16_t)(stack_op ? arg * (SW * BLOCK) : arg * N);
        ++j;
    }
    ops[j] = (uint8_t)MK_OP_END;
    offs[j] = 0;
}

// One modal step for all U = UB*V units (unit u: block u/V): publish this
// thread's W world words, read the group's words, combine with this
// thread's edge rows of the unit's block.
template <int N, int W, int UB, int V, bool BOX>
__device__ __forceinline__ void modal_ws(uint32_t (&A)[UB * V][W], const uint32_t (&E)[UB][W][N], uint32_t *xw,
                                         int xo, int jw0, bool active) {
    constexpr int RN = WS<N, W>::RN, XW = WS<N, W>::XW, U = UB * V;
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int w = 0; w < W; ++w)
            if (active) xw[u * XW + xo + jw0 + w] = A[u][w];
    __syncwarp();
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint4 *p = reinterpret_cast<const uint4 *>(xw + u * XW + xo);
        uint32_t t[RN];
#pragma unroll
        for (int q = 0; q < RN / 4; ++q) {
            const uint4 v = p[q];
            t[4 * q] = v.x;
            t[4 * q + 1] = v.y;
            t[4 * q + 2] = v.z;
            t[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint32_t acc = BOX ? 0xFFFFFFFFu : 0u;
#pragma unroll
            for (int v = 0; v < N; ++v) {
                if (BOX) acc &= t[v] | ~E[u / V][w][v];
                else acc |= t[v] & E[u / V][w][v];
            }
            A[u][w] = acc;
        }
    }
    __syncwarp();
}

// Run a decoded program on this thread's W worlds of U = UB*V units, unit
// u being block u/V under valuation x + u%V (xs[v] = (x + v) >> jw0).
// Every thread of a warp runs the same program, so the __syncwarp of the
// modal steps is reached by all 32 lanes.
template <int N, int W, int UB, int V, int BLOCK>
__device__ __forceinline__ void run_ws(const uint8_t *ops, const uint16_t *offs, const uint32_t (&xs)[V],
                                       const uint32_t (&E)[UB][W][N], uint32_t *stack, uint32_t *xw, int xo, int jw0,
                                       bool active, uint32_t (&A)[UB * V][W]) {
    constexpr int U = UB * V;
    uint32_t op = ops[0], off = offs[0];
    for (int pc = 1;; ++pc) {
        const uint32_t op_next = ops[pc], off_next = offs[pc];
        uint32_t *st = stack + off;
        if (op & MK_DEC_PUSH) {                         // folded PUSH: save A first
            uint32_t *ps = stack + (op >> 6) * (U * W * BLOCK);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int w = 0; w < W; ++w) ps[(u * W + w) * BLOCK] = A[u][w];
            op &= MK_DEC_PUSH - 1u;
        }
        // atom truth word of p_i at world jw0+w under unit u's valuation:
        // only variable operands (off = i*N < 16) are shifts
#define MK_ATOM(u, w) (0u - ((xs[(u) % V] >> (off + (w))) & 1u))
#define MK_EACH for (int u = 0; u < U; ++u) _Pragma("unroll") for (int w = 0; w < W; ++w)
        switch (op) {
        case MK_OP_LDV:
#pragma unroll
            MK_EACH A[u][w] = MK_ATOM(u, w);
            break;
        case MK_OP_LDT:
#pragma unroll
            MK_EACH A[u][w] = 0xFFFFFFFFu;
            break;
        case MK_OP_LDF:
#pragma unroll
            MK_EACH A[u][w] = 0u;
            break;
        case MK_OP_NOT:
#pragma unroll
            MK_EACH A[u][w] = ~A[u][w];
            break;
        case MK_OP_BOX:
            modal_ws<N, W, UB, V, true>(A, E, xw, xo, jw0, active);
            break;
        case MK_OP_DIA:
            modal_ws<N, W, UB, V, false>(A, E, xw, xo, jw0, active);
            break;
        case MK_OP_PUSH:
#pragma unroll
            MK_EACH st[(u * W + w) * BLOCK] = A[u][w];
            break;
        case MK_OP_AND_S:
#pragma unroll
            MK_EACH A[u][w] &= st[(u * W + w) * BLOCK];
            break;
        case MK_OP_OR_S:
#pragma unroll
            MK_EACH A[u][w] |= st[(u * W + w) * BLOCK];
            break;
        case MK_OP_IMP_S:
#pragma unroll
            MK_EACH A[u][w] = ~st[(u * W + w) * BLOCK] | A[u][w];
            break;
        case MK_OP_RIMP_S:
#pragma unroll
            MK_EACH A[u][w] = ~A[u][w] | st[(u * W + w) * BLOCK];
            break;
        case MK_OP_IFF_S:
#pragma unroll
            MK_EACH A[u][w] = ~(A[u][w] ^ st[(u * W + w) * BLOCK]);
            break;
        case MK_OP_AND_V:
#pragma unroll
            MK_EACH A[u][w] &= MK_ATOM(u, w);
            break;
        case MK_OP_OR_V:
#pragma unroll
            MK_EACH A[u][w] |= MK_ATOM(u, w);
            break;
        case MK_OP_IMP_V:
#pragma unroll
            MK_EACH A[u][w] = ~A[u][w] | MK_ATOM(u, w);
            break;
        case MK_OP_RIMP_V:
#pragma unroll
            MK_EACH A[u][w] = ~MK_ATOM(u, w) | A[u][w];
            break;
        case MK_OP_LDNV:
#pragma unroll
            MK_EACH A[u][w] = ~MK_ATOM(u, w);
            break;
        case MK_OP_AND_NV:
#pragma unroll
            MK_EACH A[u][w] &= ~MK_ATOM(u, w);
            break;
        case MK_OP_OR_NV:
#pragma unroll
            MK_EACH A[u][w] |= ~MK_ATOM(u, w);
            break;
        case MK_OP_IMP_NV:
#pragma unroll
            MK_EACH A[u][w] = ~A[u][w] | ~MK_ATOM(u, w);
            break;
        case MK_OP_BOX_V:
        case MK_OP_DIA_V:
        case MK_OP_BOX_NV:
        case MK_OP_DIA_NV: {
            const uint32_t flip = (op == MK_OP_BOX_NV || op == MK_OP_DIA_NV) ? 0xFFFFFFFFu : 0u;
#pragma unroll
            MK_EACH A[u][w] = MK_ATOM(u, w) ^ flip;
            if (op == MK_OP_BOX_V || op == MK_OP_BOX_NV) modal_ws<N, W, UB, V, true>(A, E, xw, xo, jw0, active);
            else modal_ws<N, W, UB, V, false>(A, E, xw, xo, jw0, active);
            break;
        }
        case MK_OP_END:
            return;
        default:
            __builtin_unreachable();
        }
        op = op_next;
        off = off_next;
    }
#undef MK_EACH
#undef MK_ATOM
}

template <int N, int W, int UB, int V, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 2) stress_kernel(StressArgs a) {
    constexpr int U = UB * V;
    using SM = StressSmem<N, W, U, BLOCK>;
    using L = WS<N, W>;
    constexpr int GROUPS = (BLOCK / 32) * L::GW;
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_active;
    const int tile = a.tile;
    uint16_t *s_offs_a = (uint16_t *)smem;
    uint16_t *s_offs_b = s_offs_a + (size_t)tile * ST_OPS_STRIDE;
    uint8_t *s_ops_a = (uint8_t *)(s_offs_b + (size_t)tile * ST_OPS_STRIDE);
    uint8_t *s_ops_b = s_ops_a + (size_t)tile * ST_OPS_STRIDE;
    int *s_na = (int *)(smem + SM::code_bytes(tile));
    int *s_nb = s_na + tile;
    int *s_k = s_nb + tile;
    uint32_t *s_cnt = (uint32_t *)(s_k + tile);
    unsigned long long *s_key = (unsigned long long *)(s_cnt + tile);
    uint32_t *s_stack = (uint32_t *)(smem + SM::code_bytes(tile) + SM::meta_bytes(tile));
    uint32_t *s_xbuf = s_stack + (size_t)MK_MAX_STACK * U * W * BLOCK;

    const int tid = threadIdx.x, wi = tid >> 5, lane = tid & 31;
    const int g = lane / L::T, j = lane - g * L::T;
    const int jw0 = j * W;                         // this thread's first world
    const bool active = g < L::GW;
    const int G = wi * L::GW + (active ? g : 0);
    const uint64_t cta_b0 = a.blk_lo + (uint64_t)blockIdx.x * GROUPS * UB;
    const uint32_t x_lo = blockIdx.z * a.vchunk;
    const unsigned long long floor_key = (a.index_base + (cta_b0 << 5)) << ST_KEY_S;

    if (tid == 0) s_active = 0;
    __syncthreads();
    const int p0 = blockIdx.y * tile;
    const int np = min(tile, a.npairs - p0);
    for (int i = tid; i < np; i += BLOCK) {
        const mk_program &pa = a.phi[p0 + i], &pb = a.psi[p0 + i];
        const bool first_cta = blockIdx.x == 0 && blockIdx.z == 0 && a.blk_lo == 0;
        int ok = program_ok(pa) && program_ok(pb);
        if (!ok && first_cta && !a.with_vars) atomicOr(a.status, (int)MK_ST_PROGRAM);
        const int k = pa.nvars > pb.nvars ? pa.nvars : pb.nvars;
        if (ok && (k > 0) != (a.with_vars != 0)) ok = 0;       // the other launch's pair
        if (ok && k * N > 16) {
            ok = 0;
            if (first_cta) atomicOr(a.status, (int)MK_ST_LIMIT);
        }
        if (ok && x_lo >= (1u << (k * N))) ok = 0;             // nothing in this valuation slice
        if (ok && !a.count_splits && ((volatile unsigned long long *)a.key)[p0 + i] < floor_key) ok = 0;
        s_na[i] = ok ? pa.n_instr : -1;
        s_nb[i] = pb.n_instr;
        s_k[i] = k;
        s_cnt[i] = 0;
        s_key[i] = ~0ull;
        if (ok) {
            atomicAdd(&s_active, 1);
            decode_ws<N, U * W, BLOCK>(pa, s_ops_a + i * ST_OPS_STRIDE, s_offs_a + i * ST_OPS_STRIDE);
            decode_ws<N, U * W, BLOCK>(pb, s_ops_b + i * ST_OPS_STRIDE, s_offs_b + i * ST_OPS_STRIDE);
        }
    }
    __syncthreads();
    if (s_active == 0) return;

    // this thread's rows of its UB relation blocks (padding worlds: none)
    uint32_t E[UB][W][N];
    uint32_t valid[UB];
#pragma unroll
    for (int b = 0; b < UB; ++b) {
        const uint64_t blk = cta_b0 + (uint64_t)G * UB + b;
        valid[b] = 0;
        const bool have = active && blk < a.nblocks;
        if (have) {
            const uint64_t left = a.count - (blk << 5);
            valid[b] = left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
        }
#pragma unroll
        for (int w = 0; w < W; ++w) {
            if (have && jw0 + w < N) {
                const uint32_t *row = a.words + (blk * N + (uint64_t)(jw0 + w)) * N;
#pragma unroll
                for (int v = 0; v < N; ++v) E[b][w][v] = row[v];
            } else {
#pragma unroll
                for (int v = 0; v < N; ++v) E[b][w][v] = 0u;
            }
        }
    }
    uint32_t wmask[W];                            // real worlds of this thread
#pragma unroll
    for (int w = 0; w < W; ++w) wmask[w] = jw0 + w < N ? 0xFFFFFFFFu : 0u;
    uint32_t *xw = s_xbuf + (size_t)wi * U * L::XW;
    const int xo = g * L::RN;
    uint32_t *stk = s_stack + tid;

    for (int fi = 0; fi < np; ++fi) {
        if (s_na[fi] < 0) continue;
        const uint32_t nval = 1u << (s_k[fi] * N);
        const uint32_t x_hi = min(nval, x_lo + a.vchunk);
        const uint8_t *oa = s_ops_a + fi * ST_OPS_STRIDE, *ob = s_ops_b + fi * ST_OPS_STRIDE;
        const uint16_t *fa = s_offs_a + fi * ST_OPS_STRIDE, *fb = s_offs_b + fi * ST_OPS_STRIDE;
        int best_o = UB * 32, best_w = 0;
        uint32_t best_x = 0;
        uint32_t hm[UB];
#pragma unroll
        for (int b = 0; b < UB; ++b) hm[b] = 0;
        for (uint32_t x = x_lo; x < x_hi; x += V) {
            uint32_t A[U][W], B[U][W], xs[V];
#pragma unroll
            for (int v = 0; v < V; ++v) xs[v] = (x + v) >> jw0;
            run_ws<N, W, UB, V, BLOCK>(oa, fa, xs, E, stk, xw, xo, jw0, active, A);
            run_ws<N, W, UB, V, BLOCK>(ob, fb, xs, E, stk, xw, xo, jw0, active, B);
            // blocks outer, valuations inner, worlds ascending: for one
            // relation the first difference found has the least valuation,
            // then the least world
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t vm = (x + (u % V) < x_hi) ? valid[u / V] : 0u;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const uint32_t d = (A[u][w] ^ B[u][w]) & vm & wmask[w];
                    hm[u / V] |= d;
                    if (d) {
                        const int o = (u / V) * 32 + __ffs(d) - 1;
                        if (o < best_o) {
                            best_o = o;
                            best_x = x + (u % V);
                            best_w = w;
                        }
                    }
                }
            }
        }
        if (active && best_o < UB * 32) {
            const uint64_t s = a.index_base + ((cta_b0 + (uint64_t)G * UB + (uint64_t)(best_o >> 5)) << 5) +
                               (uint64_t)(best_o & 31);
            const unsigned long long key =
                (s << ST_KEY_S) | ((uint64_t)best_x << ST_KEY_X) | (uint64_t)(jw0 + best_w);
            atomicMin(&s_key[fi], key);
        }
        if (a.count_splits) {
            // relations of the group split at any of its worlds
#pragma unroll
            for (int b = 0; b < UB; ++b)
                if (active) xw[b * L::XW + xo + j] = hm[b];
            __syncwarp();
            if (active && j == 0) {
                uint32_t c = 0;
#pragma unroll
                for (int b = 0; b < UB; ++b) {
                    uint32_t m = 0;
#pragma unroll
                    for (int t = 0; t < L::T; ++t) m |= xw[b * L::XW + xo + t];
                    c += __popc(m);
                }
                if (c) atomicAdd(&s_cnt[fi], c);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    for (int i = tid; i < np; i += BLOCK) {
        if (s_key[i] != ~0ull) atomicMin((unsigned long long *)&a.key[p0 + i], s_key[i]);
        if (a.count_splits && s_cnt[i]) atomicAdd(&a.nsplit[p0 + i], s_cnt[i]);
    }
}

// Relation words (and successor masks) of 32 relations per warp: lane l
// builds relation 32b + l, the block's words are warp ballots.
__global__ void relwords_kernel(int pack, int gen, uint64_t seed, int n, uint64_t first, uint64_t count,
                                const uint32_t *succ_in, uint32_t *words, uint32_t *succ_out) {
    const uint64_t b = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= (count + 31) / 32) return;   // whole warp
    const uint64_t i = (b << 5) + lane;
    Succ s;
    succ_clear(s);
    if (i < count) {
        if (pack) {
            const uint32_t all = full_mask(n);
            for (int w = 0; w < n; ++w) s[w] = succ_in[i * 16 + w] & all;
        } else {
            stress_relation(gen, seed, n, first + i, s);
        }
        if (succ_out)
            for (int w = 0; w < 16; ++w) succ_out[i * 16 + w] = w < n ? s[w] : 0u;
    }
    if (words) {
        for (int w = 0; w < n; ++w)
            for (int v = 0; v < n; ++v) {
                const uint32_t m = __ballot_sync(0xFFFFFFFFu, (s[w] >> v) & 1u);
                if (lane == ((w * n + v) & 31)) words[(b * n + w) * n + v] = m;
            }
    }
}

}  // namespace mkd

namespace {

using namespace mkd;

template <typename K>
void st_smem(K kern, size_t bytes) {
    // every launch of one instantiation asks for at most the tile-64 size
    ensure_dynamic_smem((const void *)kern, bytes);
}

template <int N, int W, int UB, int V>
void launch_stress_kind(StressArgs a, uint64_t blk_hi, uint32_t vz, cudaStream_t s) {
    constexpr int GROUPS = (ST_BLOCK / 32) * WS<N, W>::GW;
    using SM = StressSmem<N, W, UB * V, ST_BLOCK>;
    auto kern = stress_kernel<N, W, UB, V, ST_BLOCK>;
    st_smem(kern, SM::total(ST_MAX_TILE));
    const uint64_t per_cta = (uint64_t)GROUPS * UB;
    // ascending launches of at most 4096 CTAs: pairs split in one launch are
    // skipped by the later ones (first-split mode)
    const uint64_t chunk = per_cta * 4096;
    for (uint64_t lo = a.blk_lo; lo < blk_hi; lo += chunk) {
        StressArgs c = a;
        c.blk_lo = lo;
        const uint64_t hi = lo + chunk < blk_hi ? lo + chunk : blk_hi;
        dim3 grid((unsigned)((hi - lo + per_cta - 1) / per_cta), (unsigned)((a.npairs + a.tile - 1) / a.tile), vz);
        kern<<<grid, ST_BLOCK, SM::total(a.tile), s>>>(c);
    }
}

// Two launches over the pair list: constant pairs (one valuation) and the
// pairs with variables, each taking only its own pairs.
template <int N>
void launch_stress(StressArgs a, uint64_t blk_hi, uint32_t vz, cudaStream_t s) {
    StressArgs c0 = a;
    c0.with_vars = 0;
    c0.vchunk = 1;
    launch_stress_kind<N, 1, st_ub0<N>(), 1>(c0, blk_hi, 1, s);
    StressArgs c1 = a;
    c1.with_vars = 1;
    launch_stress_kind<N, st_w1<N>(), 1, st_v1<N>()>(c1, blk_hi, vz, s);
}

void launch_stress_n(int n, const StressArgs &a, uint64_t blk_hi, uint32_t vz, cudaStream_t s) {
    switch (n) {
    case 1: launch_stress<1>(a, blk_hi, vz, s); break;
    case 2: launch_stress<2>(a, blk_hi, vz, s); break;
    case 3: launch_stress<3>(a, blk_hi, vz, s); break;
    case 4: launch_stress<4>(a, blk_hi, vz, s); break;
    case 5: launch_stress<5>(a, blk_hi, vz, s); break;
    case 6: launch_stress<6>(a, blk_hi, vz, s); break;
    case 7: launch_stress<7>(a, blk_hi, vz, s); break;
    case 8: launch_stress<8>(a, blk_hi, vz, s); break;
    case 9: launch_stress<9>(a, blk_hi, vz, s); break;
    case 10: launch_stress<10>(a, blk_hi, vz, s); break;
    case 11: launch_stress<11>(a, blk_hi, vz, s); break;
    case 12: launch_stress<12>(a, blk_hi, vz, s); break;
    case 13: launch_stress<13>(a, blk_hi, vz, s); break;
    case 14: launch_stress<14>(a, blk_hi, vz, s); break;
    case 15: launch_stress<15>(a, blk_hi, vz, s); break;
    case 16: launch_stress<16>(a, blk_hi, vz, s); break;
    }
}

template <int N>
uint64_t per_cta_blocks() { return (uint64_t)(ST_BLOCK / 32) * WS<N, st_w1<N>()>::GW; }

uint64_t per_cta_n(int n) {
    switch (n) {
    case 1: return per_cta_blocks<1>();
    case 2: return per_cta_blocks<2>();
    case 3: return per_cta_blocks<3>();
    case 4: return per_cta_blocks<4>();
    case 5: return per_cta_blocks<5>();
    case 6: return per_cta_blocks<6>();
    case 7: return per_cta_blocks<7>();
    case 8: return per_cta_blocks<8>();
    case 9: return per_cta_blocks<9>();
    case 10: return per_cta_blocks<10>();
    case 11: return per_cta_blocks<11>();
    case 12: return per_cta_blocks<12>();
    case 13: return per_cta_blocks<13>();
    case 14: return per_cta_blocks<14>();
    case 15: return per_cta_blocks<15>();
    default: return per_cta_blocks<16>();
    }
}

}  // namespace

extern "C" int mk_template(int32_t id, int32_t n, uint32_t *succ) {
    if (!succ || n < 1 || n > MK_MAX_WORLDS_STRESS || id < 0 || id >= MK_NUM_TEMPLATES) return MK_E_ARG;
    Succ s;
    template_succ(id, n, s);
    for (int w = 0; w < n; ++w) succ[w] = s[w];
    return MK_OK;
}

extern "C" int mk_stress_relation(int32_t gen, uint64_t seed, int32_t n, uint64_t s, uint32_t *succ) {
    if (!succ) return MK_E_ARG;
    Succ r;
    if (!stress_relation(gen, seed, n, s, r)) return MK_E_ARG;
    for (int w = 0; w < n; ++w) succ[w] = r[w];
    return MK_OK;
}

extern "C" uint64_t mk_relation_words(int32_t n, uint64_t count) {
    if (n < 1 || n > MK_MAX_WORLDS_STRESS) return 0;
    return (count + 31) / 32 * (uint64_t)n * (uint64_t)n;
}

namespace {
int relwords(int pack, int gen, uint64_t seed, int n, uint64_t first, uint64_t count, const uint32_t *succ_in,
             uint32_t *words, uint32_t *succ_out, void *stream) {
    if (count == 0) return MK_OK;
    const uint64_t nb = (count + 31) / 32;
    const uint64_t warps = 8;
    if ((nb + warps - 1) / warps > 0x7FFFFFFFull) return MK_E_ARG;
    relwords_kernel<<<(unsigned)((nb + warps - 1) / warps), (unsigned)(warps * 32), 0, (cudaStream_t)stream>>>(
        pack, gen, seed, n, first, count, succ_in, words, succ_out);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}
}  // namespace

extern "C" int mk_generate_relations(int32_t gen, uint64_t seed, int32_t n, uint64_t first, uint64_t count,
                                     uint32_t *d_words, uint32_t *d_succ, void *stream) {
    if (n < 1 || n > MK_MAX_WORLDS_STRESS || gen < 0 || gen >= MK_NUM_GENERATORS) return MK_E_ARG;
    if (gen != MK_GEN_ER && n < 2) return MK_E_ARG;
    if (count && !d_words && !d_succ) return MK_E_ARG;
    return relwords(0, gen, seed, n, first, count, nullptr, d_words, d_succ, stream);
}

extern "C" int mk_pack_relations(const uint32_t *d_succ, int32_t n, uint64_t count, uint32_t *d_words,
                                 void *stream) {
    if (n < 1 || n > MK_MAX_WORLDS_STRESS) return MK_E_ARG;
    if (count && (!d_succ || !d_words)) return MK_E_ARG;
    return relwords(1, 0, 0, n, 0, count, d_succ, d_words, nullptr, stream);
}

extern "C" int mk_stress_separate(const mk_program *d_phi, const mk_program *d_psi, int32_t npairs,
                                  const uint32_t *d_words, const mk_stress_cfg *cfg, uint64_t *d_key,
                                  uint32_t *d_nsplit, int32_t *d_status, void *stream) {
    if (!cfg || npairs < 0 || !d_status) return MK_E_ARG;
    const int n = cfg->n;
    if (n < 1 || n > MK_MAX_WORLDS_STRESS) return MK_E_ARG;
    if (cfg->tune.tile > ST_MAX_TILE || (cfg->tune.block && cfg->tune.block != ST_BLOCK)) return MK_E_ARG;
    if (cfg->index_base + cfg->count >= (1ull << 44)) return MK_E_ARG;
    if (npairs == 0 || cfg->count == 0) return MK_OK;
    if (!d_phi || !d_psi || !d_key || !d_words || (cfg->count_splits && !d_nsplit)) return MK_E_ARG;

    const uint64_t nblocks = (cfg->count + 31) / 32;
    const uint64_t rel_ctas = (nblocks + per_cta_n(n) - 1) / per_cta_n(n);
    const uint64_t want = 4 * 152;   // CTAs that fill the GPU a few times over
    // Pairs per CTA: the caller's, or 16 cut down while the relation list
    // alone gives too few CTAs.
    int tile = cfg->tune.tile;
    if (tile == 0) {
        tile = 16;
        while (tile > 1 && rel_ctas * (uint64_t)((npairs + tile - 1) / tile) < want) tile /= 2;
    }
    if ((npairs + tile - 1) / tile > 65535) return MK_E_ARG;

    StressArgs a;
    std::memset(&a, 0, sizeof(a));
    a.phi = d_phi;
    a.psi = d_psi;
    a.npairs = npairs;
    a.tile = tile;
    a.words = d_words;
    a.count = cfg->count;
    a.nblocks = nblocks;
    a.blk_lo = 0;
    a.index_base = cfg->index_base;
    a.count_splits = cfg->count_splits ? 1 : 0;
    a.key = d_key;
    a.nsplit = d_nsplit;
    a.status = d_status;
    // Then cut large valuation ranges over grid.z (first-split mode only:
    // counting needs every valuation of a relation in one CTA).
    const uint64_t base_ctas = rel_ctas * (uint64_t)((npairs + tile - 1) / tile);
    uint32_t vz = 1;
    const uint32_t nval_max = 1u << (16 - 16 % n);   // largest 2^(k n) with k n <= 16
    if (!a.count_splits) {
        while (vz < 256 && base_ctas * vz < want && nval_max / (vz * 2) >= 256) vz *= 2;
    }
    a.vchunk = (nval_max + vz - 1) / vz;
    launch_stress_n(n, a, a.nblocks, vz, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? MK_OK : MK_E_CUDA;
}
