// mk_eval.cuh -- device building blocks shared by the census and the
// separation kernels: bit-sliced frames and the postfix interpreter.
//
// Layout ("frame word"): one 32-bit register word holds one bit for each of
// 32 consecutive frames, lane l <-> frame base + l.  A truth set of an
// n-world frame is then n words t[w] (bit l of t[w] = world w is in the set
// on frame base + l), and the frame itself is n*n edge words E[w*n+v]
// (bit l = R(w,v) on frame base + l).  Every Boolean connective is one
// bitwise op per world word, box and diamond are the containment and
// intersection tests of Lemma 1 written per world, i.e. n*n three-input
// logic ops for 32 frames at once:
//     box:  t'[w] = AND_v (t[v] | ~E[w][v])     (succ[w] subset of t)
//     dia:  t'[w] = OR_v  (t[v] &  E[w][v])     (succ[w] meets t)
// A valuation is the same for all 32 lanes, so atom p_i at world w is the
// all-ones or all-zeros word given by bit i*n+w of the valuation value.
#pragma once
#include <cstdint>

#include "mk.h"

namespace mkd {

// Bit b (b < 5) of the frame index across the 32 lanes of a word whose base
// index is a multiple of 32.
__device__ __forceinline__ constexpr uint32_t lane_pattern(int b) {
    return b == 0 ? 0xAAAAAAAAu : b == 1 ? 0xCCCCCCCCu : b == 2 ? 0xF0F0F0F0u
         : b == 3 ? 0xFF00FF00u : 0xFFFF0000u;
}

__device__ __forceinline__ uint32_t bit_word(uint64_t x, int b) {
    return 0u - (uint32_t)((x >> b) & 1u);
}

// K index of the reflexive frame with compact index c: the n diagonal edge
// bits are inserted as ones, the off-diagonal bits taken from c in order
// (monotone, so compact order is K order).
__host__ __device__ __forceinline__ uint64_t t_to_k(uint64_t c, int n) {
    uint64_t f = 0;
    int j = 0;
    for (int e = 0; e < n * n; ++e) {
        if (e % (n + 1) == 0) {
            f |= 1ull << e;
        } else {
            f |= ((c >> j) & 1ull) << e;
            ++j;
        }
    }
    return f;
}

// Edge words of the K-class word: frame index = 32*word + lane.
template <int N>
__device__ __forceinline__ void k_frame_word(uint64_t word, uint32_t (&E)[N * N]) {
    const uint64_t base = word << 5;
#pragma unroll
    for (int e = 0; e < N * N; ++e) E[e] = e < 5 ? lane_pattern(e) : bit_word(base, e);
}

// Edge words of the T-class word: compact index = 32*word + lane.
template <int N>
__device__ __forceinline__ void t_frame_word(uint64_t word, uint32_t (&E)[N * N]) {
    const uint64_t base = word << 5;
#pragma unroll
    for (int w = 0; w < N; ++w) {
#pragma unroll
        for (int v = 0; v < N; ++v) {
            const int j = w * N + v - w - (v > w ? 1 : 0);   // off-diagonal rank
            E[w * N + v] = (w == v) ? 0xFFFFFFFFu : (j < 5 ? lane_pattern(j) : bit_word(base, j));
        }
    }
}

// Edge words from 32 explicit K indices (lane l <- idx[l]).
template <int N>
__device__ __forceinline__ void list_frame_word(const uint64_t *idx, int count, uint32_t (&E)[N * N]) {
#pragma unroll
    for (int e = 0; e < N * N; ++e) E[e] = 0;
    for (int l = 0; l < count; ++l) {
        const uint64_t f = idx[l];
#pragma unroll
        for (int e = 0; e < N * N; ++e) E[e] |= (uint32_t)((f >> e) & 1u) << l;
    }
}

// Lanes of a word that are transitive (and, if sym, symmetric) frames.
template <int N>
__device__ __forceinline__ uint32_t preorder_mask(const uint32_t (&E)[N * N], bool sym) {
    uint32_t m = 0xFFFFFFFFu;
#pragma unroll
    for (int w = 0; w < N; ++w)
#pragma unroll
        for (int v = 0; v < N; ++v)
#pragma unroll
            for (int u = 0; u < N; ++u) m &= ~(E[w * N + v] & E[v * N + u]) | E[w * N + u];
    if (sym) {
#pragma unroll
        for (int w = 0; w < N; ++w)
#pragma unroll
            for (int v = w + 1; v < N; ++v) m &= ~(E[w * N + v] ^ E[v * N + w]);
    }
    return m;
}

// ----------------------------------------------------------- interpreter
//
// Accumulator machine of mk.h, evaluated for U "units" at once (U
// valuations of one frame word in the census, U frame words under one
// valuation in the separation search), so that every dispatched
// instruction carries U times the logic work.  A[U][N] lives in registers;
// the stack lives in shared memory, one column per thread (element (d, u,
// w) at stack[((d*U + u)*N + w) * BLOCK], bank-conflict free); atom truth
// sets come from shared-memory rows (see atom_row_word).
//
// Programs are pre-decoded when a CTA stages them (decode_program): one
// byte per instruction holding the op (MK_OP_END after the last one) and a
// 16-bit word offset holding the operand already scaled (stack entry d ->
// d * U*N*BLOCK, variable i -> i * RS), so dispatch is a table jump with no
// decoding arithmetic.  A PUSH is always followed by an instruction that
// starts a new subtree (a load, or a modal step on an atom), which does not
// read A: the decoder folds the PUSH into it as a flag (bit 5 of the op
// byte) and the stack entry (bits 6-7), and the interpreter saves A before
// executing it -- one dispatch instead of two.

constexpr uint32_t MK_DEC_PUSH = 32u;   // decoded op: save A to the stack first
constexpr int MK_OP_END = MK_NUM_OPS;

// Words per variable in an atom row (a multiple of 4 for 16-byte loads).
template <int N>
struct RowShape {
    static constexpr int RS = (N + 3) & ~3;
    static constexpr int WORDS = 4 * RS;   // MK_MAX_VARS variables
};

// Word w of variable i in the atom row of valuation value `val`: all ones
// iff p_i holds at world w (bit i*N+w of the valuation), i.e. the
// valuation's truth set of p_i, the same for all 32 frame lanes.
template <int N>
__device__ __forceinline__ uint32_t atom_row_word(uint32_t val, int idx) {
    const int i = idx / RowShape<N>::RS, w = idx % RowShape<N>::RS;
    return w < N ? 0u - ((val >> (i * N + w)) & 1u) : 0u;
}

// An op that does not read A (the ones a PUSH can be folded into).
__host__ __device__ __forceinline__ bool fresh_op(int op) {
    return op == MK_OP_LDV || op == MK_OP_LDT || op == MK_OP_LDF || op == MK_OP_LDNV || op >= MK_OP_BOX_V;
}

// Decode program p into ops[0..m] (ops[m] = END, m <= n_instr) and offs[0..m).
// FOLD: fold each PUSH into the op after it (pays off when a dispatch
// carries many units; run_program must be instantiated with the same FOLD).
template <int N, int U, int BLOCK, bool FOLD = true>
__device__ __forceinline__ void decode_program(const mk_program &p, uint8_t *ops, uint16_t *offs) {
    int j = 0;
    uint32_t push = 0;                                  // pending PUSH folded into the next op
    for (int i = 0; i < p.n_instr; ++i) {
        const int op = p.code[i] & 31, arg = p.code[i] >> 5;
        if (FOLD && op == MK_OP_PUSH && !push && i + 1 < p.n_instr && fresh_op(p.code[i + 1] & 31)) {
            push = MK_DEC_PUSH | ((uint32_t)arg << 6);
            continue;
        }
        ops[j] = (uint8_t)(op | push);
        push = 0;
        const bool stack_op = op >= MK_OP_PUSH && op <= MK_OP_IFF_S;
        offs[j] = (uint16_t)(stack_op ? arg * (U * N * BLOCK) : arg * RowShape<N>::RS);
        ++j;
    }
    ops[j] = (uint8_t)MK_OP_END;
    offs[j] = 0;
}

template <int N>
__device__ __forceinline__ void load_atom(const uint32_t *src, uint32_t (&x)[N]) {
    constexpr int RS = RowShape<N>::RS;
    const uint4 *p = reinterpret_cast<const uint4 *>(src);
    uint32_t t[RS];
#pragma unroll
    for (int q = 0; q < RS / 4; ++q) {
        const uint4 v = p[q];
        t[4 * q] = v.x;
        t[4 * q + 1] = v.y;
        t[4 * q + 2] = v.z;
        t[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int w = 0; w < N; ++w) x[w] = t[w];
}

template <int N>
__device__ __forceinline__ void box_op(uint32_t (&a)[N], const uint32_t (&E)[N * N]) {
    uint32_t t[N];
#pragma unroll
    for (int v = 0; v < N; ++v) t[v] = a[v];
#pragma unroll
    for (int w = 0; w < N; ++w) {
        uint32_t acc = 0xFFFFFFFFu;
#pragma unroll
        for (int v = 0; v < N; ++v) acc &= t[v] | ~E[w * N + v];
        a[w] = acc;
    }
}

template <int N>
__device__ __forceinline__ void dia_op(uint32_t (&a)[N], const uint32_t (&E)[N * N]) {
    uint32_t t[N];
#pragma unroll
    for (int v = 0; v < N; ++v) t[v] = a[v];
#pragma unroll
    for (int w = 0; w < N; ++w) {
        uint32_t acc = 0u;
#pragma unroll
        for (int v = 0; v < N; ++v) acc |= t[v] & E[w * N + v];
        a[w] = acc;
    }
}

// Run a decoded program on U units.  Unit u's atom row is row0 + u*ROWSTEP
// (ROWSTEP = 0: all units share one valuation); its frame word is
// E[NE == 1 ? 0 : u]; stack: this thread's column.
template <int N, int U, int NE, int BLOCK, int ROWSTEP, bool FOLD = true>
__device__ __forceinline__ void run_program(const uint8_t *ops, const uint16_t *offs, const uint32_t *row0,
                                            const uint32_t (&E)[NE][N * N], uint32_t *stack,
                                            uint32_t (&A)[U][N]) {
    uint32_t op = ops[0], off = offs[0];
    for (int pc = 1;; ++pc) {
        const uint32_t op_next = ops[pc], off_next = offs[pc];
        uint32_t *st = stack + off;
        const uint32_t *rw = row0 + off;
        if (FOLD && (op & MK_DEC_PUSH)) {               // folded PUSH: save A first
            uint32_t *ps = stack + (op >> 6) * (U * N * BLOCK);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int w = 0; w < N; ++w) ps[(u * N + w) * BLOCK] = A[u][w];
            op &= MK_DEC_PUSH - 1u;
        }
        switch (op) {
        case MK_OP_LDV:
#pragma unroll
            for (int u = 0; u < U; ++u) load_atom<N>(rw + u * ROWSTEP, A[u]);
            break;
        case MK_OP_LDT:
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] = 0xFFFFFFFFu;
            break;
        case MK_OP_LDF:
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] = 0u;
            break;
        case MK_OP_NOT:
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] = ~A[u][w];
            break;
        case MK_OP_BOX:
#pragma unroll
            for (int u = 0; u < U; ++u) box_op<N>(A[u], E[NE == 1 ? 0 : u]);
            break;
        case MK_OP_DIA:
#pragma unroll
            for (int u = 0; u < U; ++u) dia_op<N>(A[u], E[NE == 1 ? 0 : u]);
            break;
        case MK_OP_PUSH:
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int w = 0; w < N; ++w) st[(u * N + w) * BLOCK] = A[u][w];
            break;
        case MK_OP_AND_S:
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] &= st[(u * N + w) * BLOCK];
            break;
        case MK_OP_OR_S:
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] |= st[(u * N + w) * BLOCK];
            break;
        case MK_OP_IMP_S:
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] = ~st[(u * N + w) * BLOCK] | A[u][w];
            break;
        case MK_OP_RIMP_S:
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] = ~A[u][w] | st[(u * N + w) * BLOCK];
            break;
        case MK_OP_IFF_S:
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] = ~(A[u][w] ^ st[(u * N + w) * BLOCK]);
            break;
        case MK_OP_AND_V:
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t x[N];
                load_atom<N>(rw + u * ROWSTEP, x);
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] &= x[w];
            }
            break;
        case MK_OP_OR_V:
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t x[N];
                load_atom<N>(rw + u * ROWSTEP, x);
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] |= x[w];
            }
            break;
        case MK_OP_IMP_V:
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t x[N];
                load_atom<N>(rw + u * ROWSTEP, x);
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] = ~A[u][w] | x[w];
            }
            break;
        case MK_OP_RIMP_V:
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t x[N];
                load_atom<N>(rw + u * ROWSTEP, x);
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] = ~x[w] | A[u][w];
            }
            break;
        case MK_OP_LDNV:
#pragma unroll
            for (int u = 0; u < U; ++u) {
                load_atom<N>(rw + u * ROWSTEP, A[u]);
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] = ~A[u][w];
            }
            break;
        case MK_OP_AND_NV:
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t x[N];
                load_atom<N>(rw + u * ROWSTEP, x);
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] &= ~x[w];
            }
            break;
        case MK_OP_OR_NV:
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t x[N];
                load_atom<N>(rw + u * ROWSTEP, x);
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] |= ~x[w];
            }
            break;
        case MK_OP_IMP_NV:
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t x[N];
                load_atom<N>(rw + u * ROWSTEP, x);
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] = ~A[u][w] | ~x[w];
            }
            break;
        case MK_OP_BOX_V:
#pragma unroll
            for (int u = 0; u < U; ++u) {
                load_atom<N>(rw + u * ROWSTEP, A[u]);
                box_op<N>(A[u], E[NE == 1 ? 0 : u]);
            }
            break;
        case MK_OP_DIA_V:
#pragma unroll
            for (int u = 0; u < U; ++u) {
                load_atom<N>(rw + u * ROWSTEP, A[u]);
                dia_op<N>(A[u], E[NE == 1 ? 0 : u]);
            }
            break;
        case MK_OP_BOX_NV:
#pragma unroll
            for (int u = 0; u < U; ++u) {
                load_atom<N>(rw + u * ROWSTEP, A[u]);
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] = ~A[u][w];
                box_op<N>(A[u], E[NE == 1 ? 0 : u]);
            }
            break;
        case MK_OP_DIA_NV:
#pragma unroll
            for (int u = 0; u < U; ++u) {
                load_atom<N>(rw + u * ROWSTEP, A[u]);
#pragma unroll
                for (int w = 0; w < N; ++w) A[u][w] = ~A[u][w];
                dia_op<N>(A[u], E[NE == 1 ? 0 : u]);
            }
            break;
        case MK_OP_END:
            return;
        default:
            __builtin_unreachable();
        }
        op = op_next;
        off = off_next;
    }
}

// A program read from device memory is checked once by the CTA that stages
// it: every instruction must be a known op whose operand names an existing
// variable or stack entry.
__device__ __forceinline__ bool program_ok(const mk_program &p) {
    if (p.n_instr == 0 || p.n_instr > MK_MAX_CODE || p.nvars > MK_MAX_VARS || p.depth > MK_MAX_STACK)
        return false;
    for (int i = 0; i < p.n_instr; ++i) {
        const int op = p.code[i] & 31, arg = p.code[i] >> 5;
        if (op >= MK_NUM_OPS) return false;
        if (op == MK_OP_LDV || op >= MK_OP_AND_V) {
            if (arg >= p.nvars) return false;
        } else if (op >= MK_OP_PUSH) {
            if (arg >= p.depth) return false;
        } else if (arg != 0) {
            return false;
        }
    }
    return true;
}

// Separation split key: sampled << 63 | (n-1) << 60 | f << 24 | x << 3 | w
// (f < 2^36: K index or sample number; x < 2^21; w < 8).  Exhaustive sizes
// are searched before sampled ones, so the key order is the search order.
__host__ __device__ __forceinline__ uint64_t split_key(int sampled, int n, uint64_t f, uint64_t x, uint64_t w) {
    return ((uint64_t)(sampled ? 1 : 0) << 63) | ((uint64_t)(n - 1) << 60) | (f << 24) | (x << 3) | w;
}

// Valuation set of a layer: exhaustive iff S == 0, k <= 1 or 2^(k n) <= S.
__host__ __device__ __forceinline__ bool exhaustive_vals(int k, int n, uint32_t S) {
    if (S == 0 || k <= 1) return true;
    if (k * n >= 32) return false;
    return (1ull << (k * n)) <= (uint64_t)S;
}

// ---------------------------------------------------------- SplitMix64
// Steele, Lea, Flood (OOPSLA 2014): output j of the generator started at
// state s is mix(s + (j+1) * gamma).
__host__ __device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t sm_out(uint64_t state, uint64_t j) {
    return sm_mix(state + (j + 1) * 0x9E3779B97F4A7C15ull);
}
__host__ __device__ __forceinline__ uint64_t sm_stream(uint64_t seed, uint64_t tag, uint64_t n) {
    return sm_mix(seed ^ (tag << 32) ^ n);
}
// Sampled relation s on n <= 8 worlds (row-major edge mask); see mk.h.
__host__ __device__ __forceinline__ uint64_t sample_relation(uint64_t state, int n, uint64_t s) {
    const uint64_t d0 = sm_out(state, 9 * s);
    const uint64_t t = 26 + (((d0 >> 32) * 103ull) >> 32);
    uint64_t mask = 0;
    for (int g = 0; g < (n * n + 7) / 8; ++g) {
        const uint64_t d = sm_out(state, 9 * s + 1 + g);
        for (int b = 0; b < 8 && g * 8 + b < n * n; ++b)
            if (((d >> (8 * b)) & 0xFFu) < t) mask |= 1ull << (g * 8 + b);
    }
    return mask;
}

}  // namespace mkd
