// mk_relgen.cuh -- relations on up to 16 worlds for the large-frame
// separation (Sec. 7): the 39 stress templates and the six adversarial
// generators of Table 2, as successor masks (bit v of s[w] <=> R(w, v)).
//
// Every relation is a pure function of (generator, seed, n, index), drawn
// from counter-based SplitMix64 streams, so a kernel builds relation i
// without any state and the host rebuilds it for a certificate.
//
// Draws of relation i of a generator (d_j = output D*i + j of the stream):
//   Erdos-Renyi       stream tag 2, D = 9 (n <= 8) or 33: d_0 gives the
//                     threshold t = 26 + floor(hi32(d_0) * 103 / 2^32) in
//                     [26, 128] (p = t/256 in [0.1, 0.5]); edge e = w*n+v is
//                     present iff byte e%8 of d_(1+e/8) is below t.
//   other generators  stream tag 16 + gen, D = 40: d_0 -> t as above,
//                     d_1..d_32 -> one coin byte per edge as above,
//                     d_33..d_39 -> 28 16-bit choices c_j (chunk j%4 of
//                     d_(33+j/4)), pick(j, m) = floor(c_j * m / 2^16).
#pragma once
#include <cstdint>

#include "mk.h"
#include "mk_eval.cuh"

namespace mkd {

constexpr int REL_MAXN = MK_MAX_WORLDS_STRESS;
typedef uint32_t Succ[REL_MAXN];

#define MKRG __host__ __device__ __forceinline__

MKRG uint32_t full_mask(int n) { return n >= 32 ? 0xFFFFFFFFu : (1u << n) - 1u; }

MKRG void succ_clear(Succ &s) {
    for (int w = 0; w < REL_MAXN; ++w) s[w] = 0;
}
// edge w -> v, ignored when either end is outside 0..n-1
MKRG void succ_edge(Succ &s, int n, int w, int v) {
    if (w >= 0 && w < n && v >= 0 && v < n) s[w] |= 1u << v;
}

// Fork with branches 0 -> 1 -> ... -> b and 0 -> b+1 -> ... -> n-1.
MKRG void fork_succ(Succ &s, int n, int b) {
    for (int w = 0; w < b; ++w) succ_edge(s, n, w, w + 1);
    if (b + 1 < n) succ_edge(s, n, 0, b + 1);
    for (int w = b + 1; w + 1 < n; ++w) succ_edge(s, n, w, w + 1);
}

// The fixed sparse/dense templates: edge e iff byte e%8 of output e/8 of
// the stream (seed 0x5EED, tag 40 + variant, n) is below thresh.
MKRG void coin_template(Succ &s, int n, int variant, uint32_t thresh) {
    const uint64_t st = sm_stream(0x5EEDull, 40ull + (uint64_t)variant, (uint64_t)n);
    for (int e0 = 0; e0 < n * n; e0 += 8) {
        const uint64_t d = sm_out(st, (uint64_t)(e0 / 8));
        for (int b = 0; b < 8 && e0 + b < n * n; ++b)
            if (((d >> (8 * b)) & 0xFFu) < thresh) s[(e0 + b) / n] |= 1u << ((e0 + b) % n);
    }
}

// Stress template id on n worlds (h = floor(n/2), c = ceil(n/2)):
//  0 path            1 reverse path      2 reflexive path    3 path + loop at n-1
//  4 path + loop at 0  5 strict order (w<v)  6 w<=v           7 cycle
//  8 reverse cycle   9 reflexive cycle  10 two-way cycle    11 two-way path
// 12 out-star (0->v) 13 in-star         14 two-way star     15 reflexive out-star
// 16..19 forks with first branch length h, 1, 2, n-2    20 fork(h) + loops at its leaves
// 21 binary tree w -> 2w+1, 2w+2        22 its reverse      23 complete
// 24 complete without loops  25 loops only  26 empty        27 lasso: path + n-1 -> h
// 28 cycles on [0,h) and [h,n) joined by h-1 -> h
// 29..31 sparse (coin < 32)  32..34 dense (coin < 224)
// 35 comb: spine 0..c-1, teeth w -> c+w  36 w -> w+1, w+2
// 37 path + loops at odd worlds         38 reverse strict order (w>v)
// Returns false for an unknown id.
MKRG bool template_succ(int id, int n, Succ &s) {
    succ_clear(s);
    const int h = n / 2, c = (n + 1) / 2;
    const uint32_t all = full_mask(n);
    switch (id) {
    case 0: for (int w = 0; w + 1 < n; ++w) succ_edge(s, n, w, w + 1); break;
    case 1: for (int w = 1; w < n; ++w) succ_edge(s, n, w, w - 1); break;
    case 2: for (int w = 0; w < n; ++w) s[w] = ((1u << w) | (2u << w)) & all; break;
    case 3: for (int w = 0; w + 1 < n; ++w) succ_edge(s, n, w, w + 1); succ_edge(s, n, n - 1, n - 1); break;
    case 4: for (int w = 0; w + 1 < n; ++w) succ_edge(s, n, w, w + 1); succ_edge(s, n, 0, 0); break;
    case 5: for (int w = 0; w < n; ++w) s[w] = all & ~((2u << w) - 1u); break;
    case 6: for (int w = 0; w < n; ++w) s[w] = all & ~((1u << w) - 1u); break;
    case 7: for (int w = 0; w < n; ++w) succ_edge(s, n, w, (w + 1) % n); break;
    case 8: for (int w = 0; w < n; ++w) succ_edge(s, n, (w + 1) % n, w); break;
    case 9: for (int w = 0; w < n; ++w) { succ_edge(s, n, w, (w + 1) % n); succ_edge(s, n, w, w); } break;
    case 10: for (int w = 0; w < n; ++w) { succ_edge(s, n, w, (w + 1) % n); succ_edge(s, n, (w + 1) % n, w); } break;
    case 11: for (int w = 0; w + 1 < n; ++w) { succ_edge(s, n, w, w + 1); succ_edge(s, n, w + 1, w); } break;
    case 12: s[0] = all & ~1u; break;
    case 13: for (int w = 1; w < n; ++w) s[w] = 1u; break;
    case 14: s[0] = all & ~1u; for (int w = 1; w < n; ++w) s[w] = 1u; break;
    case 15: s[0] = all; for (int w = 1; w < n; ++w) s[w] = 1u << w; break;
    case 16: fork_succ(s, n, h); break;
    case 17: fork_succ(s, n, 1); break;
    case 18: fork_succ(s, n, 2); break;
    case 19: fork_succ(s, n, n - 2); break;
    case 20: fork_succ(s, n, h); succ_edge(s, n, h, h); succ_edge(s, n, n - 1, n - 1); break;
    case 21: for (int w = 0; w < n; ++w) { succ_edge(s, n, w, 2 * w + 1); succ_edge(s, n, w, 2 * w + 2); } break;
    case 22: for (int v = 1; v < n; ++v) succ_edge(s, n, v, (v - 1) / 2); break;
    case 23: for (int w = 0; w < n; ++w) s[w] = all; break;
    case 24: for (int w = 0; w < n; ++w) s[w] = all & ~(1u << w); break;
    case 25: for (int w = 0; w < n; ++w) s[w] = 1u << w; break;
    case 26: break;
    case 27: for (int w = 0; w + 1 < n; ++w) succ_edge(s, n, w, w + 1); succ_edge(s, n, n - 1, h); break;
    case 28:
        for (int w = 0; w < h; ++w) succ_edge(s, n, w, w + 1 < h ? w + 1 : 0);
        for (int w = h; w < n; ++w) succ_edge(s, n, w, w + 1 < n ? w + 1 : h);
        succ_edge(s, n, h - 1, h);
        break;
    case 29: case 30: case 31: coin_template(s, n, id - 29, 32); break;
    case 32: case 33: case 34: coin_template(s, n, id - 29, 224); break;
    case 35:
        for (int w = 0; w + 1 < c; ++w) succ_edge(s, n, w, w + 1);
        for (int w = 0; c + w < n; ++w) succ_edge(s, n, w, c + w);
        break;
    case 36: for (int w = 0; w < n; ++w) s[w] = ((2u << w) | (4u << w)) & all; break;
    case 37:
        for (int w = 0; w + 1 < n; ++w) succ_edge(s, n, w, w + 1);
        for (int w = 1; w < n; w += 2) succ_edge(s, n, w, w);
        break;
    case 38: for (int w = 0; w < n; ++w) s[w] = (1u << w) - 1u; break;
    default: return false;
    }
    return true;
}

// Draw source of one relation.
struct RelDraws {
    uint64_t st, base;
    MKRG uint64_t d(int j) const { return sm_out(st, base + (uint64_t)j); }
    MKRG uint32_t thresh() const { return 26u + (uint32_t)(((d(0) >> 32) * 103ull) >> 32); }
    MKRG uint32_t pick(int j, uint32_t m) const {
        const uint32_t cj = (uint32_t)(d(33 + j / 4) >> (16 * (j % 4))) & 0xFFFFu;
        return (uint32_t)(((uint64_t)cj * m) >> 16);
    }
};

// Edges e = w*n+v whose coin byte is below t, restricted to keep[w] & (1<<v).
MKRG void coin_edges(const RelDraws &g, int n, uint32_t t, const Succ &keep, Succ &s) {
    for (int e0 = 0; e0 < n * n; e0 += 8) {
        const uint64_t d = g.d(1 + e0 / 8);
        for (int b = 0; b < 8 && e0 + b < n * n; ++b) {
            const int w = (e0 + b) / n, v = (e0 + b) % n;
            if (((d >> (8 * b)) & 0xFFu) < t && ((keep[w] >> v) & 1u)) s[w] |= 1u << v;
        }
    }
}

MKRG void scc_succ(const RelDraws &g, int n, Succ &s) {
    const int a = 1 + (int)g.pick(0, (uint32_t)(n - 1));
    const uint32_t all = full_mask(n), lo_blk = (1u << a) - 1u, hi_blk = all & ~lo_blk;
    Succ keep;
    for (int w = 0; w < REL_MAXN; ++w) keep[w] = w < a ? lo_blk : (w < n ? hi_blk : 0u);
    succ_clear(s);
    if (a >= 2)
        for (int w = 0; w < a; ++w) succ_edge(s, n, w, w + 1 < a ? w + 1 : 0);
    if (n - a >= 2)
        for (int w = a; w < n; ++w) succ_edge(s, n, w, w + 1 < n ? w + 1 : a);
    coin_edges(g, n, g.thresh(), keep, s);
    succ_edge(s, n, a - 1, a);
}

// Relation idx of generator gen on n worlds; false for invalid arguments.
MKRG bool stress_relation(int gen, uint64_t seed, int n, uint64_t idx, Succ &s) {
    succ_clear(s);
    if (n < 1 || n > REL_MAXN || gen < 0 || gen >= MK_NUM_GENERATORS) return false;
    if (gen != MK_GEN_ER && n < 2) return false;
    Succ all_edges;
    for (int w = 0; w < REL_MAXN; ++w) all_edges[w] = w < n ? full_mask(n) : 0u;
    RelDraws g;
    if (gen == MK_GEN_ER) {
        g.st = sm_stream(seed, 2, (uint64_t)n);
        g.base = (n <= 8 ? 9ull : 33ull) * idx;
        coin_edges(g, n, g.thresh(), all_edges, s);
        return true;
    }
    g.st = sm_stream(seed, 16ull + (uint64_t)gen, (uint64_t)n);
    g.base = 40ull * idx;
    switch (gen) {
    case MK_GEN_FLIP: {
        template_succ((int)g.pick(0, MK_NUM_TEMPLATES), n, s);
        const int m = 1 + (int)g.pick(1, 4);
        for (int j = 0; j < m; ++j) {
            const uint32_t e = g.pick(2 + j, (uint32_t)(n * n));
            s[e / n] ^= 1u << (e % n);
        }
        break;
    }
    case MK_GEN_SCC:
        scc_succ(g, n, s);
        break;
    case MK_GEN_DEADEND: {
        coin_edges(g, n, g.thresh(), all_edges, s);
        const int m = 1 + (int)g.pick(0, 3);
        for (int j = 0; j < m; ++j) s[g.pick(1 + j, (uint32_t)n)] = 0u;
        break;
    }
    case MK_GEN_BACKEDGE: {
        for (int w = 0; w + 1 < n; ++w) succ_edge(s, n, w, w + 1);
        const int m = 1 + (int)g.pick(0, 4);
        for (int j = 0; j < m; ++j) {
            const int x = (int)g.pick(1 + 2 * j, (uint32_t)n), y = (int)g.pick(2 + 2 * j, (uint32_t)n);
            succ_edge(s, n, x > y ? x : y, x > y ? y : x);
        }
        break;
    }
    default: {   // MK_GEN_PERMSCC
        Succ q;
        scc_succ(g, n, q);
        int pi[REL_MAXN];
        for (int w = 0; w < REL_MAXN; ++w) pi[w] = w;
        for (int i = n - 1; i >= 1; --i) {
            const int j = (int)g.pick(4 + (n - 1 - i), (uint32_t)(i + 1));
            const int t = pi[i];
            pi[i] = pi[j];
            pi[j] = t;
        }
        for (int w = 0; w < n; ++w)
            for (int v = 0; v < n; ++v)
                if ((q[w] >> v) & 1u) s[pi[w]] |= 1u << pi[v];
        break;
    }
    }
    return true;
}

#undef MKRG

}  // namespace mkd
