/*
 * tier1.c -- the oracle's second tier: a mask evaluator for whole census
 * layers, fast enough to compute every five-world layer of a formula batch
 * on the host cores (tier 0, oracle.c, spends about a core-hour on one
 * five-world K layer with 256 valuations; tier 1 a few core-seconds).
 *
 * TEST INFRASTRUCTURE ONLY, like oracle.c: only tests/ and the scripts that
 * write the stored results under tests/golden/ use it.  It shares no code
 * with the CUDA path.  Formulas come from oracle.c's parser
 * (orc_parse_tree) and the parse tree is evaluated as it stands: no normal
 * form, no constant folding, nothing of the product's compiler.
 *
 * It is not plain.  64 consecutive K-indexed frames share one machine word
 * (bit j of word i is frame 64 i + j), so a subformula's truth set at world w
 * is one uint64_t per word: the "set of worlds as a bitmask" of Sec. 3 turned
 * sideways, one bit per frame; the evaluator walks the tree once for a
 * block of 4 words (256 frames).  Its results count only where they equal
 * tier 0's (the satisfaction clauses over explicit relations): the tests
 * compare the two on every layer through four worlds, and the script that
 * stores tier-1 results first checks it against every five-world layer tier
 * 0 has stored.
 *
 * Readings (the same as oracle.c's): R(w,v) is bit e = w n + v of the frame
 * index; p_i holds at w iff bit i n + w of the valuation index; valuations
 * are exhaustive when S == 0, k <= 1 or 2^(k n) <= S, else the S sampled
 * values in slot order; the witness is the least (frame, valuation, world).
 *
 * Edge words of word i: for e < 6, bit e of the frame index is bit e of the
 * lane index j, so the word is the fixed pattern with bit j set iff bit e of
 * j is; for e >= 6, bit e of the frame index is bit e - 6 of i, the same for
 * all 64 lanes (all ones or all zeros).  Per (word, valuation) the tree runs
 * bottom-up with one truth word per world:
 *   []a at w = AND over v of (a at v  OR  NOT E(w,v))
 *   <>a at w = OR  over v of (a at v  AND E(w,v))
 * and the Boolean connectives word by word.  Class filters are word masks:
 * reflexive = AND_w E(w,w); transitive = AND over (u,v,w) of
 * NOT (E(u,v) AND E(v,w) AND NOT E(u,w)); symmetric = AND over (u,v) of
 * NOT (E(u,v) XOR E(v,u)).
 */
#include <stdint.h>
#include <string.h>
#include <omp.h>

#define T1_MAX_NODES 256   /* oracle.c's ORC_MAX_NODES */
#define T1_MAX_N 6          /* worlds held by the evaluator (the census takes n <= 5) */

int orc_parse_tree(const char *text, int *kind, int *var, int *a, int *b, int *nn, int *root, int *nvars);

enum { K_TOP, K_BOT, K_VAR, K_NOT, K_AND, K_OR, K_IMP, K_IFF, K_BOX, K_DIA };

typedef struct {
    int kind[T1_MAX_NODES], var[T1_MAX_NODES], a[T1_MAX_NODES], b[T1_MAX_NODES];
    int nn, root, nvars;
} t1_tree;

/* the layout of oracle.c's orc_census_out */
typedef struct {
    uint64_t frames, cm_count, frames_refuted;
    int32_t found, nvals;
    uint64_t wf;
    uint32_t wv, ww;
} t1_out;

static uint64_t lane_pattern(int e) {
    uint64_t m = 0;
    for (int j = 0; j < 64; j++)
        if ((j >> e) & 1) m |= (uint64_t)1 << j;
    return m;
}

/* a block is T1_W consecutive words (64 T1_W frames): E[e][q] is edge e's
   word for word 4 b + q of block b */
#define T1_W 4

static void edge_words(uint64_t block, int n, const uint64_t *P, uint64_t (*E)[T1_W]) {
    for (int e = 0; e < n * n; e++)
        for (int q = 0; q < T1_W; q++) {
            const uint64_t word = block * T1_W + (uint64_t)q;
            E[e][q] = e < 6 ? P[e] : (((word >> (e - 6)) & 1u) ? ~(uint64_t)0 : 0);
        }
}

/* cls: 0 K, 1 T, 2 S4, 3 S5, 4 K4 (transitive), as in oracle.c */
static uint64_t class_mask(int cls, int n, const uint64_t (*E)[T1_W], int q) {
    uint64_t m = ~(uint64_t)0;
    if (cls == 0) return m;
    if (cls >= 1 && cls <= 3)
        for (int w = 0; w < n; w++) m &= E[w * n + w][q];
    if (cls >= 2)
        for (int u = 0; u < n; u++)
            for (int v = 0; v < n; v++)
                for (int w = 0; w < n; w++) m &= ~(E[u * n + v][q] & E[v * n + w][q] & ~E[u * n + w][q]);
    if (cls == 3)
        for (int u = 0; u < n; u++)
            for (int v = 0; v < n; v++) m &= ~(E[u * n + v][q] ^ E[v * n + u][q]);
    return m;
}

/* T[i][w][q] = truth word of node i at world w, word q of the block, under
   valuation x */
static void eval_tree(const t1_tree *t, int n, const uint64_t (*E)[T1_W], uint64_t x,
                      uint64_t (*T)[T1_MAX_N][T1_W]) {
    const uint64_t ONES = ~(uint64_t)0;
    for (int i = 0; i < t->nn; i++) {
        uint64_t (*A)[T1_W] = t->a[i] >= 0 ? T[t->a[i]] : NULL;
        uint64_t (*B)[T1_W] = t->b[i] >= 0 ? T[t->b[i]] : NULL;
        uint64_t (*R)[T1_W] = T[i];
        int w, v, q;
        switch (t->kind[i]) {
        case K_TOP:
            for (w = 0; w < n; w++) for (q = 0; q < T1_W; q++) R[w][q] = ONES;
            break;
        case K_BOT:
            for (w = 0; w < n; w++) for (q = 0; q < T1_W; q++) R[w][q] = 0;
            break;
        case K_VAR:
            for (w = 0; w < n; w++) {
                const uint64_t bit = ((x >> (t->var[i] * n + w)) & 1u) ? ONES : 0;
                for (q = 0; q < T1_W; q++) R[w][q] = bit;
            }
            break;
        case K_NOT:
            for (w = 0; w < n; w++) for (q = 0; q < T1_W; q++) R[w][q] = ~A[w][q];
            break;
        case K_AND:
            for (w = 0; w < n; w++) for (q = 0; q < T1_W; q++) R[w][q] = A[w][q] & B[w][q];
            break;
        case K_OR:
            for (w = 0; w < n; w++) for (q = 0; q < T1_W; q++) R[w][q] = A[w][q] | B[w][q];
            break;
        case K_IMP:
            for (w = 0; w < n; w++) for (q = 0; q < T1_W; q++) R[w][q] = ~A[w][q] | B[w][q];
            break;
        case K_IFF:
            for (w = 0; w < n; w++) for (q = 0; q < T1_W; q++) R[w][q] = ~(A[w][q] ^ B[w][q]);
            break;
        case K_BOX:
            for (w = 0; w < n; w++) {
                uint64_t r[T1_W];
                for (q = 0; q < T1_W; q++) r[q] = ONES;
                for (v = 0; v < n; v++)
                    for (q = 0; q < T1_W; q++) r[q] &= A[v][q] | ~E[w * n + v][q];
                for (q = 0; q < T1_W; q++) R[w][q] = r[q];
            }
            break;
        case K_DIA:
            for (w = 0; w < n; w++) {
                uint64_t r[T1_W];
                for (q = 0; q < T1_W; q++) r[q] = 0;
                for (v = 0; v < n; v++)
                    for (q = 0; q < T1_W; q++) r[q] |= A[v][q] & E[w * n + v][q];
                for (q = 0; q < T1_W; q++) R[w][q] = r[q];
            }
            break;
        }
    }
}

static int exhaustive(int k, int n, uint32_t S) {
    if (S == 0 || k <= 1) return 1;
    if (k * n >= 32) return 0;
    return ((uint64_t)1 << (k * n)) <= S;
}

/* Census of one formula over all class-`cls` frames on n <= 5 worlds: the
   outputs of oracle.c's orc_census (Alg. 1, Sec. 4).  Returns 0, -1 on a
   parse error, -2 on bad arguments, -3 if sampled valuations are needed and
   samp is NULL. */
int orc_census_tier1(const char *text, int cls, int n, uint32_t S, const uint32_t *samp, t1_out *out) {
    static t1_tree zero;
    t1_tree t = zero;
    memset(out, 0, sizeof(*out));
    if (n < 1 || n > 5 || cls < 0 || cls > 4) return -2;
    if (orc_parse_tree(text, t.kind, t.var, t.a, t.b, &t.nn, &t.root, &t.nvars)) return -1;
    for (int i = 0; i < t.nn; i++)
        if (t.a[i] >= i || t.b[i] >= i) return -1;      /* children first, as the parser numbers them */
    const int k = t.nvars;
    const int exh = exhaustive(k, n, S);
    if (!exh && samp == NULL) return -3;
    const uint64_t nval = exh ? (uint64_t)1 << (k * n) : S;
    const uint32_t vmask = (k * n >= 32) ? 0xFFFFFFFFu : (uint32_t)(((uint64_t)1 << (k * n)) - 1);
    const uint64_t nframes = (uint64_t)1 << (n * n);
    const uint64_t nwords = (nframes + 63) / 64;
    const uint64_t last_valid = nframes >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << nframes) - 1);
    uint64_t P[6];
    for (int e = 0; e < 6; e++) P[e] = lane_pattern(e);
    out->nvals = (int32_t)nval;

    const uint64_t nblocks = (nwords + T1_W - 1) / T1_W;
    uint64_t frames = 0, cm = 0, fr = 0, best = UINT64_MAX;
#pragma omp parallel
    {
        uint64_t T[T1_MAX_NODES][T1_MAX_N][T1_W], E[T1_MAX_N * T1_MAX_N][T1_W];
        uint64_t lbest = UINT64_MAX;
#pragma omp for schedule(dynamic, 16) reduction(+ : frames, cm, fr)
        for (int64_t bi = 0; bi < (int64_t)nblocks; bi++) {
            edge_words((uint64_t)bi, n, P, E);
            uint64_t in[T1_W], any[T1_W], best_j[T1_W], best_w[T1_W];
            int best_lane[T1_W], live = 0;
            for (int q = 0; q < T1_W; q++) {
                const uint64_t word = (uint64_t)bi * T1_W + (uint64_t)q;
                const uint64_t valid = word >= nwords ? 0 : word == nwords - 1 ? last_valid : ~(uint64_t)0;
                in[q] = class_mask(cls, n, E, q) & valid;
                frames += (uint64_t)__builtin_popcountll(in[q]);
                live |= in[q] != 0;
                any[q] = 0;
                best_lane[q] = 64;
                best_j[q] = best_w[q] = 0;
            }
            if (!live) continue;
            for (uint64_t j = 0; j < nval; j++) {
                const uint64_t x = exh ? j : (samp[j] & vmask);
                eval_tree(&t, n, (const uint64_t (*)[T1_W])E, x, T);
                for (int q = 0; q < T1_W; q++) {
                    uint64_t ref = 0;
                    for (int w = 0; w < n; w++) ref |= ~T[t.root][w][q];
                    ref &= in[q];
                    if (!ref) continue;
                    cm += (uint64_t)__builtin_popcountll(ref);
                    /* the least lane of any[q] can only fall; when it does,
                       this valuation is the first to refute that lane */
                    const uint64_t fresh = ref & ~any[q];
                    if (fresh && __builtin_ctzll(fresh) < best_lane[q]) {
                        best_lane[q] = __builtin_ctzll(fresh);
                        best_j[q] = j;
                        for (int w = 0; w < n; w++)
                            if ((~T[t.root][w][q] >> best_lane[q]) & 1u) { best_w[q] = (uint64_t)w; break; }
                    }
                    any[q] |= ref;
                }
            }
            for (int q = 0; q < T1_W; q++) {
                fr += (uint64_t)__builtin_popcountll(any[q]);
                if (any[q]) {
                    const uint64_t frame = ((uint64_t)bi * T1_W + (uint64_t)q) * 64 + (uint64_t)best_lane[q];
                    const uint64_t key = (frame << 24) | (best_j[q] << 3) | best_w[q];
                    if (key < lbest) lbest = key;
                }
            }
        }
#pragma omp critical
        {
            if (lbest < best) best = lbest;
        }
    }
    out->frames = frames;
    out->cm_count = cm;
    out->frames_refuted = fr;
    if (best != UINT64_MAX) {
        out->found = 1;
        out->wf = best >> 24;
        out->wv = (uint32_t)((best >> 3) & 0x1FFFFFu);
        out->ww = (uint32_t)(best & 7u);
    }
    return 0;
}

/* the layout of oracle.c's orc_pair_out */
typedef struct {
    int32_t found, nvals;
    uint64_t f;
    uint32_t v, w;
    int32_t phi_val, psi_val;
    uint64_t frames_disagree;
} t1_pair_out;

static int load_tree(const char *text, t1_tree *t) {
    if (orc_parse_tree(text, t->kind, t->var, t->a, t->b, &t->nn, &t->root, &t->nvars)) return -1;
    for (int i = 0; i < t->nn; i++)
        if (t->a[i] >= i || t->b[i] >= i) return -1;
    return 0;
}

/* Separation of phi and psi over the K frames on n <= 6 worlds with K index
   in [f_lo, f_hi): the least (frame, valuation, world) at which the two take
   different truth values, and the number of frames with any difference --
   the outputs of oracle.c's orc_pair_layer (Def. 2, Prop. 4).  Returns 0, -1
   on a parse error, -2 on bad arguments, -3 if sampled valuations are needed
   and samp is NULL. */
int orc_pair_tier1(const char *phi, const char *psi, int n, uint32_t S, const uint32_t *samp,
                   uint64_t f_lo, uint64_t f_hi, t1_pair_out *out) {
    static t1_tree zero;
    t1_tree ta = zero, tb = zero;
    memset(out, 0, sizeof(*out));
    if (n < 1 || n > T1_MAX_N) return -2;
    if (load_tree(phi, &ta) || load_tree(psi, &tb)) return -1;
    const int k = ta.nvars > tb.nvars ? ta.nvars : tb.nvars;
    const int exh = exhaustive(k, n, S);
    if (!exh && samp == NULL) return -3;
    const uint64_t nval = exh ? (uint64_t)1 << (k * n) : S;
    const uint32_t vmask = (k * n >= 32) ? 0xFFFFFFFFu : (uint32_t)(((uint64_t)1 << (k * n)) - 1);
    const uint64_t nframes = (uint64_t)1 << (n * n);
    if (f_hi > nframes) f_hi = nframes;
    out->nvals = (int32_t)nval;
    if (f_lo >= f_hi) return 0;
    const uint64_t b0 = f_lo / (64 * T1_W), b1 = (f_hi + 64 * T1_W - 1) / (64 * T1_W);
    uint64_t P[6];
    for (int e = 0; e < 6; e++) P[e] = lane_pattern(e);

    uint64_t dis = 0, best = UINT64_MAX;
    int best_a = 0;
#pragma omp parallel
    {
        uint64_t TA[T1_MAX_NODES][T1_MAX_N][T1_W], TB[T1_MAX_NODES][T1_MAX_N][T1_W];
        uint64_t E[T1_MAX_N * T1_MAX_N][T1_W];
        uint64_t lbest = UINT64_MAX;
        int lbest_a = 0;
#pragma omp for schedule(dynamic, 16) reduction(+ : dis)
        for (int64_t bi = (int64_t)b0; bi < (int64_t)b1; bi++) {
            edge_words((uint64_t)bi, n, P, E);
            uint64_t in[T1_W], any[T1_W], best_j[T1_W], best_w[T1_W];
            int best_lane[T1_W], best_val[T1_W];
            for (int q = 0; q < T1_W; q++) {
                /* lanes of word bi*T1_W + q whose frames lie in [f_lo, f_hi) */
                const uint64_t base = ((uint64_t)bi * T1_W + (uint64_t)q) * 64;
                uint64_t m = ~(uint64_t)0;
                if (base + 64 <= f_lo || base >= f_hi) m = 0;
                else {
                    if (f_lo > base) m &= ~(uint64_t)0 << (f_lo - base);
                    if (f_hi < base + 64) m &= ~(~(uint64_t)0 << (f_hi - base));
                }
                in[q] = m;
                any[q] = 0;
                best_lane[q] = 64;
                best_j[q] = best_w[q] = 0;
                best_val[q] = 0;
            }
            for (uint64_t j = 0; j < nval; j++) {
                const uint64_t x = exh ? j : (samp[j] & vmask);
                eval_tree(&ta, n, (const uint64_t (*)[T1_W])E, x, TA);
                eval_tree(&tb, n, (const uint64_t (*)[T1_W])E, x, TB);
                for (int q = 0; q < T1_W; q++) {
                    uint64_t d = 0;
                    for (int w = 0; w < n; w++) d |= TA[ta.root][w][q] ^ TB[tb.root][w][q];
                    d &= in[q];
                    if (!d) continue;
                    const uint64_t fresh = d & ~any[q];
                    if (fresh && __builtin_ctzll(fresh) < best_lane[q]) {
                        const int L = __builtin_ctzll(fresh);
                        best_lane[q] = L;
                        best_j[q] = j;
                        for (int w = 0; w < n; w++)
                            if (((TA[ta.root][w][q] ^ TB[tb.root][w][q]) >> L) & 1u) {
                                best_w[q] = (uint64_t)w;
                                best_val[q] = (int)((TA[ta.root][w][q] >> L) & 1u);
                                break;
                            }
                    }
                    any[q] |= d;
                }
            }
            for (int q = 0; q < T1_W; q++) {
                dis += (uint64_t)__builtin_popcountll(any[q]);
                if (any[q]) {
                    const uint64_t frame = ((uint64_t)bi * T1_W + (uint64_t)q) * 64 + (uint64_t)best_lane[q];
                    const uint64_t key = (frame << 24) | (best_j[q] << 3) | best_w[q];
                    if (key < lbest) { lbest = key; lbest_a = best_val[q]; }
                }
            }
        }
#pragma omp critical
        {
            if (lbest < best) { best = lbest; best_a = lbest_a; }
        }
    }
    out->frames_disagree = dis;
    if (best != UINT64_MAX) {
        out->found = 1;
        out->f = best >> 24;
        out->v = (uint32_t)((best >> 3) & 0x1FFFFFu);
        out->w = (uint32_t)(best & 7u);
        out->phi_val = best_a;
        out->psi_val = !best_a;
    }
    return 0;
}
