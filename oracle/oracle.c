/*
 * oracle.c -- plain, slow CPU oracle for exhaustive finite Kripke evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call
 * this file: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline
 * leg (and bench.py --impl reference) use it.  It shares no code, header,
 * table or helper with the CUDA path.
 *
 * Everything here is the textbook definition written out, over explicit
 * relations (uint8 R[w*n+v]) and explicit valuations (uint8 V[i*n+w]):
 *
 *   formulas      phi ::= T | F | p_i | ~phi | phi&phi | phi|phi | phi->phi
 *                         | []phi | <>phi                     (Sec. 2)
 *                 (phi<->psi is accepted as sugar for the biconditional of
 *                  Prop. 4.)
 *   satisfaction  w |= []phi iff for all v, R(w,v) implies v |= phi;
 *                 w |= <>phi iff some v has R(w,v) and v |= phi   (Sec. 2)
 *   classes       K all frames, T reflexive, S4 reflexive+transitive,
 *                 S5 reflexive+transitive+symmetric, K4 transitive (Sec. 2)
 *   countermodel  (F, V, w) with M,w not|= phi                  (Sec. 2)
 *   census        per (formula, class, n): the number of refuted
 *                 (frame, valuation) pairs, the number of refuted frames,
 *                 and the lexicographically least (frame, valuation, world)
 *                 witness -- the outputs of the corpus scan of Alg. 1 (Sec. 4)
 *   separation    the least (n, frame, valuation, world) at which phi and
 *                 psi take different truth values (Def. 2, Prop. 4, Sec. 7)
 *   large frames  the stress templates and adversarial relation generators
 *                 of Sec. 7 / Table 2 on up to 16 worlds, and the same
 *                 separation order over an explicit list of relations
 *
 * Readings of the paper where it is silent:
 *   - frame index f of an n-world frame: R(w,v) is bit (w*n+v) of f
 *     (so successor mask succ[w] is bits [w*n, w*n+n) of f);
 *   - valuation index x: p_i holds at w iff bit (i*n+w) of x is set;
 *   - k = 1 + the highest variable index occurring (0 if none);
 *   - valuations are exhaustive (x = 0 .. 2^(k n)-1) when S == 0, k <= 1 or
 *     2^(k n) <= S; otherwise the S sampled values samp[j] (low k n bits) are
 *     used in slot order j, counted with multiplicity;
 *   - the witness valuation index is x for exhaustive valuations and the slot
 *     j for sampled ones;
 *   - sampled 7/8-world frames come from SplitMix64 (Steele, Lea and Flood,
 *     OOPSLA 2014) in its counter form, see orc_sample_frame().
 *
 * The evaluator computes each subformula's truth value at every world by the
 * satisfaction clauses above (a bool per world, no bit tricks).  Frame loops
 * run under OpenMP; every reduction is a sum or a lexicographic minimum, so
 * the results do not depend on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <ctype.h>
#include <omp.h>

#define ORC_MAX_NODES 256
#define ORC_MAX_VARS 8
#define ORC_MAX_WORLDS 32

enum { O_TOP, O_BOT, O_VAR, O_NOT, O_AND, O_OR, O_IMP, O_IFF, O_BOX, O_DIA };

typedef struct { int kind, var, a, b; } onode;
typedef struct { onode nd[ORC_MAX_NODES]; int nn, root, nvars, err; } oform;

/* ------------------------------------------------------------------ parser */

typedef struct { const char *s; int i; oform *f; } opar;

static void skip_ws(opar *p) { while (p->s[p->i] && isspace((unsigned char)p->s[p->i])) p->i++; }

static int lit(opar *p, const char *t) {
    skip_ws(p);
    size_t L = strlen(t);
    if (strncmp(p->s + p->i, t, L) != 0) return 0;
    /* a keyword must not run into an identifier character */
    if (isalpha((unsigned char)t[0]) && isalnum((unsigned char)p->s[p->i + L])) return 0;
    p->i += (int)L;
    return 1;
}

static int mk(opar *p, int kind, int var, int a, int b) {
    oform *f = p->f;
    if (f->nn >= ORC_MAX_NODES) { f->err = 1; return 0; }
    f->nd[f->nn].kind = kind; f->nd[f->nn].var = var;
    f->nd[f->nn].a = a; f->nd[f->nn].b = b;
    return f->nn++;
}

static int p_iff(opar *p);

static int p_unary(opar *p) {
    if (p->f->err) return 0;
    if (lit(p, "~") || lit(p, "!") || lit(p, "not")) return mk(p, O_NOT, 0, p_unary(p), -1);
    if (lit(p, "[]") || lit(p, "box")) return mk(p, O_BOX, 0, p_unary(p), -1);
    if (lit(p, "<>") || lit(p, "dia")) return mk(p, O_DIA, 0, p_unary(p), -1);
    if (lit(p, "(")) {
        int e = p_iff(p);
        if (!lit(p, ")")) p->f->err = 1;
        return e;
    }
    if (lit(p, "T") || lit(p, "true")) return mk(p, O_TOP, 0, -1, -1);
    if (lit(p, "F") || lit(p, "false")) return mk(p, O_BOT, 0, -1, -1);
    skip_ws(p);
    char c = p->s[p->i];
    if (c == 'p' || c == 'q' || c == 'r' || c == 's') {
        int var;
        p->i++;
        if (c == 'p' && isdigit((unsigned char)p->s[p->i])) {
            var = 0;
            while (isdigit((unsigned char)p->s[p->i])) var = var * 10 + (p->s[p->i++] - '0');
        } else {
            var = (c == 'p') ? 0 : (c == 'q') ? 1 : (c == 'r') ? 2 : 3;
        }
        if (isalnum((unsigned char)p->s[p->i]) || var >= ORC_MAX_VARS) { p->f->err = 1; return 0; }
        if (var + 1 > p->f->nvars) p->f->nvars = var + 1;
        return mk(p, O_VAR, var, -1, -1);
    }
    p->f->err = 1;
    return 0;
}

static int p_and(opar *p) {
    int e = p_unary(p);
    while (!p->f->err && (lit(p, "&") || lit(p, "and"))) e = mk(p, O_AND, 0, e, p_unary(p));
    return e;
}

static int p_or(opar *p) {
    int e = p_and(p);
    while (!p->f->err && (lit(p, "|") || lit(p, "or"))) e = mk(p, O_OR, 0, e, p_and(p));
    return e;
}

static int p_imp(opar *p) {                 /* right associative */
    int e = p_or(p);
    skip_ws(p);
    if (!p->f->err && strncmp(p->s + p->i, "<->", 3) != 0 && lit(p, "->")) return mk(p, O_IMP, 0, e, p_imp(p));
    return e;
}

static int p_iff(opar *p) {
    int e = p_imp(p);
    while (!p->f->err && lit(p, "<->")) e = mk(p, O_IFF, 0, e, p_imp(p));
    return e;
}

static int parse(const char *text, oform *f) {
    opar p = { text, 0, f };
    memset(f, 0, sizeof(*f));
    f->root = p_iff(&p);
    skip_ws(&p);
    if (p.s[p.i] != 0) f->err = 1;
    return f->err ? -1 : 0;
}

/* ------------------------------------------------------ truth-set evaluator */

/* out[w] = 1 iff M,w |= node, for every world w of the model (R, V) on n
   worlds.  Each case is the satisfaction clause for that connective. */
static void truth(const oform *f, int id, int n, const uint8_t *R, const uint8_t *V, uint8_t *out) {
    const onode *x = &f->nd[id];
    uint8_t a[ORC_MAX_WORLDS], b[ORC_MAX_WORLDS];
    int w, v;
    switch (x->kind) {
    case O_TOP: for (w = 0; w < n; w++) out[w] = 1; return;
    case O_BOT: for (w = 0; w < n; w++) out[w] = 0; return;
    case O_VAR: for (w = 0; w < n; w++) out[w] = V[x->var * n + w]; return;
    case O_NOT:
        truth(f, x->a, n, R, V, a);
        for (w = 0; w < n; w++) out[w] = !a[w];
        return;
    case O_AND: case O_OR: case O_IMP: case O_IFF:
        truth(f, x->a, n, R, V, a);
        truth(f, x->b, n, R, V, b);
        for (w = 0; w < n; w++) {
            if (x->kind == O_AND) out[w] = a[w] && b[w];
            else if (x->kind == O_OR) out[w] = a[w] || b[w];
            else if (x->kind == O_IMP) out[w] = !a[w] || b[w];
            else out[w] = (a[w] == b[w]);
        }
        return;
    case O_BOX:   /* every R-successor satisfies the argument */
        truth(f, x->a, n, R, V, a);
        for (w = 0; w < n; w++) {
            out[w] = 1;
            for (v = 0; v < n; v++) if (R[w * n + v] && !a[v]) out[w] = 0;
        }
        return;
    case O_DIA:   /* some R-successor satisfies the argument */
        truth(f, x->a, n, R, V, a);
        for (w = 0; w < n; w++) {
            out[w] = 0;
            for (v = 0; v < n; v++) if (R[w * n + v] && a[v]) out[w] = 1;
        }
        return;
    }
}

/* ---------------------------------------------------------- frame classes */

static int reflexive(int n, const uint8_t *R) {
    for (int w = 0; w < n; w++) if (!R[w * n + w]) return 0;
    return 1;
}
static int transitive(int n, const uint8_t *R) {
    for (int w = 0; w < n; w++) for (int v = 0; v < n; v++) for (int u = 0; u < n; u++)
        if (R[w * n + v] && R[v * n + u] && !R[w * n + u]) return 0;
    return 1;
}
static int symmetric(int n, const uint8_t *R) {
    for (int w = 0; w < n; w++) for (int v = 0; v < n; v++)
        if (R[w * n + v] && !R[v * n + w]) return 0;
    return 1;
}
/* cls: 0 = K, 1 = T, 2 = S4, 3 = S5, 4 = K4 (transitive frames, the frames
   of the logic K4: Sec. 2 names K4 beside T, S4 and S5) */
static int in_class(int cls, int n, const uint8_t *R) {
    if (cls == 0) return 1;
    if (cls == 4) return transitive(n, R);
    if (!reflexive(n, R)) return 0;
    if (cls == 1) return 1;
    if (!transitive(n, R)) return 0;
    if (cls == 2) return 1;
    return symmetric(n, R);
}

static void decode_frame(uint64_t f, int n, uint8_t *R) {
    for (int e = 0; e < n * n; e++) R[e] = (uint8_t)((f >> e) & 1u);
}
static void decode_val(uint64_t x, int k, int n, uint8_t *V) {
    for (int e = 0; e < k * n; e++) V[e] = (uint8_t)((x >> e) & 1u);
}

/* The valuation set of a layer (reading listed in the header). */
static int exhaustive_vals(int k, int n, uint32_t S) {
    if (S == 0 || k <= 1) return 1;
    if (k * n >= 32) return 0;
    return ((uint64_t)1 << (k * n)) <= S;
}

/* ------------------------------------------------------------- SplitMix64 */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the generator adds the
   golden-ratio increment to its state and returns the state passed through
   the "mix13" finaliser.  The j-th output (j = 0, 1, ...) of a generator
   started at state s is therefore mix(s + (j+1)*gamma). */
#define SM_GAMMA 0x9E3779B97F4A7C15ULL
static uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
uint64_t orc_splitmix_out(uint64_t state, uint64_t j) { return sm_mix(state + (j + 1) * SM_GAMMA); }
/* the state that starts stream `tag` at frame size n for seed `seed` */
uint64_t orc_stream_state(uint64_t seed, uint64_t tag, uint64_t n) { return sm_mix(seed ^ (tag << 32) ^ n); }

/* Sampled n-world relation number s (n <= 8) of the Erdos-Renyi family with a
   per-sample edge probability in [0.1, 0.5] (Sec. 7, adversarial frames):
   nine draws per sample from stream tag 2; draw 0 gives the threshold
   t = 26 + floor(hi32(draw0) * 103 / 2^32) in [26, 128] (p = t/256); edge e
   (row-major, e = w*n+v) is present iff byte (e mod 8) of draw 1 + e/8 is
   below t.  Returns the relation as a row-major edge mask. */
uint64_t orc_sample_frame(uint64_t seed, int n, uint64_t s) {
    uint64_t st = orc_stream_state(seed, 2, (uint64_t)n);
    uint64_t d0 = orc_splitmix_out(st, 9 * s);
    uint64_t t = 26 + (((d0 >> 32) * 103ULL) >> 32);
    uint64_t mask = 0;
    for (int e = 0; e < n * n; e++) {
        uint64_t d = orc_splitmix_out(st, 9 * s + 1 + (uint64_t)(e / 8));
        uint64_t byte = (d >> (8 * (e % 8))) & 0xFFu;
        if (byte < t) mask |= (uint64_t)1 << e;
    }
    return mask;
}

/* ---------------------------------------------------------------- census */

typedef struct {
    uint64_t frames;          /* class frames in the index range            */
    uint64_t cm_count;        /* refuted (frame, valuation) pairs           */
    uint64_t frames_refuted;  /* frames with at least one refuted valuation */
    int32_t  found;
    int32_t  nvals;           /* valuations per frame                       */
    uint64_t wf;              /* witness frame (K index)                    */
    uint32_t wv;              /* witness valuation (index or sample slot)   */
    uint32_t ww;              /* witness world                              */
} orc_census_out;

/* The parse tree of `text`, for the mask evaluator of tier1.c: node i has
   kind[i] (0 T, 1 F, 2 variable, 3 not, 4 and, 5 or, 6 implies, 7 iff,
   8 box, 9 diamond), variable var[i] and children a[i], b[i] (-1: none);
   the parser numbers children before their parents.  The arrays hold
   ORC_MAX_NODES entries.  Returns 0, or -1 on a parse error. */
int orc_parse_tree(const char *text, int *kind, int *var, int *a, int *b, int *nn, int *root, int *nvars) {
    oform f;
    if (parse(text, &f)) return -1;
    for (int i = 0; i < f.nn; i++) {
        kind[i] = f.nd[i].kind;
        var[i] = f.nd[i].var;
        a[i] = f.nd[i].a;
        b[i] = f.nd[i].b;
    }
    *nn = f.nn;
    *root = f.root;
    *nvars = f.nvars;
    return 0;
}

int orc_nvars(const char *text) {
    oform f;
    if (parse(text, &f)) return -1;
    return f.nvars;
}

int orc_nodes(const char *text) {
    oform f;
    if (parse(text, &f)) return -1;
    return f.nn;
}

/* Census of one formula over the class-`cls` frames on n worlds whose K
   index lies in [f_lo, f_hi). */
int orc_census(const char *text, int cls, int n, uint32_t S, const uint32_t *samp,
               uint64_t f_lo, uint64_t f_hi, orc_census_out *out) {
    oform f;
    memset(out, 0, sizeof(*out));
    if (n < 1 || n > 6 || cls < 0 || cls > 4) return -2;
    if (parse(text, &f)) return -1;
    int k = f.nvars;
    int exh = exhaustive_vals(k, n, S);
    if (!exh && samp == NULL) return -3;
    if (exh && k * n > 30) return -4;
    uint64_t nval = exh ? ((uint64_t)1 << (k * n)) : S;
    uint32_t vmask = (k * n >= 32) ? 0xFFFFFFFFu : (uint32_t)(((uint64_t)1 << (k * n)) - 1);
    uint64_t nf = (uint64_t)1 << (n * n);
    if (f_hi > nf) f_hi = nf;
    out->nvals = (int32_t)nval;

    uint64_t frames = 0, cm = 0, fr = 0;
    uint64_t best_f = UINT64_MAX; uint32_t best_v = 0, best_w = 0;
    #pragma omp parallel
    {
        uint64_t lf = UINT64_MAX; uint32_t lv = 0, lw = 0;
        #pragma omp for schedule(dynamic, 1024) reduction(+:frames,cm,fr)
        for (int64_t fi = (int64_t)f_lo; fi < (int64_t)f_hi; fi++) {
            uint8_t R[64], V[ORC_MAX_VARS * 8], t[8];
            decode_frame((uint64_t)fi, n, R);
            if (!in_class(cls, n, R)) continue;
            frames++;
            int any = 0;
            for (uint64_t j = 0; j < nval; j++) {
                uint64_t x = exh ? j : (samp[j] & vmask);
                decode_val(x, k, n, V);
                truth(&f, f.root, n, R, V, t);
                int w0 = -1;
                for (int w = 0; w < n; w++) if (!t[w]) { w0 = w; break; }
                if (w0 >= 0) {
                    cm++;
                    any = 1;
                    if ((uint64_t)fi < lf) { lf = (uint64_t)fi; lv = (uint32_t)j; lw = (uint32_t)w0; }
                }
            }
            fr += any;
        }
        #pragma omp critical
        {
            if (lf < best_f || (lf == best_f && (lv < best_v || (lv == best_v && lw < best_w)))) {
                best_f = lf; best_v = lv; best_w = lw;
            }
        }
    }
    out->frames = frames; out->cm_count = cm; out->frames_refuted = fr;
    if (best_f != UINT64_MAX) { out->found = 1; out->wf = best_f; out->wv = best_v; out->ww = best_w; }
    return 0;
}

/* Number of class-`cls` frames on n worlds (brute force over all relations). */
uint64_t orc_class_size(int cls, int n) {
    uint64_t nf = (uint64_t)1 << (n * n), c = 0;
    #pragma omp parallel for reduction(+:c) schedule(static)
    for (int64_t fi = 0; fi < (int64_t)nf; fi++) {
        uint8_t R[64];
        decode_frame((uint64_t)fi, n, R);
        c += (uint64_t)in_class(cls, n, R);
    }
    return c;
}

/* ------------------------------------------------------------- separation */

typedef struct {
    int32_t  found;
    int32_t  nvals;
    uint64_t f;                /* K index (exhaustive) or sample index     */
    uint32_t v;                /* valuation index or sample slot           */
    uint32_t w;                /* least world where the two values differ  */
    int32_t  phi_val, psi_val; /* truth values of phi and psi at that world */
    uint64_t frames_disagree;  /* frames (in range) with any disagreement  */
} orc_pair_out;

static int pair_scan(const oform *fa, const oform *fb, int n, uint32_t S, const uint32_t *samp,
                     uint64_t lo, uint64_t hi, int sampled, uint64_t seed, orc_pair_out *out) {
    int k = fa->nvars > fb->nvars ? fa->nvars : fb->nvars;
    int exh = exhaustive_vals(k, n, S);
    if (!exh && samp == NULL) return -3;
    if (exh && k * n > 30) return -4;
    uint64_t nval = exh ? ((uint64_t)1 << (k * n)) : S;
    uint32_t vmask = (k * n >= 32) ? 0xFFFFFFFFu : (uint32_t)(((uint64_t)1 << (k * n)) - 1);
    out->nvals = (int32_t)nval;
    uint64_t best_f = UINT64_MAX; uint32_t best_v = 0, best_w = 0; int best_a = 0, best_b = 0;
    uint64_t dis = 0;
    #pragma omp parallel
    {
        uint64_t lf = UINT64_MAX; uint32_t lv = 0, lw = 0; int la = 0, lb = 0;
        #pragma omp for schedule(dynamic, 1024) reduction(+:dis)
        for (int64_t fi = (int64_t)lo; fi < (int64_t)hi; fi++) {
            uint8_t R[64], V[ORC_MAX_VARS * 8], ta[8], tb[8];
            uint64_t rel = sampled ? orc_sample_frame(seed, n, (uint64_t)fi) : (uint64_t)fi;
            decode_frame(rel, n, R);
            int any = 0;
            for (uint64_t j = 0; j < nval; j++) {
                uint64_t x = exh ? j : (samp[j] & vmask);
                decode_val(x, k, n, V);
                truth(fa, fa->root, n, R, V, ta);
                truth(fb, fb->root, n, R, V, tb);
                for (int w = 0; w < n; w++) {
                    if (ta[w] != tb[w]) {
                        any = 1;
                        if ((uint64_t)fi < lf) { lf = (uint64_t)fi; lv = (uint32_t)j; lw = (uint32_t)w; la = ta[w]; lb = tb[w]; }
                        break;
                    }
                }
            }
            dis += any;
        }
        #pragma omp critical
        {
            if (lf < best_f || (lf == best_f && (lv < best_v || (lv == best_v && lw < best_w)))) {
                best_f = lf; best_v = lv; best_w = lw; best_a = la; best_b = lb;
            }
        }
    }
    out->frames_disagree = dis;
    if (best_f != UINT64_MAX) {
        out->found = 1; out->f = best_f; out->v = best_v; out->w = best_w;
        out->phi_val = best_a; out->psi_val = best_b;
    }
    return 0;
}

/* First disagreement of phi and psi among the n-world frames with K index
   in [f_lo, f_hi). */
int orc_pair_layer(const char *phi, const char *psi, int n, uint32_t S, const uint32_t *samp,
                   uint64_t f_lo, uint64_t f_hi, orc_pair_out *out) {
    oform fa, fb;
    memset(out, 0, sizeof(*out));
    if (n < 1 || n > 6) return -2;
    if (parse(phi, &fa) || parse(psi, &fb)) return -1;
    uint64_t nf = (uint64_t)1 << (n * n);
    if (f_hi > nf) f_hi = nf;
    return pair_scan(&fa, &fb, n, S, samp, f_lo, f_hi, 0, 0, out);
}

/* First disagreement among sampled n-world relations s in [s_lo, s_hi). */
int orc_pair_sampled(const char *phi, const char *psi, int n, uint64_t seed, uint32_t S,
                     const uint32_t *samp, uint64_t s_lo, uint64_t s_hi, orc_pair_out *out) {
    oform fa, fb;
    memset(out, 0, sizeof(*out));
    if (n < 1 || n > 8) return -2;
    if (parse(phi, &fa) || parse(psi, &fb)) return -1;
    return pair_scan(&fa, &fb, n, S, samp, s_lo, s_hi, 1, seed, out);
}

/* ----------------------------------------------------------- one model */

/* Truth value of `text` at every world of the explicit model (R, V) on n
   worlds (n <= 32); V holds nvars rows of n entries. */
int orc_eval_model(const char *text, int n, const uint8_t *R, const uint8_t *V, uint8_t *out) {
    oform f;
    if (n < 1 || n > ORC_MAX_WORLDS) return -2;
    if (parse(text, &f)) return -1;
    truth(&f, f.root, n, R, V, out);
    return 0;
}

/* valid[f] = 1 iff frame f (K index) on n worlds validates `text`: the
   formula is true at every world under every valuation of its variables. */
int orc_frame_valid_all(const char *text, int n, uint8_t *valid) {
    oform f;
    if (n < 1 || n > 5) return -2;
    if (parse(text, &f)) return -1;
    int k = f.nvars;
    if (k * n > 24) return -4;
    uint64_t nf = (uint64_t)1 << (n * n), nval = (uint64_t)1 << (k * n);
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t fi = 0; fi < (int64_t)nf; fi++) {
        uint8_t R[64], V[ORC_MAX_VARS * 8], t[8];
        decode_frame((uint64_t)fi, n, R);
        int ok = 1;
        for (uint64_t x = 0; x < nval && ok; x++) {
            decode_val(x, k, n, V);
            truth(&f, f.root, n, R, V, t);
            for (int w = 0; w < n; w++) if (!t[w]) ok = 0;
        }
        valid[fi] = (uint8_t)ok;
    }
    return 0;
}

/* 1 iff the relation R on n worlds is in class cls. */
int orc_in_class(int cls, int n, const uint8_t *R) { return in_class(cls, n, R); }

int orc_threads(void) { return omp_get_max_threads(); }

/* ================================================ large frames (Sec. 7)
 *
 * Separation beyond the exhaustive sizes runs over explicit relations on
 * n <= 16 worlds: the named stress templates (paths, reverse paths, loops,
 * forks, cycles, stars, sparse and dense frames) and the adversarial relation
 * generators of Table 2.  The paper names these families without fixing a
 * construction; the readings below are the ones this project uses.  A
 * relation is returned as successor masks:
 * bit v of succ[w] is set iff R(w, v).
 */

#define ORC_STRESS_MAX 16
#define ORC_NUM_TEMPLATES 39

static void rel_clear(int n, uint8_t *R) { memset(R, 0, (size_t)n * n); }
static void rel_add(int n, uint8_t *R, int w, int v) { if (w >= 0 && w < n && v >= 0 && v < n) R[w * n + v] = 1; }
static void rel_to_succ(int n, const uint8_t *R, uint32_t *succ) {
    for (int w = 0; w < n; w++) {
        succ[w] = 0;
        for (int v = 0; v < n; v++) if (R[w * n + v]) succ[w] |= 1u << v;
    }
}

/* forks: branch 0 -> 1 -> ... -> b and branch 0 -> b+1 -> ... -> n-1 */
static void fork_rel(int n, int b, uint8_t *R) {
    for (int i = 0; i < b && i + 1 < n; i++) rel_add(n, R, i, i + 1);
    if (b + 1 < n) rel_add(n, R, 0, b + 1);
    for (int i = b + 1; i + 1 < n; i++) rel_add(n, R, i, i + 1);
}

/* the fixed sparse / dense templates: byte (e mod 8) of output e/8 of the
   SplitMix64 stream (seed 0x5EED, tag 40 + variant, n) decides edge e */
static void coin_rel(int n, int variant, int thresh, uint8_t *R) {
    uint64_t st = orc_stream_state(0x5EED, 40 + (uint64_t)variant, (uint64_t)n);
    for (int e = 0; e < n * n; e++) {
        uint64_t d = orc_splitmix_out(st, (uint64_t)(e / 8));
        if ((int)((d >> (8 * (e % 8))) & 0xFFu) < thresh) R[e] = 1;
    }
}

/* Template `id` (0 .. 38) on n worlds, as a 0/1 matrix.  h = n/2 rounded
   down, c = n/2 rounded up. */
static int template_rel(int id, int n, uint8_t *R) {
    int h = n / 2, c = (n + 1) / 2, w, v;
    rel_clear(n, R);
    switch (id) {
    case 0: for (w = 0; w + 1 < n; w++) rel_add(n, R, w, w + 1); break;                 /* path */
    case 1: for (w = 0; w + 1 < n; w++) rel_add(n, R, w + 1, w); break;                 /* reverse path */
    case 2: for (w = 0; w < n; w++) { rel_add(n, R, w, w); rel_add(n, R, w, w + 1); } break; /* reflexive path */
    case 3: for (w = 0; w + 1 < n; w++) rel_add(n, R, w, w + 1); rel_add(n, R, n - 1, n - 1); break; /* looped path */
    case 4: for (w = 0; w + 1 < n; w++) rel_add(n, R, w, w + 1); rel_add(n, R, 0, 0); break;  /* rooted loop */
    case 5: for (w = 0; w < n; w++) for (v = w + 1; v < n; v++) rel_add(n, R, w, v); break;  /* strict order */
    case 6: for (w = 0; w < n; w++) for (v = w; v < n; v++) rel_add(n, R, w, v); break;      /* preorder chain */
    case 7: for (w = 0; w < n; w++) rel_add(n, R, w, (w + 1) % n); break;                   /* cycle */
    case 8: for (w = 0; w < n; w++) rel_add(n, R, (w + 1) % n, w); break;                   /* reverse cycle */
    case 9: for (w = 0; w < n; w++) { rel_add(n, R, w, (w + 1) % n); rel_add(n, R, w, w); } break;
    case 10: for (w = 0; w < n; w++) { rel_add(n, R, w, (w + 1) % n); rel_add(n, R, (w + 1) % n, w); } break;
    case 11: for (w = 0; w + 1 < n; w++) { rel_add(n, R, w, w + 1); rel_add(n, R, w + 1, w); } break;
    case 12: for (v = 1; v < n; v++) rel_add(n, R, 0, v); break;                            /* out-star */
    case 13: for (v = 1; v < n; v++) rel_add(n, R, v, 0); break;                            /* in-star */
    case 14: for (v = 1; v < n; v++) { rel_add(n, R, 0, v); rel_add(n, R, v, 0); } break;
    case 15: for (v = 1; v < n; v++) rel_add(n, R, 0, v); for (w = 0; w < n; w++) rel_add(n, R, w, w); break;
    case 16: fork_rel(n, h, R); break;
    case 17: fork_rel(n, 1, R); break;
    case 18: fork_rel(n, 2, R); break;
    case 19: fork_rel(n, n - 2, R); break;
    case 20: fork_rel(n, h, R); rel_add(n, R, h, h); rel_add(n, R, n - 1, n - 1); break;    /* looped fork */
    case 21: for (w = 0; w < n; w++) { rel_add(n, R, w, 2 * w + 1); rel_add(n, R, w, 2 * w + 2); } break;
    case 22: for (w = 0; w < n; w++) { rel_add(n, R, 2 * w + 1, w); rel_add(n, R, 2 * w + 2, w); } break;
    case 23: for (w = 0; w < n; w++) for (v = 0; v < n; v++) rel_add(n, R, w, v); break;    /* complete */
    case 24: for (w = 0; w < n; w++) for (v = 0; v < n; v++) if (w != v) rel_add(n, R, w, v); break;
    case 25: for (w = 0; w < n; w++) rel_add(n, R, w, w); break;                            /* identity */
    case 26: break;                                                                         /* empty */
    case 27: for (w = 0; w + 1 < n; w++) rel_add(n, R, w, w + 1); rel_add(n, R, n - 1, h); break; /* lasso */
    case 28:                                                                                 /* two cycles */
        for (w = 0; w < h; w++) rel_add(n, R, w, (w + 1) % h);
        for (w = h; w < n; w++) rel_add(n, R, w, w + 1 < n ? w + 1 : h);
        if (h >= 1) rel_add(n, R, h - 1, h);
        break;
    case 29: case 30: case 31: coin_rel(n, id - 29, 32, R); break;                          /* sparse */
    case 32: case 33: case 34: coin_rel(n, id - 29, 224, R); break;                         /* dense */
    case 35: for (w = 0; w + 1 < c; w++) rel_add(n, R, w, w + 1);                           /* comb */
             for (w = 0; w < n - c; w++) rel_add(n, R, w, c + w);
             break;
    case 36: for (w = 0; w < n; w++) { rel_add(n, R, w, w + 1); rel_add(n, R, w, w + 2); } break; /* skip path */
    case 37: for (w = 0; w + 1 < n; w++) rel_add(n, R, w, w + 1);                           /* half-reflexive path */
             for (w = 1; w < n; w += 2) rel_add(n, R, w, w);
             break;
    case 38: for (w = 0; w < n; w++) for (v = 0; v < w; v++) rel_add(n, R, w, v); break;    /* reverse strict order */
    default: return -1;
    }
    return 0;
}

int orc_template(int id, int n, uint32_t *succ) {
    uint8_t R[ORC_STRESS_MAX * ORC_STRESS_MAX];
    if (n < 1 || n > ORC_STRESS_MAX) return -2;
    if (template_rel(id, n, R)) return -1;
    rel_to_succ(n, R, succ);
    return 0;
}

/* Adversarial relation generators (Table 2), relation number s of generator
 * gen at n worlds (2 <= n <= 16; Erdos-Renyi also n = 1):
 *
 *   0 Erdos-Renyi    stream tag 2, D = 9 draws per relation for n <= 8 and
 *                    33 above (so that n <= 8 is the sampled family of
 *                    orc_sample_frame): t = 26 + floor(hi32(d0) * 103 / 2^32),
 *                    edge e present iff byte (e mod 8) of d(1 + e/8) < t.
 *   others           stream tag 16 + gen, D = 40 draws per relation: d0 gives
 *                    t as above, d1..d32 the edge coins (byte e mod 8 of
 *                    d(1 + e/8)), d33..d39 the choices c_0..c_27 (16-bit chunk
 *                    i mod 4 of d(33 + i/4)); r(i, m) = floor(c_i * m / 2^16).
 *   1 edge flip      template r(0, 39), then 1 + r(1, 4) flips, flip i
 *                    toggling edge e = r(2 + i, n*n) (in that order).
 *   2 SCC bottleneck a = 1 + r(0, n-1); blocks [0, a) and [a, n); a block of
 *                    two or more worlds gets the cycle lo -> lo+1 -> ... ->
 *                    hi-1 -> lo; every intra-block pair (self-loops included)
 *                    whose coin is below t is added; one bridge a-1 -> a.
 *   3 dead ends      the coin relation (edge e iff coin e < t), then
 *                    1 + r(0, 3) worlds r(1 + i, n) lose every successor.
 *   4 back edges     the path 0 -> 1 -> ... -> n-1 plus 1 + r(0, 4) edges
 *                    max(x, y) -> min(x, y), x = r(1 + 2i, n), y = r(2 + 2i, n).
 *   5 permuted       the SCC-bottleneck relation built from this generator's
 *     bottleneck     own draws, relabelled by the permutation pi obtained by
 *                    Fisher-Yates from the identity: for i = n-1 down to 1,
 *                    swap pi[i] and pi[r(4 + n-1-i, i+1)]; R'(pi(w), pi(v)) =
 *                    R(w, v).
 */
typedef struct { uint64_t st, base; } ogen;

static uint64_t g_draw(const ogen *g, int i) { return orc_splitmix_out(g->st, g->base + (uint64_t)i); }
static int g_coin(const ogen *g, int e) { return (int)((g_draw(g, 1 + e / 8) >> (8 * (e % 8))) & 0xFFu); }
static uint32_t g_r(const ogen *g, int i, uint32_t m) {
    uint32_t c = (uint32_t)((g_draw(g, 33 + i / 4) >> (16 * (i % 4))) & 0xFFFFu);
    return (uint32_t)(((uint64_t)c * m) >> 16);
}
static int g_thresh(const ogen *g) { return 26 + (int)(((g_draw(g, 0) >> 32) * 103ULL) >> 32); }

static void scc_rel(const ogen *g, int n, uint8_t *R) {
    int a = 1 + (int)g_r(g, 0, (uint32_t)(n - 1)), t = g_thresh(g);
    int lo[2] = {0, a}, hi[2] = {a, n};
    rel_clear(n, R);
    for (int b = 0; b < 2; b++) {
        if (hi[b] - lo[b] >= 2) {
            for (int w = lo[b]; w < hi[b]; w++) rel_add(n, R, w, w + 1 < hi[b] ? w + 1 : lo[b]);
        }
        for (int w = lo[b]; w < hi[b]; w++)
            for (int v = lo[b]; v < hi[b]; v++)
                if (g_coin(g, w * n + v) < t) rel_add(n, R, w, v);
    }
    rel_add(n, R, a - 1, a);
}

int orc_stress_relation(int gen, uint64_t seed, int n, uint64_t s, uint32_t *succ) {
    uint8_t R[ORC_STRESS_MAX * ORC_STRESS_MAX], Q[ORC_STRESS_MAX * ORC_STRESS_MAX];
    if (n < 1 || n > ORC_STRESS_MAX || (gen != 0 && n < 2)) return -2;
    ogen g;
    rel_clear(n, R);
    if (gen == 0) {
        uint64_t D = n <= 8 ? 9 : 33;
        g.st = orc_stream_state(seed, 2, (uint64_t)n);
        g.base = D * s;
        int t = g_thresh(&g);
        for (int e = 0; e < n * n; e++) if (g_coin(&g, e) < t) R[e] = 1;
        rel_to_succ(n, R, succ);
        return 0;
    }
    if (gen < 0 || gen > 5) return -1;
    g.st = orc_stream_state(seed, 16 + (uint64_t)gen, (uint64_t)n);
    g.base = 40 * s;
    int t = g_thresh(&g);
    if (gen == 1) {
        template_rel((int)g_r(&g, 0, ORC_NUM_TEMPLATES), n, R);
        int m = 1 + (int)g_r(&g, 1, 4);
        for (int i = 0; i < m; i++) {
            int e = (int)g_r(&g, 2 + i, (uint32_t)(n * n));
            R[e] = (uint8_t)!R[e];
        }
    } else if (gen == 2) {
        scc_rel(&g, n, R);
    } else if (gen == 3) {
        for (int e = 0; e < n * n; e++) if (g_coin(&g, e) < t) R[e] = 1;
        int m = 1 + (int)g_r(&g, 0, 3);
        for (int i = 0; i < m; i++) {
            int w = (int)g_r(&g, 1 + i, (uint32_t)n);
            for (int v = 0; v < n; v++) R[w * n + v] = 0;
        }
    } else if (gen == 4) {
        for (int w = 0; w + 1 < n; w++) rel_add(n, R, w, w + 1);
        int m = 1 + (int)g_r(&g, 0, 4);
        for (int i = 0; i < m; i++) {
            int x = (int)g_r(&g, 1 + 2 * i, (uint32_t)n), y = (int)g_r(&g, 2 + 2 * i, (uint32_t)n);
            rel_add(n, R, x > y ? x : y, x > y ? y : x);
        }
    } else {
        int pi[ORC_STRESS_MAX];
        scc_rel(&g, n, Q);
        for (int i = 0; i < n; i++) pi[i] = i;
        for (int i = n - 1; i >= 1; i--) {
            int j = (int)g_r(&g, 4 + (n - 1 - i), (uint32_t)(i + 1));
            int tmp = pi[i]; pi[i] = pi[j]; pi[j] = tmp;
        }
        for (int w = 0; w < n; w++)
            for (int v = 0; v < n; v++)
                if (Q[w * n + v]) R[pi[w] * n + pi[v]] = 1;
    }
    rel_to_succ(n, R, succ);
    return 0;
}

/* Separation over explicit relations: for relations s = 0 .. count-1 (given
   as successor masks succ[s*16 + w]), valuations x = 0 .. 2^(k n)-1 and
   worlds w, the least (s, x, w) at which phi and psi differ (the order of
   Def. 2 with relations in list order), and the number of relations on
   which they differ at all.  Exhaustive valuations only: k*n <= 16. */
typedef struct {
    int32_t found, nvals;
    uint64_t s;
    uint32_t x, w;
    uint64_t nsplit;
} orc_stress_out;

int orc_stress_pair(const char *phi, const char *psi, int n, const uint32_t *succ, uint64_t count,
                    orc_stress_out *out) {
    oform fa, fb;
    memset(out, 0, sizeof(*out));
    if (n < 1 || n > ORC_STRESS_MAX) return -2;
    if (parse(phi, &fa) || parse(psi, &fb)) return -1;
    int k = fa.nvars > fb.nvars ? fa.nvars : fb.nvars;
    if (k * n > 16) return -4;
    uint64_t nval = (uint64_t)1 << (k * n);
    out->nvals = (int32_t)nval;
    uint64_t best_s = UINT64_MAX, nsplit = 0;
    uint32_t best_x = 0, best_w = 0;
    #pragma omp parallel
    {
        uint64_t ls = UINT64_MAX; uint32_t lx = 0, lw = 0;
        #pragma omp for schedule(dynamic, 16) reduction(+:nsplit)
        for (int64_t si = 0; si < (int64_t)count; si++) {
            uint8_t R[ORC_STRESS_MAX * ORC_STRESS_MAX], V[ORC_MAX_VARS * ORC_STRESS_MAX];
            uint8_t ta[ORC_STRESS_MAX], tb[ORC_STRESS_MAX];
            for (int w = 0; w < n; w++)
                for (int v = 0; v < n; v++) R[w * n + v] = (uint8_t)((succ[si * 16 + w] >> v) & 1u);
            int hit = 0;
            for (uint64_t x = 0; x < nval && !hit; x++) {
                decode_val(x, k, n, V);
                truth(&fa, fa.root, n, R, V, ta);
                truth(&fb, fb.root, n, R, V, tb);
                for (int w = 0; w < n; w++) {
                    if (ta[w] != tb[w]) {
                        hit = 1;
                        if ((uint64_t)si < ls) { ls = (uint64_t)si; lx = (uint32_t)x; lw = (uint32_t)w; }
                        break;
                    }
                }
            }
            nsplit += (uint64_t)hit;
        }
        #pragma omp critical
        {
            if (ls < best_s) { best_s = ls; best_x = lx; best_w = lw; }
        }
    }
    out->nsplit = nsplit;
    if (best_s != UINT64_MAX) { out->found = 1; out->s = best_s; out->x = best_x; out->w = best_w; }
    return 0;
}

/* ================================ frame correspondents (Sec. 10, Table 9)
 *
 * Recovering a first-order frame condition for a formula compares, over all
 * frames of at most N worlds, the frames that validate the formula
 * (orc_frame_valid_all) with the frames that satisfy a condition from a
 * fixed library.  Each condition below is its first-order definition over
 * the relation R, written out with quantifiers as loops.  Ids:
 *    0 every frame             1 no frame               2 reflexive
 *    3 irreflexive             4 serial                 5 transitive
 *    6 symmetric               7 Euclidean              8 partially functional
 *    9 functional             10 dense                 11 directed (confluent)
 *   12 antisymmetric          13 asymmetric            14 weakly connected
 *   15 shift reflexive        16 empty relation        17 coreflexive
 */
#define ORC_NUM_CONDITIONS 18

static int condition_holds(int c, int n, const uint8_t *R) {
    int w, v, u, x;
#define RR(a, b) (R[(a) * n + (b)])
    switch (c) {
    case 0: return 1;
    case 1: return 0;
    case 2: for (w = 0; w < n; w++) if (!RR(w, w)) return 0; return 1;
    case 3: for (w = 0; w < n; w++) if (RR(w, w)) return 0; return 1;
    case 4:                                   /* forall w exists v: wRv */
        for (w = 0; w < n; w++) {
            int any = 0;
            for (v = 0; v < n; v++) any |= RR(w, v);
            if (!any) return 0;
        }
        return 1;
    case 5: return transitive(n, R);
    case 6: return symmetric(n, R);
    case 7:                                   /* wRv and wRu imply vRu */
        for (w = 0; w < n; w++) for (v = 0; v < n; v++) for (u = 0; u < n; u++)
            if (RR(w, v) && RR(w, u) && !RR(v, u)) return 0;
        return 1;
    case 8:                                   /* wRv and wRu imply v = u */
        for (w = 0; w < n; w++) for (v = 0; v < n; v++) for (u = 0; u < n; u++)
            if (RR(w, v) && RR(w, u) && v != u) return 0;
        return 1;
    case 9: return condition_holds(4, n, R) && condition_holds(8, n, R);
    case 10:                                  /* wRv implies exists u: wRu and uRv */
        for (w = 0; w < n; w++) for (v = 0; v < n; v++) {
            if (!RR(w, v)) continue;
            int any = 0;
            for (u = 0; u < n; u++) any |= RR(w, u) && RR(u, v);
            if (!any) return 0;
        }
        return 1;
    case 11:                                  /* wRv and wRu imply exists x: vRx and uRx */
        for (w = 0; w < n; w++) for (v = 0; v < n; v++) for (u = 0; u < n; u++) {
            if (!(RR(w, v) && RR(w, u))) continue;
            int any = 0;
            for (x = 0; x < n; x++) any |= RR(v, x) && RR(u, x);
            if (!any) return 0;
        }
        return 1;
    case 12:                                  /* wRv and vRw imply w = v */
        for (w = 0; w < n; w++) for (v = 0; v < n; v++) if (w != v && RR(w, v) && RR(v, w)) return 0;
        return 1;
    case 13:                                  /* wRv implies not vRw */
        for (w = 0; w < n; w++) for (v = 0; v < n; v++) if (RR(w, v) && RR(v, w)) return 0;
        return 1;
    case 14:                                  /* wRv and wRu imply vRu or v = u or uRv */
        for (w = 0; w < n; w++) for (v = 0; v < n; v++) for (u = 0; u < n; u++)
            if (RR(w, v) && RR(w, u) && !(RR(v, u) || v == u || RR(u, v))) return 0;
        return 1;
    case 15:                                  /* wRv implies vRv */
        for (w = 0; w < n; w++) for (v = 0; v < n; v++) if (RR(w, v) && !RR(v, v)) return 0;
        return 1;
    case 16:
        for (w = 0; w < n * n; w++) if (R[w]) return 0;
        return 1;
    case 17:                                  /* wRv implies w = v */
        for (w = 0; w < n; w++) for (v = 0; v < n; v++) if (w != v && RR(w, v)) return 0;
        return 1;
    }
#undef RR
    return -1;
}

/* out[f] = 1 iff the n-world frame with K index f satisfies condition c. */
int orc_frame_condition(int c, int n, uint8_t *out) {
    if (n < 1 || n > 5) return -2;
    if (c < 0 || c >= ORC_NUM_CONDITIONS) return -1;
    uint64_t nf = (uint64_t)1 << (n * n);
    #pragma omp parallel for schedule(static, 4096)
    for (int64_t fi = 0; fi < (int64_t)nf; fi++) {
        uint8_t R[64];
        decode_frame((uint64_t)fi, n, R);
        out[fi] = (uint8_t)condition_holds(c, n, R);
    }
    return 0;
}

/* ============================== failure-density atlas (Sec. 9, Fig. atlas)
 *
 * D_ij = the fraction of (valuation, world) pairs at which formula i is
 * false on frame j.  The oracle returns the integer numerator for every
 * n-world frame (K index order); the denominator is 2^(k n) * n, with all
 * valuations of the formula's k variables. */
int orc_atlas(const char *text, int n, uint32_t *count, uint64_t *denom) {
    oform f;
    if (n < 1 || n > 4) return -2;
    if (parse(text, &f)) return -1;
    int k = f.nvars;
    if (k * n > 16) return -4;
    uint64_t nf = (uint64_t)1 << (n * n), nval = (uint64_t)1 << (k * n);
    *denom = nval * (uint64_t)n;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t fi = 0; fi < (int64_t)nf; fi++) {
        uint8_t R[64], V[ORC_MAX_VARS * 8], t[8];
        decode_frame((uint64_t)fi, n, R);
        uint32_t c = 0;
        for (uint64_t x = 0; x < nval; x++) {
            decode_val(x, k, n, V);
            truth(&f, f.root, n, R, V, t);
            for (int w = 0; w < n; w++) c += !t[w];
        }
        count[fi] = c;
    }
    return 0;
}
