"""Seeded synthetic workloads shaped like the paper's.

This module only makes inputs: formula texts, formula pairs and the tables of
sampled valuations.  It holds none of the evaluation arithmetic, so both the
CUDA path and the CPU oracle can take their inputs from it.

Workloads:

* ``pr1_formulas``      -- 64 random formulas over p, q (length <= 12, modal
  depth <= 3) plus the K, T and 4 axioms; census over n <= 3, all valuations.
* ``census5_formulas``  -- 5,621 random formulas (length 3-24, depth 1-4,
  0-3 variables) plus K, T, 4: the five-world census standing in for the
  paper's 5,624-formula corpus (Sec. 6), whose files are not available.
* ``uneven_formulas``   -- 20,000 formulas, length and depth log-uniform in
  [3, 64] and [1, 8], each with its own class and n_max (config "uneven").
* ``separation_pairs``  -- 1,024 variable-free pairs: the 32 context pairs
  (C^m b, C^(m+1) b) of the active-synthesis protocol (Sec. 7), (alpha_5,
  alpha_6), and 991 seeded random pairs, half of them one-edit mutations.
* ``proposal_formulas`` -- 10,000 formulas: 2,000 bases (length <= 21, depth
  <= 10) and 8,000 Boolean compositions of them (Sec. 9 retrieval corpus).
* ``sampled_valuations`` -- the S sampled valuations of layer n: output j of
  the SplitMix64 stream (Steele, Lea, Flood 2014) for (seed, tag 1, n).

Formula syntax: atoms ``p0``..``p3`` (``p``, ``q`` = p0, p1), ``T``, ``F``;
unary ``~``, ``[]``, ``<>``; binary ``&``, ``|``, ``->`` (right
associative).  Generated texts are fully parenthesised.
"""
import math
import random

import numpy as np

K_AXIOM = "[](p -> q) -> ([]p -> []q)"
T_AXIOM = "[]p -> p"
FOUR_AXIOM = "[]p -> [][]p"
AXIOMS = (K_AXIOM, T_AXIOM, FOUR_AXIOM)

_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def _mix(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def splitmix_state(seed, tag, n):
    """Start state of the SplitMix64 stream for (seed, tag, n)."""
    return _mix((seed ^ (tag << 32) ^ n) & _M64)


def splitmix_out(state, j):
    """Output j (0-based) of SplitMix64 started at ``state``."""
    return _mix((state + (j + 1) * _GAMMA) & _M64)


def sampled_valuations(seed, n, S):
    """uint32[S]: the sampled valuations of layer n (their low k*n bits are
    used by a k-variable formula)."""
    st = splitmix_state(seed, 1, n)
    return np.array([splitmix_out(st, j) & 0xFFFFFFFF for j in range(S)], dtype=np.uint32)


def valuation_table(seed, S, n_max=8):
    """uint32[n_max+1][S]: row n = sampled_valuations(seed, n, S) (row 0 unused)."""
    t = np.zeros((n_max + 1, max(S, 1)), dtype=np.uint32)
    for n in range(1, n_max + 1):
        if S:
            t[n] = sampled_valuations(seed, n, S)
    return t


# ------------------------------------------------------------ formula trees

def _feasible(L, d):
    """Productions that can root a tree with exactly L nodes and modal depth
    exactly d."""
    out = []
    if L == 1:
        return ["leaf"] if d == 0 else []
    if L - 1 >= d + 1 or (d == 0 and L - 1 >= 1):
        out.append("~")
    if d >= 1 and L - 1 >= d:
        out += ["[]", "<>"]
    if L >= 3 and L - 2 >= d + 1:
        out += ["&", "|", "->"]
    return out


def _tree(rng, L, d):
    prods = _feasible(L, d)
    if not prods:
        raise ValueError("no tree with %d nodes and depth %d" % (L, d))
    p = rng.choice(prods)
    if p == "leaf":
        return ["leaf"]
    if p == "~":
        return ["~", _tree(rng, L - 1, d)]
    if p in ("[]", "<>"):
        return [p, _tree(rng, L - 1, d - 1)]
    # binary: one side carries depth d, the other any feasible depth <= d
    while True:
        a = rng.randint(1, L - 2)
        b = L - 1 - a
        if rng.random() < 0.5:
            if a >= d + 1:
                da, db = d, rng.randint(0, min(d, b - 1))
                break
        else:
            if b >= d + 1:
                da, db = rng.randint(0, min(d, a - 1)), d
                break
    return [p, _tree(rng, a, da), _tree(rng, b, db)]


def _leaves(t, acc):
    if t[0] == "leaf":
        acc.append(t)
    else:
        for c in t[1:]:
            _leaves(c, acc)
    return acc


def _text(t):
    op = t[0]
    if op == "leaf":
        return t[1]
    if op in ("~", "[]", "<>"):
        return op + _text(t[1])
    return "(" + _text(t[1]) + " " + op + " " + _text(t[2]) + ")"


def random_formula(rng, length, depth, k, const_p=0.2, atoms=None):
    """A formula with exactly ``length`` nodes, modal depth exactly ``depth``
    and highest variable p_(k-1) (variable-free when k == 0)."""
    depth = min(depth, length - 1)
    t = _tree(rng, length, depth)
    leaves = _leaves(t, [])
    if atoms is None:
        atoms = ["p%d" % i for i in range(k)]
    for lf in leaves:
        if not atoms or rng.random() < const_p:
            lf.append(rng.choice(["T", "F"]))
        else:
            lf.append(rng.choice(atoms))
    if k > 0:
        rng.choice(leaves)[1:] = [atoms[k - 1]]
    return _text(t)


def pr1_formulas(seed=1, count=64):
    """64 formulas over p, q, T, F (length <= 12, depth <= 3) + K, T, 4."""
    rng = random.Random(seed)
    out = []
    for _ in range(count):
        L = rng.randint(3, 12)
        d = rng.randint(0, 3)
        k = rng.randint(0, 2)
        out.append(random_formula(rng, L, d, k, const_p=0.25,
                                  atoms=["p", "q"][:k] if k else None))
    return out + list(AXIOMS)


def census5_formulas(seed=2, count=5621):
    """Five-world census corpus: length 3-24, depth 1-4, 0-3 variables."""
    rng = random.Random(seed)
    out = []
    for _ in range(count):
        L = rng.randint(3, 24)
        d = rng.randint(1, 4)
        k = rng.randint(0, 3)
        out.append(random_formula(rng, L, d, k))
    return out + list(AXIOMS)


def atlas_formulas(seed=9, count=100000):
    """The ten-times display corpus of Sec. 9 (deterministically generated):
    the five-world corpus recipe (length 3-24, depth 1-4, 0-3 variables)
    drawn `count` times from its own seed."""
    rng = random.Random(seed)
    out = []
    for _ in range(count):
        L = rng.randint(3, 24)
        out.append(random_formula(rng, L, rng.randint(1, 4), rng.randint(0, 3)))
    return out


def _log_uniform_int(rng, lo, hi):
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def uneven_formulas(seed=3, count=20000):
    """Uneven batch: (text, class, n_max) with length log-uniform 3-64, depth
    log-uniform 1-8 (at most length-1), classes uniform over K/T/S4/S5 and
    n_max uniform over {3, 4, 5}."""
    rng = random.Random(seed)
    out = []
    for _ in range(count):
        L = _log_uniform_int(rng, 3, 64)
        d = min(_log_uniform_int(rng, 1, 8), L - 1)
        k = rng.randint(0, 3)
        cls = rng.choice(["K", "T", "S4", "S5"])
        nmax = rng.choice([3, 4, 5])
        out.append((random_formula(rng, L, d, k), cls, nmax))
    return out


def alpha(m):
    """alpha_m = ([]<>)^m T."""
    return "[]<>" * m + "T"


def context_pairs():
    """The 32 active-synthesis pairs (C^m b, C^(m+1) b) of Sec. 7."""
    out = []
    for C in ("[]<>", "<>[]", "[][]", "<><>"):
        for b in ("T", "F"):
            for m in range(1, 5):
                out.append((C * m + b, C * (m + 1) + b))
    return out


def _mutate(rng, text):
    """One edit of a modal word over a constant: flip, insert or delete one
    operator, or flip the base constant."""
    body, base = text[:-1], text[-1]
    ops = [body[i:i + 2] for i in range(0, len(body), 2)]
    r = rng.random()
    if r < 0.1:
        base = "F" if base == "T" else "T"
    elif r < 0.5 and ops:
        i = rng.randrange(len(ops))
        ops[i] = "<>" if ops[i] == "[]" else "[]"
    elif r < 0.75 or not ops:
        ops.insert(rng.randrange(len(ops) + 1), rng.choice(["[]", "<>"]))
    else:
        del ops[rng.randrange(len(ops))]
    return "".join(ops) + base


def separation_pairs(seed=4, count=1024):
    """1,024 variable-free pairs: 32 context pairs, (alpha_5, alpha_6), then
    seeded random pairs (half independent, half one-edit mutations)."""
    rng = random.Random(seed)
    out = context_pairs() + [(alpha(5), alpha(6))]
    ctx = context_pairs()
    while len(out) < count:
        if len(out) % 2 == 0:
            a, b = rng.choice(ctx)
            src = rng.choice([a, b])
            out.append((src, _mutate(rng, src)))
        else:
            L1, L2 = rng.randint(3, 14), rng.randint(3, 14)
            d1, d2 = rng.randint(1, min(6, L1 - 1)), rng.randint(1, min(6, L2 - 1))
            out.append((random_formula(rng, L1, d1, 0), random_formula(rng, L2, d2, 0)))
    return out[:count]


def context_word_formulas(max_nodes=21, max_depth=10):
    """Every distinct C^m b: a modal context word C over {[], <>} of length
    1-3 iterated m >= 1 times over a base b in {T, F, p0, ~p0}, with modal
    depth <= max_depth and at most max_nodes nodes (the active-synthesis and
    mining families of Sec. 7), in a fixed order."""
    out, seen = [], set()
    words = [""]
    for _ in range(3):
        words = [w + c for w in words for c in ("[]", "<>")] + words
    words = sorted({w for w in words if w}, key=lambda w: (len(w), w))
    for C in words:
        cl = len(C) // 2
        for b in ("T", "F", "p0", "~p0"):
            bn = 2 if b == "~p0" else 1
            m = 1
            while cl * m <= max_depth and cl * m + bn <= max_nodes:
                t = C * m + b
                if t not in seen:
                    seen.add(t)
                    out.append(t)
                m += 1
    return out


MINING_BASES = ("T", "F", "p", "(p->p)", "(p&~p)", "(~p|p)")


def mining_candidates(max_nodes=21):
    """Context-word mining candidates of Sec. 7: for every context word C
    over {[], <>} of length 1-3, every base b in {T, F, p, p->p, p&~p,
    ~p|p} and every m >= 1 with |C^(m+1) b| <= max_nodes, the pair
    (C^m b, C^(m+1) b).  Returns (phi, psi, word_length) triples in a fixed
    order (words by length, then text; bases in the order above; m up)."""
    words = [""]
    for _ in range(3):
        words = [w + c for w in words for c in ("[]", "<>")] + words
    words = sorted({w for w in words if w}, key=lambda w: (len(w), w))
    out = []
    for C in words:
        cl = len(C) // 2
        for b in MINING_BASES:
            bn = nodes(b)
            m = 1
            while cl * (m + 1) + bn <= max_nodes:
                out.append((C * m + b, C * (m + 1) + b, cl))
                m += 1
    return out


def proposal_formulas(seed=5, count=10000, bases=2000):
    """Retrieval corpus, like the paper's corpus of representatives of
    sizes 1-21 and modal depths 0-10, most with a Boolean connective (Sec. 9):
    ``bases`` base formulas -- every iterated modal context word over T, F,
    p0, ~p0 (context_word_formulas), then random trees (length 2-21, depth
    0-10, variable-free with probability 0.6, else over p0) -- and Boolean
    compositions (&, |, -> of two bases, or ~).  Duplicate texts are
    skipped.  At most one variable keeps every exact check at 6-8 worlds
    affordable (2^n valuations)."""
    rng = random.Random(seed)
    base = context_word_formulas()[:bases]
    seen = set(base)
    tries = 0
    while len(base) < bases and tries < 100 * bases:
        tries += 1
        L = rng.randint(2, 21)
        d = rng.randint(0, min(10, L - 1))
        k = 0 if rng.random() < 0.6 else 1
        t = random_formula(rng, L, d, k, const_p=0.3)
        if t not in seen:
            seen.add(t)
            base.append(t)
    out = list(base)
    tries = 0
    while len(out) < count and tries < 100 * count:
        tries += 1
        a = rng.choice(base)
        if rng.random() < 0.1:
            t = "~(" + a + ")"
        else:
            t = "(" + a + ") " + rng.choice(["&", "|", "->"]) + " (" + rng.choice(base) + ")"
        if t not in seen:
            seen.add(t)
            out.append(t)
    return out


def nodes(text):
    """Node count |phi| of a generated text (atoms, constants, operators)."""
    import re
    return len(re.findall(r"p\d+|[pqrs](?!\d)|T|F|~|\[\]|<>|&|\||->", text))


def pointed_models(seed=5, counts=(32, 96, 640, 1280, 2048)):
    """Seeded pointed models for truth vectors: counts[n-1] models on n
    worlds (each a multiple of 32, so every group of 32 has one n), with a
    per-model edge probability in [0.1, 0.6], uniform valuations of four
    variables and a uniform pointed world; drawn from the SplitMix64 stream
    (seed, tag 3, n).  Returns (models as a record array in mk_model layout,
    the n of every 32-model group)."""
    dtype = np.dtype([("frame", "<u8"), ("val", "<u4"), ("n", "u1"), ("world", "u1"), ("reserved", "<u2")])
    out, groups = [], []
    for n, cnt in enumerate(counts, start=1):
        assert cnt % 32 == 0
        st = splitmix_state(seed, 3, n)
        j = 0
        for _ in range(cnt):
            d = [splitmix_out(st, j + i) for i in range(3)]
            j += 3
            p = 0.1 + 0.5 * ((d[0] >> 11) / float(1 << 53))
            frame = 0
            r = d[1]
            for e in range(n * n):
                if e % 16 == 0 and e:
                    r = splitmix_out(st, j)
                    j += 1
                if ((r >> (4 * (e % 16))) & 0xF) < int(p * 16):
                    frame |= 1 << e
            val = d[2] & ((1 << (4 * n)) - 1)
            world = (d[2] >> 40) % n
            out.append((frame, val, n, world, 0))
        groups += [n] * (cnt // 32)
    return np.array(out, dtype=dtype), np.array(groups, np.int32)


# ------------------------------------------- matched single-formula shapes

def t_frame_kindex(c, n):
    """K index of the reflexive n-world frame with compact index c (the
    diagonal bits set, the off-diagonal bits taken from c in order)."""
    f, j = 0, 0
    for e in range(n * n):
        if e % (n + 1) == 0:
            f |= 1 << e
        else:
            f |= ((c >> j) & 1) << e
            j += 1
    return f


# K index just past the 304th transitive five-world frame: Table 4's K4 row
# filters 304 frames, read as the first 304 transitive frames in K order
# (the tests count them with the oracle)
K4_TABLE4_HI = 653

_CHAIN3 = "[](p0 -> p1) & [](p1 -> p2) -> ([]p0 -> []p2)"
_CHAIN4 = "[](p0 -> p1) & [](p1 -> p2) & [](p2 -> p3) -> ([]p0 -> []p3)"


def matched_rows():
    """Single-formula workloads on five-world frames with every valuation:
    Table 1's matched case and the shapes of Table 4's ablation (frames x
    valuations per row), plus the three-variable depth-ten stress of Sec. 8
    (34.36 G evaluations: 2^20 frames x 2^15 valuations).  The paper names
    the formula of Table 1 only; the others are chosen here to have the
    row's operator count, modal depth or variable count.  Frames are a
    prefix in K-index order (T: the first compact indices; K4: the first
    transitive frames).  'h100' is the
    paper's measured rate for the row in G evaluations/s, for context.

    Returns dicts: name, text, cls, lo, hi (K-index window), frames,
    valuations, h100."""
    K = "K"
    rows = [
        ("Table 1: matched formula", "[](p -> q) -> (<>p -> <>q)", K, 262144, 1024, 38.33),
        ("Table 4: length 2 ops", "[]p -> p", K, 65536, 32, 14.87),
        ("Table 4: length 5 ops", "[](p -> <>p) -> []p", K, 65536, 32, 11.88),
        ("Table 4: length 11 ops", "[](p -> <>p) -> (<>[]p -> [](<>p | ~p))", K, 65536, 32, 5.50),
        ("Table 4: modal depth 1", "<>p -> []p", K, 65536, 32, 7.45),
        ("Table 4: modal depth 4", "[]<>[]<>p -> p", K, 65536, 32, 6.89),
        ("Table 4: modal depth 8", "[]<>[]<>[]<>[]<>p -> p", K, 65536, 32, 11.56),
        ("Table 4: 1 variable", "[](p0 -> <>p0) -> <>p0", K, 65536, 32, 15.72),
        ("Table 4: 2 variables", "[](p0 -> p1) -> ([]p0 -> []p1)", K, 8192, 1024, 7.15),
        ("Table 4: 3 variables, underfilled", _CHAIN3, K, 512, 32768, 0.400),
        ("Table 4: 3 variables, saturated", _CHAIN3, K, 8192, 32768, 6.38),
        ("Table 4: 4 variables, underfilled", _CHAIN4, K, 32, 1048576, 0.0207),
        ("Table 4: frame filter K", "[]p -> [][]p", K, 65536, 32, 7.21),
        ("Table 4: frame filter T", "[]p -> [][]p", "T", 2049, 32, 0.240),
        ("Table 4: frame filter K4", "[]p -> [][]p", "K4", 304, 32, 0.0343),
        ("Sec. 8: semantic stress (3 vars, depth 10)", "[]<>[]<>[]<>[]<>[]<>(p0 & p1 -> p2) -> <>p0",
         K, 1 << 20, 32768, 24.08),
    ]
    out = []
    for name, text, cls, frames, vals, h100 in rows:
        if cls == K:
            hi = frames
        elif cls == "T":
            hi = t_frame_kindex(frames, 5)
        else:
            hi = K4_TABLE4_HI
        out.append({"name": name, "text": text, "cls": cls, "lo": 0, "hi": hi, "frames": frames,
                    "valuations": vals, "h100": h100})
    return out
