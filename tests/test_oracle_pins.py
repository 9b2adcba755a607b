"""Pins for the CPU oracle: facts the paper and the mathematics fix.

Each test checks oracle.c against something other than itself: values the
paper prints, closed forms, published counts, textbook frame
correspondences, or brute force by the pure-Python second path (pyref) on
tiny inputs.  A dropped term, a wrong sign or index or a transposed operand in
the oracle fails at least one of them.
"""
import itertools
import math
import random

import numpy as np
import pytest

import golden_fixtures as G
import oracle
from oracle import pyref
from paper_2606_15437_gb300 import workloads as W

ALL = 2 ** 64 - 1


def alpha(m):
    return W.alpha(m)


# ---------------------------------------------------------------- generator

def test_splitmix64_published_first_outputs():
    # SplitMix64 (Steele, Lea, Flood 2014) seeded with 0: the reference
    # implementation's first outputs.
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [oracle.splitmix_out(0, j) for j in range(4)] == want
    # the input generator's own implementation agrees
    assert [W.splitmix_out(0, j) for j in range(4)] == want


def test_sampled_frames_edge_density():
    # p_s is uniform on [26/256, 128/256]; the mean edge density over many
    # samples is (26+128)/2/256 ~ 0.30, and each sample stays in range.
    n = 8
    dens = [bin(oracle.sample_frame(7, n, s)).count("1") / 64.0 for s in range(4000)]
    assert 0.28 < np.mean(dens) < 0.32
    assert min(dens) >= 0.0 and max(dens) <= 0.75
    m7 = [oracle.sample_frame(7, 7, s) for s in range(200)]
    assert all(x < (1 << 49) for x in m7)


# ------------------------------------------------------- valid formulas (0)

@pytest.mark.parametrize("cls", ["K", "T", "S4", "S5"])
@pytest.mark.parametrize("n", [1, 2, 3])
def test_k_axiom_valid_everywhere(cls, n):
    r = oracle.census(W.K_AXIOM, cls, n)
    assert r["cm_count"] == 0 and r["frames_refuted"] == 0 and r["witness"] is None


def test_k_axiom_valid_four_worlds():
    assert oracle.census(W.K_AXIOM, "K", 4)["cm_count"] == 0


@pytest.mark.parametrize("t", ["p | ~p", "p -> p", "((p -> q) -> p) -> p", "~(p & ~p)",
                               "(p -> q) | (q -> p)", "[]T", "~<>F", "[](p | ~p)"])
def test_tautologies(t):
    for n in (1, 2, 3):
        assert oracle.census(t, "K", n)["cm_count"] == 0


# --------------------------------------------------------------- T axiom

def _t_axiom_closed_form(n):
    # valid (R, V) pairs: worlds in V(p) have any successor row, worlds
    # outside need a successor outside V(p)
    valid = sum(math.comb(n, s) * (2 ** n) ** s * (2 ** n - 2 ** s) ** (n - s)
                for s in range(n + 1))
    return 2 ** (n * n) * 2 ** n - valid


def test_t_axiom_one_world_irreflexive():
    r = oracle.census(W.T_AXIOM, "K", 1)
    assert r["cm_count"] == 1 and r["witness"] == (0, 0, 0)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_t_axiom_counts(n):
    r = oracle.census(W.T_AXIOM, "K", n)
    assert r["cm_count"] == _t_axiom_closed_form(n)
    assert r["frames_refuted"] == 2 ** (n * n) - 2 ** (n * n - n)   # non-reflexive frames
    assert [1, 23, 1609][n - 1:n] in ([], [r["cm_count"]])


@pytest.mark.parametrize("cls", ["T", "S4", "S5"])
def test_t_axiom_valid_on_reflexive(cls):
    for n in (1, 2, 3, 4):
        assert oracle.census(W.T_AXIOM, cls, n)["cm_count"] == 0


# ------------------------------------------------------------- 4 axiom

TRANSITIVE = {1: 2, 2: 13, 3: 171, 4: 3994}   # OEIS A006905


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_four_axiom_refutes_exactly_intransitive(n):
    r = oracle.census(W.FOUR_AXIOM, "K", n)
    assert r["frames_refuted"] == 2 ** (n * n) - TRANSITIVE[n]
    for cls in ("S4", "S5"):
        assert oracle.census(W.FOUR_AXIOM, cls, n)["cm_count"] == 0


def test_transitive_counts_brute_force():
    for n in (1, 2, 3):
        c = sum(1 for _, R in pyref.all_frames(n)
                if all((w, u) in R for (w, v) in R for (x, u) in R if v == x))
        assert c == TRANSITIVE[n]


# ---------------------------------------------------------- class sizes

PREORDERS = [1, 4, 29, 355, 6942]         # OEIS A000798, n = 1..5
BELL = [1, 2, 5, 15, 52]                   # equivalence relations, n = 1..5


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_class_sizes(n):
    assert oracle.class_size("K", n) == 2 ** (n * n)
    assert oracle.class_size("T", n) == 2 ** (n * n - n)
    assert oracle.class_size("S4", n) == PREORDERS[n - 1]
    assert oracle.class_size("S5", n) == BELL[n - 1]


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_bottom_is_refuted_on_every_class_frame(n):
    # F is false everywhere, so every class frame is refuted by its single
    # valuation: frames_refuted == cm_count == class size
    for cls, size in (("T", 2 ** (n * n - n)), ("S4", PREORDERS[n - 1]), ("S5", BELL[n - 1])):
        r = oracle.census("F", cls, n)
        assert r["frames_refuted"] == r["cm_count"] == r["frames"] == size


# ------------------------------------------------ constants and seriality

@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_dia_top_refutes_non_serial(n):
    r = oracle.census("<>T", "K", n)
    assert r["frames_refuted"] == 2 ** (n * n) - (2 ** n - 1) ** n


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_box_bot_valid_only_on_empty_relation(n):
    assert oracle.census("[]F", "K", n)["frames_refuted"] == 2 ** (n * n) - 1


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_b_axiom_valid_exactly_on_symmetric(n):
    r = oracle.census("p -> []<>p", "K", n)
    assert r["frames_refuted"] == 2 ** (n * n) - 2 ** (n * (n + 1) // 2)


# ------------------------------------------- frame correspondence (Table 9)

def _conds(n):
    def R(f, w, v):
        return (f >> (w * n + v)) & 1
    W_ = range(n)
    return {
        "reflexive": lambda f: all(R(f, w, w) for w in W_),
        "serial": lambda f: all(any(R(f, w, v) for v in W_) for w in W_),
        "transitive": lambda f: all(not (R(f, w, v) and R(f, v, u)) or R(f, w, u)
                                    for w in W_ for v in W_ for u in W_),
        "euclidean": lambda f: all(not (R(f, w, v) and R(f, w, u)) or R(f, v, u)
                                   for w in W_ for v in W_ for u in W_),
        "symmetric": lambda f: all(not R(f, w, v) or R(f, v, w) for w in W_ for v in W_),
        "partial_function": lambda f: all(sum(R(f, w, v) for v in W_) <= 1 for w in W_),
        "dense": lambda f: all(not R(f, w, v) or any(R(f, w, u) and R(f, u, v) for u in W_)
                               for w in W_ for v in W_),
        "confluent": lambda f: all(not (R(f, w, v) and R(f, w, u))
                                   or any(R(f, v, x) and R(f, u, x) for x in W_)
                                   for w in W_ for v in W_ for u in W_),
    }


# Table 9's landmarks (tests/golden), with this file's names for the conditions
_NAMES = {"reflexive": "reflexive", "serial": "serial", "transitive": "transitive", "Euclidean": "euclidean",
          "symmetric": "symmetric", "partially functional": "partial_function", "dense": "dense",
          "directed": "confluent"}
CORRESPONDENCES = [(f, _NAMES[c]) for _, f, c in G.table9() if c is not None]
MCKINSEY = [f for _, f, c in G.table9() if c is None]


@pytest.mark.parametrize("axiom,cond", CORRESPONDENCES)
@pytest.mark.parametrize("n", [1, 2, 3])
def test_correspondence(axiom, cond, n):
    valid = oracle.frame_valid_all(axiom, n)
    c = _conds(n)[cond]
    want = np.array([c(f) for f in range(2 ** (n * n))], np.uint8)
    assert np.array_equal(valid, want)


def test_mckinsey_matches_no_library_condition():
    n = 3
    assert MCKINSEY == ["[]<>p -> <>[]p"]
    valid = oracle.frame_valid_all(MCKINSEY[0], n)
    for name, c in _conds(n).items():
        want = np.array([c(f) for f in range(2 ** (n * n))], np.uint8)
        assert not np.array_equal(valid, want), name


# ------------------------------------------------------ alpha family (Sec. 7)

def test_alpha1_alpha2_first_split_at_four():
    # Table 3: m = 1 is UNSAT through 3 worlds, first SAT at 4
    m, through, first = G.table3()[0]
    assert (m, through, first) == (1, 3, 4)
    for n in range(1, through + 1):
        assert oracle.pair_layer(alpha(1), alpha(2), n)["split"] is None
    r = oracle.pair_layer(alpha(1), alpha(2), first)
    f, v, w, a, b = r["split"]
    # the brute-force second path agrees on the first split
    assert pyref.first_split(alpha(1), alpha(2), 4) == (f, v, w)
    assert (f, w) == (328, 1)
    assert r["frames_disagree"] == 768


@pytest.mark.slow
def test_alpha2_alpha3_agree_through_five_split_at_six():
    # Prop. 5: agreement on every frame of at most five worlds ...
    m, through, first = G.table3()[1]
    assert (m, through, first) == (2, 5, 6)
    for n in range(1, through + 1):
        assert oracle.pair_layer(alpha(2), alpha(3), n)["split"] is None
    # ... and a split at six worlds; the first one in K-index order:
    r = oracle.pair_layer(alpha(2), alpha(3), 6, f_lo=0, f_hi=17335329)
    f, v, w, a, b = r["split"]
    assert (f, w, a, b) == (17335328, 2, 1, 0)
    # the pure-Python path confirms that frame separates the pair at world 2
    R = {(x, y) for x in range(6) for y in range(6) if (f >> (x * 6 + y)) & 1}
    tr = pyref.parse(alpha(2)), pyref.parse(alpha(3))
    assert [pyref.sat(R, {}, 2, t) for t in tr] == [True, False]


def _nodes(tree):
    return 1 + sum(_nodes(c) for c in tree[1:] if isinstance(c, tuple))


def test_paper_certificate_alpha2_alpha3_path():
    # Prop. 5: successor masks (2,4,8,16,32,0), falsifying world w0
    cert = G.keyed("prop5_alpha_path_certificate.txt")
    phi, psi = cert["phi"], cert["psi"]
    assert (phi, psi) == (alpha(2), alpha(3))
    # Prop. 5 gives the formulas five and seven nodes
    assert (_nodes(pyref.parse(phi)), _nodes(pyref.parse(psi))) == (int(cert["phi_nodes"]), int(cert["psi_nodes"]))
    succ = [int(x) for x in cert["succ"].split()]
    w0 = int(cert["world"])
    n = len(succ)
    R = np.array([[(succ[w] >> v) & 1 for v in range(n)] for w in range(n)], np.uint8)
    f = sum(((succ[w] >> v) & 1) << (w * n + v) for w in range(n) for v in range(n))
    assert f == 541098242
    assert oracle.eval_model(phi, R)[w0] == 1
    assert oracle.eval_model(psi, R)[w0] == 0
    # the pure-Python path agrees
    Rs = {(x, y) for x in range(n) for y in range(n) if R[x, y]}
    assert [pyref.sat(Rs, {}, w0, pyref.parse(t)) for t in (phi, psi)] == [True, False]


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
def test_lemma8_path_family(m):
    # Lemma 2: on a directed path, alpha_m is false exactly at worlds with
    # r in {1, 3, ..., 2m-1} edges remaining to the dead end
    for L in (2 * m + 2, 2 * m + 5, 32):
        R = np.zeros((L, L), np.uint8)
        for w in range(L - 1):
            R[w, w + 1] = 1
        t = oracle.eval_model(alpha(m), R)
        for w in range(L):
            r = L - 1 - w
            assert t[w] == (0 if (r % 2 == 1 and r <= 2 * m - 1) else 1), (m, L, w)
    # the (2m+2)-world path separates alpha_m from alpha_(m+1) at its root
    L = 2 * m + 2
    R = np.zeros((L, L), np.uint8)
    for w in range(L - 1):
        R[w, w + 1] = 1
    assert oracle.eval_model(alpha(m), R)[0] == 1
    assert oracle.eval_model(alpha(m + 1), R)[0] == 0


def test_alpha3_alpha4_agree_through_four():
    # Table 3: m = 3 is UNSAT through 7 worlds (exhaustive check to 4 here),
    # first SAT at 8 worlds: the 8-world path of Lemma 2 separates them
    m, through, first = G.table3()[2]
    assert (m, through, first) == (3, 7, 8)
    for n in (1, 2, 3, 4):
        assert oracle.pair_layer(alpha(3), alpha(4), n)["split"] is None
    R = np.zeros((first, first), np.uint8)
    for w in range(first - 1):
        R[w, w + 1] = 1
    assert (oracle.eval_model(alpha(3), R)[0], oracle.eval_model(alpha(4), R)[0]) == (1, 0)


def test_table1_matched_workload_size():
    # Table 1: 262,144 five-world frames x all valuations of p, q = 268,435,456
    # cases; the formula is a K theorem, so no prefix of frames refutes it
    wl = G.keyed("table1_matched_workload.txt")
    r = oracle.census(wl["formula"], "K", int(wl["worlds"]), f_lo=0, f_hi=64)
    assert r["nvals"] == int(wl["valuations"])
    assert int(wl["frames"]) * r["nvals"] == int(wl["cases"])
    assert (r["cm_count"], r["frames_refuted"], r["witness"]) == (0, 0, None)
    # the bench's matched row is this workload
    row = W.matched_rows()[0]
    assert (row["text"], row["frames"], row["valuations"], row["hi"]) == \
        (wl["formula"], int(wl["frames"]), int(wl["valuations"]), int(wl["frames"]))


# ------------------------------------------------------ brute force (pyref)

def _random_texts(seed, count):
    rng = random.Random(seed)
    out = []
    for _ in range(count):
        L = rng.randint(1, 9)
        d = rng.randint(0, min(3, L - 1))
        k = rng.randint(0, 2)
        out.append(W.random_formula(rng, L, d, k, const_p=0.2))
    return out


@pytest.mark.parametrize("cls", ["K", "T", "S4", "S5"])
def test_brute_force_census_tiny(cls):
    for text in _random_texts(11, 40):
        for n in (1, 2):
            r = oracle.census(text, cls, n)
            cm, fr, wit = pyref.census(text, cls, n)
            assert (r["cm_count"], r["frames_refuted"], r["witness"]) == (cm, fr, wit), text


def test_brute_force_census_three_worlds():
    for text in _random_texts(12, 6):
        if pyref.nvars(pyref.parse(text)) > 1:
            continue
        for cls in ("K", "S4"):
            r = oracle.census(text, cls, 3)
            assert (r["cm_count"], r["frames_refuted"], r["witness"]) == pyref.census(text, cls, 3)


def test_brute_force_sampled_valuations():
    # k = 2 on 3 worlds has 64 valuations; with 16 samples they are sampled
    samples = W.sampled_valuations(99, 3, 16)
    for text in ["(p0 -> []p1)", "<>(p0 & ~p1) | []p1", "(p -> q) -> <>p"]:
        r = oracle.census(text, "K", 3, samples=samples)
        assert r["nvals"] == 16
        assert (r["cm_count"], r["frames_refuted"], r["witness"]) == \
            pyref.census_sampled(text, "K", 3, samples)
        # counts are additive over disjoint sample lists
        a = oracle.census(text, "K", 3, samples=samples[:8])["cm_count"]
        b = oracle.census(text, "K", 3, samples=samples[8:])["cm_count"]
        assert a + b == r["cm_count"]


def test_exhaustive_rule():
    # exhaustive when 2^(k n) <= S or k <= 1
    samples = W.sampled_valuations(1, 4, 256)
    assert oracle.census("p0 & p1", "K", 2, samples=samples)["nvals"] == 16
    assert oracle.census("p0 & p1", "K", 4, samples=samples)["nvals"] == 256   # 2^8 == S
    assert oracle.census("p0 & p2", "K", 3, samples=samples)["nvals"] == 256   # sampled
    assert oracle.census("[]p0", "K", 5, samples=samples)["nvals"] == 32


def test_frame_range_is_additive():
    text = "<>p -> [](q | p)"
    full = oracle.census(text, "T", 3)
    a = oracle.census(text, "T", 3, f_lo=0, f_hi=200)
    b = oracle.census(text, "T", 3, f_lo=200, f_hi=ALL)
    assert a["cm_count"] + b["cm_count"] == full["cm_count"]
    assert a["frames"] + b["frames"] == full["frames"] == 64
    assert min(x["witness"] for x in (a, b) if x["witness"]) == full["witness"]


def test_brute_force_first_split_tiny():
    rng = random.Random(5)
    for _ in range(20):
        a = W.random_formula(rng, rng.randint(2, 7), rng.randint(1, 3), 0)
        b = W.random_formula(rng, rng.randint(2, 7), rng.randint(1, 3), 0)
        for n in (1, 2):
            r = oracle.pair_layer(a, b, n)
            want = pyref.first_split(a, b, n)
            assert (r["split"][:3] if r["split"] else None) == want, (a, b, n)


def test_sampled_pair_scan_matches_explicit_frames():
    # the sampled scan evaluates exactly the relations sample_frame returns
    a, b = alpha(1), alpha(2)
    r = oracle.pair_sampled(a, b, 7, 3, 0, 3000)
    first = None
    for s in range(3000):
        m = oracle.sample_frame(3, 7, s)
        R = oracle.frame_matrix(m, 7)
        ta, tb = oracle.eval_model(a, R), oracle.eval_model(b, R)
        d = np.nonzero(ta != tb)[0]
        if len(d):
            first = (s, 0, int(d[0]))
            break
    assert (r["split"][:3] if r["split"] else None) == first


# ------------------------------------------------- frontier (Sec. 6, Prop. 3)

def _constant_free(nodes):
    """Every formula text over p, q with ~, [], <>, &, |, -> of exactly
    `nodes` nodes (atoms included)."""
    if nodes == 1:
        return ["p", "q"]
    out = []
    for u in ("~", "[]", "<>"):
        out += [u + "(" + a + ")" for a in _constant_free(nodes - 1)]
    for i in range(1, nodes - 1):
        for a in _constant_free(i):
            for b in _constant_free(nodes - 1 - i):
                out += ["(" + a + " " + op + " " + b + ")" for op in ("&", "|", "->")]
    return out


def test_frontier_refutable_formulas_need_at_most_two_worlds():
    # Prop. 3 and Sec. 6: no K-refutable constant-free formula over two
    # variables in the bounded corpus needs three worlds.  Checked for every
    # such formula of at most six nodes (7,040 of them), through three worlds.
    forms = [f for n in range(1, 7) for f in _constant_free(n)]
    assert len(forms) == 2 + 6 + 30 + 162 + 954 + 5886
    least = {}
    for f in forms:
        for n in (1, 2, 3):
            if oracle.census(f, "K", n)["cm_count"]:
                least[n] = least.get(n, 0) + 1
                break
    assert 3 not in least
    assert least[1] > 0 and least[2] > 0


def test_matched_rows_have_the_table_shapes():
    # Table 4's frames x valuations per row: the valuation count is all
    # valuations of the row's variables on five worlds, and the T row's
    # window holds exactly its 2,049 reflexive frames (counted by the oracle)
    for r in W.matched_rows():
        assert 2 ** (5 * oracle.nvars(r["text"])) == r["valuations"], r["name"]
        if r["cls"] == "K":
            assert (r["lo"], r["hi"]) == (0, r["frames"])
    t = [r for r in W.matched_rows() if r["cls"] == "T"][0]
    got = oracle.census(t["text"], "T", 5, f_lo=t["lo"], f_hi=t["hi"])
    assert got["frames"] == t["frames"] == 2049


# ------------------------------------------------------------------ K4 frames

def test_k4_class_is_the_transitive_frames():
    # K4's frames are the transitive relations (Sec. 2 names K4 beside T, S4,
    # S5): their number on n labelled points is OEIS A006905
    assert [oracle.class_size("K4", n) for n in range(1, 5)] == [2, 13, 171, 3994]
    assert [pyref.frames_in_class("K4", n) for n in range(1, 4)] == [2, 13, 171]


def test_k4_correspondences():
    # 4 = []p -> [][]p is valid exactly on transitive frames, so on every K4
    # frame; T = []p -> p is valid exactly on reflexive frames, so on K4 it is
    # refuted on the transitive frames that are not reflexive (K4 minus S4)
    for n in range(1, 5):
        assert oracle.census("[]p -> [][]p", "K4", n)["cm_count"] == 0
        r = oracle.census("[]p -> p", "K4", n)
        assert r["frames_refuted"] == oracle.class_size("K4", n) - oracle.class_size("S4", n)
    # and the K4 census agrees with the set-based path by brute force
    for t in ("[]p -> p", "<>[]p -> []<>p", "[](p -> q) | <>~q", "<>T -> []<>T"):
        for n in (1, 2, 3):
            a = oracle.census(t, "K4", n)
            assert (a["cm_count"], a["frames_refuted"], a["witness"]) == pyref.census(t, "K4", n), (t, n)


def test_k4_window_of_table4():
    # Table 4's K4 row filters 304 frames: read as the first 304 transitive
    # five-world frames in K order, which end below K index 653
    r = [x for x in W.matched_rows() if x["cls"] == "K4"][0]
    assert r["frames"] == 304 and (r["lo"], r["hi"]) == (0, 653)
    got = oracle.census(r["text"], "K4", 5, f_lo=0, f_hi=653)
    assert got["frames"] == 304
    assert oracle.census(r["text"], "K4", 5, f_lo=0, f_hi=652)["frames"] == 303
