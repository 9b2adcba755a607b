"""The oracle's tier-1 mask evaluator against tier 0.

``oracle.census_tier1`` (oracle/tier1.c: 64 frames per machine word, the
parse tree evaluated as it stands) computes the same census outputs as
``oracle.census`` (tier 0: the satisfaction clauses of Sec. 2 over explicit
relations, the scan of Alg. 1).  It is used only where it has been shown to
agree with tier 0; these tests pin it on the CPU: every layer through four
worlds for formulas of the five-world batch and hand-written ones with every
connective, every class, exhaustive and sampled valuations; the class sizes
through five worlds; and five-world layers that tier 0 has stored.
"""
import random

import pytest

import golden_fixtures as G
import oracle
from paper_2606_15437_gb300 import workloads as W

CLASSES = ("K", "T", "S4", "S5", "K4")


@pytest.fixture(scope="module", autouse=True)
def _oracle():
    oracle.build()


@pytest.fixture(scope="module")
def batch():
    texts = W.census5_formulas(2)
    samples = {n: W.sampled_valuations(2, n, 256) for n in range(1, 6)}
    return texts, samples


def test_tier1_equals_tier0_through_four_worlds_on_the_batch(batch):
    texts, samples = batch
    rng = random.Random(12)
    by_k = {k: [p for p, t in enumerate(texts) if oracle.nvars(t) == k] for k in range(4)}
    picks = [p for k in range(4) for p in rng.sample(by_k[k], 3)] + [len(texts) - 3, len(texts) - 1]
    for p in picks:
        for c in CLASSES:
            for n in range(1, 5):
                want = oracle.census(texts[p], c, n, samples=samples[n])
                got = oracle.census_tier1(texts[p], c, n, samples=samples[n])
                assert got == want, (p, texts[p], c, n)


@pytest.mark.parametrize("text", [
    "(p <-> q) -> ([]p <-> []q)",
    "~(<>p & []~p) | (p -> <>[]q)",
    "[](p | ~p) & <>T",
    "((p -> q) <-> (~q -> ~p)) & F",
    "<>(p & <>(q & <>r)) -> [][]p",
    "p2 | ~p2",
    "[]F",
])
def test_tier1_equals_tier0_on_every_connective(text):
    for n in range(1, 4):
        samples = W.sampled_valuations(9, n, 64)
        for c in CLASSES:
            want = oracle.census(text, c, n, samples=samples)
            assert oracle.census_tier1(text, c, n, samples=samples) == want, (text, c, n)
            want0 = oracle.census(text, c, n)
            assert oracle.census_tier1(text, c, n) == want0, (text, c, n, "exhaustive")


def test_tier1_class_sizes_through_five_worlds():
    for c in CLASSES:
        for n in range(1, 6):
            assert oracle.census_tier1("T", c, n)["frames"] == oracle.class_size(c, n), (c, n)


def test_tier1_reproduces_stored_five_world_layers(batch):
    """Five-world layers that tier 0 computed and stored: a variable-free K
    layer, K and T layers with sampled valuations, and S4/S5 layers."""
    texts, samples = batch
    subset = G.census_rows("census5_n5_subset.tsv")
    k0 = G.census_rows("census5_n5_k0.tsv")
    picks = [u for u in sorted(subset) if u[1] in ("K", "T") and oracle.nvars(texts[u[0]]) >= 2
             and len(texts[u[0]]) < 24][:2]
    picks += [next(u for u in sorted(k0) if u[1] == "K")]
    picks += [u for u in sorted(subset) if u[1] in ("S4", "S5")][:4]
    assert len(picks) == 7
    for p, c, n in picks:
        want = subset.get((p, c, n)) or k0[(p, c, n)]
        r = oracle.census_tier1(texts[p], c, n, samples=samples[n])
        assert (r["cm_count"], r["frames_refuted"], r["witness"]) == want, (p, texts[p], c)


def test_tier1_pair_scan_equals_tier0():
    """oracle.pair_tier1 (the separation of Def. 2 / Prop. 4 by the mask
    evaluator) against tier 0's pair_layer: workload pairs through four worlds
    and on a ragged five-world window, and pairs with variables (exhaustive
    and sampled valuations)."""
    pairs = W.separation_pairs(4)
    rng = random.Random(21)
    for i in rng.sample(range(len(pairs)), 16) + [0, 1, 32]:
        a, b = pairs[i]
        for n in range(1, 5):
            assert oracle.pair_tier1(a, b, n) == oracle.pair_layer(a, b, n), (i, n)
        lo, hi = 2000001, 2000001 + 30013
        assert oracle.pair_tier1(a, b, 5, f_lo=lo, f_hi=hi) == oracle.pair_layer(a, b, 5, f_lo=lo, f_hi=hi), i
    for a, b in (("[]p -> p", "<>p | ~p"), ("[](p -> q)", "[]p -> []q"), ("<>(p & q)", "<>p & <>q")):
        for n in range(1, 4):
            samples = W.sampled_valuations(9, n, 64)
            assert oracle.pair_tier1(a, b, n) == oracle.pair_layer(a, b, n), (a, b, n)
            assert oracle.pair_tier1(a, b, n, samples=samples) == oracle.pair_layer(a, b, n, samples=samples)


def test_tier1_pair_scan_finds_the_six_world_alpha_split():
    """alpha_2 / alpha_3 agree on every frame of at most five worlds and first
    split at six worlds on K index 17,335,328, world 2 (Prop. 5; tier 0 and
    the pure-Python path give the same): tier 1 finds it scanning the first
    2^27 six-world frames."""
    a, b = "[]<>[]<>T", "[]<>[]<>[]<>T"
    for n in range(1, 6):
        assert oracle.pair_tier1(a, b, n)["split"] is None
    r = oracle.pair_tier1(a, b, 6, f_lo=0, f_hi=1 << 27)
    assert r["split"] == (17335328, 0, 2, 1, 0)
