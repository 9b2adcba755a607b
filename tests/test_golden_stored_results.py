"""The stored oracle results of the benchmarked workloads reproduce.

tests/golden/make_*_golden.py wrote these files from ``oracle/`` and the
seeded input generators; the GPU tests compare the bench's launches with
them.  Here, on the CPU: the input hashes in their headers still match the
generators, and a seeded sample of the cheaper rows (layers of at most three
worlds, the five-world S5 layer, four-world uneven layers, separation splits
through four worlds) is computed again by the oracle and equals the stored
row.  A change to the generators or to the oracle's arithmetic that would
make the stored values stale fails here first.
"""
import hashlib
import os
import random

import pytest

import golden_fixtures as G
import oracle
from paper_2606_15437_gb300 import workloads as W


CENSUS_FILES = ("census5_n1to4.tsv.gz", "census5_n5_subset.tsv", "census5_n5_k0.tsv",
                "census5_n5_s4s5.tsv.gz")


@pytest.fixture(scope="module", autouse=True)
def _oracle():
    oracle.build()


@pytest.fixture(scope="module")
def census5():
    texts = W.census5_formulas(2)
    samples = {n: W.sampled_valuations(2, n, 256) for n in range(1, 6)}
    return texts, samples


def _present(names):
    return [n for n in names if os.path.exists(os.path.join(G.HERE, n))]


def _row(r):
    return (r["cm_count"], r["frames_refuted"], r["witness"])


@pytest.mark.parametrize("name", _present(CENSUS_FILES))
def test_census_file_inputs_and_sampled_rows_reproduce(name, census5):
    texts, samples = census5
    assert G.header_values(name)["texts_sha256"] == hashlib.sha256("\n".join(texts).encode()).hexdigest()
    want = G.census_rows(name)
    assert want
    # cheap rows only: n <= 3 on any class, or the 52-frame S5 layer at n = 5
    cheap = sorted(u for u in want if u[2] <= 3 or (u[1] == "S5" and u[2] == 5))
    assert cheap, name
    for p, c, n in random.Random(name).sample(cheap, min(6, len(cheap))):
        got = oracle.census(texts[p], c, n, samples=samples[n])
        assert _row(got) == want[(p, c, n)], (name, p, texts[p], c, n)


def test_census_n1to4_file_covers_every_layer(census5):
    name = "census5_n1to4.tsv.gz"
    if not _present([name]):
        pytest.fail("golden file %s is missing" % name)
    texts, _ = census5
    want = G.census_rows(name)
    assert set(want) == {(p, c, n) for p in range(len(texts)) for c in ("K", "T", "S4", "S5")
                         for n in range(1, 5)}


def test_uneven_file_inputs_and_sampled_rows_reproduce():
    name = "uneven_subset.tsv"
    items = W.uneven_formulas(3)
    sha = hashlib.sha256("\n".join("%s\t%s\t%d" % it for it in items).encode()).hexdigest()
    assert G.header_values(name)["items_sha256"] == sha
    want = G.census_rows(name)
    four = sorted(u for u in want if u[2] == 4 and u[1] != "K")
    samples = W.sampled_valuations(3, 4, 64)
    for j, c, n in random.Random(7).sample(four, 4):
        got = oracle.census(items[j][0], c, n, samples=samples)
        assert _row(got) == want[(j, c, n)], (j, items[j])


def test_separation_file_inputs_and_early_splits_reproduce():
    name = "separation_first_splits.tsv"
    pairs = W.separation_pairs(4)
    sha = hashlib.sha256("\n".join(a + "\t" + b for a, b in pairs).encode()).hexdigest()
    assert G.header_values(name)["pairs_sha256"] == sha
    want = G.separation_rows(name)
    early = sorted(i for i, w in want.items() if w["le5"] is not None and w["le5"][0] <= 4)
    assert len(early) > 700
    for i in random.Random(4).sample(early, 12):
        a, b = pairs[i]
        first = None
        for n in range(1, 5):
            r = oracle.pair_layer(a, b, n)
            if r["split"] is not None:
                first = (n,) + tuple(r["split"][:3])
                break
        assert first == want[i]["le5"], (i, a, b)


def test_tier1_file_inputs_and_sampled_rows_reproduce(census5):
    """The tier-1 K/T file: input hash, one row per class for every variable
    count, computed again by the tier-1 evaluator."""
    name = "census5_n5_tier1.tsv.gz"
    if not _present([name]):
        pytest.fail("golden file %s is missing" % name)
    texts, samples = census5
    assert G.header_values(name)["texts_sha256"] == hashlib.sha256("\n".join(texts).encode()).hexdigest()
    want = G.census_rows(name)
    assert len(want) == 2 * len(texts)
    rng = random.Random(5)
    for k in range(4):
        ps = [p for p in range(len(texts)) if oracle.nvars(texts[p]) == k and len(texts[p]) < 30]
        p = rng.choice(ps)
        for c in ("T", "K") if k < 2 else ("T",):
            got = oracle.census_tier1(texts[p], c, 5, samples=samples[5])
            assert _row(got) == want[(p, c, 5)], (p, texts[p], c)


def test_uneven_small_file_inputs_and_sampled_rows_reproduce():
    """The uneven batch's one-to-three-world file: input hash, every such
    layer of every job, and a seeded sample computed again by tier 0."""
    name = "uneven_n1to3.tsv.gz"
    if not _present([name]):
        pytest.fail("golden file %s is missing" % name)
    items = W.uneven_formulas(3)
    sha = hashlib.sha256("\n".join("%s\t%s\t%d" % it for it in items).encode()).hexdigest()
    assert G.header_values(name)["items_sha256"] == sha
    want = G.census_rows(name)
    assert set(want) == {(j, items[j][1], n) for j in range(len(items)) for n in (1, 2, 3)}
    samples = {n: W.sampled_valuations(3, n, 64) for n in (1, 2, 3)}
    for j, c, n in random.Random(10).sample(sorted(want), 40):
        got = oracle.census(items[j][0], c, n, samples=samples[n])
        assert _row(got) == want[(j, c, n)], (j, items[j], n)


def test_uneven_tier1_file_inputs_and_sampled_rows_reproduce():
    """The uneven batch's tier-1 file: input hash, one layer per job with
    n_max >= 4, and a seeded sample of its cheaper rows computed again."""
    name = "uneven_tier1.tsv.gz"
    if not _present([name]):
        pytest.fail("golden file %s is missing" % name)
    items = W.uneven_formulas(3)
    sha = hashlib.sha256("\n".join("%s\t%s\t%d" % it for it in items).encode()).hexdigest()
    assert G.header_values(name)["items_sha256"] == sha
    want = G.census_rows(name)
    assert set(want) == {(j, items[j][1], n) for j in range(len(items)) for n in range(4, items[j][2] + 1)}
    samples = {n: W.sampled_valuations(3, n, 64) for n in (4, 5)}
    cheap = sorted(u for u in want if u[2] == 4 or u[1] != "K")
    for j, c, n in random.Random(9).sample(cheap, 8):
        got = oracle.census_tier1(items[j][0], c, n, samples=samples[n])
        assert _row(got) == want[(j, c, n)], (j, items[j], n)


def test_separation_context_file_inputs_and_a_window_reproduce():
    """The context-pair file: input hash, and no six-world split in the
    first 2^24 frames of each listed pair unless the file has one there."""
    name = "separation_context_pairs.tsv"
    if not _present([name]):
        pytest.fail("golden file %s is missing" % name)
    pairs = W.separation_pairs(4)
    sha = hashlib.sha256("\n".join(a + "\t" + b for a, b in pairs).encode()).hexdigest()
    assert G.header_values(name)["pairs_sha256"] == sha
    for r in G.rows(name):
        a, b = pairs[int(r[0])]
        got = oracle.pair_tier1(a, b, 6, f_lo=0, f_hi=1 << 24)["split"]
        if r[1] == "-" or int(r[1].split(",")[0]) >= 1 << 24:
            assert got is None, r
        else:
            assert ",".join(str(x) for x in got[:3]) == r[1], r
