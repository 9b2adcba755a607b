"""The benchmarked workloads against the oracle's stored results.

The five-world census batch (5,624 formulas, K/T/S4/S5, S = 256) runs exactly
as bench.py launches it (engine.CENSUS5_CALLS), and every count, refuted-
frame count and witness key is compared with the values
tests/golden/make_census5_golden.py wrote from the oracle: all formulas at
n = 1..4; full five-world layers of a stratified subset (every variable
count, the longest and deepest formulas, the three axioms) and of every
variable-free formula; every formula's five-world S4 and S5 layers; and every formula's five-world
K and T layers as the oracle's tier-1 mask evaluator computed them (after
it had reproduced every five-world layer stored from tier 0).  The separation
workload (1,024 pairs) runs exactly as bench.py searches it
(engine.SEPARATION_SEARCH), and every first split is compared with the
oracle's: all of them through five worlds, six-world splits below K index
2^27, and the first sampled 7- and 8-world splits below sample 2^21 for the
pairs the oracle finds no earlier split for.  Every split is certified.
The uneven batch (20,000 jobs) runs in one persistent launch, and its layers
of four and five worlds are compared with the stored results: 440 of them
from tier 0, all of them from tier 1.
"""
import hashlib
import os

import numpy as np
import pytest

import golden_fixtures as G
from paper_2606_15437_gb300 import build as mkbuild
from paper_2606_15437_gb300 import mk
from paper_2606_15437_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CLS = ("K", "T", "S4", "S5")


@pytest.fixture(scope="module", autouse=True)
def _built():
    mkbuild.build()
    assert torch.cuda.is_available()


def _need(name):
    if not os.path.exists(os.path.join(G.HERE, name)):
        pytest.fail("golden file %s is missing (tests/golden/make_*_golden.py writes it)" % name)


def _key(w):
    return mk.NO_KEY if w is None else (w[0] << 27) | (w[1] << 3) | w[2]


@pytest.fixture(scope="module")
def census5():
    from paper_2606_15437_gb300 import engine as E
    texts = W.census5_formulas(2)
    progs = mk.compile_batch(texts)
    dev = torch.device("cuda", 0)
    table = W.valuation_table(2, 256, 5)
    d_progs = torch.from_numpy(progs.view(np.uint8).copy()).to(dev)
    d_samples = torch.from_numpy(table.view(np.uint8).reshape(-1).copy()).to(dev)
    plan = E.census_call_plan(progs, 256, d_samples.data_ptr(), dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    E.run_census_plan(plan, d_progs.data_ptr(), len(progs), status.data_ptr(),
                      torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return texts, progs, table, E.gather_census_plan(plan, len(progs))


def test_census_batch_n1_to_4_equals_the_oracle(census5):
    name = "census5_n1to4.tsv.gz"
    _need(name)
    texts, _, _, res = census5
    assert G.header_values(name)["texts_sha256"] == hashlib.sha256("\n".join(texts).encode()).hexdigest()
    want = G.census_rows(name)
    assert len(want) == len(texts) * 4 * 4
    bad = []
    for (p, c, n), (cm, fr, w) in want.items():
        got = tuple(int(x) for x in res[p, CLS.index(c), n - 1])
        if got != (cm, fr, _key(w)):
            bad.append((p, c, n, got, (cm, fr, _key(w))))
    assert not bad, bad[:5]


def test_census_batch_five_world_subset_equals_the_oracle(census5):
    name = "census5_n5_subset.tsv"
    _need(name)
    texts, progs, table, res = census5
    assert G.header_values(name)["texts_sha256"] == hashlib.sha256("\n".join(texts).encode()).hexdigest()
    want = G.census_rows(name)
    formulas = sorted({p for p, _, _ in want})
    assert len(want) == 4 * len(formulas)
    assert {int(progs[p]["nvars"]) for p in formulas} == {0, 1, 2, 3}
    for (p, c, n), (cm, fr, w) in want.items():
        got = tuple(int(x) for x in res[p, CLS.index(c), n - 1])
        assert got == (cm, fr, _key(w)), (p, texts[p], c)
        if w is not None:
            cert = mk.witness_cert(mk.program_at(progs, p), texts[p], c, 5, 256, table[5], got[2])
            assert mk.certify_struct(cert) == 1


def test_separation_workload_first_splits_equal_the_oracle():
    from paper_2606_15437_gb300 import engine as E
    name = "separation_first_splits.tsv"
    _need(name)
    pairs = W.separation_pairs(4)
    hv = G.header_values(name)
    assert hv["pairs_sha256"] == hashlib.sha256("\n".join(a + "\t" + b for a, b in pairs).encode()).hexdigest()
    b6, bs = int(hv["n6_bound"]), int(hv["sampled_bound"])
    assert int(hv["sampled_seed"]) == E.SEPARATION_SEARCH["seed"]
    job = E.SeparateJob(pairs, **E.SEPARATION_SEARCH)
    keys = [int(k) for k in job.run()]
    want = G.separation_rows(name)
    assert len(want) == len(pairs)
    checked = {"le5": 0, "n6": 0, "n7": 0, "n8": 0, "unsplit through 5": 0}
    for i, key in enumerate(keys):
        w = want[i]
        if key != mk.NO_KEY:
            assert mk.certify_struct(job.certificate(i, key)) == 1, i
        if w["le5"] is not None:
            n, f, v, x = w["le5"]
            assert key == mk.split_key(False, n, f, v, x), (i, pairs[i])
            checked["le5"] += 1
            continue
        checked["unsplit through 5"] += 1
        assert key == mk.NO_KEY or mk.split_n(key) >= 6, (i, pairs[i])
        if w["n6"] is not None:
            f, v, x = w["n6"]
            assert key == mk.split_key(False, 6, f, v, x), (i, pairs[i])
            checked["n6"] += 1
            continue
        # no six-world split below b6: the GPU's, if any, lies above it
        if key != mk.NO_KEY and not mk.split_sampled(key):
            assert mk.split_n(key) == 6 and (key >> 24) & ((1 << 36) - 1) >= b6, (i, pairs[i])
            continue
        # no six-world split at all: the sampled sizes, in order
        for n, col in ((7, "n7"), (8, "n8")):
            s = w[col]
            if key != mk.NO_KEY and mk.split_n(key) < n:
                break
            if s is not None:
                assert key == mk.split_key(True, n, s[0], s[1], s[2]), (i, pairs[i], n)
                checked[col] += 1
                break
            # none below bs at this size: the GPU's split, if at this size, lies above it
            if key != mk.NO_KEY and mk.split_n(key) == n:
                assert (key >> 24) & ((1 << 36) - 1) >= bs, (i, pairs[i], n)
                break
    print("separation splits checked against the oracle:", checked)
    assert checked["le5"] > 800 and checked["n6"] > 0


def test_uneven_batch_larger_layers_equal_the_oracle():
    """The uneven batch (20,000 jobs, own class and n_max each, S = 64) in one
    persistent launch: the four- and five-world layers of a seeded subset of
    jobs against the oracle's stored results (tests/golden/make_uneven_golden.py),
    and a graph replay of the same call gives the same results."""
    from paper_2606_15437_gb300 import engine as E
    name = "uneven_subset.tsv"
    _need(name)
    items = W.uneven_formulas(3)
    sha = hashlib.sha256("\n".join("%s\t%s\t%d" % it for it in items).encode()).hexdigest()
    assert G.header_values(name)["items_sha256"] == sha
    t = E.UNEVEN_TUNE
    job = E.UnevenJob(items, samples=64, seed=3, tiles=tuple(t["tiles"]), tune={"units": t["units"], "block": t["block"]})
    job.launch()
    res = job.results().copy()
    want = G.census_rows(name)
    assert len(want) == 440
    for (j, c, n), (cm, fr, w) in want.items():
        assert items[j][1] == c and items[j][2] >= n
        got = tuple(int(x) for x in res[j, n - 1])
        assert got == (cm, fr, _key(w)), (j, items[j], n)
        if w is not None:
            cert = mk.witness_cert(mk.program_at(job.progs, j), items[j][0], c, n, 64, job.sample_table[n], got[2])
            assert mk.certify_struct(cert) == 1
    job.capture()
    job.replay()
    assert np.array_equal(job.results(), res)


def test_census_batch_variable_free_five_world_layers_equal_the_oracle(census5):
    """Every variable-free formula of the batch (one valuation per frame): its
    full five-world K, T, S4 and S5 layers against the oracle's stored results."""
    name = "census5_n5_k0.tsv"
    _need(name)
    texts, progs, _, res = census5
    assert G.header_values(name)["texts_sha256"] == hashlib.sha256("\n".join(texts).encode()).hexdigest()
    want = G.census_rows(name)
    k0 = [p for p in range(len(texts)) if int(progs[p]["nvars"]) == 0]
    assert sorted({p for p, _, _ in want}) == k0 and len(want) == 4 * len(k0)
    bad = [(p, c) for (p, c, n), (cm, fr, w) in want.items()
           if tuple(int(x) for x in res[p, CLS.index(c), n - 1]) != (cm, fr, _key(w))]
    assert not bad, bad[:5]


def test_census_batch_every_formula_on_the_five_world_s4_s5_layers(census5):
    """Every formula of the batch on the full five-world S4 (6,942 frames) and
    S5 (52 frames) layers, from the device-built frame lists, against the
    oracle's stored results."""
    name = "census5_n5_s4s5.tsv.gz"
    _need(name)
    texts, _, _, res = census5
    assert G.header_values(name)["texts_sha256"] == hashlib.sha256("\n".join(texts).encode()).hexdigest()
    want = G.census_rows(name)
    assert len(want) == 2 * len(texts)
    bad = [(p, c) for (p, c, n), (cm, fr, w) in want.items()
           if tuple(int(x) for x in res[p, CLS.index(c), n - 1]) != (cm, fr, _key(w))]
    assert not bad, bad[:5]


def test_census_batch_every_formula_on_the_five_world_k_t_layers(census5):
    """Every formula of the batch on the full five-world K (2^25 frames) and T
    (2^20 frames) layers -- the launches that are 97 % of the bench's work --
    against the stored results of the oracle's tier-1 mask evaluator, which
    reproduced every five-world layer stored from tier 0 before writing them."""
    name = "census5_n5_tier1.tsv.gz"
    _need(name)
    texts, _, _, res = census5
    assert G.header_values(name)["texts_sha256"] == hashlib.sha256("\n".join(texts).encode()).hexdigest()
    want = G.census_rows(name)
    assert len(want) == 2 * len(texts) and {c for _, c, _ in want} == {"K", "T"}
    bad = [(p, c) for (p, c, n), (cm, fr, w) in want.items()
           if tuple(int(x) for x in res[p, CLS.index(c), n - 1]) != (cm, fr, _key(w))]
    assert not bad, bad[:5]


def test_uneven_batch_every_small_layer_equals_the_oracle():
    """Every layer of one to three worlds of every job of the uneven batch,
    from one persistent launch, against tier 0's stored results."""
    from paper_2606_15437_gb300 import engine as E
    name = "uneven_n1to3.tsv.gz"
    _need(name)
    items = W.uneven_formulas(3)
    sha = hashlib.sha256("\n".join("%s\t%s\t%d" % it for it in items).encode()).hexdigest()
    assert G.header_values(name)["items_sha256"] == sha
    t = E.UNEVEN_TUNE
    job = E.UnevenJob(items, samples=64, seed=3, tiles=tuple(t["tiles"]), tune={"units": t["units"], "block": t["block"]})
    job.launch()
    res = job.results().copy()
    want = G.census_rows(name)
    assert len(want) == 3 * len(items)
    bad = [(j, c, n) for (j, c, n), (cm, fr, w) in want.items()
           if items[j][1] != c or tuple(int(x) for x in res[j, n - 1]) != (cm, fr, _key(w))]
    assert not bad, bad[:5]


def test_uneven_batch_every_four_and_five_world_layer_equals_the_oracle():
    """Every four- and five-world layer of every job of the uneven batch
    (n = 4 .. n_max, the job's own class), from one persistent launch, against
    the stored results of the oracle's tier-1 mask evaluator, which first
    reproduced the layers stored from tier 0 (uneven_subset.tsv)."""
    from paper_2606_15437_gb300 import engine as E
    name = "uneven_tier1.tsv.gz"
    _need(name)
    items = W.uneven_formulas(3)
    sha = hashlib.sha256("\n".join("%s\t%s\t%d" % it for it in items).encode()).hexdigest()
    assert G.header_values(name)["items_sha256"] == sha
    t = E.UNEVEN_TUNE
    job = E.UnevenJob(items, samples=64, seed=3, tiles=tuple(t["tiles"]), tune={"units": t["units"], "block": t["block"]})
    job.launch()
    res = job.results().copy()
    want = G.census_rows(name)
    assert len(want) == sum(max(0, m - 3) for _, _, m in items)
    bad = [(j, c, n) for (j, c, n), (cm, fr, w) in want.items()
           if items[j][1] != c or tuple(int(x) for x in res[j, n - 1]) != (cm, fr, _key(w))]
    assert not bad, bad[:5]


def test_separation_context_pairs_full_ranges_equal_the_oracle():
    """The workload's unsplit alternating context pairs (the alpha family and
    its variants that no frame-independent law makes equal), searched exactly
    as the bench searches them, against the oracle over the search's whole
    range: every six-world frame (tier 1) and sampled relations [0, 10^8) of
    seven and eight worlds (tier 0)."""
    from paper_2606_15437_gb300 import engine as E
    name = "separation_context_pairs.tsv"
    _need(name)
    pairs = W.separation_pairs(4)
    hv = G.header_values(name)
    assert hv["pairs_sha256"] == hashlib.sha256("\n".join(a + "\t" + b for a, b in pairs).encode()).hexdigest()
    assert int(hv["sampled_range"]) == E.SEPARATION_SEARCH["frames_per_n"]
    rows = [r for r in G.rows(name)]
    assert rows
    idx = [int(r[0]) for r in rows]
    job = E.SeparateJob([pairs[i] for i in idx], **E.SEPARATION_SEARCH)
    keys = [int(k) for k in job.run()]
    for (i, n6, n7, n8, _), key in zip(rows, keys):
        if n6 != "-":
            f, v, w = (int(x) for x in n6.split(","))
            want = mk.split_key(False, 6, f, v, w)
        elif n7 != "-":
            f, v, w = (int(x) for x in n7.split(","))
            want = mk.split_key(True, 7, f, v, w)
        elif n8 != "-":
            f, v, w = (int(x) for x in n8.split(","))
            want = mk.split_key(True, 8, f, v, w)
        else:
            want = mk.NO_KEY
        assert key == want, (i, pairs[int(i)])
