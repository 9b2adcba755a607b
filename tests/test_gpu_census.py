"""GPU parity of mk_census against the CPU oracle (bit-exact).

Every count, refuted-frame count and witness key is compared element by
element with oracle.census on the same seeded inputs; every witness is
re-checked by mk_certify.  Sizes: the PR1 configuration in full (n <= 3),
random formulas through n = 4 with sampled valuations, five-world layers on
K-index windows, closed forms on full five-world layers, and the
five-world census batch in the launch configuration bench.py times, checked
on sampled outputs.
"""
import math
import random

import numpy as np
import pytest

import oracle
from paper_2606_15437_gb300 import build as mkbuild
from paper_2606_15437_gb300 import mk
from paper_2606_15437_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CLS = ("K", "T", "S4", "S5")


@pytest.fixture(scope="module", autouse=True)
def _built():
    mkbuild.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def engine():
    from paper_2606_15437_gb300 import engine as E
    return E


def oracle_key(r):
    if r["witness"] is None:
        return mk.NO_KEY
    f, v, w = r["witness"]
    return (f << 27) | (v << 3) | w


def check_against_oracle(job, res, texts, n_values, classes=CLS, certify=True, **rng):
    for p, text in enumerate(texts):
        for ci, c in enumerate(job.classes):
            if c not in classes:
                continue
            for n in n_values:
                ni = n - job.n_min
                samples = job.sample_table[n] if job.S else None
                want = oracle.census(text, c, n, samples=samples, **rng)
                got = tuple(int(x) for x in res[p, ci, ni])
                assert got == (want["cm_count"], want["frames_refuted"], oracle_key(want)), (text, c, n)
                if certify and got[2] != mk.NO_KEY:
                    cert = job.certificate(p, c, n, got[2])
                    assert mk.certify_struct(cert) == 1, (text, c, n)


def test_pr1_config_full():
    texts = W.pr1_formulas()
    job = engine().CensusJob(texts, CLS, 1, 3, samples=0)
    res = job.run()
    check_against_oracle(job, res, texts, (1, 2, 3))


@pytest.mark.parametrize("tile,block,units", [(1, 128, 2), (7, 256, 4), (16, 256, 8), (64, 128, 4)])
def test_random_formulas_sampled_valuations(tile, block, units):
    rng = random.Random(tile)
    texts = [W.random_formula(rng, rng.randint(1, 20), rng.randint(0, 4), rng.randint(0, 4))
             for _ in range(37)]
    job = engine().CensusJob(texts, CLS, 1, 4, samples=16, seed=tile,
                             tune={"tile": tile, "block": block, "units": units})
    res = job.run()
    check_against_oracle(job, res, texts, (1, 2, 3))
    # n = 4 on a subset (the oracle pays 2^16 frames each)
    check_against_oracle(job, res, texts[:6], (4,))


def test_long_formulas_many_registers():
    rng = random.Random(99)
    texts = []
    while len(texts) < 12:
        t = W.random_formula(rng, rng.randint(40, 64), rng.randint(1, 8), rng.randint(0, 2))
        if mk.compile(t).depth >= 2:
            texts.append(t)
    t = "p"
    for _ in range(5):
        t = "(%s & %s)" % (t, t.replace("p", "q"))
    texts.append(t)
    job = engine().CensusJob(texts, CLS, 1, 3, samples=0)
    check_against_oracle(job, job.run(), texts, (1, 2, 3))


def test_five_world_windows():
    # K and T layers at n = 5 restricted to K-index windows; the oracle
    # computes the same windows
    rng = random.Random(5)
    texts = [W.random_formula(rng, rng.randint(3, 24), rng.randint(1, 4), rng.randint(0, 3))
             for _ in range(10)] + list(W.AXIOMS)
    for lo in (0, 123457, 2 ** 25 - 5000):
        hi = lo + 5000
        job = engine().CensusJob(texts, ("K", "T", "S4"), 5, 5, samples=256, seed=2,
                                 frame_lo=lo, frame_hi=hi)
        check_against_oracle(job, job.run(), texts, (5,), f_lo=lo, f_hi=hi)


def _t_axiom(n):
    valid = sum(math.comb(n, s) * (2 ** n) ** s * (2 ** n - 2 ** s) ** (n - s) for s in range(n + 1))
    return 2 ** (n * n) * 2 ** n - valid


def test_closed_forms_full_five_worlds():
    texts = [W.T_AXIOM, W.FOUR_AXIOM, "<>T", "[]F", "p -> []<>p", W.K_AXIOM, "F"]
    job = engine().CensusJob(texts, CLS, 1, 5, samples=256)
    res = job.run()
    K, T, S4, S5 = 0, 1, 2, 3
    for n in range(1, 6):
        i = n - 1
        assert int(res[0, K, i, 0]) == _t_axiom(n)
        assert int(res[0, K, i, 1]) == 2 ** (n * n) - 2 ** (n * n - n)
        assert int(res[0, T, i, 0]) == int(res[0, S4, i, 0]) == int(res[0, S5, i, 0]) == 0
        transitive = [2, 13, 171, 3994, 154303][i]           # OEIS A006905
        assert int(res[1, K, i, 1]) == 2 ** (n * n) - transitive
        assert int(res[1, S4, i, 0]) == int(res[1, S5, i, 0]) == 0
        assert int(res[2, K, i, 1]) == 2 ** (n * n) - (2 ** n - 1) ** n
        assert int(res[3, K, i, 1]) == 2 ** (n * n) - 1
        assert int(res[4, K, i, 1]) == 2 ** (n * n) - 2 ** (n * (n + 1) // 2)
        assert int(res[5, :, i, 0].sum()) == 0 and int(res[5, K, i, 2]) == mk.NO_KEY
        sizes = [2 ** (n * n), 2 ** (n * n - n), [1, 4, 29, 355, 6942][i], [1, 2, 5, 15, 52][i]]
        assert [int(res[6, c, i, 1]) for c in range(4)] == sizes
    assert int(res[0, K, 0, 2]) == 0     # witness (frame 0, valuation 0, world 0)


def test_bench_workload_sampled_outputs():
    """The five-world census batch as bench.py launches it (5,624 formulas,
    K/T/S4/S5, n <= 5, S = 256), checked on sampled outputs: every sampled
    witness is certified and minimal (oracle scan of the frames before it),
    and all counts of sampled formulas at n <= 3 equal the oracle's."""
    texts = W.census5_formulas()
    job = engine().CensusJob(texts, CLS, 1, 5, samples=256, seed=2)
    res = job.run()
    rng = random.Random(0)
    picks = rng.sample(range(len(texts)), 24) + [len(texts) - 3, len(texts) - 2, len(texts) - 1]
    for p in picks:
        text = texts[p]
        for ci, c in enumerate(CLS):
            for n in (1, 2, 3):
                samples = job.sample_table[n]
                want = oracle.census(text, c, n, samples=samples)
                got = tuple(int(x) for x in res[p, ci, n - 1])
                assert got == (want["cm_count"], want["frames_refuted"], oracle_key(want)), (text, c, n)
            for n in (4, 5):
                key = int(res[p, ci, n - 1, 2])
                if key == mk.NO_KEY:
                    assert int(res[p, ci, n - 1, 0]) == 0
                    continue
                cert = job.certificate(p, c, n, key)
                assert mk.certify_struct(cert) == 1
                f = key >> 27
                if f < 200000:
                    # no earlier frame refutes it, and this frame's witness matches
                    want = oracle.census(text, c, n, samples=job.sample_table[n], f_lo=0, f_hi=f + 1)
                    assert oracle_key(want) == key, (text, c, n)


def test_empty_and_ragged_batches():
    E = engine()
    job = E.CensusJob([], CLS, 1, 2, samples=0, progs=np.zeros(0, mk.PROGRAM_DTYPE))
    assert job.run().shape == (0, 4, 2, 3)
    texts = W.pr1_formulas()[:17]
    job = E.CensusJob(texts, ("S5",), 3, 3, samples=0, tune={"tile": 16})
    check_against_oracle(job, job.run(), texts, (3,))


def test_malformed_program_sets_status():
    E = engine()
    progs = mk.compile_batch(["p", "q"])
    progs["code"][1][0] = 250          # not an instruction
    job = E.CensusJob(["p", "q"], ("K",), 1, 2, samples=0, progs=progs)
    with pytest.raises(mk.MkError) as e:
        job.run()
    assert e.value.code == -8


# --------------------------------------------- valuations split over CTAs

SPLIT_CASES = [
    # (formula, class, n, K window, samples): few frames, many valuations
    ("[](p0 -> p1) & <>(p1 & ~p2) -> [](p2 | <>p0)", "K", 4, (0, 1024), 0),
    ("[]<>p0 & <>(p1 -> []p2) -> <>[]p3", "K", 4, (5000, 5040), 0),    # ragged words
    ("<>(p0 & []p1) -> [](p2 -> <>p0)", "T", 4, (0, 34816), 0),       # T compact 0..255
    ("[](p0 -> <>p1) -> <>[]p0 | p2", "S4", 4, (0, mk.NO_KEY), 0),
    ("[]p0 & <>p1 -> <>(p2 & p3)", "K", 5, (0, 2048), 256),
    ("<>[](p0 -> <>(p1 & ~p2)) -> [][]p0", "K", 5, (96, 192), 0),
    # four variables at five worlds, all 2^20 valuations, on a part-filled word
    ("<>(p0 & p1) -> [](p2 | ~p3)", "K", 5, (3, 7), 0),
]


@pytest.mark.parametrize("text,cls,n,win,samples", SPLIT_CASES)
def test_valuation_split_matches_oracle(text, cls, n, win, samples):
    """A layer too small to fill the GPU splits its valuations over grid.z
    (automatically, or as forced); every split gives the oracle's counts,
    refuted frames and least witness."""
    E = engine()
    want = None
    ws = {}
    for vsplit in (0, 1, 2, 5, 4096):
        job = E.CensusJob([text], (cls,), n, n, samples=samples, seed=n, frame_lo=win[0], frame_hi=win[1],
                          vsplit=vsplit)
        ws[vsplit] = job.ws_bytes
        res = job.run()
        if want is None:
            samp = job.sample_table[n] if samples else None
            r = oracle.census(text, cls, n, samples=samp, f_lo=win[0], f_hi=win[1])
            want = (r["cm_count"], r["frames_refuted"], oracle_key(r))
            assert r["frames"] > 0
        assert tuple(int(x) for x in res[0, 0, 0]) == want, (vsplit, text, cls, n)
    # the automatic choice did split (its workspace holds the frame bitmap)
    assert ws[0] > ws[1]


def test_matched_single_formula_workload():
    """Table 1's matched workload: [](p -> q) -> (<>p -> <>q) on the first
    262,144 five-world frames under all 1,024 valuations.  It is a theorem of
    K, so no countermodel exists; the oracle confirms it on a prefix."""
    import golden_fixtures as G
    E = engine()
    wl = G.keyed("table1_matched_workload.txt")
    text = wl["formula"]
    job = E.CensusJob([text], ("K",), 5, 5, samples=0, frame_lo=0, frame_hi=int(wl["frames"]))
    res = job.run()
    assert tuple(int(x) for x in res[0, 0, 0]) == (0, 0, mk.NO_KEY)
    r = oracle.census(text, "K", 5, f_lo=0, f_hi=2048)
    assert (r["cm_count"], r["frames_refuted"], r["witness"]) == (0, 0, None)
    # a refutable neighbour on the same window: the split census against the oracle
    text2 = "[](p -> q) -> (<>q -> <>p)"
    job2 = E.CensusJob([text2], ("K",), 5, 5, samples=0, frame_lo=0, frame_hi=4096)
    got = tuple(int(x) for x in job2.run()[0, 0, 0])
    r2 = oracle.census(text2, "K", 5, f_lo=0, f_hi=4096)
    assert got == (r2["cm_count"], r2["frames_refuted"], oracle_key(r2))


def test_resumable_census_on_the_gpu(tmp_path):
    """The checkpointed census driver with mk_census as its unit runner: a
    run stopped by a failure after a few units, then resumed, merges to the
    one-call census bit for bit, and the resume runs only the missing
    units."""
    E = engine()
    texts = W.census5_formulas()[:40] + list(W.AXIOMS)
    kw = dict(samples=256, seed=2, tile=16, frame_chunk=1 << 12)
    d = str(tmp_path / "ckpt")
    units = E.census_units(len(texts), CLS, 1, 4, kw["tile"], kw["frame_chunk"])

    class Stop(Exception):
        pass

    def stop_after(u, seen=[]):
        seen.append(u)
        if len(seen) == 7:
            raise Stop()

    with pytest.raises(Stop):
        E.resumable_census(texts, CLS, 1, 4, d, after_unit=stop_after, **kw)
    ran = E.resumable_census(texts, CLS, 1, 4, d, **kw)
    assert len(ran) == len(units) - 7
    got = E.merge_census_journal(texts, CLS, 1, 4, d, **kw)
    want = E.CensusJob(texts, CLS, 1, 4, samples=256, seed=2).run()
    assert np.array_equal(got, want)


def test_k4_class_against_the_oracle():
    """K4 frames (transitive relations, listed on the device by filtering
    the K frames): every count and witness against the oracle through four
    worlds, with sampled valuations, and every witness certified in class
    K4."""
    texts = (["<>T -> []<>T", "[](p0 -> p1) & <>p2 -> <>(p1 & p2)"] + list(W.AXIOMS) +
             W.pr1_formulas()[:30])
    job = engine().CensusJob(texts, ("K4",), 1, 4, samples=16, seed=4)
    res = job.run()
    check_against_oracle(job, res, texts, (1, 2, 3), classes=("K4",))
    # four worlds (3,994 transitive frames) for the first formulas: results are
    # compared by position, so a prefix of the batch
    check_against_oracle(job, res, texts[:9], (4,), classes=("K4",))


def test_k4_closed_forms_through_five_worlds():
    # class sizes (OEIS A006905), 4 valid on every transitive frame, T
    # refuted exactly on the transitive frames that are not reflexive
    texts = ["F", W.FOUR_AXIOM, W.T_AXIOM]
    job = engine().CensusJob(texts, ("K4", "S4"), 1, 5, samples=0)
    res = job.run()
    sizes = [2, 13, 171, 3994, 154303]
    for n in range(1, 6):
        assert int(res[0, 1, n - 1, 1]) == sizes[n - 1]
        assert int(res[1, 1, n - 1, 0]) == 0 and int(res[1, 1, n - 1, 2]) == mk.NO_KEY
        assert int(res[2, 1, n - 1, 1]) == sizes[n - 1] - int(res[0, 0, n - 1, 1])


def test_k4_window_of_table4_matched_row():
    # Table 4's K4 row: the first 304 transitive five-world frames (K index < 653)
    r = [x for x in W.matched_rows() if x["cls"] == "K4"][0]
    job = engine().CensusJob(["F", r["text"], "[]p -> p"], ("K4",), 5, 5, samples=0, frame_lo=r["lo"],
                             frame_hi=r["hi"])
    res = job.run()
    assert int(res[0, 0, 0, 1]) == r["frames"] == 304
    for i, t in enumerate(["F", r["text"], "[]p -> p"]):
        want = oracle.census(t, "K4", 5, f_lo=r["lo"], f_hi=r["hi"])
        assert tuple(int(x) for x in res[i, 0, 0]) == (want["cm_count"], want["frames_refuted"], oracle_key(want))


def test_matched_rows_equal_the_oracle_at_full_shape():
    """Every matched single-formula row (Table 1, Table 4, Sec. 8) as the
    matched bench launches it -- one formula on its K-index window, every
    valuation, the valuations split over CTAs where the frames cannot fill
    the GPU -- against the oracle on the same window; the Sec. 8 stress row
    (3.4e10 evaluations) on its first 2,048 frames."""
    E = engine()
    for r in W.matched_rows():
        lo, hi = r["lo"], r["hi"]
        if r["frames"] * r["valuations"] > 3e8:
            hi = lo + 2048
        job = E.CensusJob([r["text"]], (r["cls"],), 5, 5, samples=0, frame_lo=lo, frame_hi=hi)
        got = tuple(int(x) for x in job.run()[0, 0, 0])
        want = oracle.census(r["text"], r["cls"], 5, f_lo=lo, f_hi=hi)
        assert got == (want["cm_count"], want["frames_refuted"], oracle_key(want)), r["name"]
        if got[2] != mk.NO_KEY:
            assert mk.certify_struct(job.certificate(0, r["cls"], 5, got[2])) == 1, r["name"]
