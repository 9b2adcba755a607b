"""GPU parity of mk_separate against the CPU oracle (bit-exact first splits)."""
import random

import numpy as np
import pytest

import oracle
from paper_2606_15437_gb300 import build as mkbuild
from paper_2606_15437_gb300 import mk
from paper_2606_15437_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    mkbuild.build()
    assert torch.cuda.is_available()


def engine():
    from paper_2606_15437_gb300 import engine as E
    return E


def oracle_first_split(a, b, sizes, samples_table=None):
    for n in sizes:
        r = oracle.pair_layer(a, b, n, samples=None if samples_table is None else samples_table[n])
        if r["split"]:
            f, v, w, _, _ = r["split"]
            return mk.split_key(False, n, f, v, w)
    return mk.NO_KEY


def test_random_pairs_through_four_worlds():
    pairs = W.separation_pairs()[:200]
    job = engine().SeparateJob(pairs, 1, 4)
    got = job.run()
    for i, (a, b) in enumerate(pairs):
        want = oracle_first_split(a, b, (1, 2, 3, 4))
        assert int(got[i]) == want, (a, b)
        if want != mk.NO_KEY:
            assert mk.certify_struct(job.certificate(i, got[i])) == 1


def test_pairs_with_variables_sampled_valuations():
    rng = random.Random(3)
    pairs = [(W.random_formula(rng, rng.randint(2, 10), rng.randint(0, 3), rng.randint(0, 3)),
              W.random_formula(rng, rng.randint(2, 10), rng.randint(0, 3), rng.randint(0, 3)))
             for _ in range(40)]
    job = engine().SeparateJob(pairs, 1, 3, samples=16, seed=9)
    got = job.run()
    for i, (a, b) in enumerate(pairs):
        want = oracle_first_split(a, b, (1, 2, 3), job.sample_table)
        assert int(got[i]) == want, (a, b)


def test_alpha_family_exhaustive_six_worlds():
    # Prop. 5 / Table 3: alpha_1/alpha_2 split first at 4 worlds (K index
    # 328, world 1), alpha_2/alpha_3 at 6 worlds (K index 17,335,328, world 2)
    pairs = [(W.alpha(1), W.alpha(2)), (W.alpha(2), W.alpha(3))]
    job = engine().SeparateJob(pairs, 1, 6)
    got = [mk.decode_split(int(k)) for k in job.run()]
    assert got[0] == (4, 328, 0, 1)
    assert got[1] == (6, 17335328, 0, 2)
    for i in range(2):
        assert mk.certify_struct(job.certificate(i, job.d_split.cpu().numpy().view(np.uint64)[i])) == 1


def test_sampled_relations_first_split():
    # exhaustive sizes 1..2, then sampled 7- and 8-world relations; the
    # oracle regenerates the same relations and scans them in order
    pairs = [(W.alpha(1), W.alpha(2)), ("<><><>T", "<><><><>T"), ("[]<>T", "<>[]T"), ("[][]F", "[]F")]
    job = engine().SeparateJob(pairs, 1, 2, 7, 8, frames_per_n=100000, seed=11)
    got = job.run()
    for i, (a, b) in enumerate(pairs):
        want = oracle_first_split(a, b, (1, 2))
        if want == mk.NO_KEY:
            for n in (7, 8):
                r = oracle.pair_sampled(a, b, n, 11, 0, 100000)
                if r["split"]:
                    s, v, w, _, _ = r["split"]
                    want = mk.split_key(True, n, s, v, w)
                    break
        assert int(got[i]) == want, (a, b)
        if want != mk.NO_KEY:
            assert mk.certify_struct(job.certificate(i, got[i])) == 1


def test_equivalent_pair_never_splits():
    pairs = [("[][]T", "T"), ("<>F", "F"), ("~<>~T", "T"), ("p | ~p", "T")]
    job = engine().SeparateJob(pairs, 1, 5, 7, 7, frames_per_n=50000, seed=1)
    assert all(int(k) == mk.NO_KEY for k in job.run())


def test_sampled_six_world_split_certifies():
    # a split found on a sampled 6-world relation carries the sampled flag,
    # decodes to that relation and certifies (sampled sizes may include 6)
    pairs = [("<><><>T", "<><><><>T"), (W.alpha(1), W.alpha(2)), ("[][][]F", "[][][][]F")]
    job = engine().SeparateJob(pairs, 1, 2, 6, 7, frames_per_n=200000, seed=13)
    got = job.run()
    for i, (a, b) in enumerate(pairs):
        want = mk.NO_KEY
        for n in (6, 7):
            r = oracle.pair_sampled(a, b, n, 13, 0, 200000)
            if r["split"]:
                s, v, w, _, _ = r["split"]
                want = mk.split_key(True, n, s, v, w)
                break
        assert int(got[i]) == want, (a, b)
        if want != mk.NO_KEY:
            assert mk.split_sampled(got[i]) and mk.split_n(got[i]) in (6, 7)
            assert mk.certify_struct(job.certificate(i, got[i])) == 1


def test_unaligned_window_first_splits():
    """A K-index window that starts and ends inside frame words (the search
    rounds its first word down to a multiple of its unit count and masks the
    frames before frame_lo): first splits within the window equal the
    oracle's, for pairs splitting early, late and not at all in it."""
    pairs = [(W.alpha(1), W.alpha(2)), ("<><>T", "<>[]T"), ("[]<>[]F", "[][]F"), ("[]F", "~<>T"),
             ("<>(<>T & []F)", "<>[]F")] + W.separation_pairs()[32:60]
    for n, lo, hi in ((4, 333, 40001), (5, 12345, 12345 + 70000), (5, 2 ** 25 - 9999, 2 ** 25)):
        job = engine().SeparateJob(pairs, n, n, frame_lo=lo, frame_hi=hi)
        got = job.run()
        for i, (a, b) in enumerate(pairs):
            r = oracle.pair_layer(a, b, n, f_lo=lo, f_hi=hi)
            want = mk.NO_KEY
            if r["split"]:
                f, v, w, _, _ = r["split"]
                want = mk.split_key(False, n, f, v, w)
            assert int(got[i]) == want, (a, b, n, lo)


def _balanced(d, a, b):
    """A balanced &/| tree of depth d over the leaves a, b: its postfix
    program needs d stack entries."""
    if d == 0:
        return a
    x, y = _balanced(d - 1, a, b), _balanced(d - 1, b, a)
    return "(%s %s %s)" % (x, "&" if d % 2 else "|", y)


def test_deepest_stack_and_empty_batch():
    """Programs that need every stack entry (MK_MAX_STACK = 4) size the
    search's shared-memory stack; their first splits through four worlds
    equal the oracle's.  An empty batch returns nothing and launches
    nothing."""
    deep = _balanced(4, "<>p", "[]q")
    assert mk.compile(deep).depth == 4
    pairs = [(deep, _balanced(4, "[]q", "<>p")), (deep, _balanced(3, "<>p", "[]q")),
             (_balanced(3, "<>p", "[]q"), "<>p & []q"), (deep, deep.replace("[]q", "<>q"))]
    job = engine().SeparateJob(pairs, 1, 4, samples=16, seed=5)
    assert job.cfg.max_depth == 4
    got = job.run()
    for i, (a, b) in enumerate(pairs):
        want = oracle_first_split(a, b, (1, 2, 3, 4), job.sample_table)
        assert int(got[i]) == want, (a, b)
    assert len(engine().SeparateJob([], 1, 3).run()) == 0
