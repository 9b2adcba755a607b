"""GPU parity of the uneven-batch path (persistent work queue, CUDA graph).

Every job's results from mk_census_uneven must equal, bit for bit, those of
per-bucket plain mk_census launches on the same formulas, the CPU oracle
where it is cheap (n <= 3), and a CUDA-graph replay of the same call.
"""
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
    assert torch.cuda.is_available()


def _items(seed, count, n_choices=(2, 3, 4)):
    rng = random.Random(seed)
    out = []
    for _ in range(count):
        L = rng.randint(2, 40)
        d = rng.randint(0, min(8, L - 1))
        k = rng.randint(0, 3)
        out.append((W.random_formula(rng, L, d, k), rng.choice(CLS), rng.choice(n_choices)))
    return out


def _per_bucket(job):
    from paper_2606_15437_gb300.engine import CensusJob
    want = np.zeros((job.njobs, 6, 3), np.uint64)
    want[:, :, 2] = mk.NO_KEY
    for (c, nmax), js in job.buckets().items():
        cj = CensusJob([job.texts[j] for j in js], (c,), 1, nmax, samples=job.S, seed=job.seed,
                       sample_table=job.sample_table)
        r = cj.run()
        for i, j in enumerate(js):
            want[j, :nmax] = r[i, 0]
    return want


@pytest.mark.parametrize("units,block", [(8, 256), (4, 128)])
def test_uneven_matches_per_bucket_launches(units, block):
    from paper_2606_15437_gb300.engine import UnevenJob
    items = _items(7, 300)
    job = UnevenJob(items, samples=64, seed=3, tiles=(4, 8, 16, 32),
                    tune={"units": units, "block": block})
    job.launch()
    got = job.results()
    assert np.array_equal(got, _per_bucket(job))


def test_uneven_matches_oracle_small():
    from paper_2606_15437_gb300.engine import UnevenJob
    items = _items(8, 60, n_choices=(1, 2, 3))
    job = UnevenJob(items, samples=16, seed=5)
    job.launch()
    got = job.results()
    for j, (t, c, nmax) in enumerate(items):
        for n in range(1, nmax + 1):
            want = oracle.census(t, c, n, samples=job.sample_table[n])
            key = mk.NO_KEY
            if want["witness"]:
                f, v, w = want["witness"]
                key = (f << 27) | (v << 3) | w
            assert tuple(int(x) for x in got[j, n - 1]) == (want["cm_count"], want["frames_refuted"], key)
        for n in range(nmax + 1, 7):
            assert int(got[j, n - 1, 0]) == 0 and int(got[j, n - 1, 2]) == mk.NO_KEY


def test_uneven_graph_replay_identical():
    from paper_2606_15437_gb300.engine import UnevenJob
    items = _items(9, 200, n_choices=(3, 4, 5))
    job = UnevenJob(items, samples=64, seed=3)
    job.launch()
    first = job.results().copy()
    job.capture()
    job.d_out.fill_(-1)
    job.replay()
    assert np.array_equal(job.results(), first)
    job.replay()
    assert np.array_equal(job.results(), first)
    # the five-world witnesses certify
    for j in range(0, job.njobs, 7):
        t, c, nmax = items[j]
        key = int(first[j, nmax - 1, 2])
        if key != mk.NO_KEY:
            cert = mk.witness_cert(mk.program_at(job.progs, j), t, c, nmax, job.S,
                                   job.sample_table[nmax], key)
            assert mk.certify_struct(cert) == 1


def test_autotuner_choice_is_on_the_grid_exact_and_cached(tmp_path, monkeypatch):
    """The autotuner returns a point of its swept grid (the fastest trial it
    timed), the chosen tune gives bit-identical results to the default one,
    and the choice is cached under the GPU's name and SM count and the
    batch's shape: a second call returns it without timing anything."""
    from paper_2606_15437_gb300 import engine as E
    items = W.uneven_formulas(3)[:900]
    cache = str(tmp_path / "tune.json")
    choice = E.autotune_uneven(items, samples=64, seed=3, sample_size=300, use_cache=True, cache_path=cache)
    assert choice["units"] in E.TUNE_UNITS and choice["block"] in E.TUNE_BLOCKS
    assert len(choice["tiles"]) == 4 and all(t in E.TUNE_TILES for t in choice["tiles"])
    assert choice["ms_sample"] == min(t["ms"] for t in choice["trials"])
    tuned = E.UnevenJob(items, samples=64, seed=3, tiles=tuple(choice["tiles"]),
                        tune={"units": choice["units"], "block": choice["block"]})
    tuned.launch()
    default = E.UnevenJob(items, samples=64, seed=3)
    default.launch()
    assert np.array_equal(tuned.results(), default.results())
    props = torch.cuda.get_device_properties(0)
    key = E.tune_cache_key(props.name, props.multi_processor_count, 64, [n for _, _, n in items])
    assert E._load_cache(cache)[key]["tiles"] == choice["tiles"]

    def no_timing(*a, **k):
        raise AssertionError("a cached tune must not be timed again")
    monkeypatch.setattr(E, "_time_graph", no_timing)
    assert E.autotune_uneven(items, samples=64, seed=3, sample_size=300, cache_path=cache) == choice
