"""GPU parity of the failure-density atlas (Sec. 9) against the CPU oracle:
exact counts, the FP64 Gram matrix and principal axis (to rounding), the
device sort (exact, ties by index), A(pi) (exact integer sums), and the
binned density view (exact counts from the same FP64 cell rule)."""
import random

import numpy as np
import pytest

import oracle
from oracle import atlas as OA
from paper_2606_15437_gb300 import build as mkbuild
from paper_2606_15437_gb300 import mk
from paper_2606_15437_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    mkbuild.build()
    assert torch.cuda.is_available()


def E():
    from paper_2606_15437_gb300 import engine
    return engine


@pytest.mark.parametrize("n,count", [(1, 40), (2, 60), (3, 300), (4, 12)])
def test_counts_match_oracle(n, count):
    rng = random.Random(n)
    texts = ["T", "F", "p", "[]p -> p"] + [W.random_formula(rng, rng.randint(3, 20), rng.randint(1, 4),
                                                           rng.randint(0, 4 if n <= 3 else 3))
                                          for _ in range(count)]
    texts = [t for t in texts if oracle.nvars(t) * n <= 16]
    a = E().Atlas(texts, n)
    got = a.compute().cpu().numpy().view(np.uint32)
    a.check_status()
    want_c, want_d = OA.atlas_counts(texts, n)
    assert np.array_equal(got, want_c)
    assert np.array_equal(a.denom, want_d)


@pytest.fixture(scope="module")
def corpus_atlas():
    texts = W.census5_formulas()[:1500]
    a = E().Atlas(texts, 3)
    a.compute()
    cnt, den = OA.atlas_counts(texts, 3)
    return a, OA.density(cnt, den)


def test_gram_and_principal_axis(corpus_atlas):
    a, D = corpus_atlas
    V, U = a.principal_axes(2)
    Dc = D - D.mean(axis=0, keepdims=True)
    assert np.allclose(a.d_mean.cpu().numpy(), D.mean(axis=0), rtol=0, atol=1e-12)
    assert np.allclose(a.gram.cpu().numpy(), Dc.T @ Dc, rtol=1e-10, atol=1e-9)
    col, row, v, u = OA.seriation(D)
    vg = V[0].cpu().numpy()
    assert abs(float(vg @ v)) > 1 - 1e-9 and np.allclose(vg, v, atol=1e-6)    # same sign convention
    assert np.allclose(U[0].cpu().numpy(), u, atol=1e-6)
    # second axis: orthogonal to the first, and the second right singular vector up to sign
    _, s, vt = np.linalg.svd(Dc, full_matrices=False)
    v2 = V[1].cpu().numpy()
    assert abs(float(v2 @ vg)) < 1e-9 and abs(abs(float(v2 @ vt[1])) - 1) < 1e-6


def test_seriation_orders_and_adjacent_variation(corpus_atlas):
    a, D = corpus_atlas
    colg, rowg, vg, ug = a.seriation()
    colg, vg = colg.cpu().numpy(), vg.cpu().numpy()
    # the device sort is exact on the device keys
    assert list(colg) == list(np.lexsort((np.arange(len(vg)), vg)))
    col, _, _, _ = OA.seriation(D)
    # the two orders may differ only among frames with identical columns
    # (equal keys): the seriated displays are the same matrix
    assert np.array_equal(D[:, colg], D[:, col])
    A_dev, A_orc = a.adjacent_variation(colg), OA.adjacent_variation(D, col)
    assert A_dev == pytest.approx(A_orc, abs=1e-12)
    rng = np.random.default_rng(0)
    for _ in range(3):
        p = rng.permutation(a.F).astype(np.int32)
        assert a.adjacent_variation(p) == pytest.approx(OA.adjacent_variation(D, p), rel=1e-12)
    deg = np.array([bin(f).count("1") for f in range(a.F)])
    by_deg = np.lexsort((np.arange(a.F), deg)).astype(np.int32)
    assert A_dev < a.adjacent_variation(by_deg) < a.adjacent_variation(rng.permutation(a.F).astype(np.int32))


def test_sort_keys_with_ties():
    rng = np.random.default_rng(5)
    for n in (1, 7, 1000, 4097):
        keys = np.round(rng.normal(size=n), 1)          # many ties
        d = torch.tensor(keys, dtype=torch.float64, device="cuda")
        a = E().Atlas(["T"], 1)
        got = a.order(d).cpu().numpy()
        assert list(got) == list(np.lexsort((np.arange(n), keys)))


def test_adjacent_variation_flags_bad_permutation(corpus_atlas):
    a, _ = corpus_atlas
    p = np.arange(a.F, dtype=np.int32)
    p[7] = a.F + 3
    with pytest.raises(mk.MkError):
        a.adjacent_variation(p)
    a.d_status.zero_()


def test_histogram_and_stats():
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(0.2, 0.05, 20000), rng.uniform(-1, 2, 5000), [np.nan, 1.0, 0.0]])
    y = np.concatenate([rng.normal(0.7, 0.02, 20000), rng.uniform(-1, 2, 5000), [0.5, 1.0, 0.0]])
    dx = torch.tensor(x, dtype=torch.float64, device="cuda")
    dy = torch.tensor(y, dtype=torch.float64, device="cuda")
    G = 256
    st = E().density_view(dx, dy, 0.0, 1.0, G=G, radius=2)
    h = st["hist"].cpu().numpy()
    xx = np.where(np.isnan(x), -1.0, x)                   # the device maps NaN to cell 0
    want = OA.bins2d(xx, y, 0.0, 1.0, G)
    assert np.array_equal(h, want)
    occ = want > 0
    assert st["occupied_bins"] == int(occ.sum()) and st["largest_bin"] == int(want.max())
    assert st["shared_fraction"] * len(x) == pytest.approx(float(want[want > 1].sum()))
    pad = np.pad(occ, 2)
    cov = np.zeros_like(occ)
    for dyy in range(-2, 3):
        for dxx in range(-2, 3):
            cov |= pad[2 + dyy:2 + dyy + G, 2 + dxx:2 + dxx + G]
    assert st["covered_pixels"] == int(cov.sum())
