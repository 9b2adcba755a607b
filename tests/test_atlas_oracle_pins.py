"""Pins of the oracle's atlas part (Sec. 9): exact failure counts against
closed forms and the pure-Python evaluator, the seriation against a rank-one
matrix whose principal axis is known, A(pi) and the binning on hand-worked
cases."""
import random

import numpy as np
import pytest

import oracle
from oracle import atlas, pyref


def succ_sets(f, n):
    return [{v for v in range(n) if (f >> (w * n + v)) & 1} for w in range(n)]


@pytest.mark.parametrize("n", (1, 2, 3))
def test_closed_forms(n):
    F = 1 << (n * n)
    c, d = atlas.atlas_counts(["T", "F", "p", "[]F", "<>T", "[]p -> p"], n)
    assert list(d) == [n, n, 2 ** n * n, n, n, 2 ** n * n]
    assert (c[0] == 0).all() and (c[1] == n).all() and (c[2] == 2 ** n * n // 2).all()
    for f in range(F):
        s = succ_sets(f, n)
        assert c[3, f] == sum(1 for w in range(n) if s[w])                       # []F fails where w has a successor
        assert c[4, f] == sum(1 for w in range(n) if not s[w])                   # <>T fails at dead ends
        # []p -> p fails at w iff w has no loop, p is false at w and true on succ(w)
        assert c[5, f] == sum(2 ** (n - 1 - len(s[w])) for w in range(n) if w not in s[w])


def test_brute_force_two_worlds():
    rng = random.Random(3)
    atoms = ["p", "q", "T", "F"]

    def rand(d):
        if d == 0 or rng.random() < 0.3:
            return rng.choice(atoms)
        op = rng.choice(["~", "[]", "<>", "&", "|", "->"])
        if op in ("~", "[]", "<>"):
            return op + "(" + rand(d - 1) + ")"
        return "(" + rand(d - 1) + op + rand(d - 1) + ")"

    texts = [rand(4) for _ in range(12)]
    c, d = atlas.atlas_counts(texts, 2)
    for i, t in enumerate(texts):
        tree = pyref.parse(t)
        k = pyref.nvars(tree)
        assert d[i] == (1 << (2 * k)) * 2
        for f, R in pyref.all_frames(2):
            want = sum(1 for _, V in pyref.all_valuations(k, 2) for w in range(2) if not pyref.sat(R, V, w, tree))
            assert c[i, f] == want, (t, f)


def test_seriation_rank_one():
    rng = np.random.default_rng(0)
    a = rng.random(40)
    b = rng.random(25) - 0.3
    col, row, v, u = atlas.seriation(np.outer(a, b))
    bn = b / np.linalg.norm(b)
    if bn[np.argmax(np.abs(bn))] < 0:
        bn = -bn
    assert np.allclose(v, bn, atol=1e-12)
    assert list(col) == list(np.argsort(bn, kind="stable"))
    assert list(row) == list(np.argsort(u, kind="stable"))


def test_adjacent_variation_and_bins():
    D = np.array([[0.0, 1.0, 0.0], [0.5, 0.5, 1.0]])
    assert atlas.adjacent_variation(D, [0, 1, 2]) == pytest.approx((1 + 1 + 0 + 0.5) / 4)
    assert atlas.adjacent_variation(D, [0, 2, 1]) == pytest.approx((0 + 1 + 0.5 + 0.5) / 4)
    h = atlas.bins2d([0.0, 0.24, 0.25, 0.999, 1.5, -1], [0.0, 0.0, 0.5, 0.999, 0.1, 0.9], 0.0, 1.0, 4)
    assert h[0, 0] == 2 and h[2, 1] == 1 and h[3, 3] == 1 and h[0, 3] == 1 and h[3, 0] == 1 and h.sum() == 6
