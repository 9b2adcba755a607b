"""Pins of the oracle's correspondence part (Sec. 10, Table 9): the
first-order condition library against closed-form counts and against the
pure-Python set comprehensions of pyref, and the recovery procedure against
Table 9 (every Sahlqvist landmark recovered, McKinsey unmatched)."""
from math import comb

import numpy as np
import pytest

import golden_fixtures as G
import oracle
from oracle import pyref


def closed_form(name, n):
    return {
        "every frame": 2 ** (n * n),
        "no frame": 0,
        "reflexive": 2 ** (n * n - n),
        "irreflexive": 2 ** (n * n - n),
        "serial": (2 ** n - 1) ** n,
        "symmetric": 2 ** (n * (n + 1) // 2),
        "partially functional": (n + 1) ** n,
        "functional": n ** n,
        "antisymmetric": 2 ** n * 3 ** (n * (n - 1) // 2),
        "asymmetric": 3 ** (n * (n - 1) // 2),
        "empty relation": 1,
        "coreflexive": 2 ** n,
        # choose the looped worlds S; every world's successors lie in S
        "shift reflexive": sum(comb(n, s) * 2 ** (s * (n - 1)) for s in range(n + 1)),
        "transitive": [1, 2, 13, 171, 3994][n],            # OEIS A006905
    }.get(name)


@pytest.mark.parametrize("n", (1, 2, 3, 4))
def test_condition_counts_closed_forms(n):
    for name in oracle.CONDITIONS:
        want = closed_form(name, n)
        if want is not None:
            assert int(oracle.frame_condition(name, n).sum()) == want, (name, n)


@pytest.mark.parametrize("n", (1, 2, 3))
def test_conditions_match_set_comprehensions(n):
    frames = list(pyref.all_frames(n))
    for name in oracle.CONDITIONS:
        got = oracle.frame_condition(name, n)
        want = np.array([pyref.condition(name, n, R) for _, R in frames], np.uint8)
        assert np.array_equal(got, want), (name, n)


def test_inclusions_between_conditions():
    # functional = serial and partially functional; empty implies every
    # universal-free condition's vacuous cases; coreflexive implies symmetric
    for n in (2, 3, 4):
        c = {name: oracle.frame_condition(name, n).astype(bool) for name in oracle.CONDITIONS}
        assert np.array_equal(c["functional"], c["serial"] & c["partially functional"])
        assert not (c["coreflexive"] & ~c["symmetric"]).any()
        assert not (c["reflexive"] & ~c["serial"]).any()
        assert not (c["reflexive"] & ~c["dense"]).any()
        assert not (c["asymmetric"] & ~c["irreflexive"]).any()
        assert np.array_equal(c["symmetric"] & c["transitive"], c["symmetric"] & c["Euclidean"])


# Table 9's landmarks and its McKinsey control, from tests/golden
TABLE9 = [(f, c) for _, f, c in G.table9() if c is not None]
MCKINSEY = [f for _, f, c in G.table9() if c is None][0]


@pytest.mark.parametrize("N", (3, 4))
def test_table9_recovery(N):
    for text, cond in TABLE9:
        assert cond in oracle.recover(text, N), (text, cond)
    assert oracle.recover(MCKINSEY, N) == []          # McKinsey: no match in the library
