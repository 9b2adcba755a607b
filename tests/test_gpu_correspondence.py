"""GPU parity of the correspondence path (Sec. 10, Table 9) against the CPU
oracle: per-frame validity bitmaps (mk_frame_validity), the condition
library's extensions (mk_frame_conditions), mismatch counts
(mk_bitmap_mismatch), and the recovery procedure end to end."""
import random

import numpy as np
import pytest

import golden_fixtures as G
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


def E():
    from paper_2606_15437_gb300 import engine
    return engine


def packed(u8):
    """Pack a 0/1 array over frames into little-endian uint32 words."""
    b = np.packbits(u8.astype(np.uint8), bitorder="little")
    b = np.concatenate([b, np.zeros((-len(b)) % 4, np.uint8)])
    return b.view(np.uint32)


def _formulas(seed, count, kmax):
    rng = random.Random(seed)
    out = ["[]p -> p", "p & ~p", "p | ~p", "<>T", "[]F", "[]p -> [][]p", "[]<>p -> <>[]p"]
    while len(out) < count:
        k = rng.randint(0, kmax)
        L = rng.randint(3, 14)
        out.append(W.random_formula(rng, L, rng.randint(1, min(4, L - 1)), k))
    return out


@pytest.mark.parametrize("N", (3, 4))
def test_validity_bitmaps_match_oracle(N):
    texts = _formulas(N, 60, 3 if N == 3 else 2)
    cj = E().Correspondence(texts, N)
    v = cj.validity().cpu().numpy().view(np.uint32)
    cj.check_status()
    for i, t in enumerate(texts):
        for n in range(1, N + 1):
            want = packed(oracle.frame_valid_all(t, n))
            got = v[i, cj.offs[n - 1]:cj.offs[n]]
            assert np.array_equal(got, want), (t, n)


def test_validity_five_worlds_sample():
    texts = ["[]p -> p", "<>p -> []<>p", "[][]p -> []p", "<>T -> [](<>T)", "p -> []p"]
    cj = E().Correspondence(texts, 5)
    v = cj.validity(sizes=[5]).cpu().numpy().view(np.uint32)
    cj.check_status()
    for i, t in enumerate(texts):
        assert np.array_equal(v[i, cj.offs[4]:cj.offs[5]], packed(oracle.frame_valid_all(t, 5))), t


@pytest.mark.parametrize("n", (1, 2, 3, 4))
def test_condition_bitmaps_match_oracle(n):
    cj = E().Correspondence(["T"], n)
    c = cj.conditions().cpu().numpy().view(np.uint32)
    for ci, name in enumerate(mk.CONDITION_NAMES):
        assert name == oracle.CONDITIONS[ci]
        want = packed(oracle.frame_condition(name, n))
        assert np.array_equal(c[ci, cj.offs[n - 1]:cj.offs[n]], want), (name, n)


def test_condition_bitmaps_five_worlds():
    cj = E().Correspondence(["T"], 5)
    c = cj.conditions().cpu().numpy().view(np.uint32)
    for name in ("reflexive", "serial", "symmetric", "partially functional", "coreflexive", "shift reflexive"):
        ci = mk.CONDITION_NAMES.index(name)
        assert np.array_equal(c[ci, cj.offs[4]:cj.offs[5]], packed(oracle.frame_condition(name, 5))), name


def test_mismatch_counts():
    rng = np.random.default_rng(1)
    a = rng.integers(0, 2 ** 32, size=(7, 300), dtype=np.uint64).astype(np.uint32)
    b = rng.integers(0, 2 ** 32, size=(5, 310), dtype=np.uint64).astype(np.uint32)
    conj = np.array([[0, 0], [1, 3], [4, 2], [2, 5], [-1, 0]], np.int32)
    da = torch.from_numpy(a.view(np.int32)).cuda()
    db = torch.from_numpy(b.view(np.int32)).cuda()
    dc = torch.from_numpy(conj.reshape(-1)).cuda()
    out = torch.empty((7, 5), dtype=torch.int32, device="cuda")
    words = 290
    mk.bitmap_mismatch_raw(da.data_ptr(), 7, 300, db.data_ptr(), 5, 310, dc.data_ptr(), 5, words, out.data_ptr(), 0)
    got = out.cpu().numpy().view(np.uint32)
    for i in range(7):
        for j, (c1, c2) in enumerate(conj):
            if c1 < 0 or c2 >= 5:
                assert got[i, j] == 0xFFFFFFFF
                continue
            x = a[i, :words] ^ (b[c1, :words] & b[c2, :words])
            assert got[i, j] == sum(bin(int(w)).count("1") for w in x)


# Table 9's landmarks and its McKinsey control, from tests/golden
TABLE9 = [(f, c) for _, f, c in G.table9() if c is not None]
MCKINSEY = [f for _, f, c in G.table9() if c is None][0]


def test_table9_recovery_and_confirmation():
    texts = [t for t, _ in TABLE9] + [MCKINSEY, "([]p -> p) & ([]p -> [][]p)", "p | ~p", "p"]
    rows, stats = E().recover_correspondents(texts, N=4, confirm_n=5)
    for (t, cond), r in zip(TABLE9, rows):
        assert cond in r["matches"] and r["confirmed"], (t, r)
    assert rows[8]["matches"] == []                                     # McKinsey: none in the library
    assert "reflexive & transitive" in rows[9]["matches"] and rows[9]["confirmed"]
    assert rows[10]["trivial"] and "every frame" in rows[10]["matches"]
    assert rows[11]["trivial"] and "no frame" in rows[11]["matches"]
    assert stats["unmatched"] == 1 and stats["trivial"] == 2


def test_recovery_agrees_with_oracle_on_corpus_sample():
    rng = random.Random(7)
    texts = rng.sample(W.census5_formulas(), 40)
    texts = [t for t in texts if oracle.nvars(t) <= 2][:25]
    rows, _ = E().recover_correspondents(texts, N=3, confirm_n=None)
    for t, r in zip(texts, rows):
        singles = [m for m in r["matches"] if " & " not in m]
        assert singles == oracle.recover(t, 3), t
