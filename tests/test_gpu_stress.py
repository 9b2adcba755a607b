"""GPU parity of the large-frame path (Sec. 7 stress templates, Table 2
adversarial generators) against the CPU oracle: relations drawn on the
device, their bit-sliced words, and mk_stress_separate's first splits and
split counts, bit-exact, at sizes that span several CTAs and ragged tails,
every n from 1 to 16, and valuation ranges cut over grid.z."""
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


def E():
    from paper_2606_15437_gb300 import engine
    return engine


def slice_words(succ, n):
    """Bit-sliced words of a [count, 16] successor-mask array, as
    mk_relation_words lays them out (numpy, independent of the library)."""
    count = len(succ)
    nb = (count + 31) // 32
    out = np.zeros((nb, n, n), np.uint32)
    for i in range(count):
        b, l = divmod(i, 32)
        for w in range(n):
            for v in range(n):
                if (int(succ[i, w]) >> v) & 1:
                    out[b, w, v] |= np.uint32(1 << l)
    return out.reshape(-1)


@pytest.mark.parametrize("gen", mk.GENERATORS)
@pytest.mark.parametrize("n", (2, 6, 9, 16))
def test_generated_relations_match_oracle(gen, n):
    count, first = 1000, 5
    words = torch.zeros(mk.relation_words(n, count), dtype=torch.int32, device="cuda")
    succ = torch.zeros((count, 16), dtype=torch.int32, device="cuda")
    mk.generate_relations_raw(gen, 31, n, first, count, words.data_ptr(), succ.data_ptr(), 0)
    torch.cuda.synchronize()
    want = oracle.stress_relations(gen, 31, n, first, count)
    got = succ.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, want)
    assert np.array_equal(words.cpu().numpy().view(np.uint32), slice_words(want, n))


def test_pack_relations_masks_extra_bits():
    rng = np.random.default_rng(3)
    for n in (1, 5, 13, 16):
        raw = rng.integers(0, 1 << 32, size=(77, 16), dtype=np.uint64).astype(np.uint32)
        rels = E().RelationSet.from_succ(raw, n)
        torch.cuda.synchronize()
        masked = raw & np.uint32((1 << n) - 1)
        masked[:, n:] = 0
        assert np.array_equal(rels.d_words.cpu().numpy().view(np.uint32), slice_words(masked, n))


def _pairs(seed, count, k_max, n):
    rng = random.Random(seed)
    out = []
    for i in range(count):
        k = rng.randint(0, k_max)
        a = W.random_formula(rng, rng.randint(3, 16), rng.randint(1, 5), k)
        b = W.random_formula(rng, rng.randint(3, 16), rng.randint(1, 5), k) if i % 3 else W.alpha(2) if k == 0 \
            else a.replace("p0", "~p0", 1) if "p0" in a else "p0"
        out.append((a, b))
    out += [("<>" * m + "T", "<>" * (m + 1) + "T") for m in range(1, min(n, 6))]
    out += [(W.alpha(2), W.alpha(3)), ("T", "T")]
    return out


def _oracle(pairs, n, succ):
    keys, cnts = [], []
    for a, b in pairs:
        r = oracle.stress_pair(a, b, n, succ)
        keys.append(mk.NO_KEY if r["split"] is None else (r["split"][0] << 20) | (r["split"][1] << 4) | r["split"][2])
        cnts.append(r["nsplit"])
    return np.array(keys, np.uint64), np.array(cnts)


@pytest.mark.parametrize("n,gen,count,k_max", [(1, "er", 77, 2), (3, "er", 700, 2), (6, "scc", 3000, 1),
                                               (7, "deadend", 1500, 1), (9, "flip", 600, 1), (11, "scc", 700, 1),
                                               (12, "backedge", 100, 1), (12, "permscc", 2500, 0),
                                               (16, "er", 5000, 0), (16, "flip", 70, 1)])
def test_first_split_and_counts_match_oracle(n, gen, count, k_max):
    pairs = _pairs(n * 101 + count, 24, k_max, n)
    job = E().StressJob(pairs)
    idx = job.eligible(n)
    assert len(idx) == len(pairs)
    rels = E().RelationSet.generated(gen, 8, n, 0, count)
    want_k, want_c = _oracle(pairs, n, oracle.stress_relations(gen, 8, n, 0, count))
    keys, cnt = job.run(rels, count_splits=True)
    assert np.array_equal(keys, want_k)
    assert np.array_equal(cnt, want_c)
    keys1, _ = job.run(rels, count_splits=False, tile=5)
    assert np.array_equal(keys1, want_k)
    for i, key in enumerate(keys):
        if key != mk.NO_KEY:
            assert job.certify(i, int(key), rels)


def test_chunks_with_index_base_merge_to_one_scan():
    n, count = 16, 5000
    pairs = _pairs(5, 30, 0, n)
    job = E().StressJob(pairs)
    whole = E().RelationSet.generated("er", 2, n, 0, count)
    want, _ = job.run(whole)
    d_key = torch.full((len(pairs),), -1, dtype=torch.int64, device="cuda")
    for lo, hi in ((2500, 5000), (0, 2500)):          # later chunk first: the minimum still wins
        part = E().RelationSet.generated("er", 2, n, lo, hi - lo)
        cfg = mk.stress_cfg(n, hi - lo, index_base=lo)
        mk.stress_separate_raw(job.d_pa.data_ptr(), job.d_pb.data_ptr(), len(pairs), part.d_words.data_ptr(),
                               cfg, d_key.data_ptr(), 0, job.d_status.data_ptr(), 0)
    torch.cuda.synchronize()
    job.check_status()
    assert np.array_equal(d_key.cpu().numpy().view(np.uint64), want)


@pytest.mark.parametrize("n", (10, 12, 16))
def test_one_variable_pairs_on_templates(n):
    # 2^n valuations over two relation blocks: the valuation range is cut
    # over grid.z, the keys merge to the oracle's least (relation, x, w)
    rng = random.Random(n)
    pairs = [("p", "<>p"), ("[]p", "[][]p"), ("[]<>p", "<>[]p"), ("<>(p->p)", "<><>(p->p)")]
    # splits that need high valuation bits: p at the path's last worlds
    pairs += [("[]F", "[]F & ~p"), ("<>[]F", "<>[]F & ~p"), ("p & <>p", "F")]
    pairs += [(W.random_formula(rng, 9, 3, 1), W.random_formula(rng, 9, 3, 1)) for _ in range(4)]
    rels_n = 39 if n <= 12 else 3
    tpl = [oracle.template(t, n) for t in range(rels_n)]
    job = E().StressJob(pairs)
    rels = E().RelationSet.from_succ(tpl, n)
    keys, _ = job.run(rels)
    want, _ = _oracle(pairs, n, np.array([t + [0] * (16 - n) for t in tpl], np.uint32))
    assert np.array_equal(keys, want)


def test_limit_and_empty_cases():
    job = E().StressJob([("p0 & p1", "p1 & p0"), ("<>T", "<><>T")])
    rels = E().RelationSet.templates(9)
    job.d_status.zero_()
    d_key, _ = job.launch(rels)
    torch.cuda.synchronize()
    st = int(job.d_status.item())
    assert st & 2                                       # MK_ST_LIMIT: k*n = 18 > 16
    k = d_key.cpu().numpy().view(np.uint64)
    assert k[0] == mk.NO_KEY and mk.decode_stress_key(int(k[1]))[0] == 0   # the path splits <>T / <><>T
    # zero relations and zero pairs launch nothing and succeed
    cfg = mk.stress_cfg(9, 0)
    mk.stress_separate_raw(job.d_pa.data_ptr(), job.d_pb.data_ptr(), 2, rels.d_words.data_ptr(), cfg,
                           d_key.data_ptr(), 0, job.d_status.data_ptr(), 0)
    mk.stress_separate_raw(0, 0, 0, 0, mk.stress_cfg(9, 10), 0, 0, job.d_status.data_ptr(), 0)
    torch.cuda.synchronize()


def test_context_word_mining_recovers_the_paper_hits():
    rows = E().mine_context_words()
    top = [(r["phi"], r["psi"]) for r in rows[:2]]
    # the top exact five-indistinguishable hits are the path-depth families
    assert top == [("<><><><><>T", "<><><><><><>T"), ("[][][][][]F", "[][][][][][]F")]
    for r in rows[:2]:
        assert r["a"] == 5 and r["template"][0] == 6
    # alpha_2 / alpha_3 is recovered with the six-world path witness
    (al,) = [r for r in rows if (r["phi"], r["psi"]) == (W.alpha(2), W.alpha(3))]
    assert al["a"] == 5 and al["template"][:2] == (6, 0)
    # the prefix agrees with the oracle through four worlds on a sample
    rng = random.Random(0)
    for r in rng.sample(rows, 40):
        want = None
        for n in range(1, 5):
            if oracle.pair_layer(r["phi"], r["psi"], n)["split"]:
                want = n
                break
        assert (r["a"] + 1 if r["a"] < 4 else None) == want, r
    # template witnesses are the oracle's first template splits
    for r in [r for r in rows if r["template"] is not None][:12]:
        n, s, x, w = r["template"]
        tpl = np.array([oracle.template(t, n) + [0] * (16 - n) for t in range(39)], np.uint32)
        got = oracle.stress_pair(r["phi"], r["psi"], n, tpl)["split"]
        assert got == (s, x, w)
        for m in range(6, n):
            tpl = np.array([oracle.template(t, m) + [0] * (16 - m) for t in range(39)], np.uint32)
            k = max(oracle.nvars(r["phi"]), oracle.nvars(r["psi"]))
            if k * m <= 16:
                assert oracle.stress_pair(r["phi"], r["psi"], m, tpl)["split"] is None
