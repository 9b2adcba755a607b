"""Pins of the oracle's large-frame part (Sec. 7, Table 2): the stress
templates, the adversarial relation generators and the separation scan over
explicit relations, each checked against what the construction's name and
the mathematics fix -- graph structure computed by networkx / scipy, closed
forms of Lemma 2 on paths, the sampled family at n <= 8, and brute force by
the pure-Python evaluator.
"""
import random

import numpy as np
import pytest

import oracle
from oracle import pyref

nx = pytest.importorskip("networkx")
csgraph = pytest.importorskip("scipy.sparse.csgraph")


def graph(succ, n):
    g = nx.DiGraph()
    g.add_nodes_from(range(n))
    g.add_edges_from((w, v) for w in range(n) for v in range(n) if (succ[w] >> v) & 1)
    return g


def edges(succ, n):
    return {(w, v) for w in range(n) for v in range(n) if (succ[w] >> v) & 1}


def sccs(succ, n):
    m = np.zeros((n, n), np.int8)
    for w, v in edges(succ, n):
        m[w, v] = 1
    k, lab = csgraph.connected_components(m, directed=True, connection="strong")
    return k, lab


SIZES = (6, 7, 10, 13, 16)


@pytest.mark.parametrize("n", SIZES)
def test_templates_have_their_named_shape(n):
    T = {i: graph(oracle.template(i, n), n) for i in range(oracle.NUM_TEMPLATES)}
    path = nx.path_graph(n, create_using=nx.DiGraph)
    cyc = nx.cycle_graph(n, create_using=nx.DiGraph)
    assert nx.utils.graphs_equal(T[0], path)
    assert nx.utils.graphs_equal(T[1], path.reverse())
    assert set(T[2].edges) == set(path.edges) | {(w, w) for w in range(n)}
    assert set(T[3].edges) == set(path.edges) | {(n - 1, n - 1)}
    assert set(T[4].edges) == set(path.edges) | {(0, 0)}
    assert set(T[5].edges) == set(nx.transitive_closure_dag(path).edges)
    assert set(T[6].edges) == set(T[5].edges) | {(w, w) for w in range(n)}
    assert nx.utils.graphs_equal(T[7], cyc)
    assert nx.utils.graphs_equal(T[8], cyc.reverse())
    assert set(T[9].edges) == set(cyc.edges) | {(w, w) for w in range(n)}
    assert set(T[10].edges) == set(cyc.edges) | set(cyc.reverse().edges)
    assert set(T[11].edges) == set(path.edges) | set(path.reverse().edges)
    star = nx.star_graph(n - 1, create_using=nx.DiGraph)   # hub 0 -> leaves
    assert set(T[12].edges) == set(star.edges)
    assert set(T[13].edges) == set(star.reverse().edges)
    assert set(T[14].edges) == set(star.edges) | set(star.reverse().edges)
    assert set(T[15].edges) == set(star.edges) | {(w, w) for w in range(n)}
    for i in (16, 17, 18, 19):   # forks: an arborescence from 0 with exactly two leaves
        g = T[i]
        assert nx.is_arborescence(g) and g.out_degree(0) == 2
        assert sum(1 for v in g if g.out_degree(v) == 0) == 2
    assert nx.is_arborescence(T[21])
    assert all(T[21].out_degree(w) <= 2 for w in range(n))
    assert nx.utils.graphs_equal(T[22], T[21].reverse())
    assert T[23].number_of_edges() == n * n
    assert T[24].number_of_edges() == n * (n - 1) and nx.number_of_selfloops(T[24]) == 0
    assert set(T[25].edges) == {(w, w) for w in range(n)}
    assert T[26].number_of_edges() == 0
    # lasso: a tail into one cycle of n - n//2 worlds
    k, lab = sccs(oracle.template(27, n), n)
    assert sorted(np.bincount(lab))[-1] == n - n // 2 and len(list(nx.simple_cycles(T[27]))) == 1
    # two cycles joined by one bridge: two strongly connected blocks
    k, lab = sccs(oracle.template(28, n), n)
    assert k == 2 and sorted(np.bincount(lab)) == sorted([n // 2, n - n // 2])
    dens = [T[i].number_of_edges() / n ** 2 for i in range(29, 35)]
    assert all(d < 0.3 for d in dens[:3]) and all(d > 0.7 for d in dens[3:])
    assert nx.is_arborescence(T[35]) and nx.is_directed_acyclic_graph(T[36])
    assert set(T[37].edges) == set(path.edges) | {(w, w) for w in range(1, n, 2)}
    assert nx.utils.graphs_equal(T[38], T[5].reverse())
    # 39 distinct templates at every size >= 6
    assert len({tuple(oracle.template(i, n)) for i in range(oracle.NUM_TEMPLATES)}) == 39


def test_erdos_renyi_is_the_sampled_family_up_to_eight_worlds():
    for n in (1, 3, 6, 7, 8):
        for s in (0, 1, 5, 999, 123456):
            m = oracle.sample_frame(11, n, s)
            succ = oracle.stress_relation("er", 11, n, s)
            assert succ == [(m >> (w * n)) & ((1 << n) - 1) for w in range(n)]


@pytest.mark.parametrize("n", (10, 16))
def test_erdos_renyi_density(n):
    # p_s = t/256 with t uniform on [26, 128]: mean edge density 77/256
    a = oracle.stress_relations("er", 3, n, 0, 1500)
    d = np.array([sum(bin(int(x)).count("1") for x in row) for row in a]) / n ** 2
    assert abs(d.mean() - 77 / 256) < 0.01
    assert d.min() > 0.02 and d.max() < 0.65 and d.std() > 0.08


@pytest.mark.parametrize("n", (6, 9, 16))
def test_scc_bottleneck_structure(n):
    for s in range(60):
        succ = oracle.stress_relation("scc", 5, n, s)
        k, lab = sccs(succ, n)
        assert k == 2, (n, s, succ)
        blk0 = {w for w in range(n) if lab[w] == lab[0]}
        a = len(blk0)
        assert blk0 == set(range(a))                   # a prefix block, then the rest
        cross = [(w, v) for (w, v) in edges(succ, n) if (w in blk0) != (v in blk0)]
        assert cross == [(a - 1, a)]                   # one bridge edge, first block -> second


@pytest.mark.parametrize("n", (6, 11, 16))
def test_permuted_bottleneck_structure(n):
    prefix = 0
    for s in range(60):
        succ = oracle.stress_relation("permscc", 5, n, s)
        k, lab = sccs(succ, n)
        assert k == 2
        cross = [(w, v) for (w, v) in edges(succ, n) if lab[w] != lab[v]]
        assert len(cross) == 1
        blk0 = {w for w in range(n) if lab[w] == lab[cross[0][0]]}
        prefix += blk0 == set(range(len(blk0)))
    assert prefix < 20                                  # the labels really are permuted


@pytest.mark.parametrize("n", (6, 16))
def test_dead_end_and_back_edge_structure(n):
    for s in range(60):
        succ = oracle.stress_relation("deadend", 2, n, s)
        assert 1 <= sum(1 for w in range(n) if succ[w] == 0)
        succ = oracle.stress_relation("backedge", 2, n, s)
        e = edges(succ, n)
        path = {(w, w + 1) for w in range(n - 1)}
        assert path <= e
        extra = e - path
        assert 1 <= len(extra) <= 4 and all(w >= v for (w, v) in extra)


@pytest.mark.parametrize("n", (6, 12))
def test_edge_flip_is_near_a_template(n):
    temps = [edges(oracle.template(i, n), n) for i in range(oracle.NUM_TEMPLATES)]
    dist = []
    for s in range(80):
        e = edges(oracle.stress_relation("flip", 9, n, s), n)
        dist.append(min(len(e ^ t) for t in temps))
    assert max(dist) <= 4 and sum(1 for d in dist if d > 0) > 60


def _succs(rels):
    a = np.zeros((len(rels), 16), np.uint32)
    for i, r in enumerate(rels):
        a[i, :len(r)] = r
    return a


@pytest.mark.parametrize("n", (6, 9, 16))
def test_path_depth_pairs_split_on_paths(n):
    # <>^m T holds at world w of the n-world path iff n-1-w >= m; on a cycle
    # every world has paths of every length, so the pair never splits there
    path, cyc = oracle.template(0, n), oracle.template(7, n)
    for m in range(1, n):
        phi, psi = "<>" * m + "T", "<>" * (m + 1) + "T"
        r = oracle.stress_pair(phi, psi, n, _succs([cyc, path]))
        assert r["split"] == (1, 0, n - 1 - m) and r["nsplit"] == 1
        phi, psi = "[]" * m + "F", "[]" * (m + 1) + "F"
        r = oracle.stress_pair(phi, psi, n, _succs([cyc, path]))
        assert r["split"] == (1, 0, n - 1 - m)


@pytest.mark.parametrize("n", (6, 8, 11, 16))
def test_alpha_family_on_paths_lemma2(n):
    # Lemma 2: on a directed path, alpha_m = ([]<>)^m T is false exactly at
    # the worlds with r in {1, 3, ..., 2m-1} remaining edges
    path = oracle.template(0, n)
    for m in (1, 2, 3):
        a, b = "[]<>" * m + "T", "[]<>" * (m + 1) + "T"
        fa = {w for w in range(n) if (n - 1 - w) in range(1, 2 * m, 2)}
        fb = {w for w in range(n) if (n - 1 - w) in range(1, 2 * m + 2, 2)}
        diff = sorted(fa ^ fb)
        r = oracle.stress_pair(a, b, n, _succs([path]))
        if diff:
            assert r["split"] == (0, 0, diff[0])
        else:
            assert r["split"] is None


def test_brute_force_on_generated_relations():
    rng = random.Random(4)
    atoms = ["p", "T", "F"]

    def rand(d):
        if d == 0 or rng.random() < 0.25:
            return rng.choice(atoms)
        op = rng.choice(["~", "[]", "<>", "&", "|", "->"])
        if op in ("~", "[]", "<>"):
            return op + "(" + rand(d - 1) + ")"
        return "(" + rand(d - 1) + op + rand(d - 1) + ")"

    for n, gen in ((6, "er"), (6, "scc"), (7, "backedge"), (6, "deadend")):
        rels = [oracle.stress_relation(gen, 21, n, s) for s in range(4)]
        for _ in range(5):
            phi, psi = rand(4), rand(4)
            want = None
            cnt = 0
            k = max(pyref.nvars(pyref.parse(phi)), pyref.nvars(pyref.parse(psi)))
            for s, succ in enumerate(rels):
                R = edges(succ, n)
                hit = None
                for x, V in pyref.all_valuations(k, n):
                    for w in range(n):
                        if pyref.sat(R, V, w, pyref.parse(phi)) != pyref.sat(R, V, w, pyref.parse(psi)):
                            hit = (s, x, w)
                            break
                    if hit:
                        break
                if hit:
                    cnt += 1
                    want = want or hit
            r = oracle.stress_pair(phi, psi, n, _succs(rels))
            assert r["split"] == want and r["nsplit"] == cnt, (phi, psi, n, gen)
