"""CPU tests of libmk's host side: the ABI exports, mk_compile, mk_certify.

No GPU and no compute kernel is called here.  The compiled programs are
checked by interpreting their instruction set (as mk.h defines it) in plain
Python over explicit truth sets and comparing with the oracle on small
frames, so register allocation and constant folding are covered on CPU.
"""
import os
import random
import re

import numpy as np
import pytest

import oracle
from oracle import pyref
from paper_2606_15437_gb300 import build as mkbuild
from paper_2606_15437_gb300 import mk
from paper_2606_15437_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    mkbuild.build()


def test_exports_every_declared_symbol():
    header = open(os.path.join(ROOT, "include", "mk.h")).read()
    declared = set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(mk_\w+)\s*\(", header, re.M))
    assert {"mk_compile", "mk_census", "mk_separate", "mk_certify"} <= declared
    L = mk.lib()
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert set(mk.declared_symbols()) <= declared
    assert mk.lib().mk_version() == 1


def test_struct_sizes():
    import ctypes
    assert ctypes.sizeof(mk.mk_program) == 104
    assert ctypes.sizeof(mk.mk_census_cfg) == 48
    assert ctypes.sizeof(mk.mk_result) == 24


# ------------------------------------------------------ program semantics

def run_program(prog, n, R, V):
    """Interpret a compiled program (mk.h's accumulator machine) over
    explicit truth sets (sets of worlds)."""
    full = set(range(n))
    succ = [{v for v in range(n) if R[w][v]} for w in range(n)]
    atom = [{w for w in range(n) if V[i][w]} for i in range(mk.MK_MAX_VARS)]
    A, st = set(), [None] * mk.MK_MAX_STACK
    for c in list(prog.code)[:prog.n_instr]:
        op, arg = c & 31, c >> 5
        if op == 0:
            A = set(atom[arg])
        elif op == 1:
            A = set(full)
        elif op == 2:
            A = set()
        elif op == 3:
            A = full - A
        elif op == 4:
            A = {w for w in full if succ[w] <= A}
        elif op == 5:
            A = {w for w in full if succ[w] & A}
        elif op == 6:
            st[arg] = set(A)
        elif 7 <= op <= 11:
            S = st[arg]
            A = [S & A, S | A, (full - S) | A, (full - A) | S, full - (S ^ A)][op - 7]
        elif 12 <= op <= 15:
            a = atom[arg]
            A = [A & a, A | a, (full - A) | a, (full - a) | A][op - 12]
        elif 16 <= op <= 19:
            na = full - atom[arg]
            A = [na, A & na, A | na, (full - A) | na][op - 16]
        else:
            t = atom[arg] if op in (20, 21) else full - atom[arg]
            if op in (20, 22):
                A = {w for w in full if succ[w] <= t}
            else:
                A = {w for w in full if succ[w] & t}
    return A


def _texts(seed, count, maxlen=14):
    rng = random.Random(seed)
    return [W.random_formula(rng, rng.randint(1, maxlen), rng.randint(0, 4), rng.randint(0, 3))
            for _ in range(count)]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_compiled_programs_match_oracle(seed):
    rng = np.random.default_rng(seed)
    for text in _texts(seed, 60) + list(W.AXIOMS) + [W.alpha(3), "T", "F", "~T", "p <-> []p"]:
        prog = mk.compile(text)
        k = prog.nvars
        for _ in range(6):
            n = int(rng.integers(1, 5))
            R = rng.integers(0, 2, (n, n)).astype(np.uint8)
            V = rng.integers(0, 2, (4, n)).astype(np.uint8)
            got = run_program(prog, n, R, V)
            want = oracle.eval_model(text, R, V)
            assert got == {w for w in range(n) if want[w]}, text
        assert prog.nvars == oracle.nvars(text)
        assert prog.nodes == W.nodes(text) or "<->" in text


def test_compile_iff_is_biconditional():
    prog = mk.compile_iff(W.alpha(2), W.alpha(3))
    R = np.zeros((6, 6), np.uint8)
    for w in range(5):
        R[w, w + 1] = 1
    got = run_program(prog, 6, R, np.zeros((4, 6), np.uint8))
    a, b = oracle.eval_model(W.alpha(2), R), oracle.eval_model(W.alpha(3), R)
    assert got == {w for w in range(6) if a[w] == b[w]}


def test_register_bound_for_64_nodes():
    rng = random.Random(7)
    worst = 0
    for _ in range(500):
        t = W.random_formula(rng, 64, rng.randint(1, 8), rng.randint(0, 4))
        p = mk.compile(t)
        worst = max(worst, p.depth)
        assert p.depth <= mk.MK_MAX_STACK and p.n_instr <= mk.MK_MAX_CODE
    # a complete binary tree of 32 atoms (63 nodes) needs the deepest stack
    t = "p"
    for d in range(5):
        t = "(%s & %s)" % (t, t.replace("p", "q"))
    assert mk.compile(t).depth == mk.MK_MAX_STACK


@pytest.mark.parametrize("bad,code", [("p &", -1), ("(p", -1), ("p4", -3), ("x", -1), ("p & & q", -1),
                                      ("[]" * 70 + "p", -2)])
def test_compile_errors(bad, code):
    with pytest.raises(mk.MkError) as e:
        mk.compile(bad)
    assert e.value.code == code


def test_precedence_and_associativity():
    # -> is right associative and binds loosest; & binds tighter than |
    for a, b in [("p -> q -> r", "p -> (q -> r)"), ("p | q & r", "p | (q & r)"),
                 ("~p & q", "(~p) & q"), ("[]p -> q", "([]p) -> q"), ("p & q -> r | s", "(p & q) -> (r | s)")]:
        pa, pb = mk.compile(a), mk.compile(b)
        for f in range(64):
            R = oracle.frame_matrix(f % 16, 2)
            V = np.array([[(f >> (i * 2 + w)) & 1 for w in range(2)] for i in range(4)], np.uint8)
            assert run_program(pa, 2, R, V) == run_program(pb, 2, R, V), (a, b)


# ------------------------------------------------------------ certify

def test_certify_paper_certificate():
    succ = [2, 4, 8, 16, 32, 0]
    assert mk.certify(W.alpha(3), 6, succ, world=0) == 1       # alpha_3 false at w0
    assert mk.certify(W.alpha(2), 6, succ, world=0) == 0       # alpha_2 true there
    assert mk.certify(W.alpha(2), 6, succ, world=0, psi=W.alpha(3)) == 1
    assert mk.certify(W.alpha(2), 6, succ, world=1, psi=W.alpha(3)) == 0


def test_certify_checks_class():
    # T axiom countermodel on the one-world irreflexive frame is valid in K
    # but the frame is not in T
    assert mk.certify("[]p -> p", 1, [0], [0], 0, cls="K") == 1
    assert mk.certify("[]p -> p", 1, [0], [0], 0, cls="T") == 0
    # a non-transitive reflexive frame is not S4
    assert mk.certify("[]p -> [][]p", 3, [0b011, 0b110, 0b100], [0b011], 0, cls="T") == 1
    assert mk.certify("[]p -> [][]p", 3, [0b011, 0b110, 0b100], [0b011], 0, cls="S4") == 0


def test_certify_rejects_malformed():
    with pytest.raises(mk.MkError):
        mk.certify("p &", 2, [0, 0])
    with pytest.raises(mk.MkError):
        mk.certify("p", 2, [4, 0])          # successor outside the frame
    with pytest.raises(mk.MkError):
        mk.certify("p", 2, [0, 0], world=3)


def test_certify_agrees_with_oracle_on_random_models():
    rng = np.random.default_rng(3)
    for text in _texts(9, 80):
        n = int(rng.integers(1, 6))
        R = rng.integers(0, 2, (n, n)).astype(np.uint8)
        V = rng.integers(0, 2, (4, n)).astype(np.uint8)
        succ = [int(sum(int(R[w, v]) << v for v in range(n))) for w in range(n)]
        val = [int(sum(int(V[i, w]) << w for w in range(n))) for i in range(4)]
        truth = oracle.eval_model(text, R, V)
        for w in range(n):
            assert mk.certify(text, n, succ, val, w) == (0 if truth[w] else 1), text


def test_certify_long_path_lemma8():
    for m in (1, 2, 3, 5, 10):
        L = 2 * m + 2
        succ = [1 << (w + 1) for w in range(L - 1)] + [0]
        assert mk.certify(W.alpha(m), L, succ, world=0, psi=W.alpha(m + 1)) == 1


def test_sample_relation_matches_oracle_generator():
    for n in (7, 8):
        for s in (0, 1, 2, 1000, 123456789):
            assert mk.sample_relation(42, n, s) == oracle.sample_frame(42, n, s)


def test_class_frames():
    assert [mk.class_frames("S4", n) for n in range(1, 7)] == [1, 4, 29, 355, 6942, 209527]
    assert [mk.class_frames("S5", n) for n in range(1, 7)] == [1, 2, 5, 15, 52, 203]
    assert mk.class_frames("T", 5) == 2 ** 20 and mk.class_frames("K", 6) == 2 ** 36


def test_witness_cert_decoding():
    prog = mk.compile("[]p -> p")
    key = (0 << 27) | (0 << 3) | 0
    c = mk.witness_cert(prog, "[]p -> p", "K", 1, 0, None, key)
    assert c.n == 1 and c.succ[0] == 0 and c.val[0] == 0 and mk.certify_struct(c) == 1


def test_valuation_split_plan():
    """Host planning of the valuation split (no GPU calls): a one-formula
    layer of 32 frame words is far below a full grid, so it splits and needs
    a 32-word frame bitmap and a tile counter after the lists, but no extra
    launch; a layer forced unsplit, or whose formulas have too few
    valuations to share out, needs neither."""
    cfg_auto = mk.census_cfg(("K",), 4, 4, 0, 0, 0, 1024, None, max_depth=4)
    cfg_one = mk.census_cfg(("K",), 4, 4, 0, 0, 0, 1024, None, max_depth=4, vsplit=1)
    lists = mk.census_workspace_size(cfg_one, 1)
    assert lists > 0
    assert mk.census_workspace_size(cfg_auto, 1) == -(-lists // 256) * 256 + 256
    assert mk.census_launches(cfg_auto, 1) == mk.census_launches(cfg_one, 1) == 2
    # at most one variable: 16 valuations at n = 4, one 128-row block, no split
    cfg_k1 = mk.census_cfg(("K",), 4, 4, 0, 0, 0, 1024, None, max_depth=4, max_vars=1)
    assert mk.census_workspace_size(cfg_k1, 1) == lists
    cfg_k2 = mk.census_cfg(("K",), 4, 4, 0, 0, 0, 1024, None, max_depth=4, max_vars=2)
    assert mk.census_workspace_size(cfg_k2, 1) > lists
    # 5 formulas: the bitmap holds 5 x 32 words
    assert mk.census_workspace_size(cfg_auto, 5) == -(-lists // 256) * 256 + 5 * 32 * 4 + (256 - 5 * 32 * 4 % 256) % 256
    # a layer that fills the GPU (every five-world K frame, 64 formulas) does not split
    full5 = mk.census_cfg(("K",), 5, 5, 0, 0, 0, mk.NO_KEY, None, max_depth=4)
    full5_one = mk.census_cfg(("K",), 5, 5, 0, 0, 0, mk.NO_KEY, None, max_depth=4, vsplit=1)
    assert mk.census_workspace_size(full5, 64) == mk.census_workspace_size(full5_one, 64)
    # T window: at n = 4 the diagonal is bits 0, 5, 10, 15 and compact index 255
    # sets the off-diagonal bits 1-4 and 6-9, so K index 34,815 = 2^15 + 2^10 +
    # (2^10 - 1); the T frames below 34,816 are compact indices [0, 256), 8 words
    t_auto = mk.census_cfg(("T",), 4, 4, 0, 0, 0, 34816, None, max_depth=4)
    t_one = mk.census_cfg(("T",), 4, 4, 0, 0, 0, 34816, None, max_depth=4, vsplit=1)
    lt = mk.census_workspace_size(t_one, 3)
    assert mk.census_workspace_size(t_auto, 3) == -(-lt // 256) * 256 + 256   # 3 x 8 words = 96 B
    # more than 4096 chunks is an argument error
    bad = mk.census_cfg(("K",), 4, 4, 0, 0, 0, 1024, None, max_depth=4, vsplit=4097)
    assert mk.census_workspace_size(bad, 1) == 0


def test_c_program_uses_the_abi(tmp_path):
    """The header is plain C: a C99 program (tests/c_abi_check.c) compiles
    against include/mk.h with -pedantic -Werror, links libmk.so and gets the
    same answers as the binding (host-only calls)."""
    import shutil
    import subprocess
    from paper_2606_15437_gb300 import build as mkbuild
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = mkbuild.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "c_abi_check")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_check.c"), "-o", exe, "-L", libdir, "-lmk",
                    "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {line.split()[0]: line.split()[1:] for line in out.splitlines()}
    assert got["version"] == ["1"]
    prog = mk.compile("[]p -> p")
    assert got["compile"] == ["0", "nvars", str(int(prog.nvars)), "nodes", str(int(prog.nodes))]
    assert got["syntax"] == ["-1", "ok"]
    assert got["strerror"] == ["set"]
    assert got["certify"] == ["1"] and got["certify_dead_end"] == ["0"]
    assert got["s4_5"] == ["6942"] and got["s5_5"] == ["52"]
    assert got["workspace"] == ["positive"] and got["workspace_bad"] == ["0"]


def test_uneven_plan_covers_every_layer_once():
    """mk_plan_uneven (host only): over its work items, every job's layers
    (its class at n = 1 .. its n_max) are covered exactly once, frame word
    by frame word, and no item holds jobs of another class or a smaller
    n_max."""
    rng = random.Random(17)
    texts = [W.random_formula(rng, rng.randint(1, 30), rng.randint(0, 5), rng.randint(0, 3)) for _ in range(120)]
    progs = mk.compile_batch(texts)
    jobs = np.zeros(len(texts), mk.JOB_DTYPE)
    jobs["prog"] = np.arange(len(texts))
    jobs["cls"] = [rng.randrange(4) for _ in texts]
    jobs["n_max"] = [rng.choice((2, 3, 4, 5)) for _ in texts]
    for tiles in (None, (4, 8, 16, 32)):
        plan, info = mk.plan_uneven(progs, jobs, 64, tiles=tiles)
        jl = plan[info.list_off:info.list_off + 4 * info.nlist].view(np.uint32)
        item = np.dtype([("lbeg", "<u4"), ("np", "<u2"), ("n", "u1"), ("cls", "u1"), ("w0", "<u8"), ("w1", "<u8")])
        items = plan[info.items_off:info.items_off + info.nitems * 24].view(item)
        cover = {}
        for it in items:
            for j in jl[int(it["lbeg"]):int(it["lbeg"]) + int(it["np"])]:
                assert jobs["cls"][j] == it["cls"] and jobs["n_max"][j] >= it["n"]
                cover.setdefault((int(j), int(it["n"])), []).append((int(it["w0"]), int(it["w1"])))
        names = ("K", "T", "S4", "S5")
        for j in range(len(texts)):
            for n in range(1, int(jobs["n_max"][j]) + 1):
                words = -(-mk.class_frames(names[jobs["cls"][j]], n) // 32)
                spans = sorted(cover.pop((j, n)))
                assert spans[0][0] == 0 and spans[-1][1] == words
                assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
        assert not cover


def test_compiled_programs_match_oracle_on_every_small_formula():
    """Every constant-free formula over p, q of at most six nodes (7,040 of
    them, with their nested negations, modalities and connectives in every
    arrangement): its compiled program, run by the interpreter above on
    seeded random models of 1-3 worlds, gives the oracle's truth sets, and
    its node count is the text's."""
    def texts(nodes):
        if nodes == 1:
            return ["p", "q"]
        out = []
        for u in ("~", "[]", "<>"):
            out += [u + "(" + a + ")" for a in texts(nodes - 1)]
        for i in range(1, nodes - 1):
            for a in texts(i):
                for b in texts(nodes - 1 - i):
                    out += ["(" + a + " " + op + " " + b + ")" for op in ("&", "|", "->")]
        return out
    rng = np.random.default_rng(11)
    forms = [f for n in range(1, 7) for f in texts(n)]
    assert len(forms) == 7040
    for text in forms:
        prog = mk.compile(text)
        assert prog.nodes == W.nodes(text)
        for n in (1, 2, 3):
            R = rng.integers(0, 2, (n, n)).astype(np.uint8)
            V = rng.integers(0, 2, (4, n)).astype(np.uint8)
            want = oracle.eval_model(text, R, V)
            assert run_program(prog, n, R, V) == {w for w in range(n) if want[w]}, (text, n)
