"""Why the separation workload's pairs that never split agree everywhere.

The search reports no split for 148 of the 1,024 pairs (seed 4).  The
oracle's stored scans (tests/golden/separation_first_splits.tsv) confirm
that answer on every frame of at most five worlds, on the six-world frames
below K index 2^27 and on the first 2^21 sampled relations of seven and
eight worlds; beyond those ranges the answer rests on one of these, checked
here on the CPU for every such pair:

* the pair is in tests/golden/separation_context_pairs.tsv, which the oracle
  scanned over the search's whole range;
* both formulas fold to the same formula by laws that hold at every world of
  every frame (the Boolean constant laws, []T = T, <>F = F, and the duals
  ~<>a = []~a, ~[]a = <>~a), so they agree on every frame of every size;
* the two fold to <>^a T and <>^b T, or []^a F and []^b F, with a, b >= 8:
  on a frame of n <= 8 worlds a walk of length >= n repeats a world, so it
  extends to every length, and both hold exactly where a cycle is reachable;
* the pair is one of six argued one by one below (K-valid reasoning the
  folder does not do).

The folder works on the pure-Python oracle's parse tree (oracle/pyref.py),
not on the product's compiler.
"""
import golden_fixtures as G
from oracle import pyref
from paper_2606_15437_gb300 import workloads as W

TOP, BOT = ("top",), ("bot",)

# pair -> the argument that the two sides agree at every world of every frame
BY_HAND = {
    41: "<>(<>T | <>[]<>[]F) = <><>T | <><>[]<>[]F = <><>T (the second disjunct implies the "
        "first); <><>T & (<>T | <>[]F) = <><>T since <><>T implies <>T",
    169: "~(~[]F | []<><>T) = []F & <>~<><>T = F ([]F: no successor; <>x needs one); the other "
         "side folds to F",
    269: "[]F -> []~<>~[]<>F = []F -> [][][]F (as []<>F = []F and ~<>~ = []) = T, since a world "
         "with no successor satisfies every []x; the other side folds to T",
    323: "~(<>~F | [](F & F)) = ~<>T & ~[]F = []F & <>T = F; the other side folds to F",
    807: "<>[]<>[]F | []<>T is valid: if some successor v has no successor, []<>[]F holds at v "
         "vacuously; otherwise every successor has one and []<>T holds; the other side folds to T",
    959: "<><>[][]F & []F = F ([]F: no successor, so no <>x holds); the other side <><>F folds to F",
}


def fold(t):
    """t with the laws that hold at every world of every frame applied
    bottom-up: Boolean constants, []T = T, <>F = F and the modal duals."""
    k = t[0]
    if k in ("top", "bot", "var"):
        return t
    if k == "not":
        a = fold(t[1])
        if a == TOP:
            return BOT
        if a == BOT:
            return TOP
        if a[0] == "not":
            return a[1]
        if a[0] == "box":
            return fold(("dia", ("not", a[1])))
        if a[0] == "dia":
            return fold(("box", ("not", a[1])))
        return ("not", a)
    if k == "box":
        a = fold(t[1])
        return TOP if a == TOP else ("box", a)
    if k == "dia":
        a = fold(t[1])
        return BOT if a == BOT else ("dia", a)
    a, b = fold(t[1]), fold(t[2])
    if k == "and":
        if BOT in (a, b):
            return BOT
        if a == TOP or a == b:
            return b
        if b == TOP:
            return a
    elif k == "or":
        if TOP in (a, b):
            return TOP
        if a == BOT or a == b:
            return b
        if b == BOT:
            return a
    elif k == "imp":
        if a == BOT or b == TOP or a == b:
            return TOP
        if a == TOP:
            return b
        if b == BOT:
            return fold(("not", a))
    elif k == "iff":
        if a == b:
            return TOP
        if a == TOP:
            return b
        if b == TOP:
            return a
    return (k, a, b)


def chain(t, op, leaf):
    """m if t is op^m leaf, else -1."""
    m = 0
    while t[0] == op:
        t, m = t[1], m + 1
    return m if t == leaf else -1


def test_fold_keeps_the_truth_value_on_small_frames():
    """The folder is sound on every frame of at most two worlds for the
    workload's unsplit pairs (a check of its laws, by pyref's brute force)."""
    pairs = W.separation_pairs(4)
    rows = G.separation_rows()
    un = [i for i, r in rows.items() if all(r[c] is None for c in ("le5", "n6", "n7", "n8"))]
    untree = {"top": "T", "bot": "F"}

    def text(t):
        k = t[0]
        if k in untree:
            return untree[k]
        if k == "not":
            return "~" + text(t[1])
        if k == "box":
            return "[]" + text(t[1])
        if k == "dia":
            return "<>" + text(t[1])
        op = {"and": "&", "or": "|", "imp": "->", "iff": "<->"}[k]
        return "(%s %s %s)" % (text(t[1]), op, text(t[2]))

    for i in un[:40]:
        for x in pairs[i]:
            y = text(fold(pyref.parse(x)))
            for n in (1, 2):
                assert pyref.first_split(x, y, n) is None, (i, x, y, n)


def test_every_unsplit_pair_is_fixed_by_a_law_or_scanned_in_full():
    pairs = W.separation_pairs(4)
    rows = G.separation_rows()
    unsplit = [i for i, r in rows.items() if all(r[c] is None for c in ("le5", "n6", "n7", "n8"))]
    assert len(unsplit) == 148
    scanned = {int(r[0]) for r in G.rows("separation_context_pairs.tsv")}
    for r in G.rows("separation_context_pairs.tsv"):
        assert r[1:4] == ["-", "-", "-"], r
    kinds = {"scanned": [], "folded": [], "walk": [], "by hand": [], "none": []}
    for i in unsplit:
        a, b = (fold(pyref.parse(x)) for x in pairs[i])
        if i in scanned:
            kinds["scanned"].append(i)
        elif a == b:
            kinds["folded"].append(i)
        elif min(chain(a, "dia", TOP), chain(b, "dia", TOP)) >= 8 or \
                min(chain(a, "box", BOT), chain(b, "box", BOT)) >= 8:
            kinds["walk"].append(i)
        elif i in BY_HAND:
            kinds["by hand"].append(i)
        else:
            kinds["none"].append(i)
    assert not kinds["none"], [(i, pairs[i]) for i in kinds["none"]]
    assert sorted(kinds["by hand"]) == sorted(BY_HAND)
    assert len(kinds["scanned"]) == 6
    print({k: len(v) for k, v in kinds.items()})
