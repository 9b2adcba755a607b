"""Second, even simpler oracle path -- TEST INFRASTRUCTURE.

Pure Python, for tiny inputs only: a frame is a set of (w, v) pairs, a
valuation a dict from variable index to a set of worlds, and satisfaction is
the recursive per-world clause of Sec. 2, with no truth-set arrays, no frame
index arithmetic shared with oracle.c and its own parser.  It exists to pin
oracle.c by brute force on n <= 3.
"""
import itertools
import re

_TOK = re.compile(r"\s*(<->|->|\[\]|<>|~|!|&|\||\(|\)|p\d+|[pqrs]|T|F)")


def parse(text):
    toks, i = [], 0
    text = text.replace("box", "[]").replace("dia", "<>").replace("not", "~")
    text = text.replace(" and ", " & ").replace(" or ", " | ")
    while i < len(text):
        if text[i].isspace():
            i += 1
            continue
        m = _TOK.match(text, i)
        if not m:
            raise ValueError("bad token at %d in %r" % (i, text))
        toks.append(m.group(1))
        i = m.end()
    pos = [0]

    def peek():
        return toks[pos[0]] if pos[0] < len(toks) else None

    def take():
        pos[0] += 1
        return toks[pos[0] - 1]

    def unary():
        t = take()
        if t in ("~", "!"):
            return ("not", unary())
        if t == "[]":
            return ("box", unary())
        if t == "<>":
            return ("dia", unary())
        if t == "(":
            e = iff()
            assert take() == ")"
            return e
        if t == "T":
            return ("top",)
        if t == "F":
            return ("bot",)
        if t[0] == "p" and len(t) > 1:
            return ("var", int(t[1:]))
        return ("var", "pqrs".index(t))

    def conj():
        e = unary()
        while peek() == "&":
            take()
            e = ("and", e, unary())
        return e

    def disj():
        e = conj()
        while peek() == "|":
            take()
            e = ("or", e, conj())
        return e

    def imp():
        e = disj()
        if peek() == "->":
            take()
            return ("imp", e, imp())
        return e

    def iff():
        e = imp()
        while peek() == "<->":
            take()
            e = ("iff", e, imp())
        return e

    tree = iff()
    if pos[0] != len(toks):
        raise ValueError("trailing input in %r" % text)
    return tree


def nvars(tree):
    if tree[0] == "var":
        return tree[1] + 1
    return max([0] + [nvars(c) for c in tree[1:] if isinstance(c, tuple)])


def sat(R, V, w, t):
    """M, w |= t for the frame R (set of pairs) and valuation V."""
    op = t[0]
    if op == "top":
        return True
    if op == "bot":
        return False
    if op == "var":
        return w in V[t[1]]
    if op == "not":
        return not sat(R, V, w, t[1])
    if op == "and":
        return sat(R, V, w, t[1]) and sat(R, V, w, t[2])
    if op == "or":
        return sat(R, V, w, t[1]) or sat(R, V, w, t[2])
    if op == "imp":
        return (not sat(R, V, w, t[1])) or sat(R, V, w, t[2])
    if op == "iff":
        return sat(R, V, w, t[1]) == sat(R, V, w, t[2])
    if op == "box":
        return all(sat(R, V, v, t[1]) for (u, v) in R if u == w)
    if op == "dia":
        return any(sat(R, V, v, t[1]) for (u, v) in R if u == w)
    raise ValueError(op)


def all_frames(n):
    """Every relation on n worlds, in the same order as the K index
    (the pair (w, v) is the (w*n+v)-th binary digit)."""
    pairs = [(w, v) for w in range(n) for v in range(n)]
    for bits in range(1 << len(pairs)):
        yield bits, {pairs[e] for e in range(len(pairs)) if (bits >> e) & 1}


def in_class(cls, n, R):
    refl = all((w, w) in R for w in range(n))
    trans = all((w, u) in R for (w, v) in R for (x, u) in R if v == x)
    sym = all((v, w) in R for (w, v) in R)
    return {"K": True, "T": refl, "S4": refl and trans, "S5": refl and trans and sym, "K4": trans}[cls]


def all_valuations(k, n):
    """Every valuation of k variables on n worlds, in valuation-index order
    (p_i holds at w iff digit i*n+w is set)."""
    for x in range(1 << (k * n)):
        yield x, {i: {w for w in range(n) if (x >> (i * n + w)) & 1} for i in range(k)}


def census(text, cls, n):
    """Exhaustive census by brute force: (cm_count, frames_refuted, witness)."""
    t = parse(text)
    k = nvars(t)
    cm, fr, wit = 0, 0, None
    for f, R in all_frames(n):
        if not in_class(cls, n, R):
            continue
        any_ref = False
        for x, V in all_valuations(k, n):
            bad = [w for w in range(n) if not sat(R, V, w, t)]
            if bad:
                cm += 1
                any_ref = True
                if wit is None:
                    wit = (f, x, bad[0])
        fr += any_ref
    return cm, fr, wit


def census_sampled(text, cls, n, samples):
    """Census over the given valuation values (low k*n bits of each), in
    slot order, counted with multiplicity."""
    t = parse(text)
    k = nvars(t)
    cm, fr, wit = 0, 0, None
    for f, R in all_frames(n):
        if not in_class(cls, n, R):
            continue
        any_ref = False
        for j, x in enumerate(samples):
            x = int(x) & ((1 << (k * n)) - 1)
            V = {i: {w for w in range(n) if (x >> (i * n + w)) & 1} for i in range(k)}
            bad = [w for w in range(n) if not sat(R, V, w, t)]
            if bad:
                cm += 1
                any_ref = True
                if wit is None:
                    wit = (f, j, bad[0])
        fr += any_ref
    return cm, fr, wit


def first_split(phi, psi, n):
    a, b = parse(phi), parse(psi)
    k = max(nvars(a), nvars(b))
    for f, R in all_frames(n):
        for x, V in all_valuations(k, n):
            for w in range(n):
                if sat(R, V, w, a) != sat(R, V, w, b):
                    return (f, x, w)
    return None


def frames_in_class(cls, n):
    return sum(1 for _, R in all_frames(n) if in_class(cls, n, R))


def valuation_count(k, n):
    return sum(1 for _ in itertools.product(range(2), repeat=k * n))


def condition(name, n, R):
    """First-order frame conditions of the correspondence library, by
    direct set comprehension over the relation R (a set of pairs)."""
    W = range(n)
    succ = {w: {v for (u, v) in R if u == w} for w in W}
    if name == "every frame":
        return True
    if name == "no frame":
        return False
    if name == "reflexive":
        return all((w, w) in R for w in W)
    if name == "irreflexive":
        return not any((w, w) in R for w in W)
    if name == "serial":
        return all(succ[w] for w in W)
    if name == "transitive":
        return all((w, u) in R for (w, v) in R for u in succ[v])
    if name == "symmetric":
        return all((v, w) in R for (w, v) in R)
    if name == "Euclidean":
        return all((v, u) in R for w in W for v in succ[w] for u in succ[w])
    if name == "partially functional":
        return all(len(succ[w]) <= 1 for w in W)
    if name == "functional":
        return all(len(succ[w]) == 1 for w in W)
    if name == "dense":
        return all(any(u in succ[w] and v in succ[u] for u in W) for (w, v) in R)
    if name == "directed":
        return all(succ[v] & succ[u] for w in W for v in succ[w] for u in succ[w])
    if name == "antisymmetric":
        return all(w == v or (v, w) not in R for (w, v) in R)
    if name == "asymmetric":
        return all((v, w) not in R for (w, v) in R)
    if name == "weakly connected":
        return all(v == u or (v, u) in R or (u, v) in R for w in W for v in succ[w] for u in succ[w])
    if name == "shift reflexive":
        return all((v, v) in R for (w, v) in R)
    if name == "empty relation":
        return not R
    if name == "coreflexive":
        return all(w == v for (w, v) in R)
    raise ValueError(name)
