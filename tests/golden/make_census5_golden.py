"""Writes the oracle's census results for the five-world census batch.

The batch is the seeded synthetic corpus that stands in for the paper's
5,624-formula census of Sec. 6 (5,621 random formulas of length 3-24, modal
depth 1-4 and 0-3 variables, plus the K, T and 4 axioms), over classes
K/T/S4/S5 with S = 256 sampled valuations per layer (seed 2).  Every value
written here comes from ``oracle.census`` (the recursive satisfaction of
Sec. 2 over explicit relations, the corpus scan of Alg. 1 in Sec. 4); the
inputs come from the seeded generators of ``workloads``.  Nothing of the CUDA
path is imported.

Five files:

* ``census5_n1to4.tsv.gz`` -- every formula, every class, n = 1..4;
* ``census5_n5_subset.tsv`` -- full five-world layers (all 2^25 K frames,
  2^20 T frames, the 6,942 S4 and 52 S5 frames) for a stratified subset:
  per variable count k = 0..3 the longest formula and the deepest of the
  longest, seeded random picks (40 / 20 / 2 / 2 for k = 0 / 1 / 2 / 3), and
  the three axioms;
* ``census5_n5_k0.tsv`` -- the same full five-world layers for every
  variable-free formula of the batch (one valuation per frame);
* ``census5_n5_s4s5.tsv.gz`` -- every formula on the full five-world S4
  (6,942 frames) and S5 (52 frames) layers;
* ``census5_n5_tier1.tsv.gz`` -- every formula on the full five-world K
  (2^25 frames) and T (2^20 frames) layers, computed by the oracle's tier-1
  mask evaluator (``oracle.census_tier1``, 64 frames per machine word)
  after it has reproduced every five-world layer the files above hold from
  tier 0 (the run stops at the first difference).

Rows: formula index, class, n, cm_count, frames_refuted, witness as
"frame,valuation,world" (K index; valuation index or sample slot; least
world) or "-".  The header carries the SHA-256 of the formula texts so a test
can tell that its inputs are the ones these values were computed for.

Run from the repository root (hours of CPU for the n = 5 part; the script
resumes from its partial file):

    python tests/golden/make_census5_golden.py --part n1to4
    python tests/golden/make_census5_golden.py --part n5
    python tests/golden/make_census5_golden.py --part n5k0
    python tests/golden/make_census5_golden.py --part n5s4s5 --procs 8
    python tests/golden/make_census5_golden.py --part n5tier1
"""
import argparse
import gzip
import hashlib
import multiprocessing
import os
import random
import re
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle                                          # noqa: E402
from paper_2606_15437_gb300 import workloads as W      # noqa: E402  (inputs only)

HERE = os.path.dirname(os.path.abspath(__file__))
SEED, S = 2, 256
CLASSES = ("K", "T", "S4", "S5")
SUBSET_RANDOM = {0: 40, 1: 20, 2: 2, 3: 2}


def texts_sha(texts):
    return hashlib.sha256("\n".join(texts).encode()).hexdigest()


def modal_depth(text):
    """Largest nesting of [] / <> in a generated text (fully parenthesised,
    unary operators prefixed)."""
    toks = re.findall(r"\[\]|<>|~|\(|\)|&|\||->|p\d+|[pqrs]|T|F", text)
    pos = 0

    def unary():
        nonlocal pos
        t = toks[pos]
        if t in ("[]", "<>"):
            pos += 1
            return 1 + unary()
        if t == "~":
            pos += 1
            return unary()
        if t == "(":
            pos += 1
            d = binary()
            pos += 1                      # ")"
            return d
        pos += 1                          # atom or constant
        return 0

    def binary():
        nonlocal pos
        d = unary()
        while pos < len(toks) and toks[pos] in ("&", "|", "->"):
            pos += 1
            d = max(d, unary())
        return d

    return binary()


def n5_subset(texts):
    """Indices of the stratified five-world subset (sorted)."""
    ncore = len(texts) - len(W.AXIOMS)
    info = [(oracle.nvars(t), W.nodes(t), modal_depth(t)) for t in texts[:ncore]]
    rng = random.Random(5)
    pick = set()
    for k in range(4):
        idx = [i for i in range(ncore) if info[i][0] == k]
        pick.add(max(idx, key=lambda i: (info[i][1], -i)))                  # longest
        pick.add(max(idx, key=lambda i: (info[i][2], info[i][1], -i)))      # deepest, then longest
        rest = [i for i in idx if i not in pick]
        pick.update(rng.sample(rest, SUBSET_RANDOM[k]))
    pick.update(range(ncore, len(texts)))
    return sorted(pick)


def fmt(p, c, n, r):
    w = "-" if r["witness"] is None else "%d,%d,%d" % r["witness"]
    return "%d\t%s\t%d\t%d\t%d\t%s" % (p, c, n, r["cm_count"], r["frames_refuted"], w)


def header(texts, what, source="oracle.census only"):
    return ["# Oracle census of the five-world census batch (Sec. 4 Alg. 1; Sec. 6 corpus",
            "# stand-in): %s." % what,
            "# Written by tests/golden/make_census5_golden.py from %s." % source,
            "# inputs: workloads.census5_formulas(seed=%d) (%d formulas), S = %d sampled valuations"
            % (SEED, len(texts), S),
            "# per layer from workloads.sampled_valuations(%d, n, %d)" % (SEED, S),
            "# texts_sha256\t%s" % texts_sha(texts),
            "# columns: formula\tclass\tn\tcm_count\tframes_refuted\twitness(frame,valuation,world)"]


def run(texts, units, partial, log_every=200):
    """Computes every (formula, class, n) unit not yet in ``partial``;
    returns all rows keyed by unit."""
    done = {}
    if os.path.exists(partial):
        with open(partial) as f:
            for line in f:
                p, c, n = line.split("\t")[:3]
                done[(int(p), c, int(n))] = line.rstrip("\n")
    samples = {n: W.sampled_valuations(SEED, n, S) for n in range(1, 6)}
    t0 = time.time()
    todo = [u for u in units if u not in done]
    with open(partial, "a") as f:
        for i, (p, c, n) in enumerate(todo):
            r = oracle.census(texts[p], c, n, samples=samples[n])
            line = fmt(p, c, n, r)
            f.write(line + "\n")
            f.flush()
            done[(p, c, n)] = line
            if i % log_every == 0:
                print("%d/%d units, %.0f s" % (i, len(todo), time.time() - t0), flush=True)
    return done


def _unit_worker(u):
    """One (formula, class, n) unit in a worker process (one OpenMP thread)."""
    p, c, n = u
    return u, fmt(p, c, n, oracle.census(_TEXTS[p], c, n, samples=_SAMPLES[n]))


def _init_worker():
    global _TEXTS, _SAMPLES
    _TEXTS = W.census5_formulas(SEED)
    _SAMPLES = {n: W.sampled_valuations(SEED, n, S) for n in range(1, 6)}


def run_pool(units, partial, procs, log_every=500):
    """``run`` spread over ``procs`` worker processes; rows keyed by unit."""
    done = {}
    if os.path.exists(partial):
        with open(partial) as f:
            for line in f:
                p, c, n = line.split("\t")[:3]
                done[(int(p), c, int(n))] = line.rstrip("\n")
    todo = [u for u in units if u not in done]
    t0 = time.time()
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(procs, initializer=_init_worker) as pool, open(partial, "a") as f:
        for i, (u, line) in enumerate(pool.imap_unordered(_unit_worker, todo, chunksize=4)):
            f.write(line + "\n")
            f.flush()
            done[u] = line
            if i % log_every == 0:
                print("%d/%d units, %.0f s" % (i, len(todo), time.time() - t0), flush=True)
    return done


def read_rows(path):
    """The rows of a stored census file, keyed by (formula, class, n)."""
    opener = gzip.open if path.endswith(".gz") else open
    out = {}
    with opener(path, "rt") as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p, c, n = line.split("\t")[:3]
            out[(int(p), c, int(n))] = line.rstrip("\n")
    return out


def run_tier1(texts, check, stored, units, partial, log_every=100):
    """Tier 1 on every unit of ``check`` (compared with tier 0's stored row;
    stops at the first difference), then on ``units``; rows keyed by unit,
    resumable from ``partial``."""
    done = {}
    if os.path.exists(partial):
        with open(partial) as f:
            for line in f:
                p, c, n = line.split("\t")[:3]
                done[(int(p), c, int(n))] = line.rstrip("\n")
    samples = {n: W.sampled_valuations(SEED, n, S) for n in range(1, 6)}
    t0 = time.time()
    todo = [u for u in check if u not in done] + [u for u in units if u not in done and u not in stored]
    todo = list(dict.fromkeys(todo))
    with open(partial, "a") as f:
        for i, (p, c, n) in enumerate(todo):
            line = fmt(p, c, n, oracle.census_tier1(texts[p], c, n, samples=samples[n]))
            if (p, c, n) in stored and stored[(p, c, n)] != line:
                raise SystemExit("tier 1 differs from tier 0 at %r:\n  tier 0 %s\n  tier 1 %s"
                                 % ((p, c, n), stored[(p, c, n)], line))
            f.write(line + "\n")
            f.flush()
            done[(p, c, n)] = line
            if i % log_every == 0:
                print("%d/%d units, %.0f s" % (i, len(todo), time.time() - t0), flush=True)
    return done


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--part", choices=("n1to4", "n5", "n5k0", "n5s4s5", "n5tier1"), required=True)
    ap.add_argument("--workdir", default=HERE, help="where the resumable partial file lives")
    ap.add_argument("--procs", type=int, default=1, help="worker processes (n5s4s5)")
    args = ap.parse_args()
    texts = W.census5_formulas(SEED)
    oracle.build()
    if args.part == "n1to4":
        units = [(p, c, n) for p in range(len(texts)) for c in CLASSES for n in range(1, 5)]
        partial = os.path.join(args.workdir, "census5_n1to4.partial")
        rows = run(texts, units, partial, log_every=2000)
        out = os.path.join(HERE, "census5_n1to4.tsv.gz")
        with gzip.open(out, "wt") as f:
            f.write("\n".join(header(texts, "every formula, classes K/T/S4/S5, n = 1..4")) + "\n")
            for u in units:
                f.write(rows[u] + "\n")
    elif args.part == "n5s4s5":
        os.environ["OMP_NUM_THREADS"] = "1"
        units = [(p, c, 5) for p in range(len(texts)) for c in ("S4", "S5")]
        partial = os.path.join(args.workdir, "census5_n5_s4s5.partial")
        rows = run_pool(units, partial, args.procs)
        out = os.path.join(HERE, "census5_n5_s4s5.tsv.gz")
        with gzip.open(out, "wt") as f:
            f.write("\n".join(header(texts, "every formula, classes S4/S5, n = 5")) + "\n")
            for u in units:
                f.write(rows[u] + "\n")
    elif args.part == "n5tier1":
        # tier 0's stored five-world layers, which tier 1 must reproduce first
        stored = {}
        for name in ("census5_n5_subset.tsv", "census5_n5_k0.tsv", "census5_n5_s4s5.tsv.gz"):
            path = os.path.join(HERE, name)
            if os.path.exists(path):
                stored.update(read_rows(path))
        check = sorted(stored, key=lambda u: (u[1] == "K", u[0], u[1]))
        units = [(p, c, 5) for p in range(len(texts)) for c in ("K", "T")]
        partial = os.path.join(args.workdir, "census5_n5_tier1.partial")
        rows = run_tier1(texts, check, stored, units, partial)
        out = os.path.join(HERE, "census5_n5_tier1.tsv.gz")
        with gzip.open(out, "wt") as f:
            f.write("\n".join(header(texts, "every formula, classes K/T, n = 5, by the tier-1 mask evaluator "
                                     "(oracle.census_tier1), which first reproduced all %d five-world "
                                     "layers stored from tier 0" % len(check),
                                     source="oracle.census_tier1, checked against oracle.census")) + "\n")
            for u in units:
                f.write(rows[u] + "\n")
    elif args.part == "n5k0":
        k0 = [p for p in range(len(texts)) if oracle.nvars(texts[p]) == 0]
        units = [(p, c, 5) for p in k0 for c in CLASSES]
        partial = os.path.join(args.workdir, "census5_n5_k0.partial")
        rows = run(texts, units, partial, log_every=200)
        out = os.path.join(HERE, "census5_n5_k0.tsv")
        with open(out, "w") as f:
            f.write("\n".join(header(texts, "full n = 5 layers of every variable-free formula (%d)" % len(k0)))
                    + "\n")
            for u in units:
                f.write(rows[u] + "\n")
    else:
        subset = n5_subset(texts)
        # cheapest first, so a partial run covers the most formulas
        units = [(p, c, 5) for p in subset for c in ("S5", "S4", "T", "K")]
        units.sort(key=lambda u: (u[1] == "K", oracle.nvars(texts[u[0]]), W.nodes(texts[u[0]])))
        partial = os.path.join(args.workdir, "census5_n5_subset.partial")
        rows = run(texts, units, partial, log_every=1)
        out = os.path.join(HERE, "census5_n5_subset.tsv")
        with open(out, "w") as f:
            f.write("\n".join(header(texts, "full n = 5 layers of a stratified subset of %d formulas "
                                     "(per k = 0..3: longest, deepest, seeded picks 40/20/2/2; "
                                     "the three axioms)" % len(subset))) + "\n")
            for p in subset:
                for c in CLASSES:
                    f.write(rows[(p, c, 5)] + "\n")
    if os.path.exists(partial):
        os.remove(partial)
    print("wrote", out)


if __name__ == "__main__":
    main()
