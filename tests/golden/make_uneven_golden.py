"""Writes the oracle's census results for the uneven batch.

The uneven batch (``workloads.uneven_formulas(3)``: 20,000 formulas of length
3-64 and modal depth 1-8, each with its own class and n_max in {3, 4, 5},
S = 64 sampled valuations per layer from seed 3) is the persistent,
graph-launched configuration.  Without options this script stores tier 0's
larger layers for a seeded subset of jobs (``uneven_subset.tsv``):

* 400 jobs with n_max >= 4: their class's full four-world layer;
* 40 jobs with n_max = 5: their class's full five-world layer.

Every value comes from ``oracle.census`` (the recursive satisfaction of
Sec. 2 over explicit relations, the scan of Alg. 1); nothing of the CUDA
path is imported.  Rows: job index, class, n, cm_count, frames_refuted,
witness "frame,valuation,world" or "-".

With ``--tier1`` it writes ``uneven_tier1.tsv.gz`` instead: every four- and
five-world layer of every job (n = 4 .. n_max, the job's own class),
computed by the oracle's tier-1 mask evaluator (``oracle.census_tier1``)
after it has reproduced every layer of ``uneven_subset.tsv`` (the run stops
at the first difference).

With ``--small`` it writes ``uneven_n1to3.tsv.gz``: every layer of one to
three worlds of every job (n = 1 .. min(3, n_max), the job's own class), by
``oracle.census`` (tier 0) in worker processes.

Run from the repository root (tens of minutes of CPU each; all resume from
their partial files):

    python tests/golden/make_uneven_golden.py
    python tests/golden/make_uneven_golden.py --tier1
    python tests/golden/make_uneven_golden.py --small --procs 4
"""
import argparse
import gzip
import hashlib
import multiprocessing
import os
import random
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle                                          # noqa: E402
from paper_2606_15437_gb300 import workloads as W      # noqa: E402  (inputs only)

HERE = os.path.dirname(os.path.abspath(__file__))
SEED, S = 3, 64
OUT = os.path.join(HERE, "uneven_subset.tsv")


def items_sha(items):
    return hashlib.sha256("\n".join("%s\t%s\t%d" % it for it in items).encode()).hexdigest()


def units(items):
    rng = random.Random(7)
    four = [j for j, (_, _, m) in enumerate(items) if m >= 4]
    five = [j for j, (_, _, m) in enumerate(items) if m == 5]
    out = [(j, items[j][1], 4) for j in sorted(rng.sample(four, 400))]
    out += [(j, items[j][1], 5) for j in sorted(rng.sample(five, 40))]
    return out


def fmt(u, r):
    w = "-" if r["witness"] is None else "%d,%d,%d" % r["witness"]
    return "%d\t%s\t%d\t%d\t%d\t%s" % (u[0], u[1], u[2], r["cm_count"], r["frames_refuted"], w)


def main_tier1(args, items):
    """Every four- and five-world layer of every job by tier 1, after tier 1
    has reproduced every layer tier 0 stored in uneven_subset.tsv."""
    samples = {n: W.sampled_valuations(SEED, n, S) for n in (4, 5)}
    stored = {}
    with open(OUT) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            j, c, n = line.split("\t")[:3]
            stored[(int(j), c, int(n))] = line.rstrip("\n")
    todo = [(j, items[j][1], n) for j in range(len(items)) for n in range(4, items[j][2] + 1)]
    partial = os.path.join(args.workdir, "uneven_tier1.partial")
    done = {}
    if os.path.exists(partial):
        with open(partial) as f:
            for line in f:
                j, c, n = line.split("\t")[:3]
                done[(int(j), c, int(n))] = line.rstrip("\n")
    order = [u for u in sorted(stored) if u not in done] + [u for u in todo if u not in done and u not in stored]
    t0 = time.time()
    with open(partial, "a") as f:
        for i, u in enumerate(order):
            j, c, n = u
            line = fmt(u, oracle.census_tier1(items[j][0], c, n, samples=samples[n]))
            if u in stored and stored[u] != line:
                raise SystemExit("tier 1 differs from tier 0 at %r:\n  tier 0 %s\n  tier 1 %s" % (u, stored[u], line))
            f.write(line + "\n")
            f.flush()
            done[u] = line
            if i % 500 == 0:
                print("%d/%d layers, %.0f s" % (i, len(order), time.time() - t0), flush=True)
    out = os.path.join(HERE, "uneven_tier1.tsv.gz")
    with gzip.open(out, "wt") as f:
        f.write("# Oracle census of the uneven batch (Sec. 4 Alg. 1; Sec. 8's fused uneven launch):\n"
                "# every four- and five-world layer of every job (n = 4 .. n_max, the job's own class),\n"
                "# %d layers, by the tier-1 mask evaluator (oracle.census_tier1), which first reproduced\n"
                "# all %d layers stored from tier 0 in uneven_subset.tsv.\n"
                "# Written by tests/golden/make_uneven_golden.py --tier1 from oracle.census_tier1, checked\n"
                "# against oracle.census.\n"
                "# inputs: workloads.uneven_formulas(seed=%d), S = %d sampled valuations per layer\n"
                "# from workloads.sampled_valuations(%d, n, %d)\n" % (len(todo), len(stored), SEED, S, SEED, S))
        f.write("# items_sha256\t%s\n" % items_sha(items))
        f.write("# columns: job\tclass\tn\tcm_count\tframes_refuted\twitness(frame,valuation,world)\n")
        for u in todo:
            f.write(done[u] + "\n")
    os.remove(partial)
    print("wrote", out)


_ITEMS = _SAMPLES = None


def _init_worker():
    global _ITEMS, _SAMPLES
    _ITEMS = W.uneven_formulas(SEED)
    _SAMPLES = {n: W.sampled_valuations(SEED, n, S) for n in (1, 2, 3)}


def _small_worker(u):
    j, c, n = u
    return u, fmt(u, oracle.census(_ITEMS[j][0], c, n, samples=_SAMPLES[n]))


def main_small(args, items):
    """Every layer of one to three worlds of every job, by tier 0."""
    os.environ["OMP_NUM_THREADS"] = "1"
    todo = [(j, items[j][1], n) for j in range(len(items)) for n in range(1, min(3, items[j][2]) + 1)]
    partial = os.path.join(args.workdir, "uneven_n1to3.partial")
    done = {}
    if os.path.exists(partial):
        with open(partial) as f:
            for line in f:
                j, c, n = line.split("\t")[:3]
                done[(int(j), c, int(n))] = line.rstrip("\n")
    left = [u for u in todo if u not in done]
    t0 = time.time()
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(args.procs, initializer=_init_worker) as pool, open(partial, "a") as f:
        for i, (u, line) in enumerate(pool.imap_unordered(_small_worker, left, chunksize=64)):
            f.write(line + "\n")
            done[u] = line
            if i % 5000 == 0:
                f.flush()
                print("%d/%d layers, %.0f s" % (i, len(left), time.time() - t0), flush=True)
    out = os.path.join(HERE, "uneven_n1to3.tsv.gz")
    with gzip.open(out, "wt") as f:
        f.write("# Oracle census of the uneven batch (Sec. 4 Alg. 1; Sec. 8's fused uneven launch):\n"
                "# every layer of one to three worlds of every job (n = 1 .. min(3, n_max), the job's own\n"
                "# class), %d layers.\n"
                "# Written by tests/golden/make_uneven_golden.py --small from oracle.census only.\n"
                "# inputs: workloads.uneven_formulas(seed=%d), S = %d sampled valuations per layer\n"
                "# from workloads.sampled_valuations(%d, n, %d)\n" % (len(todo), SEED, S, SEED, S))
        f.write("# items_sha256\t%s\n" % items_sha(items))
        f.write("# columns: job\tclass\tn\tcm_count\tframes_refuted\twitness(frame,valuation,world)\n")
        for u in todo:
            f.write(done[u] + "\n")
    os.remove(partial)
    print("wrote", out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workdir", default=HERE, help="where the resumable partial file lives")
    ap.add_argument("--tier1", action="store_true", help="every n >= 4 layer by the tier-1 evaluator")
    ap.add_argument("--small", action="store_true", help="every n <= 3 layer by tier 0")
    ap.add_argument("--procs", type=int, default=4, help="worker processes (--small)")
    args = ap.parse_args()
    items = W.uneven_formulas(SEED)
    oracle.build()
    if args.tier1:
        main_tier1(args, items)
        return
    if args.small:
        main_small(args, items)
        return
    samples = {n: W.sampled_valuations(SEED, n, S) for n in (4, 5)}
    todo = units(items)
    partial = os.path.join(args.workdir, "uneven_subset.partial")
    done = {}
    if os.path.exists(partial):
        with open(partial) as f:
            for line in f:
                j, c, n = line.split("\t")[:3]
                done[(int(j), c, int(n))] = line.rstrip("\n")
    t0 = time.time()
    with open(partial, "a") as f:
        for u in todo:
            if u in done:
                continue
            j, c, n = u
            r = oracle.census(items[j][0], c, n, samples=samples[n])
            w = "-" if r["witness"] is None else "%d,%d,%d" % r["witness"]
            done[u] = "%d\t%s\t%d\t%d\t%d\t%s" % (j, c, n, r["cm_count"], r["frames_refuted"], w)
            f.write(done[u] + "\n")
            f.flush()
            print("%s %.0f s" % (done[u], time.time() - t0), flush=True)
    with open(OUT, "w") as f:
        f.write("# Oracle census of a seeded subset of the uneven batch (Sec. 4 Alg. 1; Sec. 8's\n"
                "# fused uneven launch): 400 four-world layers of jobs with n_max >= 4 and 40\n"
                "# five-world layers of jobs with n_max = 5, each the job's own class.\n"
                "# Written by tests/golden/make_uneven_golden.py from oracle.census only.\n"
                "# inputs: workloads.uneven_formulas(seed=%d), S = %d sampled valuations per layer\n"
                "# from workloads.sampled_valuations(%d, n, %d)\n" % (SEED, S, SEED, S))
        f.write("# items_sha256\t%s\n" % items_sha(items))
        f.write("# columns: job\tclass\tn\tcm_count\tframes_refuted\twitness(frame,valuation,world)\n")
        for u in todo:
            f.write(done[u] + "\n")
    os.remove(partial)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
