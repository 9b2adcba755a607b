"""Writes the oracle's census results for a subset of the uneven batch.

The uneven batch (``workloads.uneven_formulas(3)``: 20,000 formulas of length
3-64 and modal depth 1-8, each with its own class and n_max in {3, 4, 5},
S = 64 sampled valuations per layer from seed 3) is the persistent,
graph-launched configuration; its layers up to three worlds are checked
against the oracle at test time.  This script stores the larger layers for
a seeded subset of jobs:

* 400 jobs with n_max >= 4: their class's full four-world layer;
* 40 jobs with n_max = 5: their class's full five-world layer.

Every value comes from ``oracle.census`` (the recursive satisfaction of
Sec. 2 over explicit relations, the scan of Alg. 1); nothing of the CUDA
path is imported.  Rows: job index, class, n, cm_count, frames_refuted,
witness "frame,valuation,world" or "-".

Run from the repository root (tens of minutes of CPU; resumes from its
partial file):

    python tests/golden/make_uneven_golden.py
"""
import argparse
import hashlib
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workdir", default=HERE, help="where the resumable partial file lives")
    args = ap.parse_args()
    items = W.uneven_formulas(SEED)
    oracle.build()
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
