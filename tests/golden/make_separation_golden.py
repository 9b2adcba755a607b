"""Writes the oracle's first splits for the 1,024-pair separation workload.

The workload is the seeded stand-in for the active-synthesis pairs of Sec. 7
(``workloads.separation_pairs(4)``: the 32 context pairs (C^m b, C^(m+1) b),
(alpha_5, alpha_6) and 991 seeded random or one-edit-mutated variable-free
pairs).  A split is the least (n, frame, valuation, world) at which the two
formulas take different truth values (Def. 2, Prop. 4): least n first, then
the least K index (sample index for the sampled sizes), valuation and world.
Every value here comes from ``oracle.pair_layer`` / ``oracle.pair_sampled``
(recursive satisfaction over explicit relations); nothing of the CUDA path
is imported.

What is pinned, per pair:

* ``le5``  -- the first split over every labelled frame of 1..5 worlds, or
  "-" when the pair agrees on all 33,620,498 of them;
* ``n6``   -- for pairs that agree through 5 worlds: the first six-world
  split among K indices [0, 2^27), or "-" when there is none below 2^27
  (the six-world layer has 2^36 frames; above 2^27 the result is pinned only
  by certificate, i.e. partially);
* ``n7``, ``n8`` -- for pairs with no six-world split below 2^27: the first
  split among sampled relations [0, 2^21) of 7 and 8 worlds (seed 4), or "-".
  They apply only if the pair has no six-world split at all.

Columns hold "n,frame,valuation,world" (le5) or "frame,valuation,world",
"-" for none and "." for not scanned.

Run from the repository root (about an hour of CPU; resumes from its partial
file):

    python tests/golden/make_separation_golden.py
"""
import argparse
import hashlib
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle                                          # noqa: E402
from paper_2606_15437_gb300 import workloads as W      # noqa: E402  (inputs only)

HERE = os.path.dirname(os.path.abspath(__file__))
SEED = 4
N6_BOUND = 1 << 27
SAMPLED_BOUND = 1 << 21
OUT = os.path.join(HERE, "separation_first_splits.tsv")


def pairs_sha(pairs):
    return hashlib.sha256("\n".join(a + "\t" + b for a, b in pairs).encode()).hexdigest()


def first_in_layer(a, b, n):
    r = oracle.pair_layer(a, b, n)
    return None if r["split"] is None else r["split"][:3]


def first_six(a, b):
    """First six-world split below N6_BOUND, scanned in doubling windows so an
    early split stops the scan."""
    lo, hi = 0, 1 << 16
    while lo < N6_BOUND:
        r = oracle.pair_layer(a, b, 6, f_lo=lo, f_hi=hi)
        if r["split"] is not None:
            return r["split"][:3]
        lo, hi = hi, min(2 * hi, N6_BOUND)
    return None


def first_sampled(a, b, n):
    lo, hi = 0, 1 << 14
    while lo < SAMPLED_BOUND:
        r = oracle.pair_sampled(a, b, n, SEED, lo, hi)
        if r["split"] is not None:
            return r["split"][:3]
        lo, hi = hi, min(2 * hi, SAMPLED_BOUND)
    return None


def fmt(t):
    return "-" if t is None else ",".join(str(int(x)) for x in t)


def row(i, a, b):
    le5 = None
    for n in range(1, 6):
        s = first_in_layer(a, b, n)
        if s is not None:
            le5 = (n,) + tuple(s)
            break
    if le5 is not None:
        return "%d\t%s\t.\t.\t." % (i, fmt(le5))
    s6 = first_six(a, b)
    if s6 is not None:
        return "%d\t-\t%s\t.\t." % (i, fmt(s6))
    s7 = first_sampled(a, b, 7)
    s8 = first_sampled(a, b, 8)
    return "%d\t-\t-\t%s\t%s" % (i, fmt(s7), fmt(s8))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workdir", default=HERE, help="where the resumable partial file lives")
    args = ap.parse_args()
    pairs = W.separation_pairs(SEED)
    oracle.build()
    partial = os.path.join(args.workdir, "separation_first_splits.partial")
    done = {}
    if os.path.exists(partial):
        with open(partial) as f:
            for line in f:
                done[int(line.split("\t")[0])] = line.rstrip("\n")
    t0 = time.time()
    with open(partial, "a") as f:
        for i, (a, b) in enumerate(pairs):
            if i in done:
                continue
            done[i] = row(i, a, b)
            f.write(done[i] + "\n")
            f.flush()
            print("%d %.0f s %s" % (i, time.time() - t0, done[i]), flush=True)
    with open(OUT, "w") as f:
        f.write("# Oracle first splits of the 1,024-pair separation workload (Sec. 7; Def. 2,\n"
                "# Prop. 4: least n, then K index or sample index, valuation, world).\n"
                "# Written by tests/golden/make_separation_golden.py from oracle.pair_layer and\n"
                "# oracle.pair_sampled only.  inputs: workloads.separation_pairs(seed=%d).\n" % SEED)
        f.write("# pairs_sha256\t%s\n" % pairs_sha(pairs))
        f.write("# n6_bound\t%d\n# sampled_bound\t%d\n# sampled_seed\t%d\n" % (N6_BOUND, SAMPLED_BOUND, SEED))
        f.write("# columns: pair\tle5(n,frame,val,world)\tn6(frame,val,world)\tn7(sample,val,world)"
                "\tn8(sample,val,world); '-' none in range, '.' not scanned\n")
        for i in range(len(pairs)):
            f.write(done[i] + "\n")
    os.remove(partial)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
