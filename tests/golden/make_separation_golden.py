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

With ``--context`` it writes ``separation_context_pairs.tsv``: for every pair
that the file above leaves unsplit and whose two formulas are alternating
context words (only []<> or <>[] steps before T or F: the alpha family and its
variants) that stay different after []T -> T and <>F -> F (laws that hold
on every frame, so pairs equal after them never split), the first
split over ALL 2^36 six-world frames, by the oracle's tier-1 mask evaluator
(``oracle.pair_tier1``, which first reproduces every six-world split of the
file above), and the first split among sampled relations [0, 10^8) of 7 and
8 worlds (the search's full sampled range), by tier 0.

Run from the repository root (about an hour of CPU, then half an hour for
--context; the first resumes from its partial file):

    python tests/golden/make_separation_golden.py
    python tests/golden/make_separation_golden.py --context
"""
import argparse
import hashlib
import os
import re
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


CONTEXT_OUT = os.path.join(HERE, "separation_context_pairs.tsv")
SAMPLED_FULL = 100_000_000
ALTERNATING = re.compile(r"((\[\]<>)+|(<>\[\])+)(<>|\[\])?[TF]")


def fold(text):
    """The text with []T -> T and <>F -> F applied until nothing changes
    (both hold on every frame)."""
    prev = None
    while prev != text:
        prev, text = text, text.replace("[]T", "T").replace("<>F", "F")
    return text


def stored_rows():
    rows = {}
    with open(OUT) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            cols = line.rstrip("\n").split("\t")
            rows[int(cols[0])] = cols[1:]
    return rows


def first_sampled_full(a, b, n):
    """First split among sampled relations [0, 10^8), in chunks of 2^22."""
    lo = 0
    while lo < SAMPLED_FULL:
        hi = min(lo + (1 << 22), SAMPLED_FULL)
        r = oracle.pair_sampled(a, b, n, SEED, lo, hi)
        if r["split"] is not None:
            return r["split"][:3]
        lo = hi
    return None


def main_context(pairs):
    rows = stored_rows()
    # tier 1 must first reproduce every six-world split tier 0 stored
    for i, cols in sorted(rows.items()):
        if cols[1] not in (".", "-"):
            want = tuple(int(x) for x in cols[1].split(","))
            a, b = pairs[i]
            got = oracle.pair_tier1(a, b, 6, f_lo=0, f_hi=want[0] + 1)["split"]
            if got is None or tuple(got[:3]) != want:
                raise SystemExit("tier 1 differs from tier 0 on pair %d: %r vs %r" % (i, got, want))
    pick = [i for i, cols in sorted(rows.items())
            if cols[0] == "-" and cols[1] == "-" and cols[2] == "-" and cols[3] == "-"
            and all(ALTERNATING.fullmatch(x) for x in pairs[i])
            and fold(pairs[i][0]) != fold(pairs[i][1])]
    t0 = time.time()
    out = []
    for i in pick:
        a, b = pairs[i]
        r6 = oracle.pair_tier1(a, b, 6)
        s6 = None if r6["split"] is None else r6["split"][:3]
        s7 = first_sampled_full(a, b, 7) if s6 is None else "."
        s8 = first_sampled_full(a, b, 8) if s6 is None and s7 is None else "."
        out.append("%d\t%s\t%s\t%s\t%d" % (i, fmt(s6), s7 if s7 == "." else fmt(s7),
                                           s8 if s8 == "." else fmt(s8), r6["frames_disagree"]))
        print("%s %.0f s" % (out[-1], time.time() - t0), flush=True)
    with open(CONTEXT_OUT, "w") as f:
        f.write("# Oracle separation of the workload's unsplit alternating context pairs (Sec. 7;\n"
                "# Def. 2, Prop. 4): pairs that separation_first_splits.tsv leaves unsplit and whose\n"
                "# two formulas are alternating context words.  n6: first split over all 2^36 six-world\n"
                "# frames by the tier-1 mask evaluator (oracle.pair_tier1, which first reproduced every\n"
                "# six-world split of separation_first_splits.tsv); n7, n8: first split among sampled\n"
                "# relations [0, 10^8) by tier 0 (oracle.pair_sampled, seed %d).\n"
                "# Written by tests/golden/make_separation_golden.py --context from oracle only.\n" % SEED)
        f.write("# pairs_sha256\t%s\n" % pairs_sha(pairs))
        f.write("# sampled_range\t%d\n" % SAMPLED_FULL)
        f.write("# columns: pair\tn6(frame,val,world)\tn7(sample,val,world)\tn8(sample,val,world)"
                "\tn6_frames_disagree; '-' none, '.' not scanned\n")
        for line in out:
            f.write(line + "\n")
    print("wrote", CONTEXT_OUT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workdir", default=HERE, help="where the resumable partial file lives")
    ap.add_argument("--context", action="store_true", help="full scans of the unsplit context pairs")
    args = ap.parse_args()
    pairs = W.separation_pairs(SEED)
    oracle.build()
    if args.context:
        main_context(pairs)
        return
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
