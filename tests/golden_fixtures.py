"""Readers of the paper-value fixtures in tests/golden/ (each file states
the passage its values come from)."""
import os

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rows(name):
    """Tab-separated rows of a fixture, comment lines skipped."""
    out = []
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.rstrip("\n")
            if line and not line.startswith("#"):
                out.append(line.split("\t"))
    return out


def table9():
    """[(axiom, formula, condition or None)] of Table 9."""
    return [(a, f, None if c == "-" else c) for a, f, c in rows("table9_frame_correspondents.tsv")]


def table3():
    """[(m, unsat_through, first_sat)] of Table 3."""
    return [tuple(int(x) for x in r) for r in rows("table3_alpha_separation_sizes.tsv")]


def keyed(name):
    """A key<TAB>value fixture as a dict of strings."""
    return {k: v for k, v in rows(name)}
