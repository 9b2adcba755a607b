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


def _open_text(name):
    import gzip
    path = os.path.join(HERE, name)
    return gzip.open(path, "rt") if name.endswith(".gz") else open(path)


def header_values(name):
    """'# key<TAB>value' header lines of a script-written fixture."""
    out = {}
    with _open_text(name) as f:
        for line in f:
            if not line.startswith("#"):
                break
            parts = line[1:].strip().split("\t")
            if len(parts) == 2:
                out[parts[0]] = parts[1]
    return out


def census_rows(name):
    """{(formula, class, n): (cm_count, frames_refuted, witness or None)}
    from a census fixture written by make_census5_golden.py."""
    out = {}
    with _open_text(name) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p, c, n, cm, fr, w = line.rstrip("\n").split("\t")
            wit = None if w == "-" else tuple(int(x) for x in w.split(","))
            out[(int(p), c, int(n))] = (int(cm), int(fr), wit)
    return out


def separation_rows(name="separation_first_splits.tsv"):
    """[pair] -> {"le5": (n, f, v, w) or None, "n6"/"n7"/"n8": (f, v, w),
    None (none in the scanned range) or "." (not scanned)}."""
    out = {}
    with _open_text(name) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            cols = line.rstrip("\n").split("\t")

            def val(x):
                return "." if x == "." else None if x == "-" else tuple(int(y) for y in x.split(","))
            out[int(cols[0])] = {"le5": val(cols[1]), "n6": val(cols[2]), "n7": val(cols[3]), "n8": val(cols[4])}
    return out
