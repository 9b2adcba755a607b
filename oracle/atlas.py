"""Failure-density atlas, seriation and density views (Sec. 9) -- TEST
INFRASTRUCTURE.

The plain definitions, written with numpy over the oracle's exact counts:

  D_ij     count_ij / denom_i, the fraction of (valuation, world) pairs at
           which formula i fails on frame j (oracle.c, orc_atlas);
  seriation  centre the columns of D, take the first right singular vector
           v (numpy SVD, float64); frames are ordered by v_j, formulas by
           (D_c v)_i, ties broken by index; the sign of v is fixed so that
           its largest-magnitude component is positive;
  A(pi)    (1 / (B (F-1))) sum_i sum_j |D_i,pi(j+1) - D_i,pi(j)|;
  bins     a point (x, y) in [lo, hi)^2 falls in cell
           floor((x - lo) / (hi - lo) * G), clamped to 0..G-1 (float64).
"""
import numpy as np

from . import _load, ctypes


def atlas_counts(texts, n=3):
    """(counts uint32 [B, 2^(n n)], denominators uint64 [B])."""
    lib = _load()
    lib.orc_atlas.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]
    F = 1 << (n * n)
    cnt = np.zeros((len(texts), F), np.uint32)
    den = np.zeros(len(texts), np.uint64)
    for i, t in enumerate(texts):
        d = ctypes.c_uint64()
        row = np.zeros(F, np.uint32)
        rc = lib.orc_atlas(t.encode(), n, row.ctypes.data_as(ctypes.c_void_p), ctypes.byref(d))
        if rc:
            raise ValueError("orc_atlas rc=%d for %r" % (rc, t))
        cnt[i], den[i] = row, d.value
    return cnt, den


def density(cnt, den):
    return cnt.astype(np.float64) / den.astype(np.float64)[:, None]


def seriation(D):
    """(frame order, formula order, v, formula coordinates)."""
    Dc = D - D.mean(axis=0, keepdims=True)
    _, _, vt = np.linalg.svd(Dc, full_matrices=False)
    v = vt[0]
    if v[np.argmax(np.abs(v))] < 0:
        v = -v
    u = Dc @ v
    col = np.lexsort((np.arange(len(v)), v))
    row = np.lexsort((np.arange(len(u)), u))
    return col, row, v, u


def adjacent_variation(D, perm):
    P = D[:, perm]
    B, F = P.shape
    return float(np.abs(np.diff(P, axis=1)).sum() / (B * (F - 1)))


def bins2d(x, y, lo, hi, G):
    """Cell counts [G, G] (row = y cell, column = x cell)."""
    def cell(z):
        c = np.floor((np.asarray(z, np.float64) - lo) / (hi - lo) * G).astype(np.int64)
        return np.clip(c, 0, G - 1)
    h = np.zeros((G, G), np.int64)
    np.add.at(h, (cell(y), cell(x)), 1)
    return h
