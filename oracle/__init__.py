"""CPU oracle for exhaustive finite Kripke evaluation -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
legs may import this package.  The product path (``paper_2606_15437_gb300``)
never imports it, and it imports nothing from the product: the two share no
code.  The arithmetic lives in ``oracle.c`` (a recursive truth-set evaluator
over explicit relations, the satisfaction clauses of Sec. 2 written out);
this module only compiles it with gcc and marshals arguments.

``pyref`` holds an even simpler pure-Python path (sets of pairs, per-world
recursion) used to pin ``oracle.c`` by brute force on tiny inputs.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_TIER1 = os.path.join(_HERE, "tier1.c")
_lock = threading.Lock()
_lib = None

CLASSES = ("K", "T", "S4", "S5", "K4")


def build(force=False):
    """Compile oracle.c (tier 0) and tier1.c (the mask evaluator) into
    _build/liboracle.so (plain gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [_SRC, _SRC_TIER1]
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(x) for x in srcs)):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                           "-o", tmp] + srcs)
    os.replace(tmp, _SO)
    return _SO


class _Census(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_uint64), ("cm_count", ctypes.c_uint64),
                ("frames_refuted", ctypes.c_uint64), ("found", ctypes.c_int32),
                ("nvals", ctypes.c_int32), ("wf", ctypes.c_uint64),
                ("wv", ctypes.c_uint32), ("ww", ctypes.c_uint32)]


class _Pair(ctypes.Structure):
    _fields_ = [("found", ctypes.c_int32), ("nvals", ctypes.c_int32),
                ("f", ctypes.c_uint64), ("v", ctypes.c_uint32), ("w", ctypes.c_uint32),
                ("phi_val", ctypes.c_int32), ("psi_val", ctypes.c_int32),
                ("frames_disagree", ctypes.c_uint64)]


class _Stress(ctypes.Structure):
    _fields_ = [("found", ctypes.c_int32), ("nvals", ctypes.c_int32), ("s", ctypes.c_uint64),
                ("x", ctypes.c_uint32), ("w", ctypes.c_uint32), ("nsplit", ctypes.c_uint64)]


NUM_TEMPLATES = 39
GENERATORS = ("er", "flip", "scc", "deadend", "backedge", "permscc")


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, u32, i32, p = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
            cs = ctypes.c_char_p
            lib.orc_census.argtypes = [cs, i32, i32, u32, p, u64, u64, ctypes.POINTER(_Census)]
            lib.orc_pair_layer.argtypes = [cs, cs, i32, u32, p, u64, u64, ctypes.POINTER(_Pair)]
            lib.orc_pair_sampled.argtypes = [cs, cs, i32, u64, u32, p, u64, u64, ctypes.POINTER(_Pair)]
            lib.orc_eval_model.argtypes = [cs, i32, p, p, p]
            lib.orc_in_class.argtypes = [i32, i32, p]
            lib.orc_class_size.argtypes = [i32, i32]
            lib.orc_class_size.restype = u64
            lib.orc_sample_frame.argtypes = [u64, i32, u64]
            lib.orc_sample_frame.restype = u64
            lib.orc_splitmix_out.argtypes = [u64, u64]
            lib.orc_splitmix_out.restype = u64
            lib.orc_stream_state.argtypes = [u64, u64, u64]
            lib.orc_stream_state.restype = u64
            lib.orc_frame_valid_all.argtypes = [cs, i32, p]
            lib.orc_template.argtypes = [i32, i32, p]
            lib.orc_stress_relation.argtypes = [i32, u64, i32, u64, p]
            lib.orc_stress_pair.argtypes = [cs, cs, i32, p, u64, ctypes.POINTER(_Stress)]
            lib.orc_frame_condition.argtypes = [i32, i32, p]
            lib.orc_nvars.argtypes = [cs]
            lib.orc_nodes.argtypes = [cs]
            lib.orc_census_tier1.argtypes = [cs, i32, i32, u32, p, ctypes.POINTER(_Census)]
            lib.orc_pair_tier1.argtypes = [cs, cs, i32, u32, p, u64, u64, ctypes.POINTER(_Pair)]
            _lib = lib
    return _lib


def _cls(c):
    return CLASSES.index(c) if isinstance(c, str) else int(c)


def _samples(samples):
    if samples is None:
        return None, 0, None
    a = np.ascontiguousarray(np.asarray(samples, dtype=np.uint32))
    return a, len(a), a.ctypes.data_as(ctypes.c_void_p)


def census(text, cls, n, samples=None, f_lo=0, f_hi=2 ** 64 - 1):
    """Census of one formula on one (class, n) layer, frames with K index in
    [f_lo, f_hi).  ``samples`` = the layer's sampled valuations (None: always
    exhaustive).  Returns a dict; ``witness`` is (frame, valuation, world)."""
    lib = _load()
    keep, S, ptr = _samples(samples)
    out = _Census()
    rc = lib.orc_census(text.encode(), _cls(cls), n, S, ptr, f_lo, f_hi, ctypes.byref(out))
    if rc:
        raise ValueError("oracle census failed (%d) for %r" % (rc, text))
    return {"frames": out.frames, "cm_count": out.cm_count,
            "frames_refuted": out.frames_refuted, "nvals": out.nvals,
            "witness": (out.wf, out.wv, out.ww) if out.found else None}


def census_tier1(text, cls, n, samples=None):
    """``census`` over all frames of one (class, n <= 5) layer, computed by
    the tier-1 mask evaluator (tier1.c: 64 frames per machine word) instead of
    tier 0's per-world recursion; the same dict.  Trusted only where it
    equals ``census`` (tests/test_tier1_oracle.py)."""
    lib = _load()
    keep, S, ptr = _samples(samples)
    out = _Census()
    rc = lib.orc_census_tier1(text.encode(), _cls(cls), n, S, ptr, ctypes.byref(out))
    if rc:
        raise ValueError("tier-1 census failed (%d) for %r" % (rc, text))
    return {"frames": out.frames, "cm_count": out.cm_count,
            "frames_refuted": out.frames_refuted, "nvals": out.nvals,
            "witness": (out.wf, out.wv, out.ww) if out.found else None}


def pair_tier1(phi, psi, n, samples=None, f_lo=0, f_hi=2 ** 64 - 1):
    """``pair_layer`` computed by the tier-1 mask evaluator (tier1.c, 64
    frames per machine word; n <= 6): the same dict.  Trusted only where it
    equals ``pair_layer`` (tests/test_tier1_oracle.py)."""
    lib = _load()
    keep, S, ptr = _samples(samples)
    out = _Pair()
    rc = lib.orc_pair_tier1(phi.encode(), psi.encode(), n, S, ptr, f_lo, f_hi, ctypes.byref(out))
    if rc:
        raise ValueError("tier-1 pair scan failed (%d) for %r / %r" % (rc, phi, psi))
    return _pair_dict(out)


def _pair_dict(out):
    return {"nvals": out.nvals, "frames_disagree": out.frames_disagree,
            "split": (out.f, out.v, out.w, out.phi_val, out.psi_val) if out.found else None}


def pair_layer(phi, psi, n, samples=None, f_lo=0, f_hi=2 ** 64 - 1):
    """First (frame, valuation, world) where phi and psi differ on n worlds."""
    lib = _load()
    keep, S, ptr = _samples(samples)
    out = _Pair()
    rc = lib.orc_pair_layer(phi.encode(), psi.encode(), n, S, ptr, f_lo, f_hi, ctypes.byref(out))
    if rc:
        raise ValueError("oracle pair_layer failed (%d)" % rc)
    return _pair_dict(out)


def pair_sampled(phi, psi, n, seed, s_lo, s_hi, samples=None):
    """First disagreement on the sampled n-world relations s in [s_lo, s_hi)."""
    lib = _load()
    keep, S, ptr = _samples(samples)
    out = _Pair()
    rc = lib.orc_pair_sampled(phi.encode(), psi.encode(), n, seed, S, ptr, s_lo, s_hi,
                              ctypes.byref(out))
    if rc:
        raise ValueError("oracle pair_sampled failed (%d)" % rc)
    return _pair_dict(out)


def eval_model(text, R, V=None):
    """Truth value at every world of the explicit model: R is an n x n 0/1
    matrix, V a (vars x n) 0/1 matrix."""
    lib = _load()
    R = np.ascontiguousarray(np.asarray(R, dtype=np.uint8))
    n = R.shape[0]
    if V is None:
        V = np.zeros((8, n), np.uint8)
    V = np.ascontiguousarray(np.asarray(V, dtype=np.uint8))
    if V.shape[0] < 8:
        V = np.ascontiguousarray(np.vstack([V, np.zeros((8 - V.shape[0], n), np.uint8)]))
    out = np.zeros(n, np.uint8)
    rc = lib.orc_eval_model(text.encode(), n, R.ctypes.data_as(ctypes.c_void_p),
                            V.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p))
    if rc:
        raise ValueError("oracle eval_model failed (%d)" % rc)
    return out


def frame_valid_all(text, n):
    """uint8[2^(n*n)]: 1 where the K-indexed frame validates ``text``."""
    lib = _load()
    out = np.zeros(1 << (n * n), np.uint8)
    rc = lib.orc_frame_valid_all(text.encode(), n, out.ctypes.data_as(ctypes.c_void_p))
    if rc:
        raise ValueError("oracle frame_valid_all failed (%d)" % rc)
    return out


def in_class(cls, R):
    lib = _load()
    R = np.ascontiguousarray(np.asarray(R, dtype=np.uint8))
    return bool(lib.orc_in_class(_cls(cls), R.shape[0], R.ctypes.data_as(ctypes.c_void_p)))


def class_size(cls, n):
    return int(_load().orc_class_size(_cls(cls), n))


def sample_frame(seed, n, s):
    """Row-major edge mask of sampled n-world relation number s."""
    return int(_load().orc_sample_frame(seed, n, s))


def splitmix_out(state, j):
    return int(_load().orc_splitmix_out(state, j))


def stream_state(seed, tag, n):
    return int(_load().orc_stream_state(seed, tag, n))


def nvars(text):
    return int(_load().orc_nvars(text.encode()))


def frame_matrix(f, n):
    """The n x n relation of K index f (R(w,v) = bit w*n+v)."""
    return np.array([[(f >> (w * n + v)) & 1 for v in range(n)] for w in range(n)], np.uint8)


def threads():
    return int(_load().orc_threads())


def template(tid, n):
    """Successor masks (list of n ints) of stress template ``tid`` on n worlds."""
    out = (ctypes.c_uint32 * 16)()
    rc = _load().orc_template(int(tid), int(n), out)
    if rc:
        raise ValueError("orc_template(%d, %d) = %d" % (tid, n, rc))
    return [int(out[w]) for w in range(n)]


def stress_relation(gen, seed, n, s):
    """Successor masks of relation ``s`` of adversarial generator ``gen``."""
    g = GENERATORS.index(gen) if isinstance(gen, str) else int(gen)
    out = (ctypes.c_uint32 * 16)()
    rc = _load().orc_stress_relation(g, int(seed), int(n), int(s), out)
    if rc:
        raise ValueError("orc_stress_relation(%d, %d, %d) = %d" % (g, n, s, rc))
    return [int(out[w]) for w in range(n)]


def stress_relations(gen, seed, n, first, count):
    """uint32 array [count, 16] of successor masks (rows >= n are zero)."""
    a = np.zeros((count, 16), np.uint32)
    for i in range(count):
        a[i, :n] = stress_relation(gen, seed, n, first + i)
    return a


def stress_pair(phi, psi, n, succ):
    """First split of (phi, psi) over the relations ``succ`` ([count, 16]
    successor masks), in (relation, valuation, world) order, and the number
    of relations on which they differ."""
    a = np.ascontiguousarray(np.asarray(succ, dtype=np.uint32).reshape(-1, 16))
    o = _Stress()
    rc = _load().orc_stress_pair(phi.encode(), psi.encode(), int(n),
                                 a.ctypes.data_as(ctypes.c_void_p), len(a), ctypes.byref(o))
    if rc:
        raise ValueError("orc_stress_pair rc=%d" % rc)
    split = (int(o.s), int(o.x), int(o.w)) if o.found else None
    return {"split": split, "nsplit": int(o.nsplit), "nvals": int(o.nvals)}


CONDITIONS = ("every frame", "no frame", "reflexive", "irreflexive", "serial", "transitive", "symmetric",
              "Euclidean", "partially functional", "functional", "dense", "directed", "antisymmetric",
              "asymmetric", "weakly connected", "shift reflexive", "empty relation", "coreflexive")


def frame_condition(cond, n):
    """uint8 array over the K indices of n-world frames: 1 iff the frame
    satisfies library condition ``cond`` (id or name)."""
    c = CONDITIONS.index(cond) if isinstance(cond, str) else int(cond)
    out = np.zeros(1 << (n * n), np.uint8)
    rc = _load().orc_frame_condition(c, int(n), out.ctypes.data_as(ctypes.c_void_p))
    if rc:
        raise ValueError("orc_frame_condition rc=%d" % rc)
    return out


def recover(text, N, conditions=None):
    """The library conditions whose extension equals the formula's validity
    set on every frame of 1..N worlds (Sec. 10): names, in library order."""
    conditions = CONDITIONS if conditions is None else conditions
    val = [frame_valid_all(text, n) for n in range(1, N + 1)]
    out = []
    for c in conditions:
        if all(np.array_equal(frame_condition(c, n), val[n - 1]) for n in range(1, N + 1)):
            out.append(c)
    return out
