"""Thin ctypes binding of libmk (include/mk.h): same names, marshalling only.

Every step of the evaluation runs in libmk's kernels; this module packs
arguments, lets PyTorch provide device memory and the current CUDA stream,
and unpacks results.  There is no CPU fallback: if libmk.so is missing or
no CUDA device is present, the device calls raise.
"""
import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmk.so")

MK_MAX_CODE = 96
MK_MAX_STACK = 4
MK_MAX_VARS = 4
MK_MAX_CERT_WORLDS = 32
CLASS_BITS = {"K": 1, "T": 2, "S4": 4, "S5": 8, "K4": 16}
CLASS_NAMES = ("K", "T", "S4", "S5")
NO_KEY = (1 << 64) - 1


class MkError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, strerror(code) if _lib else "libmk", code))


class mk_program(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_uint16), ("n_instr", ctypes.c_uint8), ("nvars", ctypes.c_uint8),
                ("modal_depth", ctypes.c_uint8), ("depth", ctypes.c_uint8),
                ("n_modal", ctypes.c_uint8), ("n_bool", ctypes.c_uint8),
                ("code", ctypes.c_uint8 * MK_MAX_CODE)]


class mk_tune(ctypes.Structure):
    _fields_ = [("block", ctypes.c_uint16), ("tile", ctypes.c_uint16), ("units", ctypes.c_uint16),
                ("persistent", ctypes.c_uint16)]


class mk_census_cfg(ctypes.Structure):
    _fields_ = [("classes", ctypes.c_uint32), ("n_min", ctypes.c_uint8), ("n_max", ctypes.c_uint8),
                ("max_depth", ctypes.c_uint8), ("max_vars", ctypes.c_uint8), ("samples", ctypes.c_uint32),
                ("vsplit", ctypes.c_uint32), ("d_samples", ctypes.c_void_p),
                ("frame_lo", ctypes.c_uint64), ("frame_hi", ctypes.c_uint64), ("tune", mk_tune)]


class mk_result(ctypes.Structure):
    _fields_ = [("cm_count", ctypes.c_uint64), ("frames_refuted", ctypes.c_uint64),
                ("witness_key", ctypes.c_uint64)]


class mk_cert(ctypes.Structure):
    _fields_ = [("phi", ctypes.c_char_p), ("psi", ctypes.c_char_p), ("n", ctypes.c_uint8),
                ("cls", ctypes.c_uint8), ("world", ctypes.c_uint8), ("reserved", ctypes.c_uint8),
                ("succ", ctypes.c_uint32 * MK_MAX_CERT_WORLDS), ("val", ctypes.c_uint32 * MK_MAX_VARS)]


class mk_job(ctypes.Structure):
    _fields_ = [("prog", ctypes.c_int32), ("cls", ctypes.c_uint8), ("n_max", ctypes.c_uint8),
                ("reserved", ctypes.c_uint16)]


class mk_plan_info(ctypes.Structure):
    _fields_ = [("bytes", ctypes.c_uint64), ("nitems", ctypes.c_uint32), ("nlist", ctypes.c_uint32),
                ("list_off", ctypes.c_uint32), ("items_off", ctypes.c_uint32), ("n_max", ctypes.c_uint8),
                ("max_depth", ctypes.c_uint8), ("block", ctypes.c_uint16), ("units", ctypes.c_uint16),
                ("tile_cap", ctypes.c_uint16), ("ops", ctypes.c_double)]


JOB_DTYPE = np.dtype([("prog", "<i4"), ("cls", "u1"), ("n_max", "u1"), ("reserved", "<u2")])
MODEL_DTYPE = np.dtype([("frame", "<u8"), ("val", "<u4"), ("n", "u1"), ("world", "u1"), ("reserved", "<u2")])


class mk_separate_cfg(ctypes.Structure):
    _fields_ = [("n_exh_min", ctypes.c_uint8), ("n_exh_max", ctypes.c_uint8),
                ("n_smp_min", ctypes.c_uint8), ("n_smp_max", ctypes.c_uint8),
                ("samples", ctypes.c_uint32), ("d_samples", ctypes.c_void_p),
                ("frames_per_n", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("frame_lo", ctypes.c_uint64), ("frame_hi", ctypes.c_uint64), ("tune", mk_tune),
                ("max_depth", ctypes.c_uint8)]


PROGRAM_DTYPE = np.dtype([("nodes", "<u2"), ("n_instr", "u1"), ("nvars", "u1"), ("modal_depth", "u1"),
                          ("depth", "u1"), ("n_modal", "u1"), ("n_bool", "u1"),
                          ("code", "u1", (MK_MAX_CODE,))])
assert PROGRAM_DTYPE.itemsize == ctypes.sizeof(mk_program) == 104

_lib = None
_lock = threading.Lock()

class mk_stress_cfg(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("count_splits", ctypes.c_int32), ("count", ctypes.c_uint64),
                ("index_base", ctypes.c_uint64), ("tune", mk_tune)]


_SIGS = {
    "mk_compile": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(mk_program), ctypes.POINTER(ctypes.c_int32)]),
    "mk_compile_iff": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(mk_program),
                                      ctypes.POINTER(ctypes.c_int32)]),
    "mk_census_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(mk_census_cfg), ctypes.c_int32]),
    "mk_census": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(mk_census_cfg),
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                 ctypes.c_void_p]),
    "mk_class_frames": (ctypes.c_uint64, [ctypes.c_uint32, ctypes.c_int32]),
    "mk_certify": (ctypes.c_int, [ctypes.POINTER(mk_cert)]),
    "mk_witness_cert": (ctypes.c_int, [ctypes.POINTER(mk_program), ctypes.c_char_p, ctypes.c_uint32,
                                       ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64,
                                       ctypes.POINTER(mk_cert)]),
    "mk_separate_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(mk_separate_cfg), ctypes.c_int32]),
    "mk_separate_launches": (ctypes.c_int64, [ctypes.POINTER(mk_separate_cfg), ctypes.c_int32]),
    "mk_separate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.POINTER(mk_separate_cfg), ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "mk_sample_relation": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint64]),
    "mk_split_cert": (ctypes.c_int, [ctypes.POINTER(mk_program), ctypes.POINTER(mk_program), ctypes.c_char_p,
                                     ctypes.c_char_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                     ctypes.c_uint64, ctypes.POINTER(mk_cert)]),
    "mk_census_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(mk_census_cfg),
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "mk_census_launches": (ctypes.c_int32, [ctypes.POINTER(mk_census_cfg), ctypes.c_int32]),
    "mk_calibrate_lop3": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32,
                                         ctypes.c_uint32, ctypes.c_void_p]),
    "mk_calibrate_ops_per_launch": (ctypes.c_uint64, [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32]),
    "mk_plan_uneven": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.c_uint32, ctypes.c_void_p, ctypes.POINTER(mk_tune), ctypes.c_void_p,
                                      ctypes.c_size_t, ctypes.POINTER(mk_plan_info)]),
    "mk_uneven_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(mk_plan_info)]),
    "mk_census_uneven": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.POINTER(mk_plan_info), ctypes.c_uint32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                        ctypes.c_void_p]),
    "mk_fingerprint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "mk_knn_workspace_size": (ctypes.c_size_t, [ctypes.c_int32]),
    "mk_hamming_knn": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.c_void_p]),
    "mk_mlp_param_count": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32]),
    "mk_mlp_workspace_size": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32]),
    "mk_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "mk_mlp_train_workspace_size": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "mk_mlp_gradient": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_size_t, ctypes.c_void_p]),
    "mk_adam_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_size_t, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_int32, ctypes.c_float, ctypes.c_void_p]),
    "mk_mlp_infer_workspace_size": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "mk_mlp_infer_bf16": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "mk_template": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
    "mk_stress_relation": (ctypes.c_int, [ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint64,
                                          ctypes.c_void_p]),
    "mk_relation_words": (ctypes.c_uint64, [ctypes.c_int32, ctypes.c_uint64]),
    "mk_generate_relations": (ctypes.c_int, [ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint64,
                                             ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "mk_pack_relations": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "mk_stress_separate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.POINTER(mk_stress_cfg), ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "mk_frame_words": (ctypes.c_uint64, [ctypes.c_int32]),
    "mk_frame_validity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]),
    "mk_frame_conditions": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "mk_bitmap_mismatch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p,
                                          ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]),
    "mk_atlas_counts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]),
    "mk_atlas_gram": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "mk_power_workspace_size": (ctypes.c_size_t, [ctypes.c_int32]),
    "mk_power_iteration": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_size_t, ctypes.c_void_p]),
    "mk_atlas_project": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "mk_sort_workspace_size": (ctypes.c_size_t, [ctypes.c_int32]),
    "mk_sort_keys": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_size_t, ctypes.c_void_p]),
    "mk_adjacent_variation": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "mk_histogram2d": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "mk_histogram_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "mk_mlp_infer_tc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "mk_mlp_w1t_bf16": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "mk_mlp_layer1_tc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "mk_mlp_layer1_mma": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "mk_mlp_w1_tiles_bytes": (ctypes.c_size_t, [ctypes.c_int32]),
    "mk_mlp_w1_tiles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "mk_mlp_layer1_tc_ws": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "mk_mlp_layer1_tc_ws_bounded": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                                   ctypes.c_void_p]),
    "mk_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "mk_status_error": (ctypes.c_int, [ctypes.c_int32]),
    "mk_version": (ctypes.c_int, []),
}


def lib():
    """Load libmk.so (built by paper_2606_15437_gb300.build); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise OSError("libmk.so not built: run paper_2606_15437_gb300.build.build() "
                              "(or __graft_entry__.build())")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def declared_symbols():
    return list(_SIGS)


def strerror(code):
    return lib().mk_strerror(code).decode()


def _check(rc, what):
    if rc != 0:
        raise MkError(rc, what)


# ------------------------------------------------------------ compile

def compile(text):
    """mk_compile: formula text -> mk_program."""
    p = mk_program()
    pos = ctypes.c_int32(-1)
    rc = lib().mk_compile(text.encode(), ctypes.byref(p), ctypes.byref(pos))
    if rc != 0:
        raise MkError(rc, "mk_compile(%r) at %d" % (text, pos.value))
    return p


def compile_iff(phi, psi):
    p = mk_program()
    pos = ctypes.c_int32(-1)
    _check(lib().mk_compile_iff(phi.encode(), psi.encode(), ctypes.byref(p), ctypes.byref(pos)),
           "mk_compile_iff")
    return p


def compile_batch(texts):
    """Compile many texts into a numpy array of PROGRAM_DTYPE records."""
    out = np.zeros(len(texts), PROGRAM_DTYPE)
    buf = out.view(np.uint8).reshape(len(texts), PROGRAM_DTYPE.itemsize)
    for i, t in enumerate(texts):
        p = compile(t)
        buf[i] = np.frombuffer(bytes(p), np.uint8)
    return out


def program_at(progs, i):
    return mk_program.from_buffer_copy(progs[i:i + 1].tobytes())


# ------------------------------------------------------------- census

def class_mask(classes):
    m = 0
    for c in classes:
        m |= CLASS_BITS[c]
    return m


def census_cfg(classes, n_min, n_max, samples=0, d_samples=0, frame_lo=0, frame_hi=NO_KEY, tune=None,
               max_depth=0, vsplit=0, max_vars=0):
    """An mk_census_cfg (field meanings in include/mk.h)."""
    cfg = mk_census_cfg()
    cfg.max_depth = max_depth
    cfg.max_vars = max_vars
    cfg.vsplit = vsplit
    cfg.classes = class_mask(classes) if not isinstance(classes, int) else classes
    cfg.n_min, cfg.n_max = n_min, n_max
    cfg.samples = samples
    cfg.d_samples = d_samples or None
    cfg.frame_lo, cfg.frame_hi = frame_lo, frame_hi
    if tune:
        for k, v in tune.items():
            setattr(cfg.tune, k, v)
    return cfg


def census_workspace_size(cfg, nprog):
    return int(lib().mk_census_workspace_size(ctypes.byref(cfg), nprog))


def census_raw(d_progs, nprog, cfg, d_out, d_status, d_ws, ws_bytes, stream):
    """mk_census on raw device pointers (ints) and a cudaStream_t (int)."""
    _check(lib().mk_census(d_progs, nprog, ctypes.byref(cfg), d_out, d_status, d_ws, ws_bytes, stream),
           "mk_census")


def census_noalloc_raw(d_progs, nprog, cfg, d_out, d_status, stream):
    """mk_census_noalloc: the census with the library's own fixed scratch
    array instead of a caller workspace (for callers that cannot allocate
    device memory).  Returns the library's code (0 = ok)."""
    return int(lib().mk_census_noalloc(d_progs, nprog, ctypes.byref(cfg), d_out, d_status, stream))


def census_launches(cfg, nprog):
    return int(lib().mk_census_launches(ctypes.byref(cfg), nprog))


def calibrate_lop3(d_sink, blocks, threads, iters, seed, stream):
    _check(lib().mk_calibrate_lop3(d_sink, blocks, threads, iters, seed, stream), "mk_calibrate_lop3")
    return int(lib().mk_calibrate_ops_per_launch(blocks, threads, iters))


def class_frames(cls, n):
    return int(lib().mk_class_frames(CLASS_BITS[cls] if isinstance(cls, str) else cls, n))


def status_error(status):
    return int(lib().mk_status_error(int(status)))


def decode_key(key):
    """Census witness key -> (frame, valuation index or slot, world)."""
    if key == NO_KEY:
        return None
    return (key >> 27, (key >> 3) & 0xFFFFFF, key & 7)


def decode_split(key):
    """Separation key -> (n, frame or sample, valuation, world)."""
    if key == NO_KEY:
        return None
    return (split_n(key), (key >> 24) & ((1 << 36) - 1), (key >> 3) & ((1 << 21) - 1), key & 7)


def split_n(key):
    """Worlds of the split a separation key encodes (0 for no split)."""
    key = int(key)
    return 0 if key == NO_KEY else ((key >> 60) & 7) + 1


def split_sampled(key):
    """True if the split was found on a sampled relation (not a K index)."""
    return int(key) != NO_KEY and bool(int(key) >> 63)


def split_key(sampled, n, f, x, w):
    """The separation key mk_separate writes for a split."""
    return (int(bool(sampled)) << 63) | ((n - 1) << 60) | (f << 24) | (x << 3) | w


# ------------------------------------------------------- certificates

def certify(phi, n, succ, val=(), world=0, cls=0, psi=None):
    """mk_certify on an explicit certificate; returns 1 / 0 (or raises)."""
    c = mk_cert()
    c.phi = phi.encode()
    c.psi = psi.encode() if psi is not None else None
    c.n, c.cls, c.world = n, (CLASS_NAMES.index(cls) if isinstance(cls, str) else cls), world
    for i, s in enumerate(succ):
        c.succ[i] = s
    for i, v in enumerate(val):
        c.val[i] = v
    rc = lib().mk_certify(ctypes.byref(c))
    if rc < 0:
        raise MkError(rc, "mk_certify")
    return rc


def certify_struct(c):
    return lib().mk_certify(ctypes.byref(c))


def witness_cert(prog, phi, cls, n, samples, h_samples_n, key):
    c = mk_cert()
    keep = None
    ptr = None
    if h_samples_n is not None:
        keep = np.ascontiguousarray(np.asarray(h_samples_n, np.uint32))
        ptr = keep.ctypes.data_as(ctypes.c_void_p)
    phi_b = phi.encode()
    _check(lib().mk_witness_cert(ctypes.byref(prog), phi_b, CLASS_BITS[cls], n, samples, ptr, key,
                                 ctypes.byref(c)), "mk_witness_cert")
    c._keep = (phi_b, keep)
    return c


def split_cert(prog_a, prog_b, phi, psi, seed, samples, h_samples_n, key):
    c = mk_cert()
    keep = None
    ptr = None
    if h_samples_n is not None:
        keep = np.ascontiguousarray(np.asarray(h_samples_n, np.uint32))
        ptr = keep.ctypes.data_as(ctypes.c_void_p)
    a, b = phi.encode(), psi.encode()
    _check(lib().mk_split_cert(ctypes.byref(prog_a), ctypes.byref(prog_b), a, b, seed, samples, ptr, key,
                               ctypes.byref(c)), "mk_split_cert")
    c._keep = (a, b, keep)
    return c


def sample_relation(seed, n, s):
    return int(lib().mk_sample_relation(seed, n, s))


# --------------------------------------------------------- separation

def separate_cfg(n_exh_min=1, n_exh_max=6, n_smp_min=0, n_smp_max=0, samples=0, d_samples=0,
                 frames_per_n=0, seed=0, frame_lo=0, frame_hi=NO_KEY, tune=None, max_depth=0):
    cfg = mk_separate_cfg()
    cfg.max_depth = max_depth
    cfg.n_exh_min, cfg.n_exh_max = n_exh_min, n_exh_max
    cfg.n_smp_min, cfg.n_smp_max = n_smp_min, n_smp_max
    cfg.samples = samples
    cfg.d_samples = d_samples or None
    cfg.frames_per_n, cfg.seed = frames_per_n, seed
    cfg.frame_lo, cfg.frame_hi = frame_lo, frame_hi
    if tune:
        for k, v in tune.items():
            setattr(cfg.tune, k, v)
    return cfg


def separate_raw(d_phi, d_psi, npairs, cfg, d_split, d_status, d_ws, ws_bytes, stream):
    _check(lib().mk_separate(d_phi, d_psi, npairs, ctypes.byref(cfg), d_split, d_status, d_ws, ws_bytes,
                             stream), "mk_separate")


def separate_workspace_size(cfg, npairs):
    return int(lib().mk_separate_workspace_size(ctypes.byref(cfg), npairs))


def separate_launches(cfg, npairs):
    """Kernel launches of one mk_separate call (its own count)."""
    return int(lib().mk_separate_launches(ctypes.byref(cfg), npairs))


# ------------------------------------------------------ uneven batches

def plan_uneven(progs, jobs, samples, tiles=None, tune=None):
    """mk_plan_uneven: returns (plan bytes as a numpy uint8 array, mk_plan_info)."""
    progs = np.ascontiguousarray(progs)
    jobs = np.ascontiguousarray(jobs)
    info = mk_plan_info()
    t = mk_tune()
    if tune:
        for k, v in tune.items():
            setattr(t, k, v)
    tl = None if tiles is None else np.ascontiguousarray(np.asarray(tiles, np.uint16))
    tl_ptr = None if tl is None else tl.ctypes.data_as(ctypes.c_void_p)
    args = (progs.ctypes.data_as(ctypes.c_void_p), len(progs), jobs.ctypes.data_as(ctypes.c_void_p),
            len(jobs), samples, tl_ptr, ctypes.byref(t))
    _check(lib().mk_plan_uneven(*args, None, 0, ctypes.byref(info)), "mk_plan_uneven")
    plan = np.zeros(int(info.bytes), np.uint8)
    _check(lib().mk_plan_uneven(*args, plan.ctypes.data_as(ctypes.c_void_p), plan.nbytes, ctypes.byref(info)),
           "mk_plan_uneven")
    return plan, info


def uneven_workspace_size(info):
    return int(lib().mk_uneven_workspace_size(ctypes.byref(info)))


def census_uneven_raw(d_progs, d_jobs, njobs, d_plan, info, samples, d_samples, d_out, d_status, d_ws,
                      ws_bytes, stream):
    _check(lib().mk_census_uneven(d_progs, d_jobs, njobs, d_plan, ctypes.byref(info), samples, d_samples,
                                  d_out, d_status, d_ws, ws_bytes, stream), "mk_census_uneven")


# ------------------------------------------------------- learned proposal

def fingerprint_raw(d_progs, nprog, d_models, group_n, d_bits, d_status, stream):
    g = np.ascontiguousarray(np.asarray(group_n, np.int32))
    _check(lib().mk_fingerprint(d_progs, nprog, d_models, g.ctypes.data_as(ctypes.c_void_p), len(g), d_bits,
                                d_status, stream), "mk_fingerprint")


def knn_workspace_size(nvec):
    return int(lib().mk_knn_workspace_size(nvec))


def hamming_knn_raw(d_bits, nvec, words, k, d_nbr, d_dist, d_ws, ws_bytes, stream):
    _check(lib().mk_hamming_knn(d_bits, nvec, words, k, d_nbr, d_dist, d_ws, ws_bytes, stream), "mk_hamming_knn")


def mlp_param_count(features, hidden):
    return int(lib().mk_mlp_param_count(features, hidden))


def mlp_forward_raw(d_params, features, hidden, d_vec, d_pa, d_pb, batch, d_logits, d_ws, ws_bytes, stream):
    _check(lib().mk_mlp_forward(d_params, features, hidden, d_vec, d_pa, d_pb, batch, d_logits, d_ws, ws_bytes,
                                stream), "mk_mlp_forward")


def mlp_workspace_size(batch, hidden):
    return int(lib().mk_mlp_workspace_size(batch, hidden))


def mlp_train_workspace_size(batch, features, hidden):
    return int(lib().mk_mlp_train_workspace_size(batch, features, hidden))


def mlp_gradient_raw(d_params, features, hidden, d_vec, d_pa, d_pb, d_y, d_w, batch, d_grad, d_loss, d_ws,
                     ws_bytes, stream):
    _check(lib().mk_mlp_gradient(d_params, features, hidden, d_vec, d_pa, d_pb, d_y, d_w, batch, d_grad, d_loss,
                                 d_ws, ws_bytes, stream), "mk_mlp_gradient")


def adam_step_raw(d_params, d_grad, d_m, d_v, n, lr, beta1, beta2, eps, step, grad_scale, stream):
    _check(lib().mk_adam_step(d_params, d_grad, d_m, d_v, n, lr, beta1, beta2, eps, step, grad_scale, stream),
           "mk_adam_step")


def mlp_infer_workspace_size(batch, features, hidden):
    return int(lib().mk_mlp_infer_workspace_size(batch, features, hidden))


def mlp_infer_bf16_raw(d_params, features, hidden, d_vec, d_pa, d_pb, batch, d_logits, d_ws, ws_bytes, stream):
    _check(lib().mk_mlp_infer_bf16(d_params, features, hidden, d_vec, d_pa, d_pb, batch, d_logits, d_ws, ws_bytes,
                                   stream), "mk_mlp_infer_bf16")


def mlp_infer_tc_raw(d_params, features, hidden, d_vec, d_pa, d_pb, batch, d_logits, d_status, d_ws, ws_bytes,
                     stream):
    _check(lib().mk_mlp_infer_tc(d_params, features, hidden, d_vec, d_pa, d_pb, batch, d_logits, d_status, d_ws,
                                 ws_bytes, stream), "mk_mlp_infer_tc")


def mlp_w1t_bf16_raw(d_params, features, hidden, d_w1t, stream):
    _check(lib().mk_mlp_w1t_bf16(d_params, features, hidden, d_w1t, stream), "mk_mlp_w1t_bf16")


def mlp_layer1_tc_raw(d_vec, features, d_pa, d_pb, batch, d_w1t, d_b1, d_h1, d_status, stream):
    _check(lib().mk_mlp_layer1_tc(d_vec, features, d_pa, d_pb, batch, d_w1t, d_b1, d_h1, d_status, stream),
           "mk_mlp_layer1_tc")


def mlp_w1_tiles_bytes(features):
    return int(lib().mk_mlp_w1_tiles_bytes(int(features)))


def mlp_w1_tiles_raw(d_params, features, hidden, d_tiles, stream):
    _check(lib().mk_mlp_w1_tiles(d_params, features, hidden, d_tiles, stream), "mk_mlp_w1_tiles")


def mlp_layer1_tc_ws_raw(d_vec, features, d_pa, d_pb, batch, d_tiles, d_b1, d_h1, d_status, stream):
    _check(lib().mk_mlp_layer1_tc_ws(d_vec, features, d_pa, d_pb, batch, d_tiles, d_b1, d_h1, d_status, stream),
           "mk_mlp_layer1_tc_ws")


def mlp_layer1_tc_ws_bounded_raw(d_vec, features, d_pa, d_pb, batch, d_tiles, d_b1, d_h1, d_status, wait_spins,
                                 stream):
    _check(lib().mk_mlp_layer1_tc_ws_bounded(d_vec, features, d_pa, d_pb, batch, d_tiles, d_b1, d_h1, d_status,
                                             wait_spins, stream), "mk_mlp_layer1_tc_ws_bounded")


def mlp_layer1_mma_raw(d_vec, features, d_pa, d_pb, batch, d_w1t, d_b1, d_h1, stream):
    _check(lib().mk_mlp_layer1_mma(d_vec, features, d_pa, d_pb, batch, d_w1t, d_b1, d_h1, stream),
           "mk_mlp_layer1_mma")


# ------------------------------------------------------------ large frames
NUM_TEMPLATES = 39
GENERATORS = ("er", "flip", "scc", "deadend", "backedge", "permscc")


def gen_index(gen):
    return GENERATORS.index(gen) if isinstance(gen, str) else int(gen)


def template(tid, n):
    """Successor masks of stress template ``tid`` on n worlds (host)."""
    out = (ctypes.c_uint32 * 16)()
    _check(lib().mk_template(int(tid), int(n), out), "mk_template")
    return [int(out[w]) for w in range(n)]


def stress_relation(gen, seed, n, s):
    """Successor masks of relation ``s`` of generator ``gen`` (host)."""
    out = (ctypes.c_uint32 * 16)()
    _check(lib().mk_stress_relation(gen_index(gen), int(seed), int(n), int(s), out), "mk_stress_relation")
    return [int(out[w]) for w in range(n)]


def relation_words(n, count):
    return int(lib().mk_relation_words(int(n), int(count)))


def generate_relations_raw(gen, seed, n, first, count, d_words, d_succ, stream):
    _check(lib().mk_generate_relations(gen_index(gen), int(seed), int(n), int(first), int(count), d_words,
                                       d_succ, stream), "mk_generate_relations")


def pack_relations_raw(d_succ, n, count, d_words, stream):
    _check(lib().mk_pack_relations(d_succ, int(n), int(count), d_words, stream), "mk_pack_relations")


def stress_cfg(n, count, index_base=0, count_splits=False, tile=0):
    c = mk_stress_cfg()
    c.n, c.count, c.index_base, c.count_splits = int(n), int(count), int(index_base), int(bool(count_splits))
    c.tune.tile = int(tile)
    return c


def stress_separate_raw(d_phi, d_psi, npairs, d_words, cfg, d_key, d_nsplit, d_status, stream):
    _check(lib().mk_stress_separate(d_phi, d_psi, int(npairs), d_words, ctypes.byref(cfg), d_key, d_nsplit,
                                    d_status, stream), "mk_stress_separate")


def decode_stress_key(key):
    """(relation index, valuation, world) of a key mk_stress_separate wrote,
    None for no split."""
    key = int(key)
    if key == NO_KEY:
        return None
    return key >> 20, (key >> 4) & 0xFFFF, key & 15


# ----------------------------------------------------- frame correspondents
CONDITION_NAMES = ("every frame", "no frame", "reflexive", "irreflexive", "serial", "transitive", "symmetric",
                   "Euclidean", "partially functional", "functional", "dense", "directed", "antisymmetric",
                   "asymmetric", "weakly connected", "shift reflexive", "empty relation", "coreflexive")


def frame_words(n):
    return int(lib().mk_frame_words(int(n)))


def frame_validity_raw(d_progs, nprog, n, max_depth, d_bits, ld_words, d_status, stream):
    _check(lib().mk_frame_validity(d_progs, int(nprog), int(n), int(max_depth), d_bits, int(ld_words), d_status,
                                   stream), "mk_frame_validity")


def frame_conditions_raw(n, d_bits, ld_words, stream):
    _check(lib().mk_frame_conditions(int(n), d_bits, int(ld_words), stream), "mk_frame_conditions")


def bitmap_mismatch_raw(d_a, na, lda, d_b, nb, ldb, d_conj, nconj, words, d_out, stream):
    _check(lib().mk_bitmap_mismatch(d_a, int(na), int(lda), d_b, int(nb), int(ldb), d_conj, int(nconj), int(words),
                                    d_out, stream), "mk_bitmap_mismatch")


# ------------------------------------------------------ failure-density atlas
def atlas_counts_raw(d_progs, nprog, n, d_counts, ld, d_status, stream):
    _check(lib().mk_atlas_counts(d_progs, int(nprog), int(n), d_counts, int(ld), d_status, stream), "mk_atlas_counts")


def atlas_gram_raw(d_counts, d_denom, B, F, ld, d_mean, d_gram, stream):
    _check(lib().mk_atlas_gram(d_counts, d_denom, int(B), int(F), int(ld), d_mean, d_gram, stream), "mk_atlas_gram")


def power_workspace_size(F):
    return int(lib().mk_power_workspace_size(int(F)))


def power_iteration_raw(d_gram, F, d_prev, nprev, iters, d_v, d_lambda, d_ws, ws_bytes, stream):
    _check(lib().mk_power_iteration(d_gram, int(F), d_prev, int(nprev), int(iters), d_v, d_lambda, d_ws,
                                    int(ws_bytes), stream), "mk_power_iteration")


def atlas_project_raw(d_counts, d_denom, B, F, ld, d_mean, d_v, d_u, stream):
    _check(lib().mk_atlas_project(d_counts, d_denom, int(B), int(F), int(ld), d_mean, d_v, d_u, stream),
           "mk_atlas_project")


def sort_workspace_size(n):
    return int(lib().mk_sort_workspace_size(int(n)))


def sort_keys_raw(d_keys, n, d_order, d_ws, ws_bytes, stream):
    _check(lib().mk_sort_keys(d_keys, int(n), d_order, d_ws, int(ws_bytes), stream), "mk_sort_keys")


def adjacent_variation_raw(d_counts, B, F, ld, d_perm, d_rowsum, d_status, stream):
    _check(lib().mk_adjacent_variation(d_counts, int(B), int(F), int(ld), d_perm, d_rowsum, d_status, stream),
           "mk_adjacent_variation")


def histogram2d_raw(d_x, d_y, npts, lo, hi, G, d_hist, stream):
    _check(lib().mk_histogram2d(d_x, d_y, int(npts), float(lo), float(hi), int(G), d_hist, stream), "mk_histogram2d")


def histogram_stats_raw(d_hist, G, radius, d_stats, stream):
    _check(lib().mk_histogram_stats(d_hist, int(G), int(radius), d_stats, stream), "mk_histogram_stats")
