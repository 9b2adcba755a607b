"""Python driver over libmk: device buffers from PyTorch, kernels from libmk.

``CensusJob`` and ``SeparateJob`` own the device memory of one batch
(programs, sampled valuations, workspace, outputs, status word) and call the
C ABI on the current torch CUDA stream.  Host-side steps are marshalling
only: compiling texts (mk_compile), uploading, launching, downloading, and
re-checking every reported witness with mk_certify.
"""
import numpy as np
import torch

from . import mk, workloads

CLASSES = ("K", "T", "S4", "S5")


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dev_bytes(arr, device):
    """Upload a numpy array as a uint8 device tensor."""
    t = torch.from_numpy(np.ascontiguousarray(arr).view(np.uint8).reshape(-1).copy())
    return t.to(device)


class CensusJob:
    """One census batch: texts x classes x n in [n_min, n_max]."""

    def __init__(self, texts=None, classes=CLASSES, n_min=1, n_max=5, samples=256, seed=2,
                 device="cuda", tune=None, frame_lo=0, frame_hi=mk.NO_KEY, progs=None,
                 sample_table=None):
        if not torch.cuda.is_available():
            raise RuntimeError("CensusJob needs a CUDA device (there is no CPU fallback)")
        self.texts = list(texts) if texts is not None else None
        self.progs = progs if progs is not None else mk.compile_batch(self.texts)
        self.nprog = len(self.progs)
        self.classes = tuple(c for c in CLASSES if c in classes)
        self.n_min, self.n_max = n_min, n_max
        self.S = samples
        self.seed = seed
        self.device = torch.device(device)
        if samples:
            self.sample_table = (sample_table if sample_table is not None
                                 else workloads.valuation_table(seed, samples, n_max))
        else:
            self.sample_table = None
        self.d_progs = _dev_bytes(self.progs, self.device)
        self.d_samples = (_dev_bytes(self.sample_table, self.device) if samples else None)
        depth = int(self.progs["depth"].max()) if self.nprog else 0
        self.cfg = mk.census_cfg(self.classes, n_min, n_max, samples,
                                 self.d_samples.data_ptr() if samples else 0, frame_lo, frame_hi, tune,
                                 max_depth=max(depth, 1))
        self.ws_bytes = mk.census_workspace_size(self.cfg, self.nprog)
        if self.ws_bytes == 0:
            raise mk.MkError(-5, "mk_census_workspace_size")
        self.d_ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.nn = n_max - n_min + 1
        self.d_out = torch.empty(self.nprog * len(self.classes) * self.nn * 3, dtype=torch.int64,
                                 device=self.device)
        self.d_status = torch.zeros(1, dtype=torch.int32, device=self.device)

    def launch(self, stream=None):
        """Enqueue the whole census on the stream (no synchronisation)."""
        self.d_status.zero_()
        mk.census_raw(self.d_progs.data_ptr(), self.nprog, self.cfg, self.d_out.data_ptr(),
                      self.d_status.data_ptr(), self.d_ws.data_ptr(), self.ws_bytes, _stream_ptr(stream))

    def check_status(self):
        st = int(self.d_status.item())
        if st:
            raise mk.MkError(mk.status_error(st), "device status 0x%x" % st)

    def results(self):
        """uint64[nprog, ncls, nn, 3]: (cm_count, frames_refuted, witness_key)."""
        torch.cuda.synchronize(self.device)
        self.check_status()
        out = self.d_out.cpu().numpy().view(np.uint64)
        return out.reshape(self.nprog, len(self.classes), self.nn, 3)

    def run(self):
        self.launch()
        return self.results()

    def evals(self):
        """Formula-frame-valuation evaluations in this census (algorithmic count)."""
        total = 0
        for p in self.progs:
            k = int(p["nvars"])
            for c in self.classes:
                for n in range(self.n_min, self.n_max + 1):
                    total += mk.class_frames(c, n) * n_valuations(k, n, self.S)
        return total

    def certificate(self, p, cls, n, key):
        """mk_cert for the witness key of program p on layer (cls, n)."""
        samples_n = self.sample_table[n] if self.S else None
        return mk.witness_cert(mk.program_at(self.progs, p), self.texts[p], cls, n, self.S, samples_n, key)


def n_valuations(k, n, S):
    """Valuations per frame of a k-variable formula on layer n."""
    if S == 0 or k <= 1 or (k * n < 32 and (1 << (k * n)) <= S):
        return 1 << (k * n)
    return S


def lop3_per_eval(prog, n):
    """Algorithmic logic ops per evaluation of the bit-sliced recurrence:
    n per Boolean connective, n*n per modal operator, n for the refutation
    test, all shared by 32 frames (one 32-bit word)."""
    return (n * int(prog["n_bool"]) + n * n * int(prog["n_modal"]) + n) / 32.0


class SeparateJob:
    """Distinguishing-pair search for a list of (phi, psi) texts."""

    def __init__(self, pairs, n_exh_min=1, n_exh_max=6, n_smp_min=0, n_smp_max=0, frames_per_n=0,
                 seed=4, samples=0, device="cuda", tune=None, frame_lo=0, frame_hi=mk.NO_KEY):
        if not torch.cuda.is_available():
            raise RuntimeError("SeparateJob needs a CUDA device (there is no CPU fallback)")
        self.pairs = list(pairs)
        self.npairs = len(self.pairs)
        self.pa = mk.compile_batch([a for a, _ in self.pairs])
        self.pb = mk.compile_batch([b for _, b in self.pairs])
        self.device = torch.device(device)
        self.seed = seed
        self.S = samples
        self.sample_table = workloads.valuation_table(seed, samples, 8) if samples else None
        self.d_pa = _dev_bytes(self.pa, self.device)
        self.d_pb = _dev_bytes(self.pb, self.device)
        self.d_samples = _dev_bytes(self.sample_table, self.device) if samples else None
        self.cfg = mk.separate_cfg(n_exh_min, n_exh_max, n_smp_min, n_smp_max, samples,
                                   self.d_samples.data_ptr() if samples else 0, frames_per_n, seed,
                                   frame_lo, frame_hi, tune)
        self.ws_bytes = mk.separate_workspace_size(self.cfg, self.npairs)
        self.d_ws = torch.empty(max(self.ws_bytes, 1), dtype=torch.uint8, device=self.device)
        self.d_split = torch.empty(self.npairs, dtype=torch.int64, device=self.device)
        self.d_status = torch.zeros(1, dtype=torch.int32, device=self.device)

    def launch(self, stream=None):
        self.d_status.zero_()
        mk.separate_raw(self.d_pa.data_ptr(), self.d_pb.data_ptr(), self.npairs, self.cfg,
                        self.d_split.data_ptr(), self.d_status.data_ptr(), self.d_ws.data_ptr(),
                        self.ws_bytes, _stream_ptr(stream))

    def results(self):
        torch.cuda.synchronize(self.device)
        st = int(self.d_status.item())
        if st:
            raise mk.MkError(mk.status_error(st), "device status 0x%x" % st)
        return self.d_split.cpu().numpy().view(np.uint64)

    def run(self):
        self.launch()
        return self.results()

    def certificate(self, i, key):
        n = int(key) >> 60
        samples_n = self.sample_table[n] if self.S else None
        a, b = self.pairs[i]
        return mk.split_cert(mk.program_at(self.pa, i), mk.program_at(self.pb, i), a, b, self.seed,
                             self.S, samples_n, int(key))


class UnevenJob:
    """An uneven batch: every formula has its own class and n_max, all of
    them evaluated by one persistent launch over a host-built work plan
    (mk_plan_uneven / mk_census_uneven).  ``capture()`` records the whole
    call (clear, lists, queue reset, persistent kernel) as one CUDA graph."""

    def __init__(self, items, samples=64, seed=3, tiles=None, tune=None, device="cuda"):
        if not torch.cuda.is_available():
            raise RuntimeError("UnevenJob needs a CUDA device (there is no CPU fallback)")
        self.items = list(items)                       # (text, class name, n_max)
        self.texts = [t for t, _, _ in self.items]
        self.progs = mk.compile_batch(self.texts)
        self.njobs = len(self.items)
        self.jobs = np.zeros(self.njobs, mk.JOB_DTYPE)
        self.jobs["prog"] = np.arange(self.njobs)
        self.jobs["cls"] = [CLASSES.index(c) for _, c, _ in self.items]
        self.jobs["n_max"] = [n for _, _, n in self.items]
        self.S = samples
        self.seed = seed
        self.device = torch.device(device)
        self.plan, self.info = mk.plan_uneven(self.progs, self.jobs, samples, tiles, tune)
        n_max = int(self.info.n_max)
        self.sample_table = workloads.valuation_table(seed, samples, n_max) if samples else None
        self.d_progs = _dev_bytes(self.progs, self.device)
        self.d_jobs = _dev_bytes(self.jobs, self.device)
        self.d_plan = _dev_bytes(self.plan, self.device)
        self.d_samples = _dev_bytes(self.sample_table, self.device) if samples else None
        self.ws_bytes = mk.uneven_workspace_size(self.info)
        self.d_ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.d_out = torch.empty(self.njobs * 6 * 3, dtype=torch.int64, device=self.device)
        self.d_status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.graph = None

    def launch(self, stream=None):
        mk.census_uneven_raw(self.d_progs.data_ptr(), self.d_jobs.data_ptr(), self.njobs,
                             self.d_plan.data_ptr(), self.info, self.S,
                             self.d_samples.data_ptr() if self.S else None, self.d_out.data_ptr(),
                             self.d_status.data_ptr(), self.d_ws.data_ptr(), self.ws_bytes, _stream_ptr(stream))

    def capture(self):
        """Record one launch as a CUDA graph (after an uncaptured warm-up)."""
        self.launch()
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(self.device)
        with torch.cuda.graph(self.graph, stream=s):
            self.launch(s)
        return self.graph

    def replay(self):
        self.graph.replay()

    def results(self):
        """uint64[njobs, 6, 3]: (cm_count, frames_refuted, witness_key) for n = 1..6."""
        torch.cuda.synchronize(self.device)
        st = int(self.d_status.item())
        if st:
            raise mk.MkError(mk.status_error(st), "device status 0x%x" % st)
        return self.d_out.cpu().numpy().view(np.uint64).reshape(self.njobs, 6, 3)

    def evals(self):
        total = 0
        for (t, c, nmax), p in zip(self.items, self.progs):
            for n in range(1, nmax + 1):
                total += mk.class_frames(c, n) * n_valuations(int(p["nvars"]), n, self.S)
        return total

    def buckets(self):
        """Jobs grouped by (class, n_max): the per-bucket plain-launch baseline."""
        groups = {}
        for j, (t, c, nmax) in enumerate(self.items):
            groups.setdefault((c, nmax), []).append(j)
        return groups


# ------------------------------------------------------------------ autotuner

_TUNE_CACHE = None


def _cache_path():
    import os
    return os.path.join(os.path.dirname(mk.LIB_PATH), "autotune.json")


def _load_cache():
    import json
    import os
    global _TUNE_CACHE
    if _TUNE_CACHE is None:
        p = _cache_path()
        _TUNE_CACHE = json.load(open(p)) if os.path.exists(p) else {}
    return _TUNE_CACHE


def _store_cache():
    import json
    json.dump(_TUNE_CACHE, open(_cache_path(), "w"), indent=1, sort_keys=True)


def _time_graph(job, reps=2):
    job.launch()
    job.results()
    job.capture()
    torch.cuda.synchronize(job.device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        job.replay()
    e1.record()
    torch.cuda.synchronize(job.device)
    return e0.elapsed_time(e1) / reps


def autotune_uneven(items, samples=64, seed=3, sample_size=2400, device="cuda", use_cache=True, log=None):
    """Pick the persistent launch's CTA size, valuations per dispatched
    instruction (units) and formulas per tile for each length bucket.

    Coordinate descent on a stratified sample of the batch (every length
    bucket and class represented in proportion): first (units, block) with
    16-formula tiles, then each bucket's tile size in {4, 8, 16, 32, 64} with
    the others fixed; each candidate is timed as a CUDA-graph replay.  The
    choice is cached per (GPU name, SM count, samples, n_max set)."""
    props = torch.cuda.get_device_properties(torch.device(device))
    nmaxes = sorted({n for _, _, n in items})
    key = "%s|%d|uneven|S=%d|n=%s" % (props.name, props.multi_processor_count, samples, nmaxes)
    cache = _load_cache()
    if use_cache and key in cache:
        return cache[key]
    step = max(1, len(items) // sample_size)
    sample = items[::step]
    trials = []

    def run(units, block, tiles):
        job = UnevenJob(sample, samples=samples, seed=seed, tiles=tiles, tune={"units": units, "block": block},
                        device=device)
        ms = _time_graph(job)
        trials.append({"units": units, "block": block, "tiles": list(tiles), "ms": ms})
        if log:
            log("autotune units=%d block=%d tiles=%s: %.2f ms" % (units, block, tiles, ms))
        return ms

    best = None
    for units in (4, 8):
        for block in (128, 256):
            ms = run(units, block, (16, 16, 16, 16))
            if best is None or ms < best[0]:
                best = (ms, units, block, [16, 16, 16, 16])
    _, units, block, tiles = best
    for b in range(4):
        for t in (4, 8, 32, 64):
            cand = list(tiles)
            cand[b] = t
            ms = run(units, block, tuple(cand))
            if ms < best[0]:
                best = (ms, units, block, cand)
                tiles = cand
    choice = {"units": best[1], "block": best[2], "tiles": best[3], "ms_sample": best[0],
              "sample_size": len(sample), "trials": trials}
    cache[key] = choice
    _store_cache()
    return choice
