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

CLASSES = ("K", "T", "S4", "S5", "K4")


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dev_bytes(arr, device):
    """Upload a numpy array as a uint8 device tensor."""
    t = torch.from_numpy(np.ascontiguousarray(arr).view(np.uint8).reshape(-1).copy())
    return t.to(device)


class CensusJob:
    """One census batch: texts x classes x n in [n_min, n_max].

    frame_lo/frame_hi restrict every layer to frames whose K index lies in
    [frame_lo, frame_hi).  vsplit steers how a layer too small to fill the
    GPU shares its valuations over the grid (0 automatic, 1 never, v > 1
    chunks); it never changes the results."""

    def __init__(self, texts=None, classes=CLASSES, n_min=1, n_max=5, samples=256, seed=2,
                 device="cuda", tune=None, frame_lo=0, frame_hi=mk.NO_KEY, progs=None,
                 sample_table=None, vsplit=0):
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
                                 max_depth=max(depth, 1), vsplit=vsplit,
                                 max_vars=int(self.progs["nvars"].max()) if self.nprog else 0)
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


_SOURCE_OPS = None


def source_op_counts(text):
    """(Boolean connectives, modal operators) of the formula as written: the
    counts of ~, &, |, ->, <-> and of [], <> in its text (before the normal
    form and constant folding the compiler applies)."""
    global _SOURCE_OPS
    if _SOURCE_OPS is None:
        import re
        _SOURCE_OPS = re.compile(r"<->|->|\[\]|<>|~|!|&|\||\b(?:not|and|or|box|dia)\b")
    nb = nm = 0
    for t in _SOURCE_OPS.findall(text):
        if t in ("[]", "<>", "box", "dia"):
            nm += 1
        else:
            nb += 1
    return nb, nm


def source_ops_per_eval(text, n):
    """Algorithmic logic ops per evaluation counted on the source formula:
    (n * #Boolean + n^2 * #modal + n) / 32 (the bit-sliced minimum of the
    recurrence of Lemma 1 for 32 frames, with the refutation test)."""
    nb, nm = source_op_counts(text)
    return (n * nb + n * n * nm + n) / 32.0


# The five-world census as three mk_census calls over one program batch:
# the dominant K n=5 layer alone (timed on its own by the bench), K at
# n = 1..4, and T/S4/S5 at n = 1..5.
CENSUS5_CALLS = ((("K",), 5, 5), (("K",), 1, 4), (("T", "S4", "S5"), 1, 5))


def census_call_plan(progs, samples, d_samples_ptr, device, calls=CENSUS5_CALLS):
    """Configurations, workspaces and output buffers of a multi-call census
    (the caller keeps the programs and the sampled-valuation table on the
    device).  Returns one dict per call: classes, n_min, n_max, cfg, ws,
    ws_bytes, out ([nprog][classes][n][3] int64), launches."""
    nprog = len(progs)
    depth = max(1, int(progs["depth"].max())) if nprog else 1
    plan = []
    for classes, lo, hi in calls:
        bits = 0
        for c in classes:
            bits |= mk.CLASS_BITS[c]
        cfg = mk.census_cfg(bits, lo, hi, samples, d_samples_ptr, max_depth=depth)
        ws = mk.census_workspace_size(cfg, nprog)
        plan.append({"classes": classes, "n_min": lo, "n_max": hi, "cfg": cfg,
                     "ws": torch.empty(max(ws, 1), dtype=torch.uint8, device=device), "ws_bytes": ws,
                     "out": torch.empty(nprog * len(classes) * (hi - lo + 1) * 3, dtype=torch.int64, device=device),
                     "launches": mk.census_launches(cfg, nprog)})
    return plan


def run_census_plan(plan, d_progs_ptr, nprog, d_status_ptr, stream_ptr, calls=None):
    """Issues the plan's mk_census calls (all, or the given indices) on the stream."""
    for i, c in enumerate(plan):
        if calls is None or i in calls:
            mk.census_raw(d_progs_ptr, nprog, c["cfg"], c["out"].data_ptr(), d_status_ptr, c["ws"].data_ptr(),
                          c["ws_bytes"], stream_ptr)


def gather_census_plan(plan, nprog, classes=CLASSES, n_min=1, n_max=5):
    """The plan's outputs as one uint64 array [nprog][classes][n][3]
    (layers no call computed stay zero)."""
    out = np.zeros((nprog, len(classes), n_max - n_min + 1, 3), np.uint64)
    for c in plan:
        r = c["out"].cpu().numpy().view(np.uint64).reshape(nprog, len(c["classes"]), c["n_max"] - c["n_min"] + 1, 3)
        for j, cls in enumerate(c["classes"]):
            for n in range(c["n_min"], c["n_max"] + 1):
                out[:, classes.index(cls), n - n_min] = r[:, j, n - c["n_min"]]
    return out


# The uneven batch's launch configuration as the autotuner chooses it on a
# GB300 (units, CTA size, formulas per tile of the four length buckets).
UNEVEN_TUNE = {"units": 4, "block": 128, "tiles": [16, 16, 8, 16]}

# The separation workload's search: every frame of 1..6 worlds, then 1e8
# sampled relations of 7 and 8 worlds (seed 4) for pairs still unsplit.
SEPARATION_SEARCH = dict(n_exh_min=1, n_exh_max=6, n_smp_min=7, n_smp_max=8, frames_per_n=100_000_000, seed=4)


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
        depth = max([1] + [int(p["depth"]) for p in self.pa] + [int(p["depth"]) for p in self.pb])
        self.cfg = mk.separate_cfg(n_exh_min, n_exh_max, n_smp_min, n_smp_max, samples,
                                   self.d_samples.data_ptr() if samples else 0, frames_per_n, seed,
                                   frame_lo, frame_hi, tune, max_depth=depth)
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
        n = mk.split_n(key)
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

# the swept grid: valuations per dispatched instruction, CTA size, and
# formulas per tile of each of the plan's four length buckets
TUNE_UNITS = (4, 8)
TUNE_BLOCKS = (128, 256)
TUNE_TILES = (4, 8, 16, 32, 64)


def _cache_path():
    import os
    return os.path.join(os.path.dirname(mk.LIB_PATH), "autotune.json")


def _load_cache(path):
    import json
    import os
    return json.load(open(path)) if os.path.exists(path) else {}


def _store_cache(path, cache):
    import json
    import os
    tmp = "%s.tmp%d" % (path, os.getpid())
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_cache_key(gpu_name, sms, samples, n_maxes):
    """Cache key of an uneven-batch tune: the GPU (name and SM count, which
    set the waves a persistent grid fills) and the batch's shape (sampled
    valuations S and the set of n_max values, which set the layers and their
    valuation counts).  The per-bucket tile sizes are part of the tune."""
    return "%s|%d|uneven|S=%d|n=%s" % (gpu_name, int(sms), int(samples), sorted({int(n) for n in n_maxes}))


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


def autotune_uneven(items, samples=64, seed=3, sample_size=2400, device="cuda", use_cache=True, log=None,
                    cache_path=None):
    """Pick the persistent launch's CTA size, valuations per dispatched
    instruction (units) and formulas per tile for each length bucket.

    Coordinate descent on a stratified sample of the batch (every length
    bucket and class represented in proportion): first (units, block) with
    16-formula tiles, then each bucket's tile size in {4, 8, 16, 32, 64} with
    the others fixed; each candidate is timed as a CUDA-graph replay.  The
    choice is cached (``cache_path``, default beside libmk) under
    tune_cache_key(GPU name, SM count, samples, n_max set)."""
    props = torch.cuda.get_device_properties(torch.device(device))
    key = tune_cache_key(props.name, props.multi_processor_count, samples, [n for _, _, n in items])
    cache_path = cache_path or _cache_path()
    cache = _load_cache(cache_path)
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
    for units in TUNE_UNITS:
        for block in TUNE_BLOCKS:
            ms = run(units, block, (16, 16, 16, 16))
            if best is None or ms < best[0]:
                best = (ms, units, block, [16, 16, 16, 16])
    _, units, block, tiles = best
    for b in range(4):
        for t in TUNE_TILES:
            if t == tiles[b]:
                continue
            cand = list(tiles)
            cand[b] = t
            ms = run(units, block, tuple(cand))
            if ms < best[0]:
                best = (ms, units, block, cand)
                tiles = cand
    choice = {"units": best[1], "block": best[2], "tiles": best[3], "ms_sample": best[0],
              "sample_size": len(sample), "trials": trials}
    cache[key] = choice
    _store_cache(cache_path, cache)
    return choice


# ----------------------------------------------------------- learned proposal

def truth_vectors(texts=None, progs=None, models=None, groups=None, seed=5, device="cuda"):
    """uint32 device tensor [len(texts)][ngroups]: formula i's truth value at
    each seeded pointed model (mk_fingerprint)."""
    if progs is None:
        progs = mk.compile_batch(texts)
    if models is None:
        models, groups = workloads.pointed_models(seed)
    dev = torch.device(device)
    d_progs = _dev_bytes(progs, dev)
    d_models = _dev_bytes(models, dev)
    bits = torch.zeros(len(progs) * len(groups), dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    mk.fingerprint_raw(d_progs.data_ptr(), len(progs), d_models.data_ptr(), groups, bits.data_ptr(),
                       status.data_ptr(), _stream_ptr(None))
    torch.cuda.synchronize(dev)
    if int(status.item()):
        raise mk.MkError(mk.status_error(int(status.item())), "mk_fingerprint")
    return bits.view(len(progs), len(groups))


def hamming_knn(bits, k):
    """Exact k nearest neighbours of every truth vector (mk_hamming_knn):
    (neighbour indices int32 [n][k], distances uint16 [n][k]) on the host."""
    n, words = bits.shape
    dev = bits.device
    ws = torch.empty(mk.knn_workspace_size(n), dtype=torch.uint8, device=dev)
    nbr = torch.empty(n * k, dtype=torch.int32, device=dev)
    dist = torch.empty(n * k, dtype=torch.int16, device=dev)
    mk.hamming_knn_raw(bits.data_ptr(), n, words, k, nbr.data_ptr(), dist.data_ptr(), ws.data_ptr(), ws.numel(),
                       _stream_ptr(None))
    torch.cuda.synchronize(dev)
    return nbr.cpu().numpy().reshape(n, k), dist.cpu().numpy().view(np.uint16).reshape(n, k)


def knn_universe(nbr, target, seed=0):
    """Candidate pairs (i < j): the union of every formula's neighbour list,
    cut or filled with seeded random pairs to ``target`` pairs."""
    n, k = nbr.shape
    i = np.repeat(np.arange(n, dtype=np.int64), k)
    j = nbr.reshape(-1).astype(np.int64)
    ok = j >= 0
    a, b = np.minimum(i[ok], j[ok]), np.maximum(i[ok], j[ok])
    code = np.unique(a * n + b)
    rng = np.random.default_rng(seed)
    if len(code) > target:
        code = np.sort(rng.choice(code, target, replace=False))
    while len(code) < target:
        x = rng.integers(0, n, size=2 * (target - len(code)))
        y = rng.integers(0, n, size=len(x))
        keep = x != y
        extra = np.minimum(x[keep], y[keep]) * n + np.maximum(x[keep], y[keep])
        code = np.unique(np.concatenate([code, extra]))[:target] if len(code) + len(extra) >= target else \
            np.unique(np.concatenate([code, extra]))
    return (code // n).astype(np.int32), (code % n).astype(np.int32)


class MLP:
    """The pair-ranking network, trained and run by libmk's kernels
    (mk_mlp_gradient + mk_adam_step for FP32 training, mk_mlp_infer_bf16 for
    scoring).  Torch only holds the device buffers."""

    def __init__(self, features, hidden=256, seed=0, device="cuda"):
        self.F, self.H = features, hidden
        self.dev = torch.device(device)
        self.n = mk.mlp_param_count(features, hidden)
        g = torch.Generator().manual_seed(seed)
        F, H = features, hidden
        parts = [torch.randn(F * H, generator=g) * (2.0 / F) ** 0.5, torch.zeros(H),
                 torch.randn(H * H, generator=g) * (2.0 / H) ** 0.5, torch.zeros(H),
                 torch.randn(H, generator=g) * (1.0 / H) ** 0.5, torch.zeros(1)]
        self.params = torch.cat(parts).float().to(self.dev)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.step = 0

    def gradient(self, vec, pa, pb, y, w=None):
        """Loss and gradient on one batch (device tensors)."""
        B = len(pa)
        ws = torch.empty(mk.mlp_train_workspace_size(B, self.F, self.H), dtype=torch.uint8, device=self.dev)
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        mk.mlp_gradient_raw(self.params.data_ptr(), self.F, self.H, vec.data_ptr(), pa.data_ptr(), pb.data_ptr(),
                            y.data_ptr(), w.data_ptr() if w is not None else None, B, self.grad.data_ptr(),
                            loss.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(None))
        return loss

    def train(self, vec, pa, pb, y, w=None, epochs=8, batch=4096, lr=1e-3, seed=0, log=None):
        """Adam on the weighted binary cross-entropy, mean over each batch."""
        n = len(pa)
        g = torch.Generator(device="cpu").manual_seed(seed)
        history = []
        for ep in range(epochs):
            perm = torch.randperm(n, generator=g).to(self.dev)
            tot = 0.0
            for s in range(0, n, batch):
                idx = perm[s:s + batch]
                bpa, bpb, by = pa[idx].contiguous(), pb[idx].contiguous(), y[idx].contiguous()
                bw = w[idx].contiguous() if w is not None else None
                loss = self.gradient(vec, bpa, bpb, by, bw)
                self.step += 1
                mk.adam_step_raw(self.params.data_ptr(), self.grad.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                 self.n, lr, 0.9, 0.999, 1e-8, self.step, 1.0 / len(idx), _stream_ptr(None))
                tot += float(loss.item())
            history.append(tot / n)
            if log:
                log("epoch %d loss %.5f" % (ep, history[-1]))
        return history

    def forward(self, vec, pa, pb):
        """FP32 logits (mk_mlp_forward)."""
        B = len(pa)
        out = torch.empty(B, dtype=torch.float32, device=self.dev)
        ws = torch.empty(mk.mlp_workspace_size(B, self.H), dtype=torch.uint8, device=self.dev)
        mk.mlp_forward_raw(self.params.data_ptr(), self.F, self.H, vec.data_ptr(), pa.data_ptr(), pb.data_ptr(), B,
                           out.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(None))
        return out

    def score(self, vec, pa, pb, batch=152 * 256 * 4, impl="tc"):
        """BF16 tensor-core logits for many pairs: first layer on tcgen05
        (mk_mlp_infer_tc), or on warp-level mma.sync (impl="mma",
        mk_mlp_infer_bf16)."""
        n = len(pa)
        out = torch.empty(n, dtype=torch.float32, device=self.dev)
        ws = torch.empty(mk.mlp_infer_workspace_size(min(batch, max(n, 1)), self.F, self.H), dtype=torch.uint8,
                         device=self.dev)
        status = torch.zeros(1, dtype=torch.int32, device=self.dev)
        for s in range(0, n, batch):
            e = min(n, s + batch)
            if impl == "tc":
                mk.mlp_infer_tc_raw(self.params.data_ptr(), self.F, self.H, vec.data_ptr(), pa[s:e].data_ptr(),
                                    pb[s:e].data_ptr(), e - s, out[s:].data_ptr(), status.data_ptr(), ws.data_ptr(),
                                    ws.numel(), _stream_ptr(None))
            else:
                mk.mlp_infer_bf16_raw(self.params.data_ptr(), self.F, self.H, vec.data_ptr(), pa[s:e].data_ptr(),
                                      pb[s:e].data_ptr(), e - s, out[s:].data_ptr(), ws.data_ptr(), ws.numel(),
                                      _stream_ptr(None))
        st = int(status.item())
        if st:
            raise mk.MkError(mk.status_error(st), "device status 0x%x" % st)
        return out


def exact_split_search(texts, pa, pb, frames_per_n=1 << 20, seed=4, chunk=8192, device="cuda"):
    """The exact judge: mk_separate over every frame of 1..5 worlds, then
    ``frames_per_n`` sampled relations at 6, 7 and 8 worlds.  Returns (split
    keys, evaluations spent per pair up to its split or to the end)."""
    keys = np.empty(len(pa), np.uint64)
    evals = np.empty(len(pa), np.float64)
    for s in range(0, len(pa), chunk):
        e = min(len(pa), s + chunk)
        pairs = [(texts[a], texts[b]) for a, b in zip(pa[s:e], pb[s:e])]
        job = SeparateJob(pairs, 1, 5, 6, 8, frames_per_n=frames_per_n, seed=seed, device=device)
        k = job.run()
        keys[s:e] = k
        for i in range(e - s):
            nv = max(int(job.pa[i]["nvars"]), int(job.pb[i]["nvars"]))
            evals[s + i] = _evals_to_split(int(k[i]), nv, frames_per_n)
    return keys, evals


def _evals_to_split(key, k, frames_per_n):
    """Pair evaluations (frame x valuation) the search spends up to and
    including the first split, or all of them if there is none."""
    tot = 0
    last_n = 8 if key == mk.NO_KEY else mk.split_n(key)
    f = None if key == mk.NO_KEY else (key >> 24) & ((1 << 36) - 1)
    for n in range(1, 9):
        frames = (1 << (n * n)) if n <= 5 else frames_per_n
        vals = n_valuations(k, n, 0)
        if key != mk.NO_KEY and n == last_n:
            tot += (f + 1) * vals
            break
        tot += frames * vals
    return float(tot)


def identical_pairs(bits_np, pa, pb):
    """Pairs whose truth vectors are equal (only these can agree on every
    frame of at most five worlds: the models have n <= 5)."""
    return np.all(bits_np[pa] == bits_np[pb], axis=1)


def budget_walk(texts, pa, pb, order, budget, frames_per_n=1 << 20, chunk=4096, max_pairs=1_000_000, seed=4,
                log=None):
    """Check ranked pairs with the exact search, in rank order, until the
    exact-evaluation budget is spent (or max_pairs pairs are checked).
    A hit is a pair whose first split is at 6-8 worlds -- it agrees on every
    frame of at most five worlds -- and whose split certificate mk_certify
    accepts.  Returns a dict of counts."""
    spent, checked, hits, certified, late_keys = 0.0, 0, 0, 0, []
    by_n = np.zeros(9, np.int64)
    pos = 0
    while pos < min(len(order), max_pairs) and spent < budget:
        idx = order[pos:pos + chunk]
        pos += len(idx)
        keys, ev = exact_split_search(texts, pa[idx], pb[idx], frames_per_n=frames_per_n, seed=seed)
        cum = spent + np.cumsum(ev)
        take = int(np.searchsorted(cum, budget, side="right"))
        take = min(take, len(idx))
        for i in range(take):
            key = int(keys[i])
            n = mk.split_n(key)
            by_n[n] += 1
            if n >= 6:
                hits += 1
                a, b = texts[pa[idx[i]]], texts[pb[idx[i]]]
                c = mk.split_cert(mk.compile(a), mk.compile(b), a, b, seed, 0, None, key)
                certified += mk.certify_struct(c) == 1
                late_keys.append((int(idx[i]), key))
        spent = float(cum[take - 1]) if take else spent
        checked += take
        if take < len(idx):
            break
        if log:
            log("  checked %d pairs, %.3g evals, %d late splits" % (checked, spent, hits))
    return {"pairs_checked": checked, "evals": spent, "late_splits": hits, "certified": certified,
            "certified_per_1e12_evals": certified / (spent / 1e12) if spent else 0.0,
            "first_split_n_hist": by_n.tolist(), "hits": late_keys}


def proposal_experiment(n_formulas=10000, universe=5_467_766, k=1024, train_identical=100_000,
                        train_other=100_000, budget=5e13, frames_per_n=1 << 20, epochs=8, seed=5,
                        train_seed=55, methods=("mlp", "random", "random_identical", "pca10"), log=None,
                        device="cuda"):
    """The learned proposal against random, filtered-random and PCA-10
    rankings at an equal exact-evaluation budget (Sec. 9's retrieval
    protocol with a learned ranker).  "random_identical" takes the pairs with
    identical truth vectors first, in random order (only they can agree on
    every model of at most five worlds), then the rest: the best a ranker
    can do from the truth vectors without a network.  Every number comes
    from libmk kernels; torch only holds buffers (and computes the PCA-10
    comparator's projection)."""
    import time
    t0 = time.time()
    say = log or (lambda *a: None)
    texts = workloads.proposal_formulas(seed, n_formulas)
    bits = truth_vectors(texts, seed=seed, device=device)
    bits_np = bits.cpu().numpy().view(np.uint32)
    nbr, _ = hamming_knn(bits, k)
    pa, pb = knn_universe(nbr, universe, seed)
    say("test universe: %d pairs (%.1f s)" % (len(pa), time.time() - t0))

    # training pairs from a disjoint corpus, labelled by the exact search
    ttexts = workloads.proposal_formulas(train_seed, n_formulas)
    tbits = truth_vectors(ttexts, seed=seed, device=device)
    tbits_np = tbits.cpu().numpy().view(np.uint32)
    tnbr, _ = hamming_knn(tbits, k)
    tpa, tpb = knn_universe(tnbr, universe, train_seed)
    test_set = set(texts)
    keep = np.array([not (ttexts[a] in test_set and ttexts[b] in test_set) for a, b in zip(tpa, tpb)])
    tpa, tpb = tpa[keep], tpb[keep]
    same = identical_pairs(tbits_np, tpa, tpb)
    rng = np.random.default_rng(train_seed)
    si = np.where(same)[0]
    so = np.where(~same)[0]
    si = rng.choice(si, min(train_identical, len(si)), replace=False)
    so = rng.choice(so, min(train_other, len(so)), replace=False)
    keys, _ = exact_split_search(ttexts, tpa[si], tpb[si], frames_per_n=frames_per_n, seed=train_seed)
    late = np.array([mk.split_n(x) >= 6 for x in keys])
    # pairs with different truth vectors split on a model of <= 5 worlds: label 0
    la = np.concatenate([tpa[si], tpa[so]]).astype(np.int32)
    lb = np.concatenate([tpb[si], tpb[so]]).astype(np.int32)
    y = np.concatenate([late.astype(np.float32), np.zeros(len(so), np.float32)])
    npos = int(y.sum())
    wpos = min(1000.0, (len(y) - npos) / max(1, npos))
    wt = np.where(y > 0, wpos, 1.0).astype(np.float32)
    say("training pairs: %d (%d identical-vector, %d late splits) (%.1f s)" % (len(y), len(si), npos,
                                                                            time.time() - t0))
    dev = torch.device(device)
    F = bits.shape[1] * 64
    net = MLP(F, 256, seed=seed, device=device)
    hist = net.train(tbits, torch.from_numpy(la).to(dev), torch.from_numpy(lb).to(dev),
                     torch.from_numpy(y).to(dev), torch.from_numpy(wt).to(dev), epochs=epochs, batch=4096,
                     lr=1e-3, seed=seed, log=say)
    say("trained (%.1f s)" % (time.time() - t0))

    # rankings of the test universe
    dpa, dpb = torch.from_numpy(pa).to(dev), torch.from_numpy(pb).to(dev)
    orders = {}
    if "mlp" in methods:
        s = net.score(bits, dpa, dpb)
        orders["mlp"] = torch.argsort(s, descending=True, stable=True).cpu().numpy()
    if "random" in methods:
        orders["random"] = np.random.default_rng(seed + 1).permutation(len(pa))
    if "random_identical" in methods:
        same_u = identical_pairs(bits_np, pa, pb)
        r = np.random.default_rng(seed + 2)
        orders["random_identical"] = np.concatenate([r.permutation(np.where(same_u)[0]),
                                                     r.permutation(np.where(~same_u)[0])])
    if "pca10" in methods:
        xf = torch.from_numpy(np.unpackbits(bits_np.view(np.uint8), axis=1, bitorder="little").astype(np.float32)).to(dev)
        xf = xf - xf.mean(0, keepdim=True)
        _, _, V = torch.pca_lowrank(xf, q=10, center=False, niter=4)
        emb = xf @ V[:, :10]
        d = ((emb[dpa.long()] - emb[dpb.long()]) ** 2).sum(1)
        orders["pca10"] = torch.argsort(d, stable=True).cpu().numpy()
    out = {"universe": len(pa), "train_pairs": len(y), "train_late": npos, "loss_history": hist,
           "identical_in_universe": int(identical_pairs(bits_np, pa, pb).sum()), "budget_evals": budget}
    for m, order in orders.items():
        r = budget_walk(texts, pa, pb, order, budget, frames_per_n=frames_per_n, seed=4)
        r.pop("hits")
        out[m] = r
        say("%s: %s (%.1f s)" % (m, r, time.time() - t0))
    return out


# ------------------------------------------------------------ sharding

# ---------------------------------------------------- frame correspondents
def library_entries():
    """The correspondence library: every condition alone, then every
    conjunction of two proper conditions (ids >= 2).  Returns
    ((c1, c2) pairs, names)."""
    conj, names = [], []
    nc = len(mk.CONDITION_NAMES)
    for c in range(nc):
        conj.append((c, c))
        names.append(mk.CONDITION_NAMES[c])
    for a in range(2, nc):
        for b in range(a + 1, nc):
            conj.append((a, b))
            names.append(mk.CONDITION_NAMES[a] + " & " + mk.CONDITION_NAMES[b])
    return conj, names


class Correspondence:
    """Validity bitmaps of a batch of formulas over every K frame of
    1..N worlds (mk_frame_validity), the condition library's extensions
    (mk_frame_conditions) and their mismatch counts (mk_bitmap_mismatch):
    the recovery procedure of Sec. 10."""

    def __init__(self, texts, N=4, device="cuda"):
        if not torch.cuda.is_available():
            raise RuntimeError("Correspondence needs a CUDA device (there is no CPU fallback)")
        self.texts = list(texts)
        self.N = N
        self.device = torch.device(device)
        self.progs = mk.compile_batch(self.texts)
        self.d_progs = _dev_bytes(self.progs, self.device)
        self.depth = int(self.progs["depth"].max()) if len(self.progs) else 1
        self.offs = [0]
        for n in range(1, N + 1):
            self.offs.append(self.offs[-1] + mk.frame_words(n))
        self.words = self.offs[-1]
        self.conj, self.names = library_entries()
        self.d_conj = torch.tensor(np.array(self.conj, np.int32).reshape(-1), device=self.device)
        self.d_status = torch.zeros(1, dtype=torch.int32, device=self.device)

    def validity(self, sizes=None, stream=None):
        """[nprog, words] int32 device bitmaps, sizes 1..N side by side."""
        sizes = range(1, self.N + 1) if sizes is None else sizes
        bits = torch.zeros((len(self.texts), self.words), dtype=torch.int32, device=self.device)
        for n in sizes:
            mk.frame_validity_raw(self.d_progs.data_ptr(), len(self.texts), n, self.depth,
                                  bits.data_ptr() + 4 * self.offs[n - 1], self.words, self.d_status.data_ptr(),
                                  _stream_ptr(stream))
        return bits

    def conditions(self, stream=None):
        bits = torch.zeros((len(mk.CONDITION_NAMES), self.words), dtype=torch.int32, device=self.device)
        for n in range(1, self.N + 1):
            mk.frame_conditions_raw(n, bits.data_ptr() + 4 * self.offs[n - 1], self.words, _stream_ptr(stream))
        return bits

    def mismatch(self, vbits, cbits, size=None, stream=None):
        """[nprog, entries] mismatch counts over sizes 1..N, or over the
        one size `size` when given."""
        off, words = (0, self.words) if size is None else (self.offs[size - 1], mk.frame_words(size))
        out = torch.empty((vbits.shape[0], len(self.conj)), dtype=torch.int32, device=self.device)
        mk.bitmap_mismatch_raw(vbits.data_ptr() + 4 * off, vbits.shape[0], vbits.shape[1],
                               cbits.data_ptr() + 4 * off, cbits.shape[0], cbits.shape[1], self.d_conj.data_ptr(),
                               len(self.conj), words, out.data_ptr(), _stream_ptr(stream))
        return out

    def check_status(self):
        st = int(self.d_status.item())
        if st:
            raise mk.MkError(mk.status_error(st), "device status 0x%x" % st)


def recover_correspondents(texts, N=4, confirm_n=5, device="cuda"):
    """Sec. 10 over a batch: for each formula the library entries whose
    extension equals its validity set on every frame of 1..N worlds.  A
    formula whose set is constant (all frames or none) is trivial; for the
    others with a match, the match is re-checked on every frame of
    confirm_n worlds (None: skipped).  Returns (rows, stats)."""
    cj = Correspondence(texts, N, device)
    v = cj.validity()
    c = cj.conditions()
    d = cj.mismatch(v, c).cpu().numpy().view(np.uint32)
    cj.check_status()
    rows = []
    for i, t in enumerate(cj.texts):
        m = np.nonzero(d[i] == 0)[0]
        names = [cj.names[j] for j in m]
        trivial = 0 in m or 1 in m
        near = int(np.argmin(d[i]))
        rows.append({"formula": t, "matches": names, "match_ids": [int(j) for j in m], "trivial": bool(trivial),
                     "nearest": cj.names[near], "nearest_mismatch": int(d[i][near]), "confirmed": None})
    todo = [i for i, r in enumerate(rows) if r["matches"] and not r["trivial"]]
    if confirm_n and todo:
        big = Correspondence([texts[i] for i in todo], confirm_n, device)
        vb = big.validity(sizes=[confirm_n])
        cb = big.conditions()
        db = big.mismatch(vb, cb, size=confirm_n).cpu().numpy().view(np.uint32)
        big.check_status()
        for r_i, i in enumerate(todo):
            rows[i]["confirmed"] = all(int(db[r_i][j]) == 0 for j in rows[i]["match_ids"])
    stats = {"formulas": len(rows), "trivial": sum(r["trivial"] for r in rows),
             "recovered": sum(1 for r in rows if r["matches"] and not r["trivial"]),
             "unmatched": sum(1 for r in rows if not r["matches"]),
             "confirmed": sum(1 for r in rows if r["confirmed"])}
    return rows, stats


# ---------------------------------------------------- failure-density atlas
class Atlas:
    """The failure-density atlas of Sec. 9 for a batch of formulas over all
    n-world frames: exact counts (mk_atlas_counts), seriation by the first
    principal axis (mk_atlas_gram, mk_power_iteration, mk_atlas_project,
    mk_sort_keys), adjacent variation (mk_adjacent_variation) and the binned
    density view (mk_histogram2d, mk_histogram_stats)."""

    def __init__(self, texts, n=3, device="cuda"):
        if not torch.cuda.is_available():
            raise RuntimeError("Atlas needs a CUDA device (there is no CPU fallback)")
        self.texts = list(texts)
        self.B, self.n, self.F = len(self.texts), n, 1 << (n * n)
        self.device = torch.device(device)
        self.progs = mk.compile_batch(self.texts)
        self.d_progs = _dev_bytes(self.progs, self.device)
        k = self.progs["nvars"].astype(np.uint64)
        self.denom = (np.uint64(1) << (k * np.uint64(n))) * np.uint64(n)
        self.d_denom = torch.from_numpy(self.denom.view(np.int64).copy()).to(self.device)
        self.d_status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.counts = None

    def check_status(self):
        st = int(self.d_status.item())
        if st:
            raise mk.MkError(mk.status_error(st), "device status 0x%x" % st)

    def compute(self, stream=None):
        """Enqueue the counts (into the same buffer on every call)."""
        if getattr(self, "counts", None) is None:
            self.counts = torch.empty((self.B, self.F), dtype=torch.int32, device=self.device)
        mk.atlas_counts_raw(self.d_progs.data_ptr(), self.B, self.n, self.counts.data_ptr(), self.F,
                            self.d_status.data_ptr(), _stream_ptr(stream))
        return self.counts

    def principal_axes(self, k=1, iters=4000, stream=None):
        """The first k principal axes of the centred D (frame loadings, [k, F])
        and the formula coordinates on them ([k, B]), FP64 on the device."""
        sp = _stream_ptr(stream)
        F, B = self.F, self.B
        self.d_mean = torch.empty(F, dtype=torch.float64, device=self.device)
        gram = torch.empty((F, F), dtype=torch.float64, device=self.device)
        mk.atlas_gram_raw(self.counts.data_ptr(), self.d_denom.data_ptr(), B, F, F, self.d_mean.data_ptr(),
                          gram.data_ptr(), sp)
        V = torch.empty((k, F), dtype=torch.float64, device=self.device)
        U = torch.empty((k, B), dtype=torch.float64, device=self.device)
        lam = torch.empty(k, dtype=torch.float64, device=self.device)
        ws = torch.empty(mk.power_workspace_size(F), dtype=torch.uint8, device=self.device)
        for a in range(k):
            mk.power_iteration_raw(gram.data_ptr(), F, V.data_ptr(), a, iters, V[a].data_ptr(), lam[a].data_ptr(),
                                   ws.data_ptr(), ws.numel(), sp)
            mk.atlas_project_raw(self.counts.data_ptr(), self.d_denom.data_ptr(), B, F, F, self.d_mean.data_ptr(),
                                 V[a].data_ptr(), U[a].data_ptr(), sp)
        self.gram, self.lam = gram, lam
        return V, U

    def order(self, keys, stream=None):
        """Indices sorted by (key, index) on the device."""
        n = keys.numel()
        out = torch.empty(n, dtype=torch.int32, device=self.device)
        ws = torch.empty(mk.sort_workspace_size(n), dtype=torch.uint8, device=self.device)
        mk.sort_keys_raw(keys.data_ptr(), n, out.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(stream))
        return out

    def adjacent_variation(self, perm, stream=None):
        """A(perm), from exact per-row integer sums."""
        d_perm = perm if torch.is_tensor(perm) else torch.tensor(np.asarray(perm, np.int32), device=self.device)
        rs = torch.empty(self.B, dtype=torch.int64, device=self.device)
        mk.adjacent_variation_raw(self.counts.data_ptr(), self.B, self.F, self.F, d_perm.data_ptr(), rs.data_ptr(),
                                  self.d_status.data_ptr(), _stream_ptr(stream))
        r = rs.cpu().numpy().view(np.uint64)
        self.check_status()
        return float(np.sum(r.astype(np.float64) / self.denom.astype(np.float64)) / (self.B * (self.F - 1)))

    def seriation(self, iters=4000):
        """(frame order, formula order, axis, coordinates) on the device."""
        V, U = self.principal_axes(1, iters)
        return self.order(V[0]), self.order(U[0]), V[0], U[0]


def density_view(x, y, lo, hi, G=1024, radius=2, device="cuda"):
    """Datashading statistics of points (x_i, y_i) binned on a G x G grid
    (Sec. 9): occupied cells, largest cell, points sharing a cell, the
    pixels square marks of the given radius cover, and the overdraw
    factor of drawing every point as such a mark."""
    hist = torch.empty((G, G), dtype=torch.int32, device=device)
    mk.histogram2d_raw(x.data_ptr(), y.data_ptr(), x.numel(), lo, hi, G, hist.data_ptr(), _stream_ptr(None))
    st = torch.empty(4, dtype=torch.int64, device=device)
    mk.histogram_stats_raw(hist.data_ptr(), G, radius, st.data_ptr(), _stream_ptr(None))
    occ, big, shared, covered = (int(v) for v in st.cpu().numpy().view(np.uint64))
    npts = x.numel()
    draws = npts * (2 * radius + 1) ** 2
    return {"points": npts, "grid": G, "occupied_bins": occ, "largest_bin": big,
            "shared_fraction": shared / npts if npts else 0.0, "covered_pixels": covered,
            "point_pixel_draws": draws, "overdraw": draws / covered if covered else 0.0,
            "draw_op_reduction": npts / occ if occ else 0.0, "hist": hist}


# ------------------------------------------------------------ large frames
class RelationSet:
    """Relations on n <= 16 worlds in device memory, bit-sliced 32 to a
    block: drawn by an adversarial generator on the device
    (mk_generate_relations) or packed from explicit successor masks
    (mk_pack_relations), e.g. the stress templates."""

    def __init__(self, n, count, d_words, succ_host=None, gen=None, seed=0, first=0):
        self.n, self.count, self.d_words = int(n), int(count), d_words
        self.succ_host, self.gen, self.seed, self.first = succ_host, gen, seed, first

    @classmethod
    def generated(cls, gen, seed, n, first, count, device="cuda", stream=None):
        words = torch.empty(max(1, mk.relation_words(n, count)), dtype=torch.int32, device=device)
        mk.generate_relations_raw(gen, seed, n, first, count, words.data_ptr(), 0, _stream_ptr(stream))
        return cls(n, count, words, gen=mk.gen_index(gen), seed=seed, first=first)

    @classmethod
    def from_succ(cls, succ, n, device="cuda", stream=None):
        a = np.zeros((len(succ), 16), np.uint32)
        for i, row in enumerate(succ):
            a[i, :len(row)] = row
        d = torch.from_numpy(a.view(np.int32)).to(device)
        words = torch.empty(max(1, mk.relation_words(n, len(a))), dtype=torch.int32, device=device)
        mk.pack_relations_raw(d.data_ptr(), n, len(a), words.data_ptr(), _stream_ptr(stream))
        obj = cls(n, len(a), words, succ_host=a)
        obj._keep = d
        return obj

    @classmethod
    def templates(cls, n, device="cuda"):
        return cls.from_succ([mk.template(t, n) for t in range(mk.NUM_TEMPLATES)], n, device)

    def relation(self, i):
        """Successor masks of relation i (host)."""
        if self.succ_host is not None:
            return [int(x) for x in self.succ_host[i, :self.n]]
        return mk.stress_relation(self.gen, self.seed, self.n, self.first + i)


class StressJob:
    """Separation of (phi, psi) pairs over relation lists on up to 16
    worlds (mk_stress_separate)."""

    def __init__(self, pairs, device="cuda"):
        if not torch.cuda.is_available():
            raise RuntimeError("StressJob needs a CUDA device (there is no CPU fallback)")
        self.pairs = list(pairs)
        self.npairs = len(self.pairs)
        self.device = torch.device(device)
        self.pa = mk.compile_batch([a for a, _ in self.pairs])
        self.pb = mk.compile_batch([b for _, b in self.pairs])
        self.k = np.maximum(self.pa["nvars"], self.pb["nvars"]).astype(np.int64)
        self.d_pa = _dev_bytes(self.pa, self.device).view(self.npairs, -1)
        self.d_pb = _dev_bytes(self.pb, self.device).view(self.npairs, -1)
        self.d_status = torch.zeros(1, dtype=torch.int32, device=self.device)

    def eligible(self, n):
        """Pairs whose valuations at n worlds are exhaustive within the
        kernel's limit (k*n <= 16)."""
        return np.nonzero(self.k * n <= 16)[0]

    def launch(self, rels, idx=None, count_splits=False, tile=0, d_key=None, d_cnt=None, stream=None):
        """Launch on the pairs idx (default: all); returns the device key and
        count tensors (keys merged by minimum into d_key if given)."""
        idx = np.arange(self.npairs) if idx is None else np.asarray(idx)
        sel = torch.from_numpy(idx.astype(np.int64)).to(self.device)
        pa = self.d_pa.index_select(0, sel).contiguous()
        pb = self.d_pb.index_select(0, sel).contiguous()
        if d_key is None:
            d_key = torch.full((len(idx),), -1, dtype=torch.int64, device=self.device)
        if count_splits and d_cnt is None:
            d_cnt = torch.zeros(len(idx), dtype=torch.int32, device=self.device)
        cfg = mk.stress_cfg(rels.n, rels.count, 0, count_splits, tile)
        mk.stress_separate_raw(pa.data_ptr(), pb.data_ptr(), len(idx), rels.d_words.data_ptr(), cfg,
                               d_key.data_ptr(), d_cnt.data_ptr() if count_splits else 0,
                               self.d_status.data_ptr(), _stream_ptr(stream))
        self._keep = (pa, pb)
        return d_key, d_cnt

    def check_status(self):
        st = int(self.d_status.item())
        if st:
            raise mk.MkError(mk.status_error(st), "device status 0x%x" % st)

    def run(self, rels, idx=None, count_splits=False, tile=0):
        """First split keys (np.uint64) and, with count_splits, the number
        of relations splitting each pair."""
        self.d_status.zero_()
        d_key, d_cnt = self.launch(rels, idx, count_splits, tile)
        torch.cuda.synchronize(self.device)
        self.check_status()
        keys = d_key.cpu().numpy().view(np.uint64)
        return keys, (d_cnt.cpu().numpy().astype(np.int64) if count_splits else None)

    def certify(self, i, key, rels):
        """mk_certify on the split that key names for pair i."""
        s, x, w = mk.decode_stress_key(key)
        n = rels.n
        full = (1 << n) - 1
        val = [(x >> (v * n)) & full for v in range(int(self.k[i]))]
        a, b = self.pairs[i]
        return mk.certify(a, n, rels.relation(s), val, w, psi=b) == 1

    def evals(self, idx, n, relations):
        """Pair evaluations (relation x valuation) of a full scan."""
        return float(sum(relations * (1 << (int(self.k[i]) * n)) for i in idx))

    def lop3(self, idx, n, relations):
        """Algorithmic logic ops of a full scan (both programs and the
        difference test, per 32 relations)."""
        tot = 0.0
        for i in idx:
            per = lop3_per_eval(self.pa[i], n) + lop3_per_eval(self.pb[i], n)
            tot += per * relations * (1 << (int(self.k[i]) * n))
        return tot


def template_similarity(succ, n):
    """Largest Jaccard similarity (shared edges over edges of either) of a
    relation to the 39 stress templates of the same size; 1 for a template
    itself.  A witness below 0.5 counts as non-template."""
    def es(rows):
        return {(w, v) for w in range(n) for v in range(n) if (rows[w] >> v) & 1}
    e = es(succ)
    best = 0.0
    for t in range(mk.NUM_TEMPLATES):
        te = es(mk.template(t, n))
        u = len(e | te)
        best = max(best, (len(e & te) / u) if u else 1.0)
    return best


def template_stress(pairs, sizes=range(6, 17), job=None, device="cuda"):
    """Challenge pairs on the 39 templates at every size (Sec. 7 mining):
    for each pair the first (n, template, valuation, world) at which it
    splits, sizes ascending, or None.  Pairs with k*n > 16 skip size n."""
    job = job or StressJob(pairs, device)
    first = [None] * job.npairs
    for n in sizes:
        todo = [i for i in job.eligible(n) if first[i] is None]
        if not todo:
            continue
        rels = RelationSet.templates(n, device)
        keys, _ = job.run(rels, todo)
        for i, key in zip(todo, keys):
            d = mk.decode_stress_key(int(key))
            if d is not None:
                assert job.certify(i, int(key), rels)
                first[i] = (n,) + d
    return first


def mine_context_words(max_nodes=21, sizes=range(6, 17), device="cuda", log=None):
    """Automated context-word mining (Sec. 7): every candidate
    (C^m b, C^(m+1) b) is scanned on every K frame through five worlds; a is
    the largest size through which the pair agrees (exact prefix); pairs
    with a = 5 are stressed on the templates at 6..16 worlds.  Score
    J = a + 2 [template witness after a] - 0.02 (|phi| + |psi|) + 0.1/|C|.
    Returns rows sorted by J (highest first)."""
    cands = workloads.mining_candidates(max_nodes)
    pairs = [(a, b) for a, b, _ in cands]
    sj = SeparateJob(pairs, 1, 5, device=device)
    keys = sj.run()
    rows = []
    for i, (a, b, cl) in enumerate(cands):
        key = int(keys[i])
        ag = 5 if key == mk.NO_KEY else mk.split_n(key) - 1
        rows.append({"phi": a, "psi": b, "word": cl, "a": ag, "nodes": workloads.nodes(a) + workloads.nodes(b),
                     "prefix_key": key, "template": None})
    surv = [i for i, r in enumerate(rows) if r["a"] == 5]
    if log:
        log("mining: %d candidates, %d agree through five worlds" % (len(rows), len(surv)))
    if surv:
        tw = template_stress([pairs[i] for i in surv], sizes, device=device)
        for i, t in zip(surv, tw):
            rows[i]["template"] = t
    for r in rows:
        late = r["template"] is not None and r["template"][0] > r["a"]
        r["J"] = r["a"] + 2.0 * late - 0.02 * r["nodes"] + 0.1 / r["word"]
    rows.sort(key=lambda r: (-r["J"], r["phi"]))
    return rows


def adversarial_search(pairs, generators=mk.GENERATORS, sizes=(6, 8, 10, 12, 14, 16), relations=1 << 18,
                       seed=6, k_max=lambda n: 1 if n <= 12 else 0, device="cuda", log=None):
    """Adversarial frame synthesis (Table 2): for every generator and size,
    `relations` relations are drawn on the device and every eligible pair
    (k <= k_max(n): one-variable pairs through 12 worlds, constant pairs
    beyond) is scanned on all of them.  Per panel: relations, pair-relation
    tests, valuation evaluations, pairs split (each first split certified by
    mk_certify), non-template witnesses, GPU seconds (CUDA events)."""
    job = StressJob(pairs, device)
    rows, first = [], [None] * job.npairs
    for gen in generators:
        for n in sizes:
            idx = np.array([i for i in job.eligible(n) if job.k[i] <= k_max(n)], np.int64)
            if len(idx) == 0:
                continue
            rels = RelationSet.generated(gen, seed, n, 0, relations, device)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            job.d_status.zero_()
            ev0.record()
            d_key, d_cnt = job.launch(rels, idx, count_splits=True)
            ev1.record()
            torch.cuda.synchronize()
            job.check_status()
            keys = d_key.cpu().numpy().view(np.uint64)
            cnt = d_cnt.cpu().numpy()
            hits = cert = nontpl = 0
            for j, i in enumerate(idx):
                key = int(keys[j])
                if key == mk.NO_KEY:
                    continue
                hits += 1
                ok = job.certify(int(i), key, rels)
                cert += ok
                s, _, _ = mk.decode_stress_key(key)
                sim = template_similarity(rels.relation(s), n)
                nontpl += sim < 0.5
                if first[i] is None or (n, gen) < first[i][:2]:
                    first[i] = (n, gen, s, sim)
            row = {"generator": gen, "n": n, "relations": relations, "pairs": len(idx),
                   "tests": len(idx) * relations, "evals": job.evals(idx, n, relations),
                   "lop3": job.lop3(idx, n, relations), "split_pairs": hits, "certified": cert,
                   "non_template": nontpl, "split_relations": int(cnt.sum()),
                   "gpu_s": ev0.elapsed_time(ev1) / 1e3}
            rows.append(row)
            if log:
                log("  %-8s n=%2d pairs=%4d split=%4d cert=%4d non-template=%4d  %.3f s" %
                    (gen, n, len(idx), hits, cert, nontpl, row["gpu_s"]))
    return rows, first


def shard_range(total, rank, world):
    """[lo, hi) of the rank-th of ``world`` near-equal contiguous shards of
    [0, total) (frame K indices for the census, pairs for separation)."""
    lo = total * rank // world
    hi = total * (rank + 1) // world
    return lo, hi


def merge_results(parts):
    """Merge census results of disjoint frame shards: counts add, the
    witness is the least key (the census's own reduction, Sec. 4)."""
    parts = [np.asarray(p, np.uint64) for p in parts]
    out = parts[0].copy()
    for p in parts[1:]:
        out[..., 0] += p[..., 0]
        out[..., 1] += p[..., 1]
        out[..., 2] = np.minimum(out[..., 2], p[..., 2])
    return out


def allreduce_results(res, group=None):
    """The same merge across ranks with torch.distributed (sum of the
    counts, min of the keys; a missing witness, all ones, maps to the
    largest int64 for the min)."""
    import torch.distributed as dist
    r = np.asarray(res, np.uint64)
    counts = torch.from_numpy(r[..., :2].astype(np.int64).copy())
    keys = r[..., 2].copy()
    none = keys == np.uint64(mk.NO_KEY)
    k64 = torch.from_numpy(np.where(none, np.int64(2 ** 63 - 1), keys.astype(np.int64)))
    dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(k64, op=dist.ReduceOp.MIN, group=group)
    out = np.empty_like(r)
    out[..., :2] = counts.numpy().astype(np.uint64)
    k = k64.numpy()
    out[..., 2] = np.where(k == 2 ** 63 - 1, np.uint64(mk.NO_KEY), k.astype(np.uint64))
    return out


# ------------------------------------------------------ checkpoint / resume
#
# A long census is cut into independent units -- a tile of formulas, one
# (class, n) layer, one K-index chunk of that layer -- whose results merge
# exactly: counts add over disjoint frame sets and the witness is the least
# key (the census's own reduction, Sec. 4).  Every finished unit is appended
# to a per-rank journal (one line per unit, flushed and fsync'd before the
# next unit starts, with a CRC so a line torn by a kill is ignored), so a
# run that is killed between units resumes by skipping every unit found in
# any rank's journal.

def census_units(nformulas, classes, n_min, n_max, tile=256, frame_chunk=1 << 22):
    """The units of a census, in a fixed order: (p0, p1, class, n, f_lo,
    f_hi) for formula tiles [p0, p1), layers (class, n) and K-index chunks
    [f_lo, f_hi) of the layer (a chunk of the K index holds the chunk's
    frames of every class)."""
    out = []
    for p0 in range(0, nformulas, tile):
        p1 = min(nformulas, p0 + tile)
        for c in classes:
            for n in range(n_min, n_max + 1):
                kf = 1 << (n * n)
                for lo in range(0, kf, frame_chunk):
                    out.append((p0, p1, c, n, lo, min(kf, lo + frame_chunk)))
    return out


def _journal_config(texts, classes, n_min, n_max, samples, seed, tile, frame_chunk):
    import hashlib
    h = hashlib.sha256()
    h.update("\n".join(texts).encode())
    h.update(repr((tuple(classes), n_min, n_max, samples, seed, tile, frame_chunk)).encode())
    return h.hexdigest()


class CensusJournal:
    """The append-only journal of one rank's finished units, in
    ``directory``/census_rank<r>.jsonl; ``finished()`` reads every rank's."""

    def __init__(self, directory, rank, config):
        import os
        self.directory = directory
        self.config = config
        os.makedirs(directory, exist_ok=True)
        self.path = os.path.join(directory, "census_rank%d.jsonl" % rank)

    @staticmethod
    def _line(obj):
        import json
        import zlib
        body = json.dumps(obj, separators=(",", ":"), sort_keys=True)
        return "%08x %s\n" % (zlib.crc32(body.encode()), body)

    @staticmethod
    def _parse(line):
        import json
        import zlib
        if not line.endswith("\n") or len(line) < 10:
            return None                          # torn: the process died while writing it
        crc, body = line[:8], line[9:-1]
        try:
            if int(crc, 16) != zlib.crc32(body.encode()):
                return None
            return json.loads(body)
        except ValueError:
            return None

    def finished(self):
        """{unit: [[cm_count, frames_refuted, key] per formula]} from every
        rank's journal; a journal written for another configuration raises."""
        import glob
        out = {}
        for path in sorted(glob.glob(self.directory + "/census_rank*.jsonl")):
            with open(path) as f:
                for line in f:
                    rec = self._parse(line)
                    if rec is None:
                        continue
                    if rec.get("config") is not None:
                        if rec["config"] != self.config:
                            raise ValueError("%s was written for another census configuration" % path)
                        continue
                    out[tuple(rec["unit"])] = rec["res"]
        return out

    def record(self, unit, res):
        import os
        new = not os.path.exists(self.path) or os.path.getsize(self.path) == 0
        torn = False
        if not new:
            with open(self.path, "rb") as f:
                f.seek(-1, os.SEEK_END)
                torn = f.read(1) != b"\n"
        with open(self.path, "a") as f:
            if torn:
                f.write("\n")                      # end a line torn by a kill; it fails its CRC
            if new:
                f.write(self._line({"config": self.config}))
            f.write(self._line({"unit": list(unit), "res": [[int(x) for x in r] for r in res]}))
            f.flush()
            os.fsync(f.fileno())


def gpu_unit_runner(texts, samples=256, seed=2, device="cuda"):
    """Runs one census unit with mk_census on the GPU: the unit's formulas
    on its layer, frames restricted to its K-index chunk."""
    def run(unit):
        p0, p1, c, n, lo, hi = unit
        job = CensusJob(texts[p0:p1], (c,), n, n, samples=samples, seed=seed, frame_lo=lo, frame_hi=hi,
                        device=device)
        return job.run()[:, 0, 0, :]
    return run


def resumable_census(texts, classes, n_min, n_max, directory, runner=None, rank=0, world=1, samples=256, seed=2,
                     tile=256, frame_chunk=1 << 22, after_unit=None):
    """Runs this rank's share of the census units (unit i belongs to rank
    i % world) that no journal in ``directory`` holds yet, recording each
    as it finishes.  ``runner(unit)`` returns the unit's [formulas][3]
    results (default: mk_census on the GPU); ``after_unit(unit)`` is called
    after each recorded unit.  Returns the units run now."""
    cfg = _journal_config(texts, classes, n_min, n_max, samples, seed, tile, frame_chunk)
    journal = CensusJournal(directory, rank, cfg)
    done = journal.finished()
    runner = runner or gpu_unit_runner(texts, samples, seed)
    ran = []
    for i, u in enumerate(census_units(len(texts), classes, n_min, n_max, tile, frame_chunk)):
        if i % world != rank or u in done:
            continue
        res = np.asarray(runner(u), np.uint64)
        journal.record(u, res)
        ran.append(u)
        if after_unit:
            after_unit(u)
    return ran


def merge_census_journal(texts, classes, n_min, n_max, directory, samples=256, seed=2, tile=256,
                         frame_chunk=1 << 22):
    """The census result [formula][class][n - n_min][3] merged from the
    journals (counts summed, least key); raises if a unit is missing."""
    cfg = _journal_config(texts, classes, n_min, n_max, samples, seed, tile, frame_chunk)
    done = CensusJournal(directory, -1, cfg).finished()
    out = np.zeros((len(texts), len(classes), n_max - n_min + 1, 3), np.uint64)
    out[..., 2] = np.uint64(mk.NO_KEY)
    missing = 0
    for u in census_units(len(texts), classes, n_min, n_max, tile, frame_chunk):
        if u not in done:
            missing += 1
            continue
        p0, p1, c, n, _, _ = u
        r = np.asarray(done[u], np.uint64)
        blk = out[p0:p1, classes.index(c), n - n_min]
        blk[:, 0] += r[:, 0]
        blk[:, 1] += r[:, 1]
        blk[:, 2] = np.minimum(blk[:, 2], r[:, 2])
    if missing:
        raise RuntimeError("%d census units have no journal entry yet" % missing)
    return out
