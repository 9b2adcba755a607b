#!/usr/bin/env python
"""Benchmark: the five-world census (exhaustive modal-formula evaluation).

One step = one complete census of the five-world workload: 5,624 seeded
formulas (length 3-24, modal depth 1-4, 0-3 variables, plus the K, T, 4
axioms) over every labelled frame of 1..5 worlds in K, T, S4 and S5, with
exhaustive valuations for formulas of <= 1 variable and 256 sampled
valuations otherwise.  Metric: G formula-frame-valuation evaluations/s
(bit-exact integer work).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mk|reference]

N > 1 runs under torchrun, one rank per GPU; every rank runs its own
independent five-world census batch (weak scaling, no data-path
collective: the barrier and the max of the timings are the only exchange).
--impl reference times the CPU oracle (oracle/, plain C over explicit
relations) on bounded samples of the same workload on the host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "G formula-frame-valuation evals/s (bit-exact)"
UNIT = "G evals/s"
WORKLOAD = ("five-world census: 5,624 seeded formulas (length 3-24, depth 1-4, 0-3 vars) x "
            "classes K/T/S4/S5 x all labelled frames n=1..5 x valuations (exhaustive if <=1 var, "
            "else 256 seeded)")
SEED = 2
S = 256
SMS = 152
SM_MAX_MHZ = 2070.0
LOP3_PER_SM_CLK = 64        # 3-input logic ops per SM per clock (4 SMSPs x 16 ALU lanes)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mk", choices=["mk", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ------------------------------------------------------------ CPU oracle leg

def oracle_sample(formulas, samples5, budget_s, start_frame=0):
    """Time the oracle on the K n=5 layer, formula by formula over frame
    windows of 4096 frames, until the budget is used.  Returns (evals, secs,
    description)."""
    import oracle
    oracle.build()
    evals, t0 = 0, time.perf_counter()
    done = []
    i = 0
    while time.perf_counter() - t0 < budget_s:
        text = formulas[i % len(formulas)]
        lo = start_frame + 4096 * (i // len(formulas))
        r = oracle.census(text, "K", 5, samples=samples5, f_lo=lo, f_hi=lo + 4096)
        evals += r["frames"] * r["nvals"]
        done.append(i)
        i += 1
    secs = time.perf_counter() - t0
    desc = ("oracle.census on the K n=5 layer: %d (formula, 4096-frame window) units of the first %d "
            "workload formulas, their full valuation sets" % (len(done), min(len(formulas), len(done))))
    return evals, secs, desc


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2606_15437_gb300 import workloads as W
    oracle.build()
    formulas = W.census5_formulas(SEED)
    samples5 = W.sampled_valuations(SEED, 5, S)
    step_s = 3.0
    for _ in range(args.warmup):
        oracle_sample(formulas, samples5, 0.5)
    tot_e, tot_s = 0, 0.0
    desc = ""
    for k in range(args.steps):
        e, s, desc = oracle_sample(formulas, samples5, step_s, start_frame=4096 * 64 * k)
        tot_e += e
        tot_s += s
    value = tot_e / tot_s / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_s / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
           "data": "synthetic (seeded; the paper's corpus is not available)",
           "config": {"workload": WORKLOAD, "sample": desc},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                            "sample": desc},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------ clock sampling

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_%d.csv" % os.getpid())
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_id), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9 and p[1].replace(".", "").isdigit():
                rows.append(p)
        if not rows:
            return None
        mhz = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3][:1].isdigit())
                if any(r[3][:1].isdigit() for r in rows) else None}


# ------------------------------------------------------------------ GPU leg

def gpu_smi_id(dev, local):
    """The nvidia-smi id of this process's GPU (its UUID when torch knows it)."""
    import torch
    u = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    if u is None:
        return str(local)
    u = str(u)
    return u if u.startswith("GPU-") else "GPU-" + u

def run_mk(args):
    import torch
    from paper_2606_15437_gb300 import build as mkbuild
    from paper_2606_15437_gb300 import mk
    from paper_2606_15437_gb300 import workloads as W
    from paper_2606_15437_gb300.engine import lop3_per_eval, n_valuations

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    mkbuild.build()

    formulas = W.census5_formulas(SEED if rank == 0 else SEED + 1000 * rank)
    progs = mk.compile_batch(formulas)
    nprog = len(progs)
    table = W.valuation_table(SEED, S, 5)

    # pinned host inputs (the e2e leg copies them every step)
    h_progs = torch.from_numpy(progs.view(np.uint8).copy()).pin_memory()
    h_samples = torch.from_numpy(table.view(np.uint8).reshape(-1).copy()).pin_memory()
    d_progs = h_progs.to(dev)
    d_samples = h_samples.to(dev)

    # one step = three census calls: the dominant K n=5 layer alone (timed
    # by its own events), K n=1..4, and T/S4/S5 n=1..5
    parts = [((mk.CLASS_BITS["K"]), 5, 5), ((mk.CLASS_BITS["K"]), 1, 4),
             (mk.CLASS_BITS["T"] | mk.CLASS_BITS["S4"] | mk.CLASS_BITS["S5"], 1, 5)]
    calls = []
    for cls, lo, hi in parts:
        cfg = mk.census_cfg(cls, lo, hi, S, d_samples.data_ptr(), max_depth=max(1, int(progs["depth"].max())))
        ws = mk.census_workspace_size(cfg, nprog)
        ncls = bin(cls).count("1")
        out = torch.empty(nprog * ncls * (hi - lo + 1) * 3, dtype=torch.int64, device=dev)
        calls.append({"cfg": cfg, "ws": torch.empty(max(ws, 1), dtype=torch.uint8, device=dev),
                      "ws_bytes": ws, "out": out, "launches": mk.census_launches(cfg, nprog)})
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    def step():
        for c in calls:
            mk.census_raw(d_progs.data_ptr(), nprog, c["cfg"], c["out"].data_ptr(), status.data_ptr(),
                          c["ws"].data_ptr(), c["ws_bytes"], sp)

    # algorithmic work
    evals = 0
    ops_dom = 0.0
    for p in progs:
        k = int(p["nvars"])
        for cls in ("K", "T", "S4", "S5"):
            for n in range(1, 6):
                evals += mk.class_frames(cls, n) * n_valuations(k, n, S)
        ops_dom += (1 << 25) * n_valuations(k, 5, S) * lop3_per_eval(p, 5)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    if int(status.item()):
        raise SystemExit("device status 0x%x" % int(status.item()))

    clocks = ClockSampler(gpu_smi_id(dev, local)) if local == 0 else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dom = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    ev0.record(stream)
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        dom[k][0].record(stream)
        c = calls[0]
        mk.census_raw(d_progs.data_ptr(), nprog, c["cfg"], c["out"].data_ptr(), status.data_ptr(),
                      c["ws"].data_ptr(), c["ws_bytes"], sp)
        dom[k][1].record(stream)
        for c in calls[1:]:
            mk.census_raw(d_progs.data_ptr(), nprog, c["cfg"], c["out"].data_ptr(), status.data_ptr(),
                          c["ws"].data_ptr(), c["ws_bytes"], sp)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks else None
    ms = ev0.elapsed_time(ev1)
    dom_ms = statistics.mean(a.elapsed_time(b) for a, b in dom)
    if int(status.item()):
        raise SystemExit("device status 0x%x" % int(status.item()))

    # e2e through the public API: pinned host inputs in, results out, every step
    h_outs = [torch.empty(c["out"].numel(), dtype=torch.int64).pin_memory() for c in calls]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for k in range(args.steps):
        d_progs.copy_(h_progs, non_blocking=True)
        d_samples.copy_(h_samples, non_blocking=True)
        step()
        for c, h in zip(calls, h_outs):
            h.copy_(c["out"], non_blocking=True)
        stream.synchronize()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1)
    h2d = h_progs.numel() + h_samples.numel()
    d2h = sum(h.numel() * 8 for h in h_outs)

    # logic-op ceiling cross-check (own calibration kernel)
    sink = torch.zeros(SMS * 8, dtype=torch.int32, device=dev)
    blocks = torch.cuda.get_device_properties(dev).multi_processor_count * 8
    cal_ops = mk.calibrate_lop3(sink.data_ptr(), blocks, 256, 2048, 7, sp)
    torch.cuda.synchronize(dev)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(3):
        mk.calibrate_lop3(sink.data_ptr(), blocks, 256, 2048, 7, sp)
    c1.record(stream)
    torch.cuda.synchronize(dev)
    cal_tops = 3 * cal_ops / (c0.elapsed_time(c1) / 1e3) / 1e12

    # max over ranks
    t = torch.tensor([ms, e2e_ms], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms, e2e_ms = float(t[0]), float(t[1])
    if rank != 0:
        torch.distributed.destroy_process_group()
        return

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tops = sms * LOP3_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
    achieved = ops_dom / (dom_ms / 1e3) / 1e12
    value = world * evals * args.steps / (ms / 1e3) / 1e9
    e2e_value = world * evals * args.steps / (e2e_ms / 1e3) / 1e9
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u32",
           "data": "synthetic (seeded formulas; the paper's corpus is not available)",
           "config": {"workload": WORKLOAD, "formulas": nprog, "classes": "K,T,S4,S5", "n_max": 5,
                      "samples": S, "evals_per_step": evals, "l2": "flushed (256 MB write) before every step",
                      "parallelism": "replicas x%d (independent batches)" % world},
           "roofline": {"bound": "alu", "kernel": "census_layer_kernel<5> (K, n=5)",
                        "achieved": achieved, "peak": peak_tops, "unit": "Tops/s (3-input logic ops)",
                        "frac": achieved / peak_tops, "traffic": None,
                        "algorithmic_ops_per_launch": ops_dom, "launch_ms": dom_ms,
                        "peak_basis": "%d SMs x %d logic ops/clk x %.0f MHz" % (sms, LOP3_PER_SM_CLK, SM_MAX_MHZ),
                        "calibrated_lop3_tops": cal_tops},
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
           "gpu_launches": sum(c["launches"] for c in calls) * args.steps,
           "clocks": clk}
    if not args.no_cpu_baseline:
        e, s, desc = oracle_sample(formulas, table[5], args.cpu_seconds)
        import oracle
        out["cpu_baseline"] = {"value": e / s / 1e9, "unit": UNIT, "cores": oracle.threads(),
                               "kind": "oracle", "sample": desc}
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_mk(args)


if __name__ == "__main__":
    main()
