"""Checkpoint and resume of a long census, on the CPU with gloo ranks.

The census is cut into units (formula tile x (class, n) layer x K-index
chunk) whose results merge exactly (counts add, least witness key).  Each
rank appends every finished unit to its journal before it starts the next
one.  Here rank 1 of two gloo ranks is killed between units; rank 0 learns
of it when its next collective fails.  A resume run skips every unit found
in any journal (a line torn by the kill is ignored) and the merged result
equals the uninterrupted census -- and the oracle's census of whole layers
-- bit for bit.  Units are computed by the CPU oracle (this host has no
GPU); on a GPU the same driver runs them with mk_census.
"""
import datetime
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

from paper_2606_15437_gb300 import workloads as W  # noqa: E402

FORMULAS = W.pr1_formulas()[:9] + ["[](p0 -> p1) & <>p2 -> <>(p0 & p2)"]
CLS = ("K", "T", "S4", "S5")
N_MIN, N_MAX, S, SEED, TILE, CHUNK = 1, 3, 16, 7, 4, 64
NO_KEY = (1 << 64) - 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def oracle_runner(calls=None):
    import oracle
    table = {n: W.sampled_valuations(SEED, n, S) for n in range(N_MIN, N_MAX + 1)}

    def run(u):
        p0, p1, c, n, lo, hi = u
        if calls is not None:
            calls.append(u)
        out = []
        for t in FORMULAS[p0:p1]:
            r = oracle.census(t, c, n, samples=table[n], f_lo=lo, f_hi=hi)
            key = NO_KEY
            if r["witness"]:
                f, v, w = r["witness"]
                key = (f << 27) | (v << 3) | w
            out.append((r["cm_count"], r["frames_refuted"], key))
        return out
    return run


def _kw():
    return dict(samples=S, seed=SEED, tile=TILE, frame_chunk=CHUNK)


def _worker(rank, world, port, directory, kill_after, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=30))
    from paper_2606_15437_gb300 import engine as E
    finished = [0]

    def after(u):
        finished[0] += 1
        if kill_after is not None and rank == 1 and finished[0] == kill_after:
            os._exit(3)          # killed between units: the journal holds every unit it finished

    ran = E.resumable_census(FORMULAS, CLS, N_MIN, N_MAX, directory, runner=oracle_runner(), rank=rank, world=world,
                             after_unit=after, **_kw())
    try:
        dist.barrier()
    except RuntimeError:
        q.put((rank, "peer lost", len(ran), None))
        q.close()
        q.join_thread()          # the queue's feeder thread must deliver before the exit
        os._exit(0)              # the process group is unusable once a peer is gone
    merged = E.merge_census_journal(FORMULAS, CLS, N_MIN, N_MAX, directory, **_kw()) if rank == 0 else None
    q.put((rank, "ok", len(ran), merged))
    dist.destroy_process_group()


def _run_ranks(directory, kill_after):
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, directory, kill_after, q)) for r in range(2)]
    # two ranks share this host's cores: one oracle thread each (read when
    # the children load their OpenMP runtime)
    old = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"
    try:
        for p in procs:
            p.start()
    finally:
        if old is None:
            del os.environ["OMP_NUM_THREADS"]
        else:
            os.environ["OMP_NUM_THREADS"] = old
    got = {}
    for _ in range(2 if kill_after is None else 1):
        r = q.get(timeout=240)
        got[r[0]] = r[1:]
    for p in procs:
        p.join(timeout=120)
    return got, [p.exitcode for p in procs]


def test_killed_rank_resumes_to_the_uninterrupted_census(tmp_path):
    from paper_2606_15437_gb300 import engine as E
    import oracle
    units = E.census_units(len(FORMULAS), CLS, N_MIN, N_MAX, TILE, CHUNK)
    assert len(units) > 20

    # the uninterrupted census, through the same journal, and pinned to the
    # oracle's census of whole layers
    full_dir = str(tmp_path / "full")
    E.resumable_census(FORMULAS, CLS, N_MIN, N_MAX, full_dir, runner=oracle_runner(), **_kw())
    full = E.merge_census_journal(FORMULAS, CLS, N_MIN, N_MAX, full_dir, **_kw())
    for p, t in enumerate(FORMULAS):
        for ci, c in enumerate(CLS):
            for n in range(N_MIN, N_MAX + 1):
                r = oracle.census(t, c, n, samples=W.sampled_valuations(SEED, n, S))
                key = NO_KEY if r["witness"] is None else (r["witness"][0] << 27) | (r["witness"][1] << 3) | r["witness"][2]
                assert tuple(int(x) for x in full[p, ci, n - N_MIN]) == (r["cm_count"], r["frames_refuted"], key)

    # two ranks; rank 1 is killed after finishing 3 units
    d = str(tmp_path / "ckpt")
    got, codes = _run_ranks(d, kill_after=3)
    assert codes[1] == 3
    assert got[0][0] == "peer lost"                  # rank 0's next collective failed
    cfg = E._journal_config(FORMULAS, CLS, N_MIN, N_MAX, S, SEED, TILE, CHUNK)
    done = E.CensusJournal(d, -1, cfg).finished()
    mine1 = [u for i, u in enumerate(units) if i % 2 == 1]
    assert sum(u in done for u in mine1) == 3        # exactly the units rank 1 finished
    with pytest.raises(RuntimeError):
        E.merge_census_journal(FORMULAS, CLS, N_MIN, N_MAX, d, **_kw())

    # the kill tore a line: it is ignored, and the next record starts afresh
    with open(os.path.join(d, "census_rank1.jsonl"), "a") as f:
        f.write('0badc0de {"res":[[1,2,3]],"unit":[0,4,"K",3,0')
    got, codes = _run_ranks(d, kill_after=None)
    assert codes == [0, 0]
    assert got[0][0] == got[1][0] == "ok"
    assert got[0][1] + got[1][1] == len(units) - len(done)      # only the missing units ran
    assert np.array_equal(got[0][2], full)

    # a third run has nothing left to do
    calls = []
    assert E.resumable_census(FORMULAS, CLS, N_MIN, N_MAX, d, runner=oracle_runner(calls), rank=1, world=2,
                              **_kw()) == []
    assert calls == []


def test_journal_refuses_another_configuration(tmp_path):
    from paper_2606_15437_gb300 import engine as E
    d = str(tmp_path / "j")
    E.resumable_census(FORMULAS[:2], ("K",), 1, 2, d, runner=oracle_runner(), **_kw())
    with pytest.raises(ValueError):
        E.resumable_census(FORMULAS[:3], ("K",), 1, 2, d, runner=oracle_runner(), **_kw())
