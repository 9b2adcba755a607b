"""The multi-rank path on the CPU: gloo, world size 2.

The census partitions into frame shards whose results merge by a sum of
the counts and a min of the witness keys.  Each rank computes its K-index
shard (here with the CPU oracle, since this host has no GPU), the ranks
merge with torch.distributed all_reduce, and the merged result must equal
the unsharded census bit for bit; bench.py's timing reduction (max over
ranks) is exercised the same way.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

FORMULAS = ["[]p -> p", "<>(p & ~q) | []q", "[]<>T", "p -> []<>p", "[](p -> q) -> ([]p -> []q)"]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _oracle_results(lo, hi, n):
    import oracle
    out = np.zeros((len(FORMULAS), 1, 1, 3), np.uint64)
    for i, t in enumerate(FORMULAS):
        r = oracle.census(t, "K", n, f_lo=lo, f_hi=hi)
        key = (1 << 64) - 1
        if r["witness"]:
            f, v, w = r["witness"]
            key = (f << 27) | (v << 3) | w
        out[i, 0, 0] = (r["cm_count"], r["frames_refuted"], key)
    return out


def _worker(rank, world, port, n, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2606_15437_gb300 import engine as E
    lo, hi = E.shard_range(1 << (n * n), rank, world)
    part = _oracle_results(lo, hi, n)
    merged = E.allreduce_results(part)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, merged, float(t.item())))
    dist.destroy_process_group()


@pytest.mark.parametrize("n", [2, 3])
def test_two_rank_shards_merge_to_the_full_census(n):
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full = _oracle_results(0, 1 << (n * n), n)
    for rank, merged, tmax in got:
        assert np.array_equal(merged, full), rank
        assert tmax == 2.0


def test_merge_results_locally():
    from paper_2606_15437_gb300 import engine as E
    n = 3
    parts = [_oracle_results(*E.shard_range(1 << 9, r, 3), n) for r in range(3)]
    assert np.array_equal(E.merge_results(parts), _oracle_results(0, 1 << 9, n))
