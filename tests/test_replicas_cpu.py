"""The multi-GPU mode of bench.py is independent replicas (one series per rank, different seeds, no
data-path collective; the time recursion does not shard).  Its host-side bookkeeping is exercised
here with two gloo ranks on the CPU: the max-over-ranks timing, the barrier, the per-rank seeds and
the whole-job aggregation."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    try:
        bench.barrier(ws)
        # max over ranks
        m = bench.allmax(ws, 10.0 * (rank + 1))
        # per-rank series: the replicas must not share their data
        w, _ = bench.workload("small", 2, seed_offset=rank, device=None)
        y = torch.as_tensor(np.asarray(w.y[:64], dtype=np.float64))
        ys = [torch.zeros_like(y) for _ in range(ws)]
        dist.all_gather(ys, y)
        same = bool(torch.equal(ys[0], ys[1]))
        out.put((rank, m, same, bench.job_value(ws, w.T, 3, m)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, same, value in res:
        assert m == 20.0                       # the slowest rank's time on every rank
        assert not same                         # different seeds per rank
        assert abs(value - ws * 2 * 3 / (20.0 / 1e3)) < 1e-9   # 2 ranks x T=2 x 3 steps in 20 ms
