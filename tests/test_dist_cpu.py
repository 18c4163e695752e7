"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1) agree on rank
0's headline mode, take the slowest rank's step time, report whole-job points/s for
weak scaling, and draw disjoint, reproducible workloads per rank (replicas: no
collective on the data path)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mode = bench.agree_on(f"mode-of-rank-{rank}", world)
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
        value = bench.job_points_per_s(1 << 20, world, ms)
        seeds, scal = bench.rank_workload(64, rank, 2)
        q.put((rank, mode, ms, value, seeds.tobytes(), scal[0].tobytes()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    modes = {r[1] for r in res}
    assert modes == {"mode-of-rank-0"}
    assert all(r[2] == 15.0 for r in res)                       # the slower rank's time
    assert all(abs(r[3] - 2 * (1 << 20) / 0.015) < 1e-3 for r in res)
    assert res[0][4] != res[1][4] and res[0][5] != res[1][5]    # disjoint workloads
    import sys
    sys.path.insert(0, ROOT)
    import bench
    seeds0, _ = bench.rank_workload(64, 0, 1)
    assert seeds0.tobytes() == res[0][4]                        # reproducible
    assert np.frombuffer(res[0][4], dtype=np.uint32).any()
