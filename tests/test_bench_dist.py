"""Host-side logic of the multi-rank benchmark on CPU ranks (gloo, world size 2): each
rank builds its own replicas of the workload (weak scaling, no data-path exchange) and the
job time is the slowest rank's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl, reps = bench.make_workload("tiny", rank)
        ms = 10.0 + 5.0 * rank
        t = bench.max_over_ranks(ms, dist)
        v = bench.job_value(reps[0].n_cr, world, 100, t)
        out[rank] = (reps[0].n_cr, float(reps[0].v_cr[-1, 0]), t, v)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    (n0, v0, t0, val0), (n1, v1, t1, val1) = out[0], out[1]
    assert n0 == n1 == 1024            # same work per rank
    assert v0 != v1                    # independent velocity draws
    assert t0 == t1 == 15.0            # the slowest rank's time on every rank
    assert val0 == pytest.approx(1024 * 2 * 100 / 15e-3)


def test_single_rank_defaults():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    wl, reps = bench.make_workload("batched", 0)
    assert len(reps) == 256
    _, reps1 = bench.make_workload("batched", 1)
    assert sum(r.n_cr for r in reps1) != sum(r.n_cr for r in reps)
