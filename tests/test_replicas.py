"""The multi-GPU path is replicas only (requests are independent; no data-path
collective): bench.py under torchrun runs one replica per rank, takes the
largest elapsed time over the ranks and reports the units of all ranks over it.
This runs that host logic as two gloo ranks on the CPU: the barrier, the
maximum over ranks, the whole-job aggregate, the configuration line's
parallelism, and the reference arm, which only rank 0 runs."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    w, r, local = bench.dist_env()
    assert (w, r, local) == (world, rank, rank)
    bench.dist_init(w, "gloo")
    bench.barrier(w)
    # rank r took 1 + r seconds for 100 units: the job is as slow as rank 1
    value, t = bench.aggregate(1.0 + rank, 100, w)
    mx = bench.max_over_ranks(float(rank), w)
    cfg = bench.config(w)
    out[rank] = (value, t, mx, cfg.get("parallelism"), cfg.get("global_batch"))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_over_the_slowest_replica():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, t, mx, par, batch = res[rank]
        assert t == 2.0 and value == pytest.approx(100 * world / 2.0)
        assert mx == 1.0
        assert par == "replicas x2" and batch == world


def _ref_rank(rank, world, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup = 1, 0

    ran = []
    bench.OracleSample = lambda: ran.append(rank) or (_ for _ in ()).throw(RuntimeError("rank 0 only"))
    try:
        bench.run_reference(Args)
        out[rank] = "returned"
    except RuntimeError:
        out[rank] = "ran"


def test_reference_arm_runs_on_rank_zero_only():
    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_ref_rank, args=(world, out), nprocs=world, join=True)
        res = dict(out)
    assert res == {0: "ran", 1: "returned"}
