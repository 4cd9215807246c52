"""Multi-GPU mode of the benchmark on CPU: world size 2 over gloo.

The path does not shard: N GPUs run N independent realisations (replicas, weak
scaling), so the only cross-rank steps are a barrier and a max-reduce of the
timings.  These run here with the gloo backend on 127.0.0.1; each rank
reports a different local time, both must see the maximum, and the job rate
counts every rank's units against the slowest rank.  Each rank also draws its
own Zel'dovich realisation (seed 1 + rank)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    from paper_2110_00328_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_init()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    local_ms = 10.0 * (rank + 1)
    mx = bench.reduce_max(local_ms, w, torch.device("cpu"))
    rate = bench.job_rate(1e6, w, mx)
    pos = inputs.zeldovich_positions(8, seed=1 + rank, sigma=1.0)
    out[rank] = (mx, rate, float(pos.sum()))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_rank_barrier_max_reduce_and_job_rate():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    (mx0, rate0, s0), (mx1, rate1, s1) = out[0], out[1]
    assert mx0 == mx1 == 20.0
    assert rate0 == rate1 == pytest.approx(1e6 * 2 / 0.020 / 1e6)
    assert s0 != s1  # independent realisations


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, 1, None) == 3.5
    bench.barrier(1)
    assert bench.job_rate(2e6, 1, 1000.0) == pytest.approx(2.0)
    assert np.isfinite(bench.job_rate(1.0, 4, 1.0))
