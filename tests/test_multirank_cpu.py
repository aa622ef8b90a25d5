"""The multi-GPU path of bench.py (replicas, weak scaling) on two gloo ranks on the CPU.

Each rank solves its own clips (no data-path collective); the only collectives
are the timing barrier and the maximum over ranks.  Checked here: per-rank
inputs are independent and reproducible, and the whole-job throughput divides
the units of all ranks by the slowest rank's time.
"""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from workloads import get_workload


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = [120.0, 150.0][rank]                       # rank 1 is the slower one
        ms, value = bench.job_throughput(ms_local, world, 8, 65536, 10, dist)
        dist.barrier()
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.array([ms, value]))
    finally:
        dist.destroy_process_group()


def test_job_throughput_is_max_over_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    want_ms = 150.0
    want = world * 8 * 65536 * 10 / (want_ms / 1e3)
    for rank in range(world):
        ms, value = np.load(tmp_path / f"rank{rank}.npy")
        assert ms == want_ms
        assert value == pytest.approx(want, rel=1e-12)


def test_single_rank_throughput_needs_no_process_group():
    ms, value = bench.job_throughput(200.0, 1, 8, 65536, 100)
    assert ms == 200.0 and value == pytest.approx(8 * 65536 * 100 / 0.2)


def test_rank_inputs_are_independent_and_reproducible():
    wl = get_workload("tones8k_n8192")
    t0, i0 = bench.rank_inputs(wl, 0)
    t1, i1 = bench.rank_inputs(wl, 1)
    t1b, i1b = bench.rank_inputs(wl, 1)
    assert t0.shape == t1.shape == (wl.batch, wl.N) and i0.shape == i1.shape
    assert np.array_equal(t1, t1b) and np.array_equal(i1, i1b)
    assert not np.allclose(t0, t1) and not np.allclose(i0, i1)
    assert np.array_equal(t0, wl.targets()) and np.array_equal(i0, wl.inits())
