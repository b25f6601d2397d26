"""Multi-process paths on the CPU (gloo, world size 2 and 4).

The benchmark runs one independent replica per GPU (TSQR needs no data-path collective inside a
GPU); across ranks it only takes the slowest rank's step time.  The sharded algebra the paper's
parallel TSQR uses between processors (Algorithm 1: each processor factors its block of rows, the
R factors are combined) is checked here with a real all-gather of the R factors between gloo
processes and the oracle as the local QR."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _timing_rank(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # rank r took 10 + 5 r ms per step
    slowest = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (slowest, bench.job_value(1e9, world, slowest))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_rank_timing_is_the_slowest_rank(world):
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_timing_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    slowest = 10.0 + 5.0 * (world - 1)
    for r in range(world):
        assert res[r][0] == slowest
        assert res[r][1] == pytest.approx(world / (slowest / 1e3))


def _allgather_rank(rank, world, port, m, n, out):
    import sys

    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from paper_0809_2407_gb300 import inputs

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    A = inputs.gaussian(m, n, inputs.seed_for(13, world))
    rows = np.array_split(np.arange(m), world)[rank]
    R_local = oracle.qr(np.ascontiguousarray(A[rows]))["R"]
    # all-gather the n x n R factors (the only exchange of the parallel TSQR) and reduce them
    gathered = [torch.empty((n, n), dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, torch.from_numpy(R_local))
    R = oracle.qr(np.vstack([g.numpy() for g in gathered]))["R"]
    out[rank] = R
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_allgather_tsqr_equals_one_qr(world):
    """Every rank ends with the R of the whole matrix (the all-reduction variant), equal to the
    oracle's single QR of all rows up to rounding."""
    import oracle
    from paper_0809_2407_gb300 import inputs

    m, n = 2000, 12
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_allgather_rank, args=(world, port, m, n, out), nprocs=world, join=True)
        res = dict(out)
    R_one = oracle.qr(inputs.gaussian(m, n, inputs.seed_for(13, world)))["R"]
    for r in range(world):
        assert np.abs(res[r] - R_one).max() <= 1e-12 * np.abs(R_one).max()
        assert np.array_equal(res[r], res[0])
