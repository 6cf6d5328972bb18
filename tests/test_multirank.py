"""The multi-process path of bench.py on CPU (gloo, world size 2).

Under torchrun every rank runs its own replica on its own seeded batch (weak
scaling, no collective on the data path). The job's step time is the
slowest rank's (a MAX all-reduce), and its throughput counts every rank's
maps. The reference arm runs on rank 0 only. Ranks are spawned processes
that rendezvous on 127.0.0.1."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    try:
        import torch.distributed as dist
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import bench
        bench.set_workload(16, "32x16")  # a small workload: 16 maps, 32 x 16 G-buffer
        local_ms = [2.0, 3.5][rank]
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        e2e = bench.max_over_ranks([4.0, 3.0][rank], dist, "cpu")
        val = bench.job_value(world, bench.N_MAPS, ms)
        w, x, g, c = bench.make_inputs(seed_offset=rank)
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, ms, e2e, val, x.copy(), w.copy(), g["pos"].copy()))
    except Exception as exc:  # reported to the parent, which fails the test
        q.put((rank, "error", repr(exc)))


def test_two_gloo_ranks_reduce_and_seed_per_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        item = q.get(timeout=180)
        assert item[1] != "error", item
        res[item[0]] = item
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        _, ms, e2e, val, _, _, _ = res[r]
        assert ms == 3.5 and e2e == 4.0  # the slowest rank, on every rank
        assert val == pytest.approx(2 * 16 / 3.5e-3)  # both ranks' maps over the slowest step
    # each rank draws its own batch and G-buffer; the network is the same
    assert not np.array_equal(res[0][4], res[1][4])
    assert not np.array_equal(res[0][6], res[1][6])
    np.testing.assert_array_equal(res[0][5], res[1][5])


def test_single_rank_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench.job_value(1, 4096, 2.0) == pytest.approx(4096 / 2e-3)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, gpus = 1, 0, 2

    bench.run_reference(Args(), rank=1)  # no work and no output on the other ranks
    assert capsys.readouterr().out == ""
