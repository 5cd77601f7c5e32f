"""Multi-rank (replicas) logic of bench.py on CPU with the gloo backend, world size 2.

One H-LU does not shard; N GPUs run N independent replicas. The only cross-rank data are the
whole-job figures: the slowest rank's time (max) and the sum of all ranks' FLOPs. These tests
run that reduction with two gloo ranks and check the per-replica seeding and that a non-zero
rank of the reference arm exits without work.
"""
import os
import socket
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import hm_workloads as W  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, fl = bench.aggregate_ranks(100.0 + 50.0 * rank, 1e9 * (rank + 1), dist, "cpu")
        np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([ms, fl]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        ms, fl = np.load(tmp_path / f"r{r}.npy")
        assert ms == 150.0          # the slowest rank's time
        assert fl == 3e9            # every rank's FLOPs
    # whole-job GFLOP/s as bench.py forms it
    assert 3e9 / (150.0 * 1e-3) * 1e-9 == pytest.approx(20.0)


def test_single_rank_aggregate_is_identity():
    assert bench.aggregate_ranks(12.5, 7.0, None, "cpu") == (12.5, 7.0)


def test_replicas_get_distinct_seeded_instances():
    cfg = W.WORKLOADS["sphere2048"]
    p0, p0b, p1 = bench.replica_points(cfg, 0), bench.replica_points(cfg, 0), bench.replica_points(cfg, 1)
    assert p0.shape == (cfg["n"], 3)
    np.testing.assert_array_equal(p0, p0b)      # deterministic per rank
    assert not np.array_equal(p0, p1)           # independent instances


def test_reference_arm_nonzero_rank_does_no_work(capsys):
    args = types.SimpleNamespace(workload="sphere2048", warmup=3, steps=2, gpus=2)
    assert bench.run_reference(args, 1) == 0
    assert capsys.readouterr().out == ""
