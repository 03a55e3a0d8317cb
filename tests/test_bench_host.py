"""Host-side logic of bench.py: byte model, kernel naming, and the multi-process
replica timing reduction (world size 2 over gloo, no GPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def test_sweep_byte_model_is_25_plus_n_words_per_voxel():
    """Five pruned sweeps with M = 2N: (n - 1) + 2 + 2 + 4 + 4 + 1 + 4 + 4 + 2 + 2 + 1 words."""
    for n_h in (2, 3, 4, 5):
        N = 64
        by = bench.sweep_bytes((N, N, N), (2 * N, 2 * N, 2 * N), n_h, fused_source=True)
        octant = (N + 1) ** 3
        words = sum(by) / 8
        assert words == (25 + n_h) * N ** 3 - N ** 3 + octant


def test_kernel_names_follow_the_engine():
    assert bench.kernel_name(2, (512, 512, 512), (1, 1, 1)).startswith("line2_conv_pipe_kernel")
    assert bench.kernel_name(2, (200, 200, 200), (0, 0, 0)).startswith("line_sweep_kernel")
    assert "source" in bench.kernel_name(0, (512, 512, 512), (1, 1, 1))
    assert bench.kernel_name(3, (200, 512, 200), (0, 1, 0)).startswith("col2_kernel inverse")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        local_ms = 10.0 * (rank + 1)
        total = bench.max_over_ranks(local_ms, world)
        value = bench.aggregate_value(voxels=1000, steps=5, world=world, total_ms=total)
        out[rank] = (total, value)
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_max_over_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        total, value = out[r]
        assert total == pytest.approx(20.0)
        # whole-job throughput: units of all ranks / slowest rank's time
        assert value == pytest.approx(1000 * 5 * world / 0.020)
