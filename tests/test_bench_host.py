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
    assert bench.kernel_name(2, (1200, 1200, 1280), (1, 1, 1)) == "line2_conv_pipe_kernel (L=1280)"
    assert bench.kernel_name(2, (200, 200, 200), (0, 0, 0)).startswith("line_sweep_kernel")
    assert "source" in bench.kernel_name(0, (512, 512, 512), (1, 1, 1))
    # after a nested source the first sweep reads f: the plain forward sweep
    assert "source" not in bench.kernel_name(0, (512, 512, 512), (1, 1, 1), fused_source=False)
    assert bench.kernel_name(3, (200, 512, 200), (0, 1, 0)).startswith("col2_kernel inverse")


def test_nested_source_bytes_read_one_field():
    """With the source formed by the nested-source kernel the first sweep reads f once."""
    N = 64
    fused = bench.sweep_bytes((N, N, N), (2 * N, 2 * N, 2 * N), 3, fused_source=True)
    plain = bench.sweep_bytes((N, N, N), (2 * N, 2 * N, 2 * N), 3, fused_source=False)
    assert fused[0] - plain[0] == 8 * N ** 3 and fused[1:] == plain[1:]


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the FP64 oracle on the host (no GPU) and prints one
    JSON line with the contract's keys."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "3",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 3
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


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


def test_contended_harmonics_are_those_started_before_the_side_stream_ended():
    import bench
    # step 0: V_k1 ends at 0.2 ms, harmonic 2 starts at 0, harmonic 3 at 0.5
    # step 1: V_k1 ends at 0.6 ms (a slow step): harmonic 3 began at 0.55, inside it
    assert bench.contended_harmonics([0.2], [{2: 0.0, 3: 0.5}]) == {2}
    assert bench.contended_harmonics([0.2, 0.6], [{2: 0.0, 3: 0.5}, {2: 0.0, 3: 0.55}]) == {2, 3}
    assert bench.contended_harmonics([], []) == set()
