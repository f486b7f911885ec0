"""Multi-process host logic of the replica runs (no GPU): the path shards
into independent replicas with no collective on the data path, so the only
cross-rank step is the timing reduction after the timed region.  Two `gloo`
ranks on the CPU exercise it."""
import os
import socket
import sys
import types

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out_dir):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        t_max = bench.max_over_ranks(times[rank], world, device="cpu")
        rate = bench.replica_rate(100, world, t_max)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{t_max!r} {rate!r}\n")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_max_over_ranks_gloo(tmp_path, world):
    """Every rank sees the slowest rank's time; throughput counts all ranks'
    units over that time."""
    times = [12.5, 40.0, 7.25][:world]
    mp.start_processes(_rank_main, args=(world, _free_port(), times, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    want = max(times)
    for r in range(world):
        t_max, rate = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert t_max == want
        assert rate == pytest.approx(world * 100 / (want / 1e3), rel=1e-12)


def test_single_rank_needs_no_process_group():
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_rate(10, 1, 5.0) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    """Under torchrun the CPU reference arm is run and printed by rank 0
    alone; the other ranks return at once without work or output."""
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = types.SimpleNamespace(gpus=2, steps=1, warmup=3, impl="reference")
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
