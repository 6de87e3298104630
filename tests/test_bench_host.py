"""Host logic of the benchmark's replica mode (one independent solve per rank), on CPU with gloo."""
import json
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each replica reports its own mean step time; every rank must see the slowest one
        got = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
        out[rank] = got
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_world_size_two():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, torch.device("cpu")) == 3.5


def test_reference_arm_prints_only_on_rank_zero(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup = 1, 0
    assert bench.run_reference(Args, 1, 2) == 0
    assert capsys.readouterr().out == ""


@pytest.mark.parametrize("key", ["metric", "unit", "higher_is_better", "scaling", "config"])
def test_reference_line_shares_the_native_contract(key, monkeypatch, capsys):
    """The oracle arm prints the same metric, unit and config as the GPU arm (tiny sample)."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "DIMS", (4, 4, 4, 4))

    class Args:
        steps, warmup = 1, 0
    assert bench.run_reference(Args, 0, 1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    expected = {"metric": "CG time-to-1e-10 residual", "unit": "ms", "higher_is_better": False,
                "scaling": "weak"}
    if key == "config":
        assert line["config"]["workload"].startswith("plain FP64 CG")
    else:
        assert line[key] == expected[key]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
