"""The N > 1 path of bench.py (independent replicas, one per rank): the timed
region is the slowest rank's, the value counts every rank's node updates, and
only rank 0 reports.  Two gloo ranks on the CPU."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist, r, ws = bench._dist("gloo")
    assert (r, ws) == (rank, world)
    ms = bench.max_over_ranks(dist, 10.0 + 5.0 * rank, device="cpu")
    value = bench.aggregate_mlups(1.0e6, 20, ws, ms)
    dist.barrier()
    if r == 0:
        with open(out, "w") as fh:
            json.dump({"ms": ms, "value": value}, fh)
    dist.destroy_process_group()


def test_replicas_report_the_slowest_rank_and_all_updates(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "rank0.json")
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    res = json.load(open(out))
    assert res["ms"] == 15.0                       # max over ranks (10 and 15 ms)
    assert res["value"] == pytest.approx(1.0e6 * 20 * 2 / 15e-3 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the reference arm (the oracle on the host cores) runs on
    rank 0 alone; the other ranks exit without work."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class Args:
        gpus, steps, warmup = 2, 1, 3
    assert bench.reference_arm(Args()) is None
    assert capsys.readouterr().out == ""
