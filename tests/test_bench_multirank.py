"""Host logic of bench.py's multi-GPU form (independent replicas), run as two
gloo ranks on the CPU: the slowest rank's step time is what every rank uses,
the whole-job value counts every rank's cells, and the reference arm does
its work on rank 0 only."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    my_ms = 1.0 + rank  # rank 1 is the slower one
    ms = bench.max_over_ranks(my_ms)
    value = bench.whole_job_value(ws, 1000, ms)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"ws": ws, "rank": r, "local": local, "ms": ms, "value": value}, f)


def test_two_gloo_ranks_agree_on_the_slowest(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, d in enumerate(res):
        assert (d["ws"], d["rank"], d["local"]) == (2, r, r)
        assert d["ms"] == 2.0  # the max over ranks, on both ranks
        assert d["value"] == pytest.approx(2 * 1000 / 2e-3)  # both ranks' cells over the slowest time


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_value(1, 8, 2.0) == pytest.approx(4000.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup = 1, 3

    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""  # rank 1 prints nothing and touches no oracle
