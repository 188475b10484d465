"""Host logic of bench.py's multi-rank path, run as two gloo ranks on the CPU.

Under torchrun every rank simulates its own replica (weak scaling): the only
exchange is the max over ranks of the step time, and the reported value is the
units all ranks processed divided by the slowest rank's time.
"""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench as b
    R = b.Ranks(rank, world, rank, backend="gloo")
    R.barrier()
    step_s = (0.5, 2.0, 1.0, 0.25)[rank]        # the second rank is the slowest
    slowest = R.max(step_s)
    rate = b.whole_job_rate(1000, world, slowest)
    R.barrier()
    R.close()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"slowest": slowest, "rate": rate, "own": step_s}, f)


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_whole_job_rate(tmp_path, world):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r in res:
        assert r["slowest"] == 2.0                  # every rank sees the slowest rank's time
        assert r["rate"] == pytest.approx(1000 * world / 2.0)
    assert res[0]["own"] != res[1]["own"]


def test_single_rank_needs_no_process_group():
    R = bench.Ranks(0, 1, 0, backend="gloo")
    assert R.dist is None
    assert R.max(3.5) == 3.5
    R.barrier()
    R.close()
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0


def test_reference_arm_prints_only_on_rank_zero(capsys):
    class Args:
        steps, warmup, gpus = 1, 1, 2
    bench.run_reference(Args(), 1)
    assert capsys.readouterr().out == ""
