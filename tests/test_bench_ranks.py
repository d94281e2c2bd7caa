"""CPU: the multi-rank (replica) path of bench.py with world size 2 over gloo,
and the reference arm's JSON line on a small workload."""
import json
import os
import socket
import sys
import types

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: timed region 10 + r ms, e2e 20 + 2r ms, 7 + r gradients, 8 + r in the e2e loop
        res = bench.aggregate_ranks(torch, dist, torch.device("cpu"), 10.0 + rank, 20.0 + 2 * rank,
                                    7 + rank, 8 + rank)
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


def test_aggregate_ranks_world2_gloo(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        with open(tmp_path / ("rank%d.json" % r)) as f:
            t_max, e2e_max, illum, illum_e2e = json.load(f)
        assert t_max == 11.0 and e2e_max == 22.0      # slowest rank's times
        assert illum == 15.0 and illum_e2e == 17.0    # all ranks' work


def test_aggregate_ranks_single_rank():
    assert bench.aggregate_ranks(torch, None, None, 5.0, 6.0, 3, 4) == (5.0, 6.0, 3.0, 4.0)


def test_reference_arm_prints_one_line_on_rank0_only(capsys):
    args = types.SimpleNamespace(workload="ls32", steps=1, warmup=0, gpus=2)
    bench.run_reference(args, world=2, rank=1)
    assert capsys.readouterr().out == ""
    bench.run_reference(args, world=2, rank=0)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == bench.UNIT and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
