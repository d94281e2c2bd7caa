"""CPU: illumination sharding of the subset gradient (Eq. 4.1) over gloo
ranks.  Each rank computes the FP64 oracle's partial gradient over its share
of the subset with the library's sharding function; after the all-reduce every
rank must hold the whole subset's gradient and loss (to rounding: the partial
sums are regrouped), for even and uneven splits and for a rank whose share is
empty."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from paper_2307_02043_gb300 import sharded  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from oracle import physics
    w = synth.small("ls32", n=8, L=6, batch=3)
    kd = synth.illumination_dirs(w)
    om = physics.Model(w.n, kd, "ls", tol=1e-12)
    xt = synth.phantom(w)
    ys = physics.simulate(om, xt, synth.noise_draws(w), w.snr_db)
    return w, om, 0.7 * xt, ys


def _rank_main(rank, world, port, out_dir, illum):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, om, x, ys = _problem()
        calls = []

        def grad_fn(mine, scale):
            calls.append(list(mine))
            loss, g = om.batch_loss_grad(x, mine, ys, scale)
            return torch.from_numpy(np.ascontiguousarray(g)), loss

        g, loss = sharded.sharded_gradient(grad_fn, illum, w.S / w.L, rank, world,
                                           lambda: torch.zeros(x.shape, dtype=torch.float64))
        np.save(os.path.join(out_dir, "g%d.npy" % rank), g.numpy())
        with open(os.path.join(out_dir, "r%d.txt" % rank), "w") as f:
            f.write("%r\n%r\n" % (loss, calls))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("illum", [[0, 1, 2, 3], [0, 2, 4, 1, 5], [3]])
def test_sharded_gradient_world2_equals_full_subset(tmp_path, illum):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), illum), nprocs=world, join=True,
                       start_method="spawn")
    w, om, x, ys = _problem()
    loss_ref, g_ref = om.batch_loss_grad(x, illum, ys, w.S / w.L)
    shares = []
    for r in range(world):
        g = np.load(tmp_path / ("g%d.npy" % r))
        with open(tmp_path / ("r%d.txt" % r)) as f:
            loss, calls = [eval(line) for line in f.read().splitlines()]
        assert np.linalg.norm(g - g_ref) <= 1e-13 * np.linalg.norm(g_ref)
        assert abs(loss - loss_ref) <= 1e-13 * abs(loss_ref)
        shares += [l for c in calls for l in c]
        assert len(calls) == (1 if sharded.shard(illum, r, world) else 0)
    assert sorted(shares) == sorted(illum)   # every illumination on exactly one rank


def test_shard_partition():
    for n_il in range(0, 9):
        il = list(range(10, 10 + n_il))
        for world in (1, 2, 3, 4):
            parts = [sharded.shard(il, r, world) for r in range(world)]
            assert sorted(sum(parts, [])) == il
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        sharded.shard([1, 2], 2, 2)
