"""GPU parity on box-shaped grids (nz x ny x nx, each transform length 2 n_d
compiled separately) against the FP64 oracle: the Green's apply at every
launch-shape tile (where a column tile reaches past 2 nx it is masked), the
truncated kernel, LS and Born gradients, the remote detector, the weighted
proximal mapping and a short outer-loop trajectory.

Tolerances as in the cubic parity tests: apply 2e-6 (max-norm), forward data
2e-5, gradient 1e-4 and loss 1e-5 at Krylov tolerance 1e-6, prox 1e-5
(norm-wise), trajectory iterates 2e-3 and objective 1e-4.
"""
import math

import numpy as np
import pytest

import synth
from oracle import bqnpm, physics
from oracle import wprox as owprox

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2307_02043_gb300 import binding  # noqa: E402

DEV = torch.device("cuda:0")
KB = math.pi / 2


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def c64(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).to(DEV)


def f32(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.float32)).to(DEV)


def box_workload(shape, model="ls", L=6, batch=3, **kw):
    w = synth.small("ls32", n=max(shape), L=L, batch=batch, model=model).with_(grid=tuple(shape), **kw)
    return w


def problem(shape, model="ls", L=6, batch=3, contrast=0.05, det_na=0.0, det_distance=0.0):
    w = box_workload(shape, model, L, batch, contrast_max=contrast)
    kd = synth.illumination_dirs(w)
    om = physics.Model(shape, kd, model, tol=1e-12, det_na=det_na, det_distance=det_distance)
    xt = synth.phantom(w)
    ys = physics.simulate(om, xt, synth.noise_draws(w), w.snr_db)
    so = np.zeros(w.L, dtype=np.int32)
    for s, ii in enumerate(synth.subsets(w)):
        so[ii] = s
    return w, kd, om, xt, ys, so


@pytest.mark.parametrize("shape", [(16, 24, 32), (32, 24, 16), (12, 8, 16), (24, 16, 48), (8, 32, 12)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_box_green_apply_matches_oracle(shape, adjoint):
    rng = np.random.default_rng(sum(shape) + adjoint)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    h = binding.MQNPM(shape, [[0.0, 0.0, 1.0]], [0], [1.0], max_batch=2)
    out = h.green_apply(c64(np.stack([v, 2 * v])).reshape(-1), adjoint=adjoint).cpu().numpy().reshape(2, *shape)
    ref = physics.green_apply(v, physics.green_hat(shape, KB), adjoint=adjoint)
    assert relmax(out[0], ref) < 2e-6 and relmax(out[1], 2 * ref) < 2e-6
    h.close()


@pytest.mark.parametrize("shape", [(12, 16, 24), (16, 32, 12)])
def test_box_every_tile_gives_the_same_apply(shape):
    """All sixteen launch-shape tiles on a box whose column tiles do not all
    divide 2 nx (the last tile of a column pass is masked there): identical
    outputs, equal to the oracle's."""
    rng = np.random.default_rng(7 + sum(shape))
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = physics.green_apply(v, physics.green_hat(shape, KB))
    first = None
    for tile in range(16):
        try:
            h = binding.MQNPM(shape, [[0.0, 0.0, 1.0]], [0], [1.0], max_batch=1, tile=tile)
        except binding.MQNPMError as err:     # a tile whose shared memory does not fit
            assert err.code == 1
            continue
        out = h.green_apply(c64(v).reshape(-1)).cpu().numpy().reshape(shape)
        h.close()
        assert relmax(out, ref) < 2e-6, tile
        if first is None:
            first = out
        else:
            assert np.array_equal(out, first), tile


def test_box_truncated_kernel_matches_oracle():
    shape = (12, 16, 24)
    rng = np.random.default_rng(12)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    h = binding.MQNPM(shape, [[0.0, 0.0, 1.0]], [0], [1.0], max_batch=1, green_kernel="truncated")
    out = h.green_apply(c64(v).reshape(-1)).cpu().numpy().reshape(shape)
    ref = physics.green_apply(v, physics.green_hat(shape, KB, 1.0, "truncated"))
    assert relmax(out, ref) < 2e-6
    h.close()


@pytest.mark.parametrize("model", ["ls", "born"])
@pytest.mark.parametrize("shape", [(12, 16, 24), (24, 16, 12)])
def test_box_forward_and_gradient_match_oracle(model, shape):
    w, kd, om, xt, ys, so = problem(shape, model)
    h = binding.MQNPM(shape, kd, so, [1.0] * w.S, model=model, krylov_tol=1e-6, max_batch=2)
    y, _ = h.forward(f32(xt).reshape(-1), [0, 3])
    for b, l in enumerate([0, 3]):
        assert rel(y[b].cpu().numpy(), om.forward(xt, l)) < 2e-5
    h.set_measurements(c64(ys).reshape(-1))
    x = 0.7 * xt
    scale = w.S / w.L
    g, loss, _ = h.grad_batch(f32(x).reshape(-1), [0, 1, 2], scale)
    lo, go = om.batch_loss_grad(x, [0, 1, 2], ys, scale)
    assert rel(g.cpu().numpy().reshape(shape), go) < 1e-4
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    h.close()


def test_box_remote_detector_matches_oracle():
    shape = (12, 16, 24)
    w, kd, om, xt, ys, so = problem(shape, "ls", det_na=0.9, det_distance=5.0)
    h = binding.MQNPM(shape, kd, so, [1.0] * w.S, krylov_tol=1e-6, max_batch=3, det_na=0.9, det_distance=5.0)
    h.set_measurements(c64(ys).reshape(-1))
    x = 0.7 * xt
    g, loss, _ = h.grad_batch(f32(x).reshape(-1), [1, 4], 1.0)
    lo, go = om.batch_loss_grad(x, [1, 4], ys, 1.0)
    assert rel(g.cpu().numpy().reshape(shape), go) < 1e-4
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    h.close()


@pytest.mark.parametrize("kind", ["iso", "aniso"])
@pytest.mark.parametrize("shape", [(16, 24, 32), (8, 12, 16)])
def test_box_wprox_matches_oracle(kind, shape):
    rng = np.random.default_rng(sum(shape) + (kind == "aniso"))
    v = rng.uniform(-0.02, 0.07, shape)
    U = rng.standard_normal((3, *shape)) * 0.05
    P0 = rng.uniform(-0.5, 0.5, (3, *shape))
    tau, c, J = 1.5, 2e-3, 12
    xo, Po, _ = owprox.wprox(v, tau, U, c, 0.0, 0.05, kind, J, P0=P0, newton_tol=1e-6)
    h = binding.MQNPM(shape, [[0.0, 0.0, 1.0]], [0], [1.0], tv=kind, box=(0.0, 0.05), dual_iters=J,
                      newton_tol=1e-6, max_batch=1)
    Pw = f32(P0).reshape(-1).clone()
    xg = h.wprox(f32(v).reshape(-1), tau, f32(U).reshape(-1), c, P_warm=Pw)
    assert rel(xg.cpu().numpy().reshape(shape), xo) < 1e-5
    assert rel(Pw.cpu().numpy().reshape(3, *shape), Po) < 1e-4
    h.close()


def test_box_step_trajectory_matches_oracle():
    """Algorithm 4.1 with SR1 on a 8 x 12 x 16 box, L = 4, S = 2, six iterations."""
    shape = (8, 12, 16)
    w, kd, om, xt, ys, so = problem(shape, "ls", L=4, batch=2, contrast=0.02)
    subs = synth.subsets(w)
    alpha = [om.lipschitz(s, w.S / w.L, synth.power_start(w), 20) for s in subs]
    opt = bqnpm.BQNPM(om, ys, subs, alpha, lam=1e-4, box=w.box, kind="iso", dual_iters=w.dual_iters,
                      gamma=w.gamma, step=w.step)
    xs = opt.run(np.zeros(shape), 6)
    h = binding.MQNPM(shape, kd, so, alpha, tv="iso", lam=1e-4, box=w.box, krylov_tol=1e-6,
                      dual_iters=w.dual_iters, gamma=w.gamma, step=w.step, max_batch=2)
    h.set_measurements(c64(ys).reshape(-1))
    x = torch.zeros(w.N, dtype=torch.float32, device=DEV)
    for k in range(1, 7):
        info = h.step(x)
        assert info["subset"] == opt.history[k - 1]["s"]
        xg = x.cpu().numpy().astype(np.float64).reshape(shape)
        assert rel(xg, xs[k]) < 2e-3, k
    assert abs(opt.full_cost(xg) - opt.full_cost(xs[6])) <= 1e-4 * abs(opt.full_cost(xs[6]))
    h.close()
