"""GPU parity at the workloads' full sizes, in the launch configuration the
bench times (batch 8 at 128^3, batch 16 at 192^3, the uneven grids 96^3 and
160^3), through outputs the oracle computes one by one and properties that
hold at any size.

Tolerances (written per test):
  * Green's apply: 2e-6 relative (max-norm), the complex64 transform floor, as
    in the small-size parity tests.
  * Born gradient: the Born loss is exactly quadratic in x, so its central
    difference equals <grad, d> for any step; only FP32/complex64 rounding of
    the fields remains: 1e-4.
  * LS gradient: central difference with step 0.02 along the phantom; the
    truncation term is ~(0.02 x phase shift)^2 ~ 1e-4 and the loss noise of a
    1e-6 Krylov tolerance ~1e-5 / 0.16 relative, so 2e-3.
  * batching: slots of one batched launch and separate launches differ only in
    the summation order of the gradient over illuminations: 1e-5.
  * against the oracle at 128^3: gradient 1e-4 norm-wise and loss 1e-5 with the
    GPU Krylov solves run to 1e-6 (the complex64 floor) and the oracle's to
    1e-9; weighted proximal map 1e-5 norm-wise at equal dual iterations (the
    tolerances of the small-size parity tests).
"""
import math

import numpy as np
import pytest

import synth
from oracle import physics
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


def subset_of(w):
    so = np.zeros(w.L, dtype=np.int32)
    for s, ii in enumerate(synth.subsets(w)):
        so[ii] = s
    return so


def handle(w, model, tol, max_batch, one_subset=False):
    """A handle for workload w; one_subset puts every illumination in one
    subset (the gradient calls below name their illuminations explicitly)."""
    so = np.zeros(w.L, dtype=np.int32) if one_subset else subset_of(w)
    S = 1 if one_subset else w.S
    return binding.MQNPM(w.n, synth.illumination_dirs(w), so, [1.0] * S, model=model,
                         krylov_tol=tol, krylov_maxit=500, max_batch=max_batch, tv=w.tv, lam=w.lam, box=w.box)


def phantom(w):
    return torch.from_numpy(synth.phantom(w).astype(np.float32)).to(DEV).reshape(-1)


def measure(h, w, xt, illum):
    """Noise-free data of the phantom for the illuminations used (others 0)."""
    y_sub, _ = h.forward(xt, illum)
    y = torch.zeros((w.L, w.n * w.n), dtype=torch.complex64, device=DEV)
    y[torch.tensor(illum, device=DEV)] = y_sub
    h.set_measurements(y.reshape(-1))


def dot64(a, b):
    return float(torch.dot(a.double(), b.double()))


def central_difference_check(h, x0, d, illum, eps, tol):
    g, f0, its = h.grad_batch(x0, illum, 1.0)
    g = g.clone()
    _, fp, _ = h.grad_batch(x0 + eps * d, illum, 1.0)
    _, fm, _ = h.grad_batch(x0 - eps * d, illum, 1.0)
    fd = (fp - fm) / (2 * eps)
    an = dot64(g, d)
    assert np.isfinite(f0) and f0 > 0
    assert abs(fd - an) <= tol * abs(an), (fd, an, abs(fd - an) / abs(an))
    return its


# --------------------------------------------------------------- Green's apply
@pytest.mark.parametrize("adjoint", [False, True])
def test_green_dense_128_matches_oracle(adjoint):
    """All outputs of G v / G^H v at 128^3 (P = 256) against the FP64 oracle."""
    n = 128
    rng = np.random.default_rng(11 + adjoint)
    v = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    w = synth.workload("ls128")
    h = handle(w, "ls", 1e-4, 1)
    out = h.green_apply(torch.from_numpy(v.astype(np.complex64)).to(DEV).reshape(-1), adjoint=adjoint)
    ref = physics.green_apply(v, physics.green_hat(n, KB), adjoint=adjoint)
    assert relmax(out.cpu().numpy().reshape(n, n, n), ref) < 2e-6
    h.close()


@pytest.mark.parametrize("n,adjoint", [(96, False), (160, False), (192, False), (192, True)])
def test_green_sampled_direct_sum(n, adjoint):
    """Grids of the uneven mix (96, 160) and of the large case (192, the largest
    transform): sampled outputs against the direct sum over a sparse support."""
    rng = np.random.default_rng(n)
    v = np.zeros((n, n, n), dtype=np.complex128)
    idx = rng.integers(0, n, size=(400, 3))
    v[idx[:, 0], idx[:, 1], idx[:, 2]] = rng.standard_normal(400) + 1j * rng.standard_normal(400)
    h = binding.MQNPM(n, [[0.0, 0.0, 1.0]], [0], [1.0], max_batch=1)
    out = h.green_apply(torch.from_numpy(v.astype(np.complex64)).to(DEV).reshape(-1), adjoint=adjoint)
    out = out.cpu().numpy().reshape(n, n, n)
    w0 = physics.self_term(KB)
    src = np.argwhere(v != 0)
    vals = v[v != 0]
    for probe in rng.integers(0, n, size=(16, 3)):
        dd = src - probe[None, :]
        r = np.sqrt(np.sum(dd * dd, axis=1).astype(np.float64))
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.exp(1j * KB * r) / (4 * math.pi * r)
        g[r == 0] = w0
        if adjoint:
            g = np.conj(g)
        ref = KB ** 2 * np.sum(g * vals)
        assert abs(out[tuple(probe)] - ref) <= 2e-6 * np.max(np.abs(out)) + 1e-6 * abs(ref), probe
    h.close()


# ------------------------------------------------------------------ gradients
def test_born128_gradient_is_the_exact_derivative():
    """born128, batch 8: the Born loss is quadratic, so the central difference
    along the phantom equals <grad, d> up to rounding."""
    w = synth.workload("born128")
    h = handle(w, "born", 1e-6, w.batch)
    xt = phantom(w)
    illum = [int(i) for i in synth.subsets(w)[0]]
    measure(h, w, xt, illum)
    central_difference_check(h, 0.5 * xt, xt, illum, 0.25, 1e-4)
    h.close()


def test_ls128_gradient_central_difference():
    """ls128, batch 8 (the measured launch shape), Krylov tolerance 1e-6."""
    w = synth.workload("ls128")
    h = handle(w, "ls", 1e-6, w.batch)
    xt = phantom(w)
    illum = [int(i) for i in synth.subsets(w)[0]]
    assert len(illum) == 8
    measure(h, w, xt, illum)
    its = central_difference_check(h, 0.5 * xt, xt, illum, 0.02, 2e-3)
    assert all(a > 0 and b > 0 for a, b in its)
    h.close()


def test_ls128_gradient_16_seeded_directions():
    """ls128 with the hand-written adjoint: the mini-batch gradient against
    central differences of the loss along 16 seeded directions, each a
    Gaussian bump (sigma 4 voxels) centred on a random voxel of the phantom
    (the voxel-direction gradient check of the autograd configuration), batch
    8, Krylov tol 1e-6."""
    w = synth.workload("ls128")
    h = handle(w, "ls", 1e-6, w.batch)
    xt = phantom(w)
    illum = [int(i) for i in synth.subsets(w)[0]]
    measure(h, w, xt, illum)
    x0 = 0.5 * xt
    g, f0, _ = h.grad_batch(x0, illum, 1.0)
    g = g.clone()
    n = w.n
    support = np.argwhere(xt.reshape(n, n, n).cpu().numpy() > 0)
    rng = np.random.default_rng(16)
    centres = support[rng.choice(len(support), 16, replace=False)]
    ax = np.arange(n, dtype=np.float64)
    for k, (cz, cy, cx) in enumerate(centres):
        bz, by, bx = (np.exp(-(ax - c) ** 2 / (2 * 4.0 ** 2)) for c in (cz, cy, cx))
        d = torch.from_numpy((bz[:, None, None] * by[None, :, None] * bx[None, None, :]).astype(np.float32)
                             .reshape(-1)).to(DEV)
        eps = 0.01
        fp, _ = h.loss_batch(x0 + eps * d, illum, 1.0)
        fm, _ = h.loss_batch(x0 - eps * d, illum, 1.0)
        fd = (fp - fm) / (2 * eps)
        an = dot64(g, d)
        assert abs(fd - an) <= 5e-3 * abs(an), (k, fd, an, abs(fd - an) / abs(an))
    assert np.isfinite(f0) and f0 > 0
    h.close()


def test_ls128_batched_equals_single_launches():
    """The bench configuration (batch 8, tolerance 1e-4): each slot of the
    batched solve gives the gradient and iteration counts of a solve alone."""
    w = synth.workload("ls128")
    hb = handle(w, "ls", w.krylov_tol, w.batch)
    h1 = handle(w, "ls", w.krylov_tol, 1)
    xt = phantom(w)
    illum = [int(i) for i in synth.subsets(w)[0]]
    measure(hb, w, xt, illum)
    measure(h1, w, xt, illum)
    x0 = 0.5 * xt
    gb, fb, itb = hb.grad_batch(x0, illum, 1.0)
    gb = gb.clone()
    acc = torch.zeros_like(gb, dtype=torch.float64)
    f1 = 0.0
    its1 = []
    for l in illum:
        g, f, it = h1.grad_batch(x0, [l], 1.0)
        acc += g.double()
        f1 += f
        its1 += it
    assert itb == its1
    assert abs(fb - f1) <= 1e-6 * abs(f1)
    assert float((gb.double() - acc).norm() / acc.norm()) < 1e-5
    hb.close()
    h1.close()


def test_ls192_batch16_gradient():
    """ls192 (the largest grid, P = 384), batch 16 workspace: the batched
    gradient of 15 illuminations is finite and a 4-illumination central
    difference matches it."""
    w = synth.workload("ls192")
    h = handle(w, "ls", 1e-6, w.batch)
    xt = phantom(w)
    illum = [int(i) for i in synth.subsets(w)[0]]
    assert len(illum) == 15
    measure(h, w, xt, illum)
    g, f, its = h.grad_batch(0.5 * xt, illum, w.S / w.L)
    assert torch.isfinite(g).all() and f > 0 and all(a > 0 and b > 0 for a, b in its)
    central_difference_check(h, 0.5 * xt, xt, illum[:4], 0.02, 2e-3)
    h.close()


@pytest.mark.parametrize("n", [96, 160])
def test_uneven_grid_gradient(n):
    """The first request of the uneven mix with grid n (its L, cone and batch
    size b as the workspace): central difference of its first subset's
    gradient.  The handle holds one subset because the mix has S = ceil(L/b)
    up to 15 and the gradient does not depend on the partition."""
    w = next(r for r in synth.uneven_requests() if r.n == n)
    h = handle(w, "ls", 1e-6, w.batch, one_subset=True)
    xt = phantom(w)
    illum = [int(i) for i in synth.subsets(w)[0]]
    measure(h, w, xt, illum)
    central_difference_check(h, 0.5 * xt, xt, illum, 0.02, 2e-3)
    h.close()


# ------------------------------------------------- against the oracle at 128^3
def test_ls128_gradient_matches_oracle():
    """ls128 in the bench's launch configuration (batch-8 workspace, the
    autotuned launch shapes): two illuminations of subset 0, F_s scaling S/L,
    at x = 0.5 x_true, against the FP64 oracle's adjoint-state gradient at the
    same (float32-rounded) x.  The measurements are zero, so the data term is
    1/2 ||S(u - u_in)||^2 and no input comes from the GPU path."""
    w = synth.workload("ls128")
    h = handle(w, "ls", 1e-6, w.batch)
    illum = [int(i) for i in synth.subsets(w)[0][:2]]
    x0 = (0.5 * synth.phantom(w)).astype(np.float32)
    h.set_measurements(torch.zeros(w.L * w.n * w.n, dtype=torch.complex64, device=DEV))
    scale = w.S / w.L
    g, f, its = h.grad_batch(torch.from_numpy(x0).to(DEV).reshape(-1), illum, scale)
    g = g.cpu().numpy().astype(np.float64).reshape(w.n, w.n, w.n)
    h.close()
    om = physics.Model(w.n, synth.illumination_dirs(w), "ls", tol=1e-9)
    ys = np.zeros((w.L, w.n * w.n), dtype=np.complex128)
    fo, go = om.batch_loss_grad(x0.astype(np.float64), illum, ys, scale)
    assert all(a > 0 and b > 0 for a, b in its)
    assert abs(f - fo) <= 1e-5 * abs(fo), (f, fo)
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go), np.linalg.norm(g - go) / np.linalg.norm(go)


@pytest.mark.parametrize("kind", ["iso", "aniso"])
def test_wprox_128_rank8_matches_oracle(kind):
    """The weighted proximal map at the bench's grid and rank (128^3, eight
    rank-one terms, 20 dual iterations, warm-started dual field).  The
    cooperative kernel's grid-stride loops take several trips per phase at this
    size (304 blocks x 256 threads x 4 voxels per trip), which no small grid
    reaches."""
    n, S_eff, J, tau, c = 128, 8, 20, 1.5, 2e-3
    rng = np.random.default_rng(128 + (kind == "aniso"))
    v = rng.uniform(-0.02, 0.07, (n, n, n))
    v[n // 4: n // 2, n // 4: 3 * n // 4, :] += 0.03
    U = rng.standard_normal((S_eff, n, n, n)) * 0.05
    P0 = rng.uniform(-0.5, 0.5, (3, n, n, n))
    h = binding.MQNPM(n, [[0.0, 0.0, 1.0]], [0], [1.0], tv=kind, box=(0.0, 0.05), dual_iters=J,
                      newton_tol=1e-6, max_batch=1)
    Pw = torch.from_numpy(P0.astype(np.float32)).to(DEV).reshape(-1)
    xg = h.wprox(torch.from_numpy(v.astype(np.float32)).to(DEV).reshape(-1), tau,
                 torch.from_numpy(U.astype(np.float32)).to(DEV).reshape(-1), c, P_warm=Pw)
    xg = xg.cpu().numpy().astype(np.float64).reshape(n, n, n)
    Pg = Pw.cpu().numpy().astype(np.float64).reshape(3, n, n, n)
    h.close()
    xo, Po, _ = owprox.wprox(v.astype(np.float32).astype(np.float64), tau,
                             U.astype(np.float32).astype(np.float64), c, 0.0, 0.05, kind, J,
                             P0=P0.astype(np.float32).astype(np.float64), newton_tol=1e-6)
    assert np.linalg.norm(xg - xo) <= 1e-5 * np.linalg.norm(xo), np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert np.linalg.norm(Pg - Po) <= 1e-4 * np.linalg.norm(Po)


def test_ls192_gradient_matches_oracle():
    """ls192 (P = 384, the largest transform) in the bench's launch
    configuration (batch-16 workspace): one illumination's gradient and loss
    against the FP64 oracle at the same x, measurements zero (no input from
    the GPU path)."""
    w = synth.workload("ls192")
    h = handle(w, "ls", 1e-6, w.batch)
    x0 = (0.5 * synth.phantom(w)).astype(np.float32)
    h.set_measurements(torch.zeros(w.L * w.n * w.n, dtype=torch.complex64, device=DEV))
    illum = [int(synth.subsets(w)[0][0])]
    g, f, its = h.grad_batch(torch.from_numpy(x0).to(DEV).reshape(-1), illum, 1.0)
    g = g.cpu().numpy().astype(np.float64).reshape(w.n, w.n, w.n)
    h.close()
    om = physics.Model(w.n, synth.illumination_dirs(w), "ls", tol=1e-9)
    fo, go = om.batch_loss_grad(x0.astype(np.float64), illum, np.zeros((w.L, w.n * w.n), np.complex128), 1.0)
    assert its[0][0] > 0 and its[0][1] > 0
    assert abs(f - fo) <= 1e-5 * abs(fo), (f, fo)
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go), np.linalg.norm(g - go) / np.linalg.norm(go)


def test_ls192_recomputed_fields_equal_stored_fields():
    """The recompute path of the autograd split at the large configuration: a
    15-illumination subset on a 4-slot workspace cannot keep its forward
    fields between the loss and the gradient call, so the gradient call
    recomputes them chunk by chunk; it equals the gradient of a 16-slot
    workspace that holds the whole subset (summation regrouped: 1e-5)."""
    w = synth.workload("ls192")
    xt = phantom(w)
    illum = [int(i) for i in synth.subsets(w)[0]]
    big = handle(w, "ls", w.krylov_tol, 16)
    measure(big, w, xt, illum)
    x0 = 0.5 * xt
    gb, fb, _ = big.grad_batch(x0, illum, w.S / w.L)
    gb = gb.clone()
    y = torch.zeros((w.L, w.n * w.n), dtype=torch.complex64, device=DEV)
    y[torch.tensor(illum, device=DEV)] = big.forward(xt, illum)[0]
    big.close()
    small = handle(w, "ls", w.krylov_tol, 4)
    small.set_measurements(y.reshape(-1))
    fs, _ = small.loss_batch(x0, illum, w.S / w.L)
    gs, reused = small.grad_fields(x0, illum, w.S / w.L)
    assert not reused
    assert abs(fs - fb) <= 1e-6 * abs(fb)
    assert float((gs.double() - gb.double()).norm() / gb.double().norm()) < 1e-5
    small.close()
