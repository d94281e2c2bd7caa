"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (written per test): the transforms run in complex64, so the Green's
apply is held to 2e-6 relative (max-norm); solves run BiCGSTAB to a relative
residual of 1e-6 in complex64 with FP64 inner products, so gradients are held to
1e-4 (norm-wise) and losses to 1e-5; the proximal mapping runs in float32 with
FP64 reductions and is held to 1e-5 (norm-wise) at equal dual iterations.
"""
import math

import numpy as np
import pytest

import synth
from oracle import physics, wprox as owprox, tv as otv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2307_02043_gb300 import binding  # noqa: E402

DEV = torch.device("cuda:0")
KB = math.pi / 2


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def relmax(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b))))


def make_handle(n, kd, subset_of, alpha, **kw):
    kw.setdefault("max_batch", 4)
    return binding.MQNPM(n, kd, subset_of, alpha, **kw)


def cone(L, deg=30.0):
    t = math.radians(deg)
    return np.array([[math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)]
                     for p in 2 * math.pi * np.arange(L) / L])


def c64(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).to(DEV)


def f32(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.float32)).to(DEV)


# ------------------------------------------------------------- Green's apply
@pytest.mark.parametrize("n", [8, 12, 16, 24, 32, 48, 64])
@pytest.mark.parametrize("adjoint", [False, True])
def test_green_apply_matches_oracle(n, adjoint):
    rng = np.random.default_rng(100 + n)
    nb = 3
    v = rng.standard_normal((nb, n, n, n)) + 1j * rng.standard_normal((nb, n, n, n))
    h = make_handle(n, cone(2), [0, 0], [1.0], max_batch=nb)
    out = h.green_apply(c64(v).reshape(-1), adjoint=adjoint).cpu().numpy().reshape(nb, n, n, n)
    kh = physics.green_hat(n, KB)
    for b in range(nb):
        ref = physics.green_apply(v[b], kh, adjoint=adjoint)
        assert relmax(out[b], ref) < 2e-6, (n, b, relmax(out[b], ref))
    h.close()


def test_green_apply_full_size_sampled():
    """n = 128 (P = 256, the measured size): sampled outputs against the direct sum."""
    n = 128
    rng = np.random.default_rng(7)
    v = np.zeros((n, n, n), dtype=np.complex128)
    # sparse random support keeps the direct sum cheap and exact
    idx = rng.integers(0, n, size=(400, 3))
    v[idx[:, 0], idx[:, 1], idx[:, 2]] = rng.standard_normal(400) + 1j * rng.standard_normal(400)
    h = make_handle(n, cone(2), [0, 0], [1.0], max_batch=1)
    out = h.green_apply(c64(v).reshape(-1)).cpu().numpy().reshape(n, n, n)
    a = (3 / (4 * math.pi)) ** (1 / 3)
    w0 = physics.self_term(KB)
    src = np.argwhere(v != 0)
    vals = v[v != 0]
    for probe in rng.integers(0, n, size=(12, 3)):
        d = src - probe[None, :]
        r = np.sqrt(np.sum(d * d, axis=1).astype(np.float64))
        with np.errstate(divide="ignore", invalid="ignore"):
            w = np.exp(1j * KB * r) / (4 * math.pi * r)
        w[r == 0] = w0
        ref = KB ** 2 * np.sum(w * vals)
        assert abs(out[tuple(probe)] - ref) <= 2e-6 * np.max(np.abs(out)) + 1e-6 * abs(ref), probe
    h.close()


# ---------------------------------------------------------------- forward/grad
@pytest.mark.parametrize("n", [12, 32])
def test_green_apply_with_host_spectrum(n):
    """A caller-provided spectrum replaces the built one: the octant of the
    oracle's DFT_P at another wavenumber gives that wavenumber's G, and the
    octant at the handle's own wavenumber reproduces the built spectrum."""
    rng = np.random.default_rng(300 + n)
    nb = 2
    v = rng.standard_normal((nb, n, n, n)) + 1j * rng.standard_normal((nb, n, n, n))
    kb2 = math.pi / 3
    kh2 = physics.green_hat(n, kb2)
    h = make_handle(n, cone(2), [0, 0], [1.0], max_batch=nb, green_hat=kh2[:n + 1, :n + 1, :n + 1])
    for adjoint in (False, True):
        out = h.green_apply(c64(v).reshape(-1), adjoint=adjoint).cpu().numpy().reshape(nb, n, n, n)
        for b in range(nb):
            ref = physics.green_apply(v[b], kh2, adjoint=adjoint)
            assert relmax(out[b], ref) < 2e-6, (n, adjoint, b, relmax(out[b], ref))
    h.close()
    kh = physics.green_hat(n, KB)
    ha = make_handle(n, cone(2), [0, 0], [1.0], max_batch=nb, green_hat=kh[:n + 1, :n + 1, :n + 1])
    hb = make_handle(n, cone(2), [0, 0], [1.0], max_batch=nb)
    oa = ha.green_apply(c64(v).reshape(-1)).cpu().numpy()
    ob = hb.green_apply(c64(v).reshape(-1)).cpu().numpy()
    assert relmax(oa, ob) < 1e-6
    ha.close()
    hb.close()


def test_host_spectrum_rejects_bad_input():
    n = 8
    bad = physics.green_hat(n, KB)[:n + 1, :n + 1, :n + 1].copy()
    bad[1, 2, 3] = np.nan
    with pytest.raises(binding.MQNPMError):
        make_handle(n, cone(2), [0, 0], [1.0], green_hat=bad)
    with pytest.raises(ValueError):
        make_handle(n, cone(2), [0, 0], [1.0], green_hat=bad[:n])


def problem(n, model, L=4, batch=2, contrast=None, seed_name="ls32"):
    w = synth.small(seed_name, n=n, L=L, batch=batch, model=model)
    if contrast is not None:
        w = w.with_(contrast_max=contrast)
    kd = synth.illumination_dirs(w)
    xt = synth.phantom(w)
    om = physics.Model(n, kd, model, tol=1e-12)
    ys = physics.simulate(om, xt, synth.noise_draws(w), w.snr_db)
    subs = synth.subsets(w)
    so = np.zeros(w.L, dtype=np.int32)
    for s, ii in enumerate(subs):
        so[ii] = s
    return w, kd, xt, om, ys, subs, so


@pytest.mark.parametrize("model", ["ls", "born"])
@pytest.mark.parametrize("n", [16, 24])
def test_forward_matches_oracle(model, n):
    w, kd, xt, om, ys, subs, so = problem(n, model, contrast=0.05)
    h = make_handle(n, kd, so, [1.0] * w.S, model=model, krylov_tol=1e-7, max_batch=3)
    illum = [0, 1, 3]
    y, its = h.forward(f32(xt).reshape(-1), illum)
    y = y.cpu().numpy()
    for b, l in enumerate(illum):
        ref = om.forward(xt, l)
        assert rel(y[b], ref) < 2e-5, (model, l, rel(y[b], ref), its)
    h.close()


@pytest.mark.parametrize("model", ["ls", "born"])
@pytest.mark.parametrize("n,nb,max_batch", [(16, 2, 2), (24, 3, 2), (32, 2, 2)])
def test_grad_batch_matches_oracle(model, n, nb, max_batch):
    w, kd, xt, om, ys, subs, so = problem(n, model, L=6, batch=3)
    h = make_handle(n, kd, so, [1.0] * w.S, model=model, krylov_tol=1e-6, max_batch=max_batch)
    h.set_measurements(c64(ys).reshape(-1))
    x = 0.7 * xt
    illum = list(range(nb))
    scale = w.S / w.L
    g, loss, its = h.grad_batch(f32(x).reshape(-1), illum, scale)
    lo, go = om.batch_loss_grad(x, illum, ys, scale)
    assert rel(g.cpu().numpy().reshape(go.shape), go) < 1e-4
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    if model == "ls":
        assert all(a > 0 and b > 0 for a, b in its)
    h.close()


@pytest.mark.parametrize("start", ["b", "zero"])
@pytest.mark.parametrize("n", [24, 32])
def test_both_adjoint_starts_match_oracle(start, n):
    """The LS adjoint solve (I - G^H X) z = G^H S^T r started at b or at 0
    (mqnpm_config.adjoint_start): the same gradient to the solver tolerance,
    against the oracle (which starts at 0)."""
    w, kd, xt, om, ys, subs, so = problem(n, "ls", L=6, batch=3)
    h = make_handle(n, kd, so, [1.0] * w.S, krylov_tol=1e-6, max_batch=3, adjoint_start=start)
    h.set_measurements(c64(ys).reshape(-1))
    x = 0.7 * xt
    illum = [0, 2, 4]
    scale = w.S / w.L
    g, loss, its = h.grad_batch(f32(x).reshape(-1), illum, scale)
    lo, go = om.batch_loss_grad(x, illum, ys, scale)
    assert rel(g.cpu().numpy().reshape(go.shape), go) < 1e-4, (start, its)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    assert all(a > 0 and b > 0 for a, b in its)
    h.close()


@pytest.mark.parametrize("start", ["refine", "stored"])
@pytest.mark.parametrize("n", [24, 32])
def test_both_forward_starts_match_oracle(start, n):
    """Warm-started LS forward solves from the stored field as is or refined
    by one fixed-point step (mqnpm_config.forward_start): a first gradient at
    x1 stores every illumination's field, a second one at a nearby x2 starts
    from them; both gradients match the oracle (cold starts) to the solver
    tolerance (1e-7 here: a refined start often stops just below it, where
    BiCGSTAB's last iteration usually overshoots)."""
    w, kd, xt, om, ys, subs, so = problem(n, "ls", L=6, batch=3)
    h = make_handle(n, kd, so, [1.0] * w.S, krylov_tol=1e-7, max_batch=3, warm_start=True, forward_start=start)
    h.set_measurements(c64(ys).reshape(-1))
    illum = [0, 2, 4]
    scale = w.S / w.L
    for x in (0.7 * xt, 0.72 * xt):
        g, loss, its = h.grad_batch(f32(x).reshape(-1), illum, scale)
        lo, go = om.batch_loss_grad(x, illum, ys, scale)
        assert rel(g.cpu().numpy().reshape(go.shape), go) < 1e-4, (start, its)
        assert abs(loss - lo) <= 1e-5 * abs(lo)
    h.close()


def test_physical_units_strong_scattering_matches_oracle():
    """The paper's simulated set-up in physical units (50 nm voxels, 406 nm,
    medium index 1.333, contrast up to (1.43/1.333)^2 - 1 = 0.15) on a 32^3
    grid: forward fields and the mini-batch gradient against the oracle with
    the same h (metres) and k_b (per metre)."""
    n = 32
    w = synth.small("sim64", n=n, L=4, batch=2)
    kd = synth.illumination_dirs(w)
    xt = synth.phantom(w)
    assert xt.max() > 0.1
    om = physics.Model(n, kd, "ls", kb=w.kb, h=w.h, tol=1e-12)
    ys = physics.simulate(om, xt, synth.noise_draws(w), w.snr_db)
    so = np.zeros(w.L, dtype=np.int32)
    for s_, ii in enumerate(synth.subsets(w)):
        so[ii] = s_
    h = make_handle(n, kd, so, [1.0] * w.S, h=w.h, kb=w.kb, krylov_tol=1e-6, max_batch=2)
    h.set_measurements(c64(ys).reshape(-1))
    y, its = h.forward(f32(xt).reshape(-1), [0, 1])
    y = y.cpu().numpy()
    for b, l in enumerate([0, 1]):
        assert rel(y[b], om.forward(xt, l)) < 1e-4, (l, its)
    x = 0.7 * xt
    g, loss, its = h.grad_batch(f32(x).reshape(-1), [0, 1], w.S / w.L)
    lo, go = om.batch_loss_grad(x, [0, 1], ys, w.S / w.L)
    assert rel(g.cpu().numpy().reshape(go.shape), go) < 1e-4
    assert abs(loss - lo) <= 1e-4 * abs(lo)
    h.close()


@pytest.mark.parametrize("model,n,na", [("ls", 16, 0.8), ("ls", 24, 0.8), ("born", 16, 0.8), ("born", 24, 0.8),
                                         ("ls", 16, 1.5)])
def test_remote_detector_matches_oracle(model, n, na):
    """Detector behind an angular-spectrum propagation with a pupil (remote
    detector reading of Section 6): forward data, mini-batch gradient and the
    Born power iteration against the oracle with the same distance and NA
    (na > 1 lets evanescent components through, decaying)."""
    dist = 6.0
    w = synth.small("ls32", n=n, L=4, batch=2, model=model)
    kd = synth.illumination_dirs(w)
    xt = synth.phantom(w)
    om = physics.Model(n, kd, model, tol=1e-12, det_distance=dist, det_na=na)
    ys = physics.simulate(om, xt, synth.noise_draws(w), w.snr_db)
    so = np.zeros(w.L, dtype=np.int32)
    for s_, ii in enumerate(synth.subsets(w)):
        so[ii] = s_
    h = make_handle(n, kd, so, [1.0] * w.S, model=model, krylov_tol=1e-7, max_batch=2,
                    det_distance=dist, det_na=na)
    h.set_measurements(c64(ys).reshape(-1))
    y, _ = h.forward(f32(xt).reshape(-1), [0, 3])
    y = y.cpu().numpy()
    for b, l in enumerate([0, 3]):
        assert rel(y[b], om.forward(xt, l)) < 2e-5, (model, l)
    x = 0.7 * xt
    illum = [0, 1, 2]                      # two chunks of the 2-slot workspace
    g, loss, _ = h.grad_batch(f32(x).reshape(-1), illum, w.S / w.L)
    lo, go = om.batch_loss_grad(x, illum, ys, w.S / w.L)
    assert rel(g.cpu().numpy().reshape(go.shape), go) < 1e-4
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    start = synth.power_start(w)
    a_gpu = h.lipschitz([0, 2], w.S / w.L, f32(start).reshape(-1), iters=10)
    mb = physics.Model(n, kd, "born", det_distance=dist, det_na=na)
    a_ref = mb.lipschitz([0, 2], w.S / w.L, start, iters=10)
    assert abs(a_gpu - a_ref) <= 1e-4 * a_ref
    h.close()


def test_maximum_batch_of_64_slots():
    """MQNPM_MAX_BATCH = 64 slots in one launch (the pass-3 slot mask is 64
    bits wide): every slot's apply against the oracle, and the 64-illumination
    gradient in one chunk against 13 chunks of 5 and against the oracle."""
    n, L = 8, 64
    kd = cone(L, 35.0)
    so = np.zeros(L, dtype=np.int32)
    rng = np.random.default_rng(64)
    h = make_handle(n, kd, so, [1.0], max_batch=64, krylov_tol=1e-7)
    v = rng.standard_normal((L, n, n, n)) + 1j * rng.standard_normal((L, n, n, n))
    out = h.green_apply(c64(v).reshape(-1)).cpu().numpy().reshape(L, n, n, n)
    kh = physics.green_hat(n, KB)
    for b in (0, 1, 31, 32, 62, 63):
        assert relmax(out[b], physics.green_apply(v[b], kh)) < 2e-6, b
    x = 0.02 * rng.random((n, n, n))
    om = physics.Model(n, kd, "ls", tol=1e-12)
    ys = np.stack([om.forward(x, l) for l in range(L)])
    ys = ys + 0.01 * np.abs(ys).max() * (rng.standard_normal(ys.shape) + 1j * rng.standard_normal(ys.shape))
    h.set_measurements(c64(ys).reshape(-1))
    illum = list(range(L))
    g1, l1, its = h.grad_batch(f32(x).reshape(-1), illum, 1.0 / L)
    h.close()
    h5 = make_handle(n, kd, so, [1.0], max_batch=5, krylov_tol=1e-7)
    h5.set_measurements(c64(ys).reshape(-1))
    g5, l5, _ = h5.grad_batch(f32(x).reshape(-1), illum, 1.0 / L)
    h5.close()
    g1 = g1.cpu().numpy().astype(np.float64)
    assert rel(g1, g5.cpu().numpy()) < 1e-5
    assert abs(l1 - l5) <= 1e-6 * abs(l5)
    lo, go = om.batch_loss_grad(x, illum, ys, 1.0 / L)
    assert rel(g1.reshape(go.shape), go) < 1e-4
    assert abs(l1 - lo) <= 1e-5 * abs(lo)
    assert len(its) == L and all(a > 0 and b > 0 for a, b in its)


def test_grad_edge_cases():
    """Zero contrast (Krylov converges at start), zero residual (adjoint RHS 0)."""
    n = 16
    w, kd, xt, om, ys, subs, so = problem(n, "ls")
    h = make_handle(n, kd, so, [1.0] * w.S, krylov_tol=1e-6)
    zero = np.zeros((n, n, n))
    ys0 = np.stack([om.forward(zero, l) for l in range(w.L)])   # exact data of x = 0
    h.set_measurements(c64(ys0).reshape(-1))
    g, loss, its = h.grad_batch(f32(zero).reshape(-1), [0, 1], 1.0)
    assert loss == 0.0 and float(g.abs().max()) == 0.0
    assert its == [(0, 0), (0, 0)]
    h.close()


def test_lipschitz_matches_oracle():
    n = 16
    w, kd, xt, om, ys, subs, so = problem(n, "ls")
    start = synth.power_start(w)
    ref = om.lipschitz(subs[0], w.S / w.L, start, iters=10)
    h = make_handle(n, kd, so, [1.0] * w.S)
    a = h.lipschitz(list(subs[0]), w.S / w.L, f32(start).reshape(-1), iters=10)
    assert abs(a - ref) <= 1e-5 * ref
    h.close()


# ------------------------------------------------------------ proximal map
@pytest.mark.parametrize("kind,S_eff,n", [(k, s, m) for k in ("iso", "aniso") for s in (0, 1, 3, 4)
                                          for m in (8, 24)] + [("iso", 9, 8), ("aniso", 12, 8), ("iso", 16, 8),
                                                               ("iso", 16, 24)])
def test_wprox_matches_oracle(kind, S_eff, n):
    rng = np.random.default_rng(10 * S_eff + n)
    v = rng.uniform(-0.02, 0.07, (n, n, n))
    v[n // 4: n // 2, n // 4: 3 * n // 4, :] += 0.03
    U = rng.standard_normal((S_eff, n, n, n)) * 0.05 if S_eff else None
    tau, c, J = 1.5, 2e-3, 12
    P0 = rng.uniform(-0.5, 0.5, (3, n, n, n))
    xo, Po, info = owprox.wprox(v, tau, U, c, 0.0, 0.05, kind, J, P0=P0, newton_tol=1e-6)
    h = make_handle(n, cone(2), [0, 0], [1.0], tv=kind, box=(0.0, 0.05), dual_iters=J, newton_tol=1e-6)
    Pw = f32(P0).reshape(-1).clone()
    xg = h.wprox(f32(v).reshape(-1), tau, None if U is None else f32(U).reshape(-1), c, P_warm=Pw)
    assert rel(xg.cpu().numpy().reshape(xo.shape), xo) < 1e-5, rel(xg.cpu().numpy().reshape(xo.shape), xo)
    assert rel(Pw.cpu().numpy().reshape(Po.shape), Po) < 1e-4
    h.close()


# ------------------------------------------------------------------ autograd
@pytest.mark.parametrize("model", ["ls", "born"])
@pytest.mark.parametrize("nb,max_batch", [(3, 4), (5, 2)])
def test_autograd_split_matches_grad_batch_and_oracle(model, nb, max_batch):
    """LSGradient: forward = loss only, backward = adjoint solves.  With the
    batch inside the workspace the backward reuses the forward fields; with a
    larger batch it recomputes them.  Both give grad_batch's loss and gradient
    and the oracle's to the gradient tolerance."""
    from paper_2307_02043_gb300.autograd import LSGradient

    n = 16
    w, kd, xt, om, ys, subs, so = problem(n, model, L=6, batch=3)
    h = make_handle(n, kd, so, [1.0] * w.S, model=model, krylov_tol=1e-6, max_batch=max_batch)
    h.set_measurements(c64(ys).reshape(-1))
    x = (0.7 * f32(xt)).reshape(n, n, n).requires_grad_(True)
    illum = list(range(nb))
    scale = w.S / w.L
    loss = LSGradient.apply(x, h, illum, scale)
    loss.backward()
    assert h.last_backward_reused == (nb <= max_batch)
    g_ref, l_ref, _ = h.grad_batch(x.detach().reshape(-1).contiguous(), illum, scale)
    assert abs(float(loss.detach()) - l_ref) <= 1e-7 * abs(l_ref)
    assert rel(x.grad.reshape(-1).cpu().numpy(), g_ref.cpu().numpy()) < 1e-6
    lo, go = om.batch_loss_grad(0.7 * xt, illum, ys, scale)
    assert rel(x.grad.cpu().numpy().reshape(go.shape), go) < 1e-4
    assert abs(float(loss.detach()) - lo) <= 1e-5 * abs(lo)
    h.close()


def test_grad_fields_recomputes_after_other_calls():
    """Stored fields are dropped by any other use of the workspace: the
    gradient is then recomputed and still equal."""
    n = 16
    w, kd, xt, om, ys, subs, so = problem(n, "ls", L=6, batch=3)
    h = make_handle(n, kd, so, [1.0] * w.S, krylov_tol=1e-6, max_batch=4)
    h.set_measurements(c64(ys).reshape(-1))
    x = f32(0.7 * xt).reshape(-1)
    h.loss_batch(x, [0, 1], 1.0)
    h.forward(x, [2])                                   # uses the workspace
    g1, reused = h.grad_fields(x, [0, 1], 1.0)
    assert not reused
    h.loss_batch(x, [0, 1], 1.0)
    g2, reused = h.grad_fields(x, [0, 1], 1.0)
    assert reused
    g3, reused = h.grad_fields(x, [0, 1], 1.0)          # the adjoint solve used the workspace
    assert not reused
    ref, _, _ = h.grad_batch(x, [0, 1], 1.0)
    for g in (g1, g2, g3):
        assert rel(g.cpu().numpy(), ref.cpu().numpy()) < 1e-6
    h.close()


@pytest.mark.parametrize("case", ["no_dual_iterations", "point_box", "tiny_c", "large_tau"])
def test_wprox_degenerate_cases(case):
    """Degenerate proximal problems against the oracle: J = 0 (x = prox of the
    box under B at the warm dual field), lo = hi (x is the constant), c -> 0
    (x -> box projection under B), and tau* >> |U|^2 (B ~ tau* I)."""
    n, S_eff = 8, 3
    rng = np.random.default_rng(77)
    v = rng.uniform(-0.02, 0.07, (n, n, n))
    U = rng.standard_normal((S_eff, n, n, n)) * 0.05
    P0 = rng.uniform(-0.5, 0.5, (3, n, n, n))
    tau, c, J, lo, hi, kind = 1.5, 2e-3, 6, 0.0, 0.05, "iso"
    if case == "no_dual_iterations":
        J = 0
    elif case == "point_box":
        lo = hi = 0.03
    elif case == "tiny_c":
        c, kind = 1e-12, "aniso"
    elif case == "large_tau":
        tau = 1e4
    xo, Po, _ = owprox.wprox(v, tau, U, c, lo, hi, kind, J, P0=P0, newton_tol=1e-6)
    h = make_handle(n, cone(2), [0, 0], [1.0], tv=kind, box=(lo, hi), dual_iters=J, newton_tol=1e-6)
    Pw = f32(P0).reshape(-1).clone()
    xg = h.wprox(f32(v).reshape(-1), tau, f32(U).reshape(-1), c, P_warm=Pw).cpu().numpy().reshape(xo.shape)
    if case == "point_box":
        assert np.all(xg == np.float32(0.03))
    else:
        assert rel(xg, xo) < 1e-5, rel(xg, xo)
    h.close()


def test_empty_and_invalid_batches_are_rejected():
    n = 16
    w, kd, xt, om, ys, subs, so = problem(n, "ls")
    h = make_handle(n, kd, so, [1.0] * w.S)
    h.set_measurements(c64(ys).reshape(-1))
    x = f32(xt).reshape(-1)
    lib = h.lib
    g = torch.empty_like(x)
    il = (binding.ctypes.c_int * 1)(0)
    assert lib.mqnpm_grad_batch(h._h, binding._ptr(x), il, 0, 1.0, binding._ptr(g), None, None) == 1
    bad = (binding.ctypes.c_int * 1)(w.L)
    assert lib.mqnpm_grad_batch(h._h, binding._ptr(x), bad, 1, 1.0, binding._ptr(g), None, None) == 1
    assert lib.mqnpm_loss_batch(h._h, binding._ptr(x), il, 0, 1.0, None, None) == 1
    h.close()


@pytest.mark.parametrize("model", ["ls", "born"])
def test_graph_replay_equals_direct_launches(model):
    """BiCGSTAB iterations replayed from captured CUDA graphs launch the same
    kernels as direct launches: identical gradients, losses, iteration counts,
    kernel counts and profiled applies."""
    n = 16
    w, kd, xt, om, ys, subs, so = problem(n, model, L=6, batch=3)
    outs = []
    for direct in (False, True):
        h = make_handle(n, kd, so, [1.0] * w.S, model=model, krylov_tol=1e-6, max_batch=2, direct_launches=direct)
        h.set_measurements(c64(ys).reshape(-1))
        x = f32(0.7 * xt).reshape(-1)
        h.grad_batch(x, [0, 1, 2], 1.0)                 # captures (graph path)
        k0 = h.launch_count
        h.profile_begin(64)
        g, loss, its = h.grad_batch(x, [0, 1, 2], 1.0)
        prof = h.profile_end()
        outs.append((g.cpu().numpy(), loss, its, h.launch_count - k0, prof["calls"], prof["slot_launches"]))
        h.close()
    (ga, la, ia, ka, ca, sa), (gb, lb, ib, kb, cb, sb) = outs
    assert np.array_equal(ga, gb) and la == lb and ia == ib
    assert ka == kb and ca == cb and sa == sb


def test_device_side_krylov_loop_equals_direct_launches():
    """Without pass timers a whole BiCGSTAB solve is one graph launch: a
    conditional WHILE node around the iteration, ended on the device when no
    slot is active.  It gives the gradients, losses and iteration counts of
    direct launches bit for bit, and launches exactly one more kernel (the
    loop condition) per pass through the loop."""
    n = 16
    w, kd, xt, om, ys, subs, so = problem(n, "ls", L=6, batch=3)
    outs = []
    for direct in (False, True):
        h = make_handle(n, kd, so, [1.0] * w.S, model="ls", krylov_tol=1e-6, max_batch=2, direct_launches=direct)
        h.set_measurements(c64(ys).reshape(-1))
        x = f32(0.7 * xt).reshape(-1)
        h.grad_batch(x, [0, 1, 2], 1.0)                 # builds the graphs
        k0 = h.launch_count
        g, loss, its = h.grad_batch(x, [0, 1, 2], 1.0)
        outs.append((g.cpu().numpy(), loss, its, h.launch_count - k0))
        h.close()
    (ga, la, ia, ka), (gb, lb, ib, kb) = outs
    assert np.array_equal(ga, gb) and la == lb and ia == ib
    passes = sum(max(1, max(ia[b][j] for b in chunk)) for chunk in ([0, 1], [2]) for j in (0, 1))
    assert ka == kb + passes, (ka, kb, passes)
