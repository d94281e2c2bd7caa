"""GPU parity of the outer loop (Algorithm 4.1 with SR1) on the small nonlinear
workload, checkpoint/resume, and failure reporting through the C ABI."""
import math

import numpy as np
import pytest

import synth
from oracle import bqnpm, physics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2307_02043_gb300 import binding  # noqa: E402

DEV = torch.device("cuda:0")


def f32(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.float32)).to(DEV)


def setup(w):
    kd = synth.illumination_dirs(w)
    om = physics.Model(w.n, kd, w.model, tol=1e-12)
    xt = synth.phantom(w)
    ys = physics.simulate(om, xt, synth.noise_draws(w), w.snr_db)
    subs = synth.subsets(w)
    so = np.zeros(w.L, dtype=np.int32)
    for s, ii in enumerate(subs):
        so[ii] = s
    return kd, om, xt, ys, subs, so


def handle(w, kd, so, alpha, **kw):
    args = dict(model=w.model, tv=w.tv, lam=w.lam, box=w.box, krylov_tol=1e-6, dual_iters=w.dual_iters,
                gamma=w.gamma, step=w.step, max_batch=w.batch)
    args.update(kw)
    return binding.MQNPM(w.n, kd, so, alpha, **args)


@pytest.fixture(scope="module")
def ls32():
    w = synth.workload("ls32")
    kd, om, xt, ys, subs, so = setup(w)
    alpha = [om.lipschitz(s, w.S / w.L, synth.power_start(w), 20) for s in subs]
    opt = bqnpm.BQNPM(om, ys, subs, alpha, lam=w.lam, box=w.box, kind=w.tv, dual_iters=w.dual_iters,
                      gamma=w.gamma, step=w.step)
    xs = opt.run(np.zeros((w.n,) * 3), w.outer_iters)
    return w, kd, om, ys, subs, so, alpha, opt, xs


@pytest.mark.parametrize("warm", [False, True])
def test_step_trajectory_matches_oracle(ls32, warm):
    """Config 1 (32^3, LS, L = 8, S = 4, 10 iterations): per-iterate error and the
    objective trajectory against the FP64 oracle run with the same inputs.  With
    warm starts the forward solves begin at the fields of the previous visit of
    each subset; the solutions stay within the Krylov tolerance, so the same
    bounds hold."""
    w, kd, om, ys, subs, so, alpha, opt, xs = ls32
    h = handle(w, kd, so, alpha, warm_start=warm)
    h.set_measurements(torch.from_numpy(ys.astype(np.complex64)).to(DEV).reshape(-1))
    x = torch.zeros(w.N, dtype=torch.float32, device=DEV)
    for k in range(1, w.outer_iters + 1):
        info = h.step(x)
        ho = opt.history[k - 1]
        assert info["subset"] == ho["s"]
        assert abs(info["tau_star"] - ho["tau_star"]) <= 1e-3 * ho["tau_star"], (k, info, ho)
        xg = x.cpu().numpy().astype(np.float64).reshape(xs[k].shape)
        err = np.linalg.norm(xg - xs[k]) / np.linalg.norm(xs[k])
        assert err < 2e-3, (k, err)
        if k in (1, w.S, w.outer_iters):
            cg, co = opt.full_cost(xg), opt.full_cost(xs[k])
            assert abs(cg - co) <= 1e-4 * abs(co), (k, cg, co)
    h.close()


def test_diagnostics_match_oracle(ls32):
    """Section 6 convergence diagnostics on the oracle's own iterates: the bias
    error e_k^2 (summed literally over s != s' by the oracle), the squared step
    ||x_k - x_{k-1}||^2 and the full data term."""
    w, kd, om, ys, subs, so, alpha, opt, xs = ls32
    h = handle(w, kd, so, alpha)
    h.set_measurements(torch.from_numpy(ys.astype(np.complex64)).to(DEV).reshape(-1))
    for k in (w.S + 1, w.outer_iters):
        sp = opt.history[k - 1]["s"]
        d = h.diagnostics(f32(xs[k - 1]).reshape(-1), sp, f32(xs[k]).reshape(-1))
        e2 = opt.bias_error(xs[k - 1], sp)
        dx2 = float(np.sum((xs[k].astype(np.float32).astype(np.float64)
                            - xs[k - 1].astype(np.float32).astype(np.float64)) ** 2))
        data = opt.full_cost(xs[k - 1]) - w.lam * physics_tv(xs[k - 1], w.tv)
        assert abs(d["bias_error"] - e2) <= 2e-4 * e2, (k, d, e2)
        assert abs(d["step_sq"] - dx2) <= 1e-5 * dx2, (k, d, dx2)
        assert abs(d["data_term"] - data) <= 1e-4 * abs(data), (k, d, data)   # objective bound
    # without x_k the step term is zero; a subset index out of range is rejected
    assert h.diagnostics(f32(xs[1]).reshape(-1), 0)["step_sq"] == 0.0
    with pytest.raises(binding.MQNPMError):
        h.diagnostics(f32(xs[1]).reshape(-1), w.S)
    h.close()


def physics_tv(x, kind):
    from oracle import tv as otv
    return otv.tv(x, kind)


def test_non_default_stream_gives_identical_results(ls32):
    """Every call runs on the caller's current stream (set per call): outer
    iterations and a gradient on a side stream equal those on the default
    stream bit for bit (captured iteration graphs, event records and copies all
    follow the caller's stream)."""
    import contextlib
    w, kd, om, ys, subs, so, alpha, _, _ = ls32
    out = []
    for side in (False, True):
        h = handle(w, kd, so, alpha, warm_start=True)
        ctx = torch.cuda.stream(torch.cuda.Stream()) if side else contextlib.nullcontext()
        with ctx:
            h.set_measurements(torch.from_numpy(ys.astype(np.complex64)).to(DEV).reshape(-1))
            x = torch.zeros(w.N, dtype=torch.float32, device=DEV)
            for _ in range(w.S + 2):
                h.step(x)
            g, loss, _ = h.grad_batch(x, [0, 1], 0.5)
            xc, gc = x.cpu(), g.cpu()
        torch.cuda.synchronize()
        out.append((xc, gc, loss))
        h.close()
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_strategy2_trajectory_matches_oracle(ls32):
    """Strategy II (s' drawn uniformly, seeded draws passed to both sides) on
    config 1: per-iterate error against the FP64 oracle."""
    w, kd, om, ys, subs, so, alpha, _, _ = ls32
    draws = synth.strategy2_draws(w, w.outer_iters)
    opt = bqnpm.BQNPM(om, ys, subs, alpha, lam=w.lam, box=w.box, kind=w.tv, dual_iters=w.dual_iters,
                      gamma=w.gamma, step=w.step, strategy=2, draws=draws)
    xs = opt.run(np.zeros((w.n,) * 3), w.outer_iters)
    h = handle(w, kd, so, alpha, strategy=2, draws=[int(d) for d in draws])
    h.set_measurements(torch.from_numpy(ys.astype(np.complex64)).to(DEV).reshape(-1))
    x = torch.zeros(w.N, dtype=torch.float32, device=DEV)
    for k in range(1, w.outer_iters + 1):
        info = h.step(x)
        assert info["subset"] == opt.history[k - 1]["s"]
        xg = x.cpu().numpy().astype(np.float64).reshape(xs[k].shape)
        err = np.linalg.norm(xg - xs[k]) / np.linalg.norm(xs[k])
        assert err < 2e-3, (k, err)
    h.close()


def test_full_batch_variant_matches_oracle():
    """S = 1 (every illumination in one subset: the full-batch variant of the
    method, Section 4.2): every iteration after the first takes the SR1 branch
    on the full gradient; per-iterate error against the FP64 oracle."""
    w = synth.small("ls32", n=16, L=4, batch=4)
    assert w.S == 1
    kd, om, xt, ys, subs, so = setup(w)
    alpha = [om.lipschitz(subs[0], 1.0 / w.L, synth.power_start(w), 20)]
    iters = 6
    opt = bqnpm.BQNPM(om, ys, subs, alpha, lam=w.lam, box=w.box, kind=w.tv, dual_iters=w.dual_iters,
                      gamma=w.gamma, step=w.step)
    xs = opt.run(np.zeros((w.n,) * 3), iters)
    assert all("sr1" in hh for hh in opt.history[1:])
    h = handle(w, kd, so, alpha)
    h.set_measurements(torch.from_numpy(ys.astype(np.complex64)).to(DEV).reshape(-1))
    x = torch.zeros(w.N, dtype=torch.float32, device=DEV)
    for k in range(1, iters + 1):
        info = h.step(x)
        assert info["subset"] == 0
        xg = x.cpu().numpy().astype(np.float64).reshape(xs[k].shape)
        err = np.linalg.norm(xg - xs[k]) / np.linalg.norm(xs[k])
        assert err < 2e-3, (k, err)
    h.close()


def test_step_trajectory_rank_above_8():
    """S = 12 subsets (L = 24, b = 2 at 16^3: the subset counts of the uneven
    request mix go up to 15): the rank-12 metric and prox follow the oracle."""
    w = synth.small("ls32", n=16, L=24, batch=2, outer_iters=26)
    assert w.S == 12
    kd, om, xt, ys, subs, so = setup(w)
    alpha = [om.lipschitz(s, w.S / w.L, synth.power_start(w), 10) for s in subs]
    opt = bqnpm.BQNPM(om, ys, subs, alpha, lam=w.lam, box=w.box, kind=w.tv, dual_iters=w.dual_iters,
                      gamma=w.gamma, step=w.step)
    xs = opt.run(np.zeros((w.n,) * 3), w.outer_iters)
    h = handle(w, kd, so, alpha)
    h.set_measurements(torch.from_numpy(ys.astype(np.complex64)).to(DEV).reshape(-1))
    x = torch.zeros(w.N, dtype=torch.float32, device=DEV)
    for k in range(1, w.outer_iters + 1):
        info = h.step(x)
        xg = x.cpu().numpy().astype(np.float64).reshape(xs[k].shape)
        err = np.linalg.norm(xg - xs[k]) / np.linalg.norm(xs[k])
        assert err < 2e-3, (k, err, info)
    assert info["rank"] > 8
    h.close()


@pytest.mark.parametrize("warm", [False, True])
def test_checkpoint_resume_is_bit_identical(ls32, warm):
    w, kd, om, ys, subs, so, alpha, opt, xs = ls32
    y = torch.from_numpy(ys.astype(np.complex64)).to(DEV).reshape(-1)
    h = handle(w, kd, so, alpha, warm_start=warm)
    h.set_measurements(y)
    x = torch.zeros(w.N, dtype=torch.float32, device=DEV)
    for _ in range(w.S + 1):
        h.step(x)
    blob = h.save_state()
    x_saved = x.clone()
    for _ in range(2):
        h.step(x)
    h2 = handle(w, kd, so, alpha, warm_start=warm)
    h2.set_measurements(y)
    h2.load_state(blob)
    x2 = x_saved.clone()
    for _ in range(2):
        h2.step(x2)
    assert torch.equal(x, x2)
    h.close()
    h2.close()


def test_warm_start_solves_to_the_same_tolerance(ls32):
    """A forward solve started from the stored field of a nearby contrast needs
    no more BiCGSTAB iterations and returns the same data to the tolerance."""
    w, kd, om, ys, subs, so, alpha, opt, xs = ls32
    hw = handle(w, kd, so, alpha, warm_start=True, krylov_tol=1e-7)
    hc = handle(w, kd, so, alpha, krylov_tol=1e-7)
    x1 = f32(xs[w.S]).reshape(-1)
    x2 = f32(xs[w.S + 1]).reshape(-1)
    illum = list(range(w.L))
    hw.forward(x1, illum)                      # stores the fields
    yw, itw = hw.forward(x2, illum)            # warm
    yc, itc = hc.forward(x2, illum)            # cold
    assert sum(itw) <= sum(itc), (itw, itc)
    for l in illum:
        ref = om.forward(xs[w.S + 1], l)
        ew = np.linalg.norm(yw[l].cpu().numpy() - ref)
        ec = np.linalg.norm(yc[l].cpu().numpy() - ref)
        # the detector data is the small scattered part of u, so a residual
        # tolerance of 1e-7 leaves ~1e-5 relative error in it, warm or cold
        assert ew <= 2e-5 * np.linalg.norm(ref), (l, ew, ec)
    blob_w = hw.save_state()
    h3 = handle(w, kd, so, alpha)              # cold handle: a warm checkpoint does not match it
    with pytest.raises(binding.MQNPMError):
        h3.load_state(blob_w)
    for hh in (hw, hc, h3):
        hh.close()


def test_failures_are_reported():
    w = synth.small("ls32", n=16, L=4, batch=2)
    kd, om, xt, ys, subs, so = setup(w)
    # invalid arguments
    with pytest.raises(binding.MQNPMError) as e:
        binding.MQNPM(20, kd, so, [1.0, 1.0])          # P = 40 has no transform plan
    assert e.value.code == 7
    with pytest.raises(binding.MQNPMError) as e:
        binding.MQNPM(16, kd, so, [1.0, -1.0])
    assert e.value.code == 1
    with pytest.raises(binding.MQNPMError) as e:
        binding.MQNPM(16, kd, so, [1.0, 1.0], max_batch=65)   # above MQNPM_MAX_BATCH
    assert e.value.code == 1
    # budget below the workspace
    with pytest.raises(binding.MQNPMError) as e:
        handle(w, kd, so, [1.0, 1.0], hbm_budget_bytes=1 << 20)
    assert e.value.code == 2
    h = handle(w, kd, so, [1.0, 1.0], krylov_maxit=1)
    # gradient before measurements
    with pytest.raises(binding.MQNPMError) as e:
        h.grad_batch(f32(xt).reshape(-1), [0], 1.0)
    assert e.value.code == 8
    h.set_measurements(torch.from_numpy(ys.astype(np.complex64)).to(DEV).reshape(-1))
    # Krylov cap of one iteration on a scattering object: NOT_CONVERGED, outputs written
    with pytest.raises(binding.NotConverged):
        h.grad_batch(f32(4 * xt).reshape(-1), [0, 1], 1.0)
    g, loss, its = h.grad_batch(f32(4 * xt).reshape(-1), [0, 1], 1.0, allow_not_converged=True)
    assert torch.isfinite(g).all() and all(a == 1 for a, _ in its)
    # non-finite input
    bad = xt.copy()
    bad[3, 4, 5] = np.nan
    with pytest.raises(binding.MQNPMError) as e:
        h.grad_batch(f32(bad).reshape(-1), [0], 1.0)
    assert e.value.code == 5
    h.close()


@pytest.mark.parametrize("warm", [False, True])
def test_step_halves_and_sharded_step_equal_step(ls32, warm):
    """mqnpm_step_subset + the caller's gradient + mqnpm_step_with_gradient (the
    path of the illumination-sharded step, here with one rank: no collective)
    give exactly what mqnpm_step gives, iterate for iterate, bit for bit."""
    from paper_2307_02043_gb300.sharded import ShardedStep

    w, kd, om, ys, subs, so, alpha, opt, xs = ls32
    ya = torch.from_numpy(ys.astype(np.complex64)).to(DEV).reshape(-1)
    h1 = handle(w, kd, so, alpha, warm_start=warm)
    h2 = handle(w, kd, so, alpha, warm_start=warm)
    h1.set_measurements(ya)
    h2.set_measurements(ya)
    x1 = torch.zeros(w.N, dtype=torch.float32, device=DEV)
    x2 = torch.zeros_like(x1)
    sharded = ShardedStep(h2)
    assert (sharded.rank, sharded.world) == (0, 1)
    for k in range(1, w.outer_iters + 1):
        sub, il = h2.step_subset()
        assert il == [int(i) for i in subs[sub]]
        i1 = h1.step(x1)
        i2 = sharded.step(x2)
        assert i1["subset"] == i2["subset"] == sub and i1["k"] == i2["k"] == k
        assert i1["loss"] == i2["loss"] and i1["tau_star"] == i2["tau_star"] and i1["rank"] == i2["rank"]
        assert torch.equal(x1, x2), k
    with pytest.raises(binding.MQNPMError):
        h2.step_with_gradient(x2, x2, 0.0)              # g must not alias x
    with pytest.raises(binding.MQNPMError):
        h2.step_with_gradient(x2, torch.zeros_like(x2), float("nan"))
    h1.close()
    h2.close()


def test_step_trajectory_in_the_rank8_regime_on_a_64_grid():
    """The regime the ls128 bench times, on a grid the oracle finishes in about
    a minute: 64^3 LS of the ls128 family (contrast up to 0.04, iso TV, box
    [0, 0.06]), L = 16 in eight subsets of two, 16 outer iterations, so that
    k = 9..16 take SR1-weighted steps whose metric grows to rank 8 (Algorithm
    4.1, Algorithm 4.2, Eq. 4.5).  Every iterate, tau*, the metric's rank and
    the objective are compared with the FP64 oracle run on the same inputs;
    the forward solves warm-start as in the bench.  Observed on GB300:
    iterate errors below 1e-5, tau* within 6e-7, objective within 4e-6; the
    bounds leave a factor of about ten."""
    w = synth.small("ls128", n=64, L=16, batch=2, outer_iters=16)
    kd = synth.illumination_dirs(w)
    om = physics.Model(w.n, kd, w.model, tol=1e-9)
    xt = synth.phantom(w)
    ys = physics.simulate(om, xt, synth.noise_draws(w), w.snr_db)
    subs = synth.subsets(w)
    so = np.zeros(w.L, dtype=np.int32)
    for s, ii in enumerate(subs):
        so[ii] = s
    alpha = [om.lipschitz(s, w.S / w.L, synth.power_start(w), 8) for s in subs]
    opt = bqnpm.BQNPM(om, ys, subs, alpha, lam=w.lam, box=w.box, kind=w.tv, dual_iters=w.dual_iters,
                      gamma=w.gamma, step=w.step)
    h = handle(w, kd, so, alpha, warm_start=True)
    h.set_measurements(torch.from_numpy(ys.astype(np.complex64)).to(DEV).reshape(-1))
    x = torch.zeros(w.N, dtype=torch.float32, device=DEV)
    xo = np.zeros((w.n,) * 3)
    for k in range(1, w.outer_iters + 1):
        xo = opt.step(xo)
        ho = opt.history[-1]
        rank_o = sum(u is not None for u in opt.u)
        info = h.step(x)
        xg = x.cpu().numpy().astype(np.float64).reshape(xo.shape)
        err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
        print(k, ho["s"], info["rank"], rank_o, info["tau_star"], ho["tau_star"], err, flush=True)
        assert info["subset"] == ho["s"]
        assert info["rank"] == rank_o, (k, info["rank"], rank_o)
        assert abs(info["tau_star"] - ho["tau_star"]) <= 5e-6 * ho["tau_star"], (k, info, ho)
        assert err < 1e-4, (k, err)
        if k in (w.S, w.outer_iters):
            cg, co = opt.full_cost(xg), opt.full_cost(xo)
            print("cost", k, cg, co, abs(cg - co) / abs(co), flush=True)
            assert abs(cg - co) <= 4e-5 * abs(co), (k, cg, co)
    assert rank_o == w.S
    h.close()
