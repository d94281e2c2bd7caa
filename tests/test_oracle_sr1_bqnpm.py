"""Pins of the SR1 estimate (Algorithm 4.2) and of the outer loop (Algorithm 4.1)."""
import math

import numpy as np
import pytest

import synth
from oracle import bqnpm, physics, sr1


def test_sr1_secant_and_bounds():
    rng = np.random.default_rng(0)
    hits = 0
    for trial in range(200):
        N = 20
        A = rng.standard_normal((N, N))
        H = A @ A.T / N + 0.1 * np.eye(N)      # SPD "Hessian"
        s = rng.standard_normal(N)
        m = H @ s
        alpha = 0.5
        tau, u, branch = sr1.sr1(s, m, 0.8, alpha, 1e3)
        assert tau >= min(sr1.DELTA2 / 2, alpha)          # proof of Lemma 5.2 (App. D)
        B = tau * np.eye(N) + (np.outer(u, u) if u is not None else 0)
        assert np.linalg.eigvalsh(B)[0] > 0
        if u is not None:
            hits += 1
            assert np.allclose(B @ s, m, rtol=1e-10, atol=1e-12)   # secant equation
            assert (m - tau * s) @ s > sr1.DELTA2 * (s @ s)
    assert hits > 150


def test_sr1_branches():
    N = 6
    s = np.ones(N)
    # <s, m> < 0 : tau <= 0 branch
    tau, u, br = sr1.sr1(s, -s, 0.8, 0.3, 1e3)
    assert (tau, u, br) == (0.3, None, "tau_nonpositive")
    # tau clipped at tau_max with m = 2s -> tau = min(4/(0.8*... )) ; skip when <m - tau s, s> = 0
    m = 2.0 * s
    tau, u, br = sr1.sr1(s, m, 1.0, 0.3, 1e3)
    assert br == "skip" and abs(tau - 2.0) < 1e-15
    # tiny curvature: halving reaches tau < delta2 -> alpha
    m = 1e-14 * s + 1e-14 * np.array([1, -1, 1, -1, 1, -1.0])
    tau, u, br = sr1.sr1(s, m, 0.8, 0.3, 1e3)
    assert br == "tau_tiny" and tau == 0.3 and u is None
    # ordinary rank-1 update
    m = np.array([3.0, 1, 1, 1, 1, 0.5])
    tau, u, br = sr1.sr1(s, m, 0.8, 0.3, 1e3)
    assert br == "rank1" and u is not None


def test_literal_sr1_test_always_skips():
    """Motivation of the |.| reading: without it the test fires whenever gamma < 1."""
    rng = np.random.default_rng(1)
    for _ in range(1000):
        s = rng.standard_normal(10)
        m = rng.standard_normal(10)
        if s @ m <= 0:
            continue
        tau = (m @ m) / (0.8 * (s @ m))
        assert (m - tau * s) @ s <= 0


def tiny_setup(n=8, model="ls", L=4, batch=2):
    w = synth.small("ls32", n=n, L=L, batch=batch, model=model)
    kd = synth.illumination_dirs(w)
    m = physics.Model(n, kd, model=model, tol=1e-12)
    xt = synth.phantom(w)
    ys = physics.simulate(m, xt, synth.noise_draws(w), w.snr_db)
    return w, m, xt, ys


def test_bqnpm_bookkeeping_and_descent():
    w, m, xt, ys = tiny_setup()
    subs = synth.subsets(w)
    alpha = [m.lipschitz(s, w.S / w.L, synth.power_start(w), 20) for s in subs]
    # reconstruct with a larger lambda so TV is active at this size
    opt = bqnpm.BQNPM(m, ys, subs, alpha, lam=1e-4, box=w.box, kind="iso",
                      dual_iters=20, gamma=0.8)
    x0 = np.zeros_like(xt)
    xs = opt.run(x0, 6)
    hist = opt.history
    assert [h["s"] for h in hist] == [0, 1, 0, 1, 0, 1]      # k<=S: s=k; then strategy I
    assert all("sr1" in h for h in hist[2:])
    # iterates stay in the box
    for x in xs:
        assert x.min() >= w.box[0] - 1e-15 and x.max() <= w.box[1] + 1e-15
    costs = [opt.full_cost(x) for x in xs]
    assert costs[-1] < 0.5 * costs[0]
    # the stored xbar/gbar are the latest per subset
    assert np.array_equal(opt.xbar[1], xs[5])


def test_bqnpm_strategy2_uses_draws():
    w, m, xt, ys = tiny_setup(n=6)
    subs = synth.subsets(w)
    draws = synth.strategy2_draws(w, 10)
    opt = bqnpm.BQNPM(m, ys, subs, [1.0, 1.0], lam=1e-4, box=w.box, strategy=2,
                      draws=draws, dual_iters=5)
    opt.run(np.zeros((6, 6, 6)), 5)
    assert [h["s"] for h in opt.history][2:] == list(draws[:3])


def test_bias_error_pins():
    """e_k^2 of Section 6, summed literally over s != s', against: the
    identity (1/S) sum_{s != s'} (grad F_s - grad F_{s'}) = grad F - grad F_{s'}
    with grad F the full-batch gradient (1/L) sum_l grad f_l (F_s = (S/L) sum
    over S_s, Eq. 4.1); zero for one subset; zero when every subset holds the
    same illuminations."""
    w, m, xt, ys = tiny_setup()
    subs = synth.subsets(w)
    opt = bqnpm.BQNPM(m, ys, subs, [1.0] * len(subs), lam=1e-4, box=w.box)
    x = 0.5 * xt
    for sp in range(len(subs)):
        e2 = opt.bias_error(x, sp)
        _, g_full = m.batch_loss_grad(x, np.arange(w.L), ys, 1.0 / w.L)
        _, g_sp = opt.grad_F(x, sp)
        d = g_full - g_sp
        assert e2 > 0
        assert abs(e2 - float(np.vdot(d, d).real)) <= 1e-12 * e2
    one = bqnpm.BQNPM(m, ys, [np.arange(w.L)], [1.0], lam=1e-4, box=w.box)
    assert one.bias_error(x, 0) == 0.0
    same = bqnpm.BQNPM(m, ys, [subs[0], subs[0]], [1.0, 1.0], lam=1e-4, box=w.box)
    assert same.bias_error(x, 1) <= 1e-30
