"""Pins of the SR1 estimate (Algorithm 4.2) and of the outer loop (Algorithm 4.1)."""
import math

import numpy as np
import pytest

import synth
from oracle import bqnpm, physics, sr1

from tests import independent as ind


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


class _FixedGradient:
    """Stand-in for the physics in the k > S pin: every subset's gradient at
    the current iterate is the prescribed g (the test fixes g = grad F_{s'}(x_{k-1}))."""

    def __init__(self, n, g):
        self.n = n
        self.shape = (n, n, n)
        self.g = g

    def batch_loss_grad(self, x, subset, ys, scale):
        return 0.0, self.g.copy()


def test_bqnpm_step_beyond_S_solves_eq_4_4():
    """One iteration k > S of Algorithm 4.1 (steps 8-10, Eq. 4.4 -> Eq. 4.5) against an
    independent ADMM solve of the model it minimises, written term by term:

        argmin_{x in C} (1/S) sum_s [ <g_s, x - x_s> + 1/(2a) ||x - x_s||^2_{B_s} ] + lam TV(x)

    with x_s = x_{k-1} and g_s = grad F_{s'}(x_{k-1}) for every s (strategy I / II reading of
    Section 4.2), B_{s'} the SR1 update of this iteration and every other B_s = tau_s I + u_s u_s^T
    left as stored.  No square is completed here, so the a S factor of v_k, the c = a S lam of the
    proximal mapping and tau* = sum_s tau_s (un-updated terms included) are all exercised."""
    rng = np.random.default_rng(21)
    n, S = 3, 3
    shape, N = (n, n, n), n ** 3
    a, lam, lo, hi = 0.7, 0.03, 0.0, 0.5
    x_prev = rng.uniform(0.05, 0.45, shape)
    g = 0.3 * rng.standard_normal(shape)
    subs = [np.array([s]) for s in range(S)]
    opt = bqnpm.BQNPM(_FixedGradient(n, g), None, subs, [0.9, 1.3, 1.1], lam=lam, box=(lo, hi),
                      kind="iso", step=a, gamma=0.8, dual_iters=4000, newton_tol=1e-13)
    # state after k = 5: every subset visited; iteration k = 6 takes s' = 2 (strategy I)
    opt.k = 5
    for s in range(S):
        opt.xbar[s] = rng.uniform(0.0, 0.5, shape)
        opt.gbar[s] = rng.standard_normal(shape)
    opt.tau = [0.8, 1.7, 1.2]
    opt.u = [0.25 * rng.standard_normal(shape), 0.25 * rng.standard_normal(shape), None]
    sp = 2
    A = rng.standard_normal((N, N))
    H = A @ A.T / N + 0.5 * np.eye(N)
    s_vec = (x_prev - opt.xbar[sp]).reshape(-1)
    m_vec = H @ s_vec
    opt.gbar[sp] = (g.reshape(-1) - m_vec).reshape(shape)
    x_new = opt.step(x_prev)
    assert opt.history[-1]["s"] == sp and opt.history[-1]["sr1"] == "rank1"
    Bs = []
    for s in range(S):
        B = opt.tau[s] * np.eye(N)
        if opt.u[s] is not None:
            B = B + np.outer(opt.u[s].reshape(-1), opt.u[s].reshape(-1))
        Bs.append(B)
    assert np.allclose(Bs[sp] @ s_vec, m_vec, rtol=1e-10, atol=1e-12)   # the SR1 secant equation
    assert opt.tau[0] == 0.8 and opt.tau[1] == 1.7                         # B_s, s != s', untouched
    # the model of Eq. 4.4 as 1/2 x^T Q x + q^T x (+ constants) + lam TV(x)
    gf, xf = g.reshape(-1), x_prev.reshape(-1)
    Q = sum(B for B in Bs) / (a * S)
    q = sum(gf - (B @ xf) / a for B in Bs) / S
    ref = ind.admm_quadratic_tv(Q, q, shape, lam, lo, hi, "iso", iters=30000)
    # the TV term and the box are both active at this solution
    unreg = np.clip(np.linalg.solve(Q, -q), lo, hi).reshape(shape)
    assert np.max(np.abs(unreg - ref)) > 1e-2
    assert np.max(np.abs(x_new - ref)) < 2e-6
