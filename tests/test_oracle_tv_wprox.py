"""Pins of the oracle's TV operators, structured weighted prox and dual solver.

Each check uses something the oracle does not: dense matrices, an exact 1D
solver, enumeration of active sets, ADMM on the primal problem, finite
differences, duality gaps and closed forms (Woodbury, Theorem 3.1 with h = 0).
"""
import math

import numpy as np
import pytest

from oracle import tv as tvops
from oracle import wprox as wp
from tests import independent as ind


def test_d_and_dT_are_adjoint_and_bounded():
    rng = np.random.default_rng(0)
    for shape in [(7,), (5, 6), (4, 5, 6)]:
        x = rng.standard_normal(shape)
        P = rng.standard_normal((len(shape),) + shape)
        assert abs(np.sum(x * tvops.d_of(P)) - np.sum(tvops.dT(x) * P)) < 1e-12
        K = ind.grad_matrix(shape)
        assert np.allclose(K @ x.reshape(-1), tvops.dT(x).reshape(-1))
        # ||d||^2 = ||K||^2 <= 4 D (Section 3.3 / Lemma 4.1)
        assert np.linalg.norm(K, 2) ** 2 <= 4 * len(shape) + 1e-12


def test_tv_values_brute_force():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 4, 5))
    iso = 0.0
    l1 = 0.0
    for z in range(3):
        for y in range(4):
            for xx in range(5):
                gx = x[z, y, xx + 1] - x[z, y, xx] if xx < 4 else 0.0
                gy = x[z, y + 1, xx] - x[z, y, xx] if y < 3 else 0.0
                gz = x[z + 1, y, xx] - x[z, y, xx] if z < 2 else 0.0
                iso += math.sqrt(gx * gx + gy * gy + gz * gz)
                l1 += abs(gx) + abs(gy) + abs(gz)
    assert abs(tvops.tv(x, "iso") - iso) < 1e-12
    assert abs(tvops.tv(x, "aniso") - l1) < 1e-12


def test_tv_dual_representation():
    """TV(x) = max_{P in dual ball} d(P)^T x (Eqs. 3.3-3.4), attained at P = dT x / |.|."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 4, 4))
    g = tvops.dT(x)
    Piso = g / np.maximum(np.sqrt(np.sum(g * g, axis=0)), 1e-300)[None]
    assert abs(np.sum(tvops.d_of(Piso) * x) - tvops.tv(x, "iso")) < 1e-10
    Pl1 = np.sign(g)
    assert abs(np.sum(tvops.d_of(Pl1) * x) - tvops.tv(x, "aniso")) < 1e-10
    for _ in range(20):      # any feasible P gives a lower bound
        Q = tvops.project_dual(rng.standard_normal(g.shape) * 3, "iso")
        assert np.sum(tvops.d_of(Q) * x) <= tvops.tv(x, "iso") + 1e-12


def rand_metric(rng, N, S, tau=0.7, scale=1.0):
    U = rng.standard_normal((N, S)) * scale
    return tau, U, tau * np.eye(N) + U @ U.T


def test_woodbury_inverse():
    rng = np.random.default_rng(3)
    tau, U, B = rand_metric(rng, 40, 4)
    binv = wp.woodbury_inverse(tau, U)
    y = rng.standard_normal(40)
    assert np.allclose(B @ binv(y), y, atol=1e-12)
    assert np.allclose(binv(y), np.linalg.solve(B, y), atol=1e-12)


@pytest.mark.parametrize("S", [1, 2, 3])
def test_prox_box_metric_vs_enumeration(S):
    rng = np.random.default_rng(10 + S)
    N = 7
    for trial in range(5):
        tau, U, B = rand_metric(rng, N, S, tau=0.5 + trial * 0.3)
        w = rng.uniform(-1.5, 1.5, N)
        x, beta, it = wp.prox_box_metric(w, U, tau, -0.5, 0.8, tol=1e-13)
        ref = ind.box_qp_enumerate(w, B, -0.5, 0.8)
        assert np.max(np.abs(x - ref)) < 1e-9, (x, ref)
        # Theorem 3.1 fixed point
        assert np.linalg.norm(wp.phi(beta, w, U, tau, -0.5, 0.8)) < 1e-10


def test_theorem31_unconstrained_gives_zero_beta():
    rng = np.random.default_rng(4)
    tau, U, B = rand_metric(rng, 30, 3)
    w = rng.standard_normal(30)
    x, beta, _ = wp.prox_box_metric(w, U, tau, -np.inf, np.inf)
    assert np.allclose(beta, 0.0) and np.allclose(x, w)


def test_moreau_envelope_gradient():
    """Eq. (3.5): grad M(x) = W (x - prox^W(x)) for h = iota_C."""
    rng = np.random.default_rng(5)
    N, S = 12, 2
    tau, U, B = rand_metric(rng, N, S)
    lo, hi = -0.3, 0.4

    def M(x):
        p, _, _ = wp.prox_box_metric(x, U, tau, lo, hi, tol=1e-14)
        e = p - x
        return 0.5 * e @ B @ e

    x = rng.uniform(-1, 1, N)
    p, _, _ = wp.prox_box_metric(x, U, tau, lo, hi, tol=1e-14)
    g = B @ (x - p)
    for _ in range(5):
        d = rng.standard_normal(N)
        h = 1e-6
        fd = (M(x + h * d) - M(x - h * d)) / (2 * h)
        assert abs(fd - g @ d) < 1e-6 * max(1.0, abs(fd))


def test_lemma41_gradient_of_T():
    rng = np.random.default_rng(6)
    shape = (3, 3, 4)
    N = 36
    tau, U, B = rand_metric(rng, N, 2, tau=1.2, scale=0.5)
    v = rng.uniform(-0.2, 0.6, shape)
    W = wp.WProx(shape, tau, U.T.reshape(2, *shape), 0.3, 0.0, 0.5, "iso", newton_tol=1e-14)
    P = rng.standard_normal((3,) + shape) * 0.5
    g = W.grad_T(v, P)
    for _ in range(4):
        d = rng.standard_normal(P.shape)
        h = 1e-6
        fd = (W.T(v, P + h * d) - W.T(v, P - h * d)) / (2 * h)
        assert abs(fd - np.sum(g * d)) < 1e-5 * max(1.0, abs(fd)), (fd, np.sum(g * d))
    # the Lipschitz bound of Lemma 4.1 holds on random pairs
    Lip = W.lipschitz_T()
    for _ in range(10):
        P2 = P + rng.standard_normal(P.shape)
        ratio = np.linalg.norm(W.grad_T(v, P2) - g) / np.linalg.norm(P2 - P)
        assert ratio <= Lip * (1 + 1e-9)


def test_unweighted_1d_against_exact_tv_prox():
    """D = 1, B = tau I: FGP on the dual reaches the exact TV prox (clipped)."""
    rng = np.random.default_rng(7)
    for trial in range(3):
        v = np.cumsum(rng.standard_normal(30)) * 0.1 + 0.2
        tau, c = 2.0, 0.15
        x, _, _ = wp.wprox(v, tau, None, c, -np.inf, np.inf, "iso", J=4000)
        ref = ind.tv1d_bvls(v, c / tau)
        assert np.max(np.abs(x - ref)) < 1e-6
        lo, hi = 0.0, 0.5
        xb, _, _ = wp.wprox(v, tau, None, c, lo, hi, "iso", J=4000)
        refb = ind.admm_wprox(v, tau * np.eye(30), c, lo, hi, "iso", iters=20000)
        assert np.max(np.abs(xb - refb)) < 1e-6
        assert np.max(np.abs(xb - np.clip(ref, lo, hi))) < 1e-6


@pytest.mark.parametrize("kind", ["iso", "aniso"])
def test_weighted_3d_against_admm(kind):
    rng = np.random.default_rng(8)
    shape = (3, 3, 3)
    N = 27
    tau, U, B = rand_metric(rng, N, 2, tau=1.0, scale=0.4)
    v = rng.uniform(-0.1, 0.7, shape)
    c = 0.05
    x, P, info = wp.wprox(v, tau, U.T.reshape(2, *shape), c, 0.0, 0.5, kind, J=3000,
                          newton_tol=1e-13)
    ref = ind.admm_wprox(v, B, c, 0.0, 0.5, kind, rho=1.0, iters=30000)
    assert np.max(np.abs(x - ref)) < 2e-6, np.max(np.abs(x - ref))
    # primal optimality gap is tiny
    W = wp.WProx(shape, tau, U.T.reshape(2, *shape), c, 0.0, 0.5, kind)
    assert W.objective(v, x) - W.objective(v, ref) < 1e-9


def test_duality_gap_decreases():
    rng = np.random.default_rng(9)
    shape = (4, 4, 4)
    N = 64
    tau, U, B = rand_metric(rng, N, 3, tau=0.8, scale=0.3)
    Ub = U.T.reshape(3, *shape)
    v = rng.uniform(-0.1, 0.7, shape)
    c = 0.04
    W = wp.WProx(shape, tau, Ub, c, 0.0, 0.5, "iso", newton_tol=1e-13)
    gaps = []
    for J in (5, 50, 500):
        x, P, _ = W.solve(v, J)
        wP = W.w_of(v, P)
        xP, _, _ = W.prox_box(wP)
        dual = 0.5 * (xP - v.reshape(-1)) @ B @ (xP - v.reshape(-1)) + c * tvops.d_of(P).reshape(-1) @ xP
        gaps.append(W.objective(v, xP.reshape(shape)) - dual)
    assert all(g >= -1e-10 for g in gaps)
    assert gaps[2] < gaps[0] * 1e-2 and gaps[2] < 1e-5, gaps


def test_appendix_a_identity():
    """argmin_{x in C} (1/S) sum_s Fbar_s(x) + lam TV(x) (Eq. 4.4) equals the WPM of Eq. (4.5)."""
    rng = np.random.default_rng(11)
    shape = (3, 3, 3)
    N = 27
    S, a, lam = 3, 0.7, 0.05
    Bs, xs, gs = [], [], []
    for s in range(S):
        u = rng.standard_normal(N) * 0.3
        tau_s = 0.4 + 0.2 * s
        Bs.append(tau_s * np.eye(N) + np.outer(u, u))
        xs.append(rng.uniform(0, 0.5, N))
        gs.append(rng.standard_normal(N) * 0.1)
    Bk = sum(Bs)
    vk = np.linalg.solve(Bk, sum(B @ x - a * g for B, x, g in zip(Bs, xs, gs)))
    # Direct form: (1/S) sum_s [<g_s, x> + 1/(2a)||x - x_s||^2_{B_s}] + lam TV is, up to a
    # constant, 1/(2 a S) x^T Bk x - (1/(a S)) <sum_s(B_s x_s - a g_s), x> + lam TV.
    # Multiplying by a S and completing the square gives the WPM with c = a S lam.
    # Check the algebra numerically on random points, then solve both forms.
    def direct(x):
        return sum(g @ x + (x - xx) @ B @ (x - xx) / (2 * a) for B, xx, g in zip(Bs, xs, gs)) / S
    def wpm(x):
        return ((x - vk) @ Bk @ (x - vk)) / (2 * a * S)
    pts = [rng.standard_normal(N) for _ in range(3)]
    diffs = [direct(p) - wpm(p) for p in pts]
    assert np.ptp(diffs) < 1e-10
    ref = ind.admm_wprox(vk.reshape(shape), Bk, a * S * lam, 0.0, 0.5, "iso", iters=30000)
    # the structured solver with B^k = tau* I + U U^T, tau* = sum tau_s
    taus = [0.4 + 0.2 * s for s in range(S)]
    # B_s - tau_s I = u_s u_s^T: recover u_s from the rank-1 factor
    us = []
    for B, t in zip(Bs, taus):
        ev, evec = np.linalg.eigh(B - t * np.eye(N))
        us.append(evec[:, -1] * math.sqrt(ev[-1]))
    x, _, _ = wp.wprox(vk.reshape(shape), sum(taus), np.stack(us).reshape(S, *shape),
                       a * S * lam, 0.0, 0.5, "iso", J=3000, newton_tol=1e-13)
    assert np.max(np.abs(x - ref)) < 2e-6
