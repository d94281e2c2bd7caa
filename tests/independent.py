"""Independent solvers used only to pin the oracle (different algorithms from
the ones the oracle runs).

* admm_wprox: ADMM on min_{x in C} 1/2||x - v||_B^2 + c TV(x) with the splitting
  z1 = grad x, z2 = x (dense linear solve for the x-step), for tiny volumes.
* tv1d_bvls: exact 1D TV prox via its dual, a bounded least-squares problem
  solved by the active-set BVLS method of scipy.
* box_qp_enumerate: min_{x in [lo,hi]^N} 1/2 ||x - w||_B^2 by enumerating all
  3^N active sets and keeping the one that satisfies the KKT conditions.
* admm_quadratic_tv: the same ADMM for min_{x in C} 1/2 x^T Q x + q^T x + c TV(x)
  with a general dense quadratic (an objective written term by term).
"""
import itertools

import numpy as np
from scipy.optimize import lsq_linear


def grad_matrix(shape):
    """Dense forward-difference (Neumann) gradient, rows ordered (d, voxel)."""
    N = int(np.prod(shape))
    D = len(shape)
    rows = []
    for d in range(D):
        ax = len(shape) - 1 - d
        K = np.zeros((N, N))
        idx = np.arange(N).reshape(shape)
        n = shape[ax]
        for i in np.ndindex(*shape):
            if i[ax] < n - 1:
                j = list(i)
                j[ax] += 1
                K[idx[i], idx[tuple(j)]] += 1.0
                K[idx[i], idx[i]] -= 1.0
        rows.append(K)
    return np.vstack(rows)


def admm_wprox(v, Bmat, c, lo, hi, kind="iso", rho=1.0, iters=20000):
    shape = v.shape
    N = v.size
    D = len(shape)
    K = grad_matrix(shape)
    vf = v.reshape(-1)
    x = np.clip(vf, lo, hi)
    z1 = K @ x
    z2 = x.copy()
    m1 = np.zeros_like(z1)
    m2 = np.zeros_like(z2)
    A = Bmat + rho * (K.T @ K) + rho * np.eye(N)
    Ainv = np.linalg.inv(A)
    Bv = Bmat @ vf
    for _ in range(iters):
        x = Ainv @ (Bv + rho * K.T @ (z1 - m1) + rho * (z2 - m2))
        kx = K @ x
        t = kx + m1
        if kind == "iso":
            g = t.reshape(D, N)
            nrm = np.sqrt(np.sum(g * g, axis=0))
            shrink = np.maximum(0.0, 1.0 - (c / rho) / np.maximum(nrm, 1e-300))
            z1 = (g * shrink[None]).reshape(-1)
        else:
            z1 = np.sign(t) * np.maximum(np.abs(t) - c / rho, 0.0)
        z2 = np.clip(x + m2, lo, hi)
        m1 += kx - z1
        m2 += x - z2
    return z2.reshape(shape)


def tv1d_bvls(v, c):
    """argmin_x 1/2 ||x - v||^2 + c sum |x_{i+1} - x_i| (exact, via the dual)."""
    n = v.size
    K = np.zeros((n - 1, n))
    for i in range(n - 1):
        K[i, i] = -1.0
        K[i, i + 1] = 1.0
    # dual: min_{|p_i| <= c} 1/2 ||K^T p - v||^2 ; x = v - K^T p
    res = lsq_linear(K.T, v, bounds=(-c, c), method="bvls", tol=1e-15, lsmr_tol=None)
    return v - K.T @ res.x


def box_qp_enumerate(w, Bmat, lo, hi):
    N = w.size
    best = None
    for pattern in itertools.product((0, 1, 2), repeat=N):   # 0 lower, 1 free, 2 upper
        pat = np.array(pattern)
        x = np.where(pat == 0, lo, np.where(pat == 2, hi, 0.0)).astype(float)
        free = pat == 1
        if free.any():
            Bff = Bmat[np.ix_(free, free)]
            rhs = (Bmat @ w)[free] - Bmat[np.ix_(free, ~free)] @ x[~free]
            x[free] = np.linalg.solve(Bff, rhs)
            if np.any(x[free] < lo - 1e-12) or np.any(x[free] > hi + 1e-12):
                continue
        g = Bmat @ (x - w)          # gradient of the objective
        ok = np.all(g[pat == 0] >= -1e-10) and np.all(g[pat == 2] <= 1e-10)
        if ok:
            val = 0.5 * (x - w) @ Bmat @ (x - w)
            if best is None or val < best[0]:
                best = (val, x)
    return best[1]


def admm_quadratic_tv(Q, q, shape, c, lo, hi, kind="iso", rho=1.0, iters=20000):
    """min_{x in [lo,hi]^N} 1/2 x^T Q x + q^T x + c TV(x) by ADMM with the same
    splitting as admm_wprox (z1 = grad x, z2 = x), for a general quadratic:
    no metric, no completed square, so a model whose objective is written as
    a sum of quadratic terms can be solved as printed."""
    N = int(np.prod(shape))
    D = len(shape)
    K = grad_matrix(shape)
    x = np.clip(np.linalg.solve(Q, -q), lo, hi)
    z1 = K @ x
    z2 = x.copy()
    m1 = np.zeros_like(z1)
    m2 = np.zeros_like(z2)
    Ainv = np.linalg.inv(Q + rho * (K.T @ K) + rho * np.eye(N))
    for _ in range(iters):
        x = Ainv @ (-q + rho * K.T @ (z1 - m1) + rho * (z2 - m2))
        kx = K @ x
        t = kx + m1
        if kind == "iso":
            g = t.reshape(D, N)
            nrm = np.sqrt(np.sum(g * g, axis=0))
            shrink = np.maximum(0.0, 1.0 - (c / rho) / np.maximum(nrm, 1e-300))
            z1 = (g * shrink[None]).reshape(-1)
        else:
            z1 = np.sign(t) * np.maximum(np.abs(t) - c / rho, 0.0)
        z2 = np.clip(x + m2, lo, hi)
        m1 += kx - z1
        m2 += x - z2
    return z2.reshape(shape)
