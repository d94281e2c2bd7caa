"""Weighted proximal mapping of c*TV + box under B = tau*I + U U^T
(FP64 oracle; test infrastructure only).

Problem (Eq. 4.5 with B^k = tau* I + U U^T, Section 4.3):
    x* = argmin_{x in C} 1/2 ||x - v||_B^2 + c TV(x),   C = [lo, hi]^N.
Steps, in the paper's order:
  * Woodbury inverse of B (Section 4.3);
  * w(P) = v - c B^{-1} d(P) (defined with Eq. 4.7);
  * prox^B_{iota_C}(w) = clip(w - U beta*/tau) with beta* the root of
    phi(beta) = U^T(w - clip(w - U beta/tau)) + beta (Theorem 3.1, '+' case,
    h = iota_C), found by semi-smooth Newton (Algorithm 4.3);
  * accelerated projected gradient on T(P) (Eq. 4.10) with the gradient of
    Lemma 4.1, step 1/Lip = omega_min/(4 D c) where omega_min(B) = tau
    (U U^T has rank <= S < N), momentum of Beck-Teboulle's FGP;
  * output x = prox^B_{iota_C}(w(P_J)).

Readings where the paper is silent (also listed in the design notes):
  * Newton picks H = I + tau^{-1} U^T diag(1[lo < z_i < hi]) U (interior voxels),
    stops at ||phi|| <= eps * max(1, ||U^T w||), and halves a step that does not
    reduce ||phi|| (at most 30 halvings).
  * FGP: t_1 = 1, t_{j+1} = (1 + sqrt(1 + 4 t_j^2))/2,
    R_{j+1} = P_j + (t_j - 1)/t_{j+1} (P_j - P_{j-1}); R_1 = P_0 (warm start).
  * Newton start of each dual iteration: with w(P) = v - (c/tau) d(P) + U gamma(P),
    gamma(P) = (c/tau^2) (I + U^T U/tau)^{-1} U^T d(P), the solve starts at
    beta_0 = beta_prev + tau (gamma - gamma_prev), which keeps
    theta = gamma - beta/tau of the previous solve (both 0 at the first one).
"""
from __future__ import annotations

import math
from typing import Optional, Tuple

import numpy as np

from . import tv as tvops


def _flatU(U: Optional[np.ndarray], N: int) -> np.ndarray:
    """U as an N x S matrix (columns u_s); an empty matrix when U is None."""
    if U is None or len(U) == 0:
        return np.zeros((N, 0))
    return np.asarray(U, dtype=np.float64).reshape(len(U), N).T


def woodbury_inverse(tau: float, U: np.ndarray):
    """Return y -> B^{-1} y for B = tau I + U U^T (U is N x S):
    B^{-1} = tau^{-1} I - tau^{-2} U (I + U^T U / tau)^{-1} U^T  (Section 4.3)."""
    S = U.shape[1]
    small = np.eye(S) + (U.T @ U) / tau

    def apply(y: np.ndarray) -> np.ndarray:
        if S == 0:
            return y / tau
        return y / tau - U @ np.linalg.solve(small, U.T @ y) / tau ** 2

    return apply


def phi(beta: np.ndarray, w: np.ndarray, U: np.ndarray, tau: float,
        lo: float, hi: float) -> np.ndarray:
    """phi(beta) of Eq. (3.6) for h = iota_C and Sigma = tau I."""
    z = w - U @ beta / tau
    return U.T @ (w - np.clip(z, lo, hi)) + beta


def prox_box_metric(w: np.ndarray, U: np.ndarray, tau: float, lo: float, hi: float,
                    beta0: Optional[np.ndarray] = None, tol: float = 1e-6,
                    maxit: int = 50) -> Tuple[np.ndarray, np.ndarray, int]:
    """prox^B_{iota_C}(w) via Theorem 3.1 and semi-smooth Newton (Algorithm 4.3).

    w is flat (N,), U is N x S.  Returns (x, beta*, newton iterations)."""
    S = U.shape[1]
    if S == 0:
        return np.clip(w, lo, hi), np.zeros(0), 0
    beta = np.zeros(S) if beta0 is None else np.asarray(beta0, dtype=np.float64).copy()
    scale = max(1.0, float(np.linalg.norm(U.T @ w)))
    it = 0
    f = phi(beta, w, U, tau, lo, hi)
    while it < maxit and np.linalg.norm(f) > tol * scale:
        z = w - U @ beta / tau
        inner = (z > lo) & (z < hi)
        Ua = U[inner]
        H = np.eye(S) + (Ua.T @ Ua) / tau
        step = -np.linalg.solve(H, f)
        t = 1.0
        nf = np.linalg.norm(f)
        for _ in range(30):
            f_new = phi(beta + t * step, w, U, tau, lo, hi)
            if np.linalg.norm(f_new) < nf:
                break
            t *= 0.5
        beta = beta + t * step
        f = f_new
        it += 1
    x = np.clip(w - U @ beta / tau, lo, hi)
    return x, beta, it


class WProx:
    """The weighted proximal mapping for one metric B = tau I + U U^T."""

    def __init__(self, shape, tau: float, U: Optional[np.ndarray], c: float,
                 lo: float, hi: float, kind: str = "iso",
                 newton_tol: float = 1e-6, newton_maxit: int = 50):
        self.shape = tuple(shape)
        self.N = int(np.prod(self.shape))
        self.D = len(self.shape)
        self.tau = float(tau)
        self.U = _flatU(U, self.N)
        self.c = float(c)
        self.lo, self.hi = float(lo), float(hi)
        self.kind = kind
        self.newton_tol = newton_tol
        self.newton_maxit = newton_maxit
        self.Binv = woodbury_inverse(self.tau, self.U)

    def B(self, y: np.ndarray) -> np.ndarray:
        """B y for flat y."""
        return self.tau * y + self.U @ (self.U.T @ y)

    def w_of(self, v: np.ndarray, P: np.ndarray) -> np.ndarray:
        """w(P) = v - c B^{-1} d(P) (flat)."""
        return v.reshape(-1) - self.c * self.Binv(tvops.d_of(P).reshape(-1))

    def gamma_of(self, P: np.ndarray) -> np.ndarray:
        """gamma(P) = (c/tau^2) (I + U^T U / tau)^{-1} U^T d(P) (the S-vector of
        the Woodbury term: w(P) = v - (c/tau) d(P) + U gamma(P))."""
        S = self.U.shape[1]
        if S == 0:
            return np.zeros(0)
        small = np.eye(S) + (self.U.T @ self.U) / self.tau
        return (self.c / self.tau ** 2) * np.linalg.solve(small, self.U.T @ tvops.d_of(P).reshape(-1))

    def prox_box(self, w: np.ndarray, beta0=None):
        return prox_box_metric(w, self.U, self.tau, self.lo, self.hi, beta0,
                               self.newton_tol, self.newton_maxit)

    def T(self, v: np.ndarray, P: np.ndarray) -> float:
        """T(P) = ||w||_B^2 - ||w - prox^B_C(w)||_B^2 (Eq. 4.10)."""
        w = self.w_of(v, P)
        x, _, _ = self.prox_box(w)
        e = w - x
        return float(w @ self.B(w) - e @ self.B(e))

    def grad_T(self, v: np.ndarray, P: np.ndarray) -> np.ndarray:
        """Lemma 4.1: grad T(P) = -2 c d^T(prox^B_C(w(P)))."""
        x, _, _ = self.prox_box(self.w_of(v, P))
        return -2.0 * self.c * tvops.dT(x.reshape(self.shape))

    def lipschitz_T(self) -> float:
        """Lemma 4.1: 8 D c^2 / omega_min with omega_min = tau."""
        return 8.0 * self.D * self.c ** 2 / self.tau

    def objective(self, v: np.ndarray, x: np.ndarray) -> float:
        """1/2 ||x - v||_B^2 + c TV(x) (x assumed in C)."""
        e = (x - v).reshape(-1)
        return float(0.5 * e @ self.B(e) + self.c * tvops.tv(x.reshape(self.shape), self.kind))

    def solve(self, v: np.ndarray, J: int, P0: Optional[np.ndarray] = None
              ) -> Tuple[np.ndarray, np.ndarray, dict]:
        """J accelerated dual projected-gradient iterations; returns (x, P_J, info)."""
        v = np.asarray(v, dtype=np.float64).reshape(self.shape)
        P_prev = np.zeros((self.D,) + self.shape) if P0 is None else np.asarray(P0, np.float64).copy()
        R = P_prev.copy()
        t = 1.0
        S = self.U.shape[1]
        beta, g_prev = np.zeros(S), np.zeros(S)
        step = self.tau / (4.0 * self.D * self.c)
        newton = []

        def solve_at(Q):
            nonlocal beta, g_prev
            g = self.gamma_of(Q)
            beta0 = beta + self.tau * (g - g_prev)   # theta = gamma - beta/tau kept from the last solve
            x, beta, it = self.prox_box(self.w_of(v, Q), beta0)
            g_prev = g
            newton.append(it)
            return x

        for _ in range(J):
            x = solve_at(R)
            P = tvops.project_dual(R + step * tvops.dT(x.reshape(self.shape)), self.kind)
            t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
            R = P + ((t - 1.0) / t_next) * (P - P_prev)
            P_prev = P
            t = t_next
        x = solve_at(P_prev)
        return x.reshape(self.shape), P_prev, {"newton": newton, "beta": beta}


def wprox(v: np.ndarray, tau: float, U: Optional[np.ndarray], c: float, lo: float,
          hi: float, kind: str, J: int, P0: Optional[np.ndarray] = None,
          newton_tol: float = 1e-6, newton_maxit: int = 50):
    """Functional form of :class:`WProx` (returns x, P_J, info)."""
    return WProx(v.shape, tau, U, c, lo, hi, kind, newton_tol, newton_maxit).solve(v, J, P0)
