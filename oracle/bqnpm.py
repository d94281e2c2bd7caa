"""Outer loop of the mini-batch quasi-Newton proximal method (Algorithm 4.1)
(FP64 oracle; test infrastructure only).

Iteration k (1-based):
  k <= S : s = k; g = grad F_s(x_{k-1}); B_s = alpha_s I;
           x_k = prox^{B_s}_{a lam TV + iota_C}(x_{k-1} - a B_s^{-1} g).
  k >  S : s' by strategy I (s' = ((k-1) mod S) + 1) or II (uniform draw);
           g = grad F_{s'}(x_{k-1}); (tau_{s'}, u_{s'}) from Algorithm 4.2 with
           s = x_{k-1} - xbar_{s'}, m = g - gbar_{s'}; then xbar_{s'}, gbar_{s'} <- x_{k-1}, g;
           B = sum_s B_s = tau* I + U U^T;  v_k = x_{k-1} - a S B^{-1} g
           (step 10 of Algorithm 4.1 with x_s^k = x_{k-1}, g_s^k = g for all s);
           x_k = prox^{B}_{a S lam TV + iota_C}(v_k)   (Eq. 4.5).
Readings: B_s = alpha_s I until subset s is revisited; tau_max = 1e3 max_s alpha_s;
the dual field P of the proximal mapping is warm-started from the previous
outer iteration (P_0 = 0 at k = 1).
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

from . import sr1 as sr1mod
from . import tv as tvops
from .physics import Model
from .wprox import WProx, woodbury_inverse


class BQNPM:
    def __init__(self, model: Model, ys: np.ndarray, subsets: Sequence[np.ndarray],
                 alpha: Sequence[float], lam: float, box, kind: str = "iso",
                 step: float = 1.0, gamma: float = 0.8, dual_iters: int = 20,
                 tau_max: Optional[float] = None, strategy: int = 1,
                 draws: Optional[Sequence[int]] = None,
                 newton_tol: float = 1e-6, newton_maxit: int = 50):
        self.model = model
        self.ys = ys
        self.subsets = [np.asarray(s) for s in subsets]
        self.S = len(self.subsets)
        self.L = int(sum(len(s) for s in self.subsets))
        self.alpha = [float(a) for a in alpha]
        self.lam = float(lam)
        self.lo, self.hi = float(box[0]), float(box[1])
        self.kind = kind
        self.a = float(step)
        self.gamma = float(gamma)
        self.J = int(dual_iters)
        self.tau_max = 1e3 * max(self.alpha) if tau_max is None else float(tau_max)
        self.strategy = strategy
        self.draws = draws
        self.newton_tol = newton_tol
        self.newton_maxit = newton_maxit
        self.shape = tuple(model.shape)
        self.k = 0
        self.xbar: List[Optional[np.ndarray]] = [None] * self.S
        self.gbar: List[Optional[np.ndarray]] = [None] * self.S
        self.tau = list(self.alpha)
        self.u: List[Optional[np.ndarray]] = [None] * self.S
        self.P: Optional[np.ndarray] = None
        self.history: List[dict] = []

    def grad_F(self, x: np.ndarray, s: int):
        """F_s = (S/L) sum_{l in S_s} f_l (Eq. 4.1)."""
        return self.model.batch_loss_grad(x, self.subsets[s], self.ys, self.S / self.L)

    def full_cost(self, x: np.ndarray) -> float:
        """Phi(x) = (1/L) sum_l f_l(x) + lam TV(x)  (Eq. 1.2)."""
        f = 0.0
        for l in range(self.L):
            r = self.model.forward(x, l) - self.ys[l]
            f += 0.5 * float(np.vdot(r, r).real)
        return f / self.L + self.lam * tvops.tv(x, self.kind)

    def bias_error(self, x_prev: np.ndarray, s_prime: int) -> float:
        """e_k^2 of the convergence validation (Section 6), taken literally:
        || (1/S) sum_{s != s'} (grad F_s(x_{k-1}) - g_s^k) ||^2 with
        g_s^k = grad F_{s'}(x_{k-1}) for every s (strategies I and II,
        Section 4.2)."""
        _, g_sp = self.grad_F(x_prev, s_prime)
        acc = np.zeros_like(g_sp)
        for s in range(self.S):
            if s != s_prime:
                _, g_s = self.grad_F(x_prev, s)
                acc += g_s - g_sp
        acc /= self.S
        return float(np.vdot(acc, acc).real)

    def pick(self, k: int) -> int:
        if k <= self.S:
            return k - 1
        if self.strategy == 1:
            return (k - 1) % self.S
        return int(self.draws[k - self.S - 1])

    def step(self, x: np.ndarray) -> np.ndarray:
        self.k += 1
        k = self.k
        s = self.pick(k)
        loss, g = self.grad_F(x, s)
        info = {"k": k, "s": s, "loss": loss}
        if k <= self.S:
            self.xbar[s], self.gbar[s] = x.copy(), g.copy()
            self.tau[s], self.u[s] = self.alpha[s], None
            tau_star, U, c = self.alpha[s], None, self.a * self.lam
            v = x - (self.a / self.alpha[s]) * g
        else:
            tau_s, u_s, branch = sr1mod.sr1(x - self.xbar[s], g - self.gbar[s], self.gamma,
                                           self.alpha[s], self.tau_max)
            self.tau[s], self.u[s] = tau_s, (None if u_s is None else u_s.reshape(self.shape))
            self.xbar[s], self.gbar[s] = x.copy(), g.copy()
            info["sr1"] = branch
            tau_star = float(sum(self.tau))
            us = [u for u in self.u if u is not None]
            U = np.stack(us) if us else None
            c = self.a * self.S * self.lam
            Um = np.zeros((x.size, 0)) if U is None else U.reshape(len(us), -1).T
            binv = woodbury_inverse(tau_star, Um)
            v = x - (self.a * self.S * binv(g.reshape(-1))).reshape(self.shape)
        prox = WProx(self.shape, tau_star, U, c, self.lo, self.hi, self.kind,
                     self.newton_tol, self.newton_maxit)
        x_new, self.P, pinfo = prox.solve(v, self.J, self.P)
        info.update(tau_star=tau_star, newton=pinfo["newton"])
        self.history.append(info)
        return x_new

    def run(self, x0: np.ndarray, iters: int) -> List[np.ndarray]:
        xs = [x0]
        x = x0
        for _ in range(iters):
            x = self.step(x)
            xs.append(x)
        return xs
