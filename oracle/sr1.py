"""Memory-efficient SR1 estimate B_s = tau I + u u^T (Algorithm 4.2)
(FP64 oracle; test infrastructure only).

Readings where the printed algorithm is ambiguous (also listed in the design
notes):
  * the skip test uses the absolute value |<m - tau s, s>| <= delta1 ||s|| ||m - tau s||
    (the standard SR1 skip rule; without it the test always fires for gamma < 1,
    by Cauchy-Schwarz, and u is never used);
  * u = (m - tau s)/sqrt(<m - tau s, s>) is evaluated once, after the damping
    loop has ended with <m - tau s, s> > delta2 ||s||^2, so its radicand is
    positive and u is defined on every exit of that branch;
  * <s, m> = 0 (no curvature information, e.g. s = 0) takes the tau <= 0 branch.
"""
from __future__ import annotations

import math
from typing import Optional, Tuple

import numpy as np

DELTA1 = 1e-8
DELTA2 = 1e-12


def sr1(s: np.ndarray, m: np.ndarray, gamma: float, alpha: float, tau_max: float,
        delta1: float = DELTA1, delta2: float = DELTA2) -> Tuple[float, Optional[np.ndarray], str]:
    """Return (tau, u or None, branch) for the pair (s, m) = (x - x_prev, g - g_prev)."""
    s = np.asarray(s, dtype=np.float64).reshape(-1)
    m = np.asarray(m, dtype=np.float64).reshape(-1)
    sm = float(s @ m)
    mm = float(m @ m)
    ss = float(s @ s)
    if sm == 0.0:
        return alpha, None, "tau_nonpositive"
    tau = mm / (gamma * sm)
    tau = min(tau, tau_max)
    if tau <= 0.0:
        return alpha, None, "tau_nonpositive"
    q = m - tau * s
    if abs(float(q @ s)) <= delta1 * math.sqrt(ss) * float(np.linalg.norm(q)):
        return tau, None, "skip"
    while float((m - tau * s) @ s) <= delta2 * ss:
        if tau < delta2:
            return alpha, None, "tau_tiny"
        tau = tau / 2.0
    q = m - tau * s
    u = q / math.sqrt(float(q @ s))
    return tau, u, "rank1"
