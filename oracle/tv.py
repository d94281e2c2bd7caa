"""Discrete total variation and its dual (FP64 oracle; test infrastructure only).

Section 3.1 defines D^d through the entries -delta[i-j] + delta[i-j-R_d]; as
printed the stride and the boundary rule are garbled.  Our reading: forward
differences along dimension d with Neumann boundary,
    (D^d x)_i = x_{i+e_d} - x_i  if i_d < R_d - 1,   0 on the last slice,
which keeps ||d||^2 <= 4D (Section 3.3 and the proof of Lemma 4.1).

Dimension d = 1 is the fastest array axis (x), d = 2 is y, d = 3 is z.  A dual
field P in R^{D x N} is stored as an array of shape (D, *x.shape) with
component q_d = P[d-1].
"""
from __future__ import annotations

import numpy as np


def _axis(x: np.ndarray, d: int) -> int:
    """Array axis of dimension d (0-based d; d = 0 is the fastest axis)."""
    return x.ndim - 1 - d


def forward_diff(x: np.ndarray, d: int) -> np.ndarray:
    """D^d x with the Neumann rule (zero on the last slice)."""
    ax = _axis(x, d)
    out = np.zeros_like(x, dtype=np.float64)
    n = x.shape[ax]
    lead = [slice(None)] * x.ndim
    nxt = [slice(None)] * x.ndim
    lead[ax] = slice(0, n - 1)
    nxt[ax] = slice(1, n)
    out[tuple(lead)] = x[tuple(nxt)] - x[tuple(lead)]
    return out


def forward_diff_T(q: np.ndarray, d: int) -> np.ndarray:
    """(D^d)^T q = q_{i-e_d} [i_d >= 1] - q_i [i_d <= R_d - 2]."""
    ax = _axis(q, d)
    n = q.shape[ax]
    out = np.zeros_like(q, dtype=np.float64)
    lead = [slice(None)] * q.ndim
    nxt = [slice(None)] * q.ndim
    lead[ax] = slice(0, n - 1)
    nxt[ax] = slice(1, n)
    out[tuple(nxt)] += q[tuple(lead)]
    out[tuple(lead)] -= q[tuple(lead)]
    return out


def d_of(P: np.ndarray) -> np.ndarray:
    """d(P) = sum_d (D^d)^T q_d (Section 3.3)."""
    out = np.zeros(P.shape[1:], dtype=np.float64)
    for d in range(P.shape[0]):
        out += forward_diff_T(P[d], d)
    return out


def dT(x: np.ndarray) -> np.ndarray:
    """Adjoint of d: d^T(x) = (D^1 x, ..., D^D x), shape (D, *x.shape)."""
    return np.stack([forward_diff(x, d) for d in range(x.ndim)])


def tv(x: np.ndarray, kind: str = "iso") -> float:
    """TV_iso (Eq. 3.1) or TV_l1 (Eq. 3.2) of x."""
    g = dT(x)
    if kind == "iso":
        return float(np.sum(np.sqrt(np.sum(g * g, axis=0))))
    return float(np.sum(np.abs(g)))


def project_dual(P: np.ndarray, kind: str = "iso") -> np.ndarray:
    """Projection onto the dual ball of Eq. (3.3) (iso: ||p_n||_2 <= 1) or
    Eq. (3.4) (anisotropic: ||p_n||_inf <= 1)."""
    if kind == "iso":
        nrm = np.sqrt(np.sum(P * P, axis=0))
        return P / np.maximum(1.0, nrm)[None]
    return np.clip(P, -1.0, 1.0)
