"""Forward model, data term and gradient (FP64 oracle; test infrastructure only).

Section 6 of the paper: the sample is probed by plane waves
u_in^l(r) = exp(j <k_l, r>) and the data term of Eq. (1.1) is
f_l(x) = 1/2 ||H_l(x) - y_l||^2.  Evaluating H_l once needs one
Lippmann-Schwinger (LS) solve and the gradient of f_l needs two; both are
solved with BiCGSTAB.  The discretisation is not printed in the paper (it is in
a supplement that is not available), so the following reading is fixed here
and in the CUDA library alike:

* voxel h, background wavenumber k_b; coordinates r = (idx - n/2) h;
* contrast x real, one value per voxel (x = (eta/eta_b)^2 - 1);
* (G v)_i = k_b^2 sum_j w_{i-j} v_j over offsets in (-n, n)^3 with
  w_D = h^3 exp(j k_b |D| h) / (4 pi |D| h) for D != 0 and the self term
  w_0 = [exp(j k_b a)(1 - j k_b a) - 1] / k_b^2, a = (3/(4 pi))^(1/3) h, the
  exact integral of the Green's function over the sphere of volume h^3;
  or, as an option, the truncated kernel (Vico, Greengard and Ferrando 2016):
  w_D from the transform of g restricted to r <= sqrt(3) n h, sampled on a
  grid of period 4 n h, which makes G v the continuous convolution of v's
  band-limited interpolant with g (spectrally accurate for smooth v);
* LS: u = u_in + G (x * u); Born: u_sc = G (x * u_in);
* detector: the scattered field u - u_in on the last z-slice (M = nx ny), or,
  with a remote detector, that slice carried a distance d further along z by
  the angular spectrum with a pupil of numerical aperture na (relative to the
  medium): D = F^-1 diag(H) F with H = exp(j k_z d) 1[kx^2 + ky^2 <= (na k_b)^2],
  k_z = sqrt(k_b^2 - kx^2 - ky^2) on the branch with Im k_z >= 0, F the 2D DFT
  of the n x n slice (periodic; frequencies 2 pi fftfreq(n, h));
* gradient: grad f = Re(conj(u) * z), z = (I - G^H X)^{-1} G^H S^T D^H r.

Arrays are indexed [z, y, x] (x fastest in memory).
"""
from __future__ import annotations

import math
import os
from typing import Callable, Sequence, Tuple

import numpy as np
import scipy.fft as sfft

# Threads of the FFT library routine: every core this process may run on.
FFT_WORKERS = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def kb_default(h: float = 1.0) -> float:
    """Background wavenumber for a wavelength of four voxels."""
    return 2.0 * math.pi / (4.0 * h)


def self_term(kb: float, h: float = 1.0) -> complex:
    """w_0: integral of exp(j kb r)/(4 pi r) over the sphere of volume h^3."""
    a = (3.0 / (4.0 * math.pi)) ** (1.0 / 3.0) * h
    return (np.exp(1j * kb * a) * (1.0 - 1j * kb * a) - 1.0) / kb ** 2


def grid_shape(n) -> Tuple[int, int, int]:
    """(nz, ny, nx) of a grid given as one edge n or as a (nz, ny, nx) triple."""
    if np.ndim(n) == 0:
        return (int(n),) * 3
    nz, ny, nx = (int(v) for v in n)
    return nz, ny, nx


def _wrapped_offsets(nd: int) -> Tuple[np.ndarray, np.ndarray]:
    """Offsets along one axis of the periodic grid of length P = 2 nd: index i
    carries i (i < nd) or i - P (i > nd); index nd (offset -nd, never reached
    by two voxels of the domain) is marked unused."""
    idx = np.arange(2 * nd)
    return np.where(idx < nd, idx, idx - 2 * nd), idx == nd


def green_kernel(n, kb: float, h: float = 1.0) -> np.ndarray:
    """k_b^2 w_D laid out on the periodic grid of edges P_d = 2 n_d (n: one
    edge or (nz, ny, nx)); every offset of the domain appears once, the unused
    index n_d of each axis is 0."""
    nz, ny, nx = grid_shape(n)
    (oz, uz), (oy, uy), (ox, ux) = (_wrapped_offsets(v) for v in (nz, ny, nx))
    dz, dy, dx = np.meshgrid(oz.astype(np.float64), oy.astype(np.float64), ox.astype(np.float64), indexing="ij")
    r = h * np.sqrt(dx ** 2 + dy ** 2 + dz ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        w = h ** 3 * np.exp(1j * kb * r) / (4.0 * math.pi * r)
    w[0, 0, 0] = self_term(kb, h)
    w[uz, :, :] = 0.0
    w[:, uy, :] = 0.0
    w[:, :, ux] = 0.0
    return kb ** 2 * w


def truncated_green_ft(s, kb: float, R: float) -> np.ndarray:
    """Fourier transform of the truncated Green's function
    g_R(r) = exp(j kb r) / (4 pi r) for r <= R and 0 beyond, at radial
    frequencies s >= 0 (the kernel of the truncated-kernel method of Vico,
    Greengard and Ferrando, J. Comput. Phys. 2016), written from its
    definition: for s > 0
        g_R^(s) = (1/s) int_0^R exp(j kb r) sin(s r) dr
                = (E(j(kb + s)) - E(j(kb - s))) / (2 j s),
        E(a)    = int_0^R exp(a r) dr = R expm1(a R) / (a R)   (E(0) = R),
    and g_R^(0) = int_0^R r exp(j kb r) dr = (exp(j kb R)(1 - j kb R) - 1) / kb^2.
    (Accurate for s R >= 1; every nonzero frequency of the grids below has
    s R >= 2.7.)"""
    s = np.asarray(s, dtype=np.float64)

    def E(a):
        z = a * R
        zs = np.where(z == 0, 1.0, z)
        return np.where(z == 0, R, R * np.expm1(zs) / zs)

    ss = np.where(s == 0, 1.0, s)
    val = (E(1j * (kb + ss)) - E(1j * (kb - ss))) / (2j * ss)
    g0 = (np.exp(1j * kb * R) * (1.0 - 1j * kb * R) - 1.0) / kb ** 2
    return np.where(s == 0, g0, val)


def truncated_periods(n, h: float = 1.0) -> Tuple[float, Tuple[int, int, int]]:
    """Truncation radius R (the diagonal of the domain, h sqrt(nz^2 + ny^2 + nx^2),
    which covers every distance between two voxels) and the sample counts T_d
    of the period T_d h along each axis: 4 n_d, raised to the next even count
    >= n_d + R/h where the domain is elongated, so that T_d h >= n_d h + R."""
    shape = grid_shape(n)
    R = h * math.sqrt(sum(v * v for v in shape))
    T = tuple(max(4 * v, 2 * math.ceil((v + R / h) / 2.0)) for v in shape)
    return R, T


def truncated_green_kernel(n, kb: float, h: float = 1.0) -> np.ndarray:
    """k_b^2 w_D on the periodic grid of edges P_d = 2 n_d for the truncated kernel.

    Voxel sums with this kernel are the continuous convolution of the band-
    limited interpolant of v with g_R: the transform of g_R is sampled on the
    frequency grid of periods T_d h (s_m = 2 pi m_d / (T_d h), m_d in
    [-T_d/2, T_d/2)), so  w_D = (h^3 / prod_d T_d h) sum_m g_R^(|s_m|)
    exp(j s_m . D h)  (an inverse DFT of length T_d per axis).  R covers every
    distance between two voxels of the domain and T_d h >= n_d h + R keeps the
    periodic copies of g_R out of the offsets the domain uses, which are laid
    out on the P grid as in green_kernel (index n_d unused, 0).  A cubic grid
    has T = 4n and R = sqrt(3) n h."""
    shape = grid_shape(n)
    R, T = truncated_periods(shape, h)
    fz, fy, fx = (2.0 * math.pi * np.fft.fftfreq(t, d=h) for t in T)
    s = np.sqrt(fz[:, None, None] ** 2 + fy[None, :, None] ** 2 + fx[None, None, :] ** 2)
    w = sfft.ifftn(truncated_green_ft(s, kb, R), workers=FFT_WORKERS)
    del s
    sel, unused = [], []
    for v, t in zip(shape, T):
        off, un = _wrapped_offsets(v)
        sel.append(off % t)
        unused.append(un)
    wp = w[np.ix_(*sel)].copy()
    wp[unused[0], :, :] = 0.0
    wp[:, unused[1], :] = 0.0
    wp[:, :, unused[2]] = 0.0
    return kb ** 2 * wp


def green_hat(n, kb: float, h: float = 1.0, kernel: str = "sampled") -> np.ndarray:
    """K_hat = DFT_P of the periodic kernel (2nz x 2ny x 2nx complex128): the sampled
    Green's function with the sphere self term ("sampled") or the truncated
    kernel ("truncated")."""
    if kernel == "truncated":
        return sfft.fftn(truncated_green_kernel(n, kb, h), workers=FFT_WORKERS)
    if kernel != "sampled":
        raise ValueError("kernel must be 'sampled' or 'truncated'")
    return sfft.fftn(green_kernel(n, kb, h), workers=FFT_WORKERS)


def green_apply(v: np.ndarray, khat: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """G v (or G^H v) by zero padding to P = 2n and circular convolution.

    Because the periodic kernel holds every offset of the domain exactly once,
    the circular convolution restricted to the domain equals the aperiodic sum.
    G is complex symmetric, so G^H uses conj(K_hat).
    """
    nz, ny, nx = v.shape
    pad = np.zeros((2 * nz, 2 * ny, 2 * nx), dtype=np.complex128)
    pad[:nz, :ny, :nx] = v
    k = np.conj(khat) if adjoint else khat
    out = sfft.ifftn(k * sfft.fftn(pad, workers=FFT_WORKERS), workers=FFT_WORKERS)
    return out[:nz, :ny, :nx]


def transfer_function(n, kb: float, h: float, distance: float, na: float) -> np.ndarray:
    """H[ky, kx] of the angular-spectrum propagation over `distance` with the
    pupil kx^2 + ky^2 <= (na kb)^2 (remote-detector reading of Section 6)."""
    _, ny, nx = grid_shape(n)
    KY, KX = np.meshgrid(2.0 * math.pi * np.fft.fftfreq(ny, d=h), 2.0 * math.pi * np.fft.fftfreq(nx, d=h),
                         indexing="ij")
    k2 = KX * KX + KY * KY
    kz = np.sqrt((kb * kb - k2).astype(np.complex128))   # principal root: Im >= 0
    return np.where(k2 <= (na * kb) ** 2, np.exp(1j * kz * distance), 0.0)


def propagate(field: np.ndarray, H: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """D f = F^-1 (H F f) on an ny x nx slice; D^H uses conj(H)."""
    return sfft.ifft2((np.conj(H) if adjoint else H) * sfft.fft2(field, workers=FFT_WORKERS), workers=FFT_WORKERS)


def incident_field(n, kdir: Sequence[float], kb: float, h: float = 1.0) -> np.ndarray:
    """u_in(r) = exp(j kb <kdir, r>), r_d = (idx_d - n_d/2) h, shape (nz, ny, nx) [z, y, x]."""
    nz, ny, nx = grid_shape(n)
    Z, Y, X = np.meshgrid((np.arange(nz) - nz / 2.0) * h, (np.arange(ny) - ny / 2.0) * h,
                          (np.arange(nx) - nx / 2.0) * h, indexing="ij")
    return np.exp(1j * kb * (kdir[0] * X + kdir[1] * Y + kdir[2] * Z))


def bicgstab(apply_a: Callable[[np.ndarray], np.ndarray], b: np.ndarray,
             x0: np.ndarray, tol: float, maxit: int) -> Tuple[np.ndarray, int, float]:
    """Unpreconditioned BiCGSTAB of van der Vorst (1992), <a, b> = sum conj(a) b.

    Stops when ||r|| <= tol ||b||.  Returns (solution, iterations, relres).
    """
    x = x0.astype(np.complex128).copy()
    r = b - apply_a(x)
    rhat = r.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(x), 0, 0.0
    rho_old = alpha = omega = 1.0 + 0.0j
    v = np.zeros_like(x)
    p = np.zeros_like(x)
    it = 0
    while it < maxit:
        if np.linalg.norm(r) <= tol * bnorm:
            break
        rho = np.vdot(rhat, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = apply_a(p)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        it += 1
        if np.linalg.norm(s) <= tol * bnorm:
            x = x + alpha * p
            r = s
            break
        t = apply_a(s)
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
    return x, it, float(np.linalg.norm(r) / bnorm)


class Model:
    """One configuration of the forward model (grid, wavenumber, directions)."""

    def __init__(self, n, kdirs: np.ndarray, model: str = "ls",
                 kb: float | None = None, h: float = 1.0,
                 tol: float = 1e-12, maxit: int = 2000,
                 det_distance: float = 0.0, det_na: float = 0.0, kernel: str = "sampled"):
        self.shape = grid_shape(n)          # (nz, ny, nx)
        self.n = n if np.ndim(n) == 0 else self.shape
        self.h = h
        self.kb = kb_default(h) if kb is None else kb
        self.kdirs = np.asarray(kdirs, dtype=np.float64)
        self.model = model
        self.tol = tol
        self.maxit = maxit
        self.khat = green_hat(n, self.kb, h, kernel)
        # remote detector (det_na > 0): angular-spectrum transfer function
        self.H = transfer_function(n, self.kb, h, det_distance, det_na) if det_na > 0 else None

    # -- operators ---------------------------------------------------------
    def G(self, v: np.ndarray) -> np.ndarray:
        return green_apply(v, self.khat)

    def GH(self, v: np.ndarray) -> np.ndarray:
        return green_apply(v, self.khat, adjoint=True)

    def u_in(self, l: int) -> np.ndarray:
        return incident_field(self.shape, self.kdirs[l], self.kb, self.h)

    def total_field(self, x: np.ndarray, l: int) -> Tuple[np.ndarray, int]:
        """u solving u = u_in + G(x u) (LS) or u = u_in (Born)."""
        uin = self.u_in(l)
        if self.model == "born":
            return uin, 0
        u, it, _ = bicgstab(lambda p: p - self.G(x * p), uin, uin, self.tol, self.maxit)
        return u, it

    def detect(self, usc: np.ndarray) -> np.ndarray:
        """S (then D for a remote detector): last z-slice of the scattered
        field, flattened [y, x] (M = n^2)."""
        sl = usc[-1]
        if self.H is not None:
            sl = propagate(sl, self.H)
        return sl.reshape(-1).copy()

    def lift(self, r: np.ndarray) -> np.ndarray:
        """S^T (after D^H for a remote detector): embed a detector vector into
        the last z-slice of a zero volume."""
        r2 = r.reshape(self.shape[1], self.shape[2])
        if self.H is not None:
            r2 = propagate(r2, self.H, adjoint=True)
        out = np.zeros(self.shape, dtype=np.complex128)
        out[-1] = r2
        return out

    def forward(self, x: np.ndarray, l: int) -> np.ndarray:
        """H_l(x): detector samples of the scattered field."""
        uin = self.u_in(l)
        if self.model == "born":
            return self.detect(self.G(x * uin))
        u, _ = self.total_field(x, l)
        return self.detect(u - uin)

    def loss_grad(self, x: np.ndarray, l: int, y: np.ndarray) -> Tuple[float, np.ndarray, Tuple[int, int]]:
        """(f_l(x), grad f_l(x), (forward its, adjoint its))."""
        uin = self.u_in(l)
        if self.model == "born":
            r = self.detect(self.G(x * uin)) - y
            z = self.GH(self.lift(r))
            return 0.5 * float(np.vdot(r, r).real), np.real(np.conj(uin) * z), (0, 0)
        u, it_f = self.total_field(x, l)
        r = self.detect(u - uin) - y
        b = self.GH(self.lift(r))
        z, it_a, _ = bicgstab(lambda q: q - self.GH(x * q), b, np.zeros_like(b), self.tol, self.maxit)
        return 0.5 * float(np.vdot(r, r).real), np.real(np.conj(u) * z), (it_f, it_a)

    def batch_loss_grad(self, x: np.ndarray, illum: Sequence[int], ys: np.ndarray,
                        scale: float) -> Tuple[float, np.ndarray]:
        """scale * sum_l f_l and scale * sum_l grad f_l; scale = S/L gives F_s (Eq. 4.1)."""
        loss = 0.0
        g = np.zeros_like(x, dtype=np.float64)
        for l in illum:
            f, gl, _ = self.loss_grad(x, int(l), ys[int(l)])
            loss += f
            g += gl
        return scale * loss, scale * g

    def born_normal(self, dx: np.ndarray, illum: Sequence[int], scale: float) -> np.ndarray:
        """scale * sum_l Re(J_l^H J_l dx) for the Born Jacobian J_l at x = 0."""
        out = np.zeros_like(dx, dtype=np.float64)
        for l in illum:
            uin = self.u_in(int(l))
            y = self.detect(self.G(dx * uin))
            out += np.real(np.conj(uin) * self.GH(self.lift(y)))
        return scale * out

    def lipschitz(self, illum: Sequence[int], scale: float, start: np.ndarray,
                  iters: int = 20) -> float:
        """alpha_s: power iteration on the Born Gauss-Newton operator of F_s.

        The paper leaves alpha_s as 'the Lipschitz constant of F_s' (Algorithm 4.1
        input); our reading estimates it by ``iters`` power steps from ``start``
        and returns the final Rayleigh quotient.
        """
        q = start / np.linalg.norm(start)
        lam = 0.0
        for _ in range(iters):
            a = self.born_normal(q, illum, scale)
            lam = float(np.vdot(q, a).real)
            q = a / np.linalg.norm(a)
        return lam


def simulate(model: Model, x_true: np.ndarray, noise: np.ndarray, snr_db: float) -> np.ndarray:
    """Measurements y_l = H_l(x_true) + sigma_l * noise_l with per-view SNR.

    sigma_l = ||H_l(x_true)|| / sqrt(M) * 10^(-snr/20) (our reading of the
    paper's noisy complex measurements).
    """
    L = model.kdirs.shape[0]
    M = model.shape[1] * model.shape[2]
    ys = np.zeros((L, M), dtype=np.complex128)
    for l in range(L):
        clean = model.forward(x_true, l)
        sigma = np.linalg.norm(clean) / math.sqrt(M) * 10.0 ** (-snr_db / 20.0)
        ys[l] = clean + sigma * noise[l]
    return ys
