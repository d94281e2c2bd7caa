"""Pins of the oracle's forward model against definitions it does not use itself.

Each test checks the FFT/BiCGSTAB oracle against an independent statement:
the O(N^2) direct Green's sum, numerical quadrature of the self term, a dense
LU solve of the discretised Lippmann-Schwinger system, the first-Born limit,
the adjoint identity and central finite differences of the data term.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import synth
from oracle import physics as ph

KB = math.pi / 2.0


def direct_green_matrix(n, kb, h=1.0):
    """Dense (N x N) matrix of G from the pairwise definition (no FFT); n is an
    edge or (nz, ny, nx)."""
    nz, ny, nx = (n, n, n) if np.ndim(n) == 0 else n
    idx = np.array([(z, y, x) for z in range(nz) for y in range(ny) for x in range(nx)], dtype=float)
    d = idx[:, None, :] - idx[None, :, :]
    r = h * np.sqrt(np.sum(d * d, axis=-1))
    with np.errstate(divide="ignore", invalid="ignore"):
        w = h ** 3 * np.exp(1j * kb * r) / (4 * math.pi * r)
    a = (3 / (4 * math.pi)) ** (1 / 3) * h
    # self term by quadrature of r exp(j kb r) over [0, a] (independent of the closed form)
    re = integrate.quad(lambda t: t * math.cos(kb * t), 0, a, epsabs=1e-14)[0]
    im = integrate.quad(lambda t: t * math.sin(kb * t), 0, a, epsabs=1e-14)[0]
    np.fill_diagonal(w, re + 1j * im)
    return kb ** 2 * w


def rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_self_term_matches_quadrature():
    for kb in (0.3, KB, 2.0):
        a = (3 / (4 * math.pi)) ** (1 / 3)
        re = integrate.quad(lambda t: t * math.cos(kb * t), 0, a, epsabs=1e-15)[0]
        im = integrate.quad(lambda t: t * math.sin(kb * t), 0, a, epsabs=1e-15)[0]
        assert abs(ph.self_term(kb) - (re + 1j * im)) < 1e-13


@pytest.mark.parametrize("n", [3, 4, 5])
def test_green_fft_equals_direct_sum(n):
    rng = np.random.default_rng(n)
    v = rand_c(rng, (n, n, n))
    Gd = direct_green_matrix(n, KB)
    ref = (Gd @ v.reshape(-1)).reshape(n, n, n)
    out = ph.green_apply(v, ph.green_hat(n, KB))
    assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) < 1e-12
    refH = (Gd.conj().T @ v.reshape(-1)).reshape(n, n, n)
    outH = ph.green_apply(v, ph.green_hat(n, KB), adjoint=True)
    assert np.max(np.abs(outH - refH)) / np.max(np.abs(refH)) < 1e-12


def test_green_is_complex_symmetric_and_khat_even():
    n = 6
    rng = np.random.default_rng(1)
    a, b = rand_c(rng, (n,) * 3), rand_c(rng, (n,) * 3)
    kh = ph.green_hat(n, KB)
    # <G a, b> = <a, G^H b>
    lhs = np.vdot(ph.green_apply(a, kh), b)
    rhs = np.vdot(a, ph.green_apply(b, kh, adjoint=True))
    assert abs(lhs - rhs) / abs(lhs) < 1e-12
    # G^T = G: sum (G a) b = sum a (G b)
    assert abs(np.sum(ph.green_apply(a, kh) * b) - np.sum(a * ph.green_apply(b, kh))) < 1e-10 * abs(lhs)
    P = 2 * n
    k = np.arange(P)
    for ax in range(3):
        flipped = np.take(kh, (-k) % P, axis=ax)
        assert np.max(np.abs(flipped - kh)) < 1e-10 * np.max(np.abs(kh))
    assert np.max(np.abs(kh - np.transpose(kh, (1, 0, 2)))) < 1e-10 * np.max(np.abs(kh))


def test_incident_field_is_plane_wave():
    n = 8
    k = np.array([0.3, -0.4, math.sqrt(1 - 0.25)])
    u = ph.incident_field(n, k, KB)
    assert np.allclose(np.abs(u), 1.0)
    # phase advance of one voxel along x is kb*kx
    assert np.allclose(u[:, :, 1:] / u[:, :, :-1], np.exp(1j * KB * k[0]))
    assert np.allclose(u[1:] / u[:-1], np.exp(1j * KB * k[2]))
    # centred coordinates: phase zero at idx = n/2
    assert abs(u[n // 2, n // 2, n // 2] - 1.0) < 1e-15


def small_problem(n=5, L=3, contrast=0.3, model="ls", seed=0):
    rng = np.random.default_rng(seed)
    x = contrast * rng.uniform(0, 1, (n, n, n))
    t = math.radians(30)
    kd = np.array([[math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)]
                   for p in 2 * math.pi * np.arange(L) / L])
    return x, ph.Model(n, kd, model=model)


def test_ls_bicgstab_equals_dense_lu():
    n = 5
    x, m = small_problem(n, contrast=0.5)
    Gd = direct_green_matrix(n, KB)
    A = np.eye(n ** 3) - Gd * x.reshape(-1)[None, :]
    for l in range(3):
        uin = m.u_in(l)
        ref = np.linalg.solve(A, uin.reshape(-1)).reshape(n, n, n)
        u, it = m.total_field(x, l)
        assert it > 1
        assert np.max(np.abs(u - ref)) / np.max(np.abs(ref)) < 1e-10


def test_fixed_point_step_residual_and_contraction():
    """The refined warm start of the forward solve: for any u0 with residual
    r0 = u_in - (I - G X) u0, the step u1 = u0 + r0 has residual exactly
    G(x r0), checked against the dense operator (n = 5).  Repeated steps
    multiply the error by G X (e_k = (G X)^k e_0), so at a weak contrast,
    where the spectral radius of G X is below 1, the iterates approach the
    dense LU solution at that rate."""
    n = 5
    x, m = small_problem(n, contrast=0.05)
    Gd = direct_green_matrix(n, KB)
    GX = Gd * x.reshape(-1)[None, :]
    A = np.eye(n ** 3) - GX
    rho = np.max(np.abs(np.linalg.eigvals(GX)))
    assert rho < 1.0
    rng = np.random.default_rng(3)
    uin = m.u_in(0).reshape(-1)
    ref = np.linalg.solve(A, uin)
    u = ref + 1e-2 * (rng.standard_normal(uin.shape) + 1j * rng.standard_normal(uin.shape))
    e0 = np.linalg.norm(u - ref)
    kappa = np.linalg.cond(np.linalg.eig(GX)[1])   # ||(GX)^k|| <= kappa rho^k
    r = uin - A @ u
    for k in range(1, 7):
        u1 = u + r
        r1 = uin - A @ u1
        assert np.linalg.norm(r1 - GX @ r) <= 1e-12 * np.linalg.norm(uin)
        u, r = u1, r1
        # the error e_k = ref - u_k = (G X)^k e_0
        assert np.linalg.norm(u - ref) <= kappa * rho ** k * e0 * (1 + 1e-9) + 1e-13


def test_born_limit_first_order():
    n = 6
    x, m = small_problem(n, contrast=1.0)
    mb = ph.Model(n, m.kdirs, model="born")
    errs = []
    eps = [1e-1, 1e-2, 1e-3]
    for e in eps:
        hls = m.forward(e * x, 0)
        hb = mb.forward(e * x, 0)
        errs.append(np.linalg.norm(hls - hb) / np.linalg.norm(hb))
    slopes = np.diff(np.log10(errs)) / np.diff(np.log10(eps))
    assert np.all(np.abs(slopes - 1.0) < 0.1), slopes


def _jvp(m, x, l, dx, h=1e-6):
    return (m.forward(x + h * dx, l) - m.forward(x - h * dx, l)) / (2 * h)


@pytest.mark.parametrize("model,remote", [("ls", False), ("born", False), ("ls", True)])
def test_gradient_central_differences(model, remote):
    n = 5
    x, m = small_problem(n, contrast=0.4, model=model)
    if remote:   # remote detector: the gradient must carry D^H through the lift
        m = ph.Model(n, m.kdirs, model=model, det_distance=3.0, det_na=0.8)
    rng = np.random.default_rng(7)
    y = rand_c(rng, n * n) * 0.05
    f0, g, _ = m.loss_grad(x, 1, y)
    for trial in range(4):
        if trial < 2:
            dx = np.zeros_like(x)
            dx[tuple(rng.integers(0, n, 3))] = 1.0      # single-voxel direction
        else:
            dx = rng.standard_normal(x.shape)
        h = 1e-5
        fp, _, _ = m.loss_grad(x + h * dx, 1, y)
        fm, _, _ = m.loss_grad(x - h * dx, 1, y)
        fd = (fp - fm) / (2 * h)
        an = float(np.sum(g * dx))
        assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-12) + 1e-12, (fd, an)


def test_adjoint_identity():
    n = 5
    x, m = small_problem(n, contrast=0.4)
    rng = np.random.default_rng(3)
    r = rand_c(rng, n * n)
    dx = rng.standard_normal(x.shape)
    # J dx by central differences of H (second order, exact up to O(h^2))
    jdx = _jvp(m, x, 0, dx, 1e-5)
    # J^H r from the gradient at y = H(x) - r: grad f = Re(J^H (H - y)) = Re(J^H r)
    y = m.forward(x, 0) - r
    _, g, _ = m.loss_grad(x, 0, y)
    lhs = float(np.real(np.vdot(r, jdx)))
    rhs = float(np.sum(dx * g))
    assert abs(lhs - rhs) <= 1e-7 * abs(lhs)


def test_lipschitz_power_iteration_matches_eigenvalue():
    n = 4
    _, m = small_problem(n, L=2, model="born")
    N = n ** 3
    A = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        A[:, j] = m.born_normal(e.reshape(n, n, n), [0, 1], 0.5).reshape(-1)
    assert np.allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    lam_max = np.linalg.eigvalsh(A)[-1]
    rng = np.random.default_rng(0)
    est = m.lipschitz([0, 1], 0.5, rng.standard_normal((n, n, n)), iters=200)
    assert abs(est - lam_max) <= 1e-6 * lam_max


def test_detector_and_lift_are_adjoint():
    n = 6
    _, m = small_problem(n)
    rng = np.random.default_rng(2)
    v = rand_c(rng, (n, n, n))
    r = rand_c(rng, n * n)
    assert abs(np.vdot(r, m.detect(v)) - np.vdot(m.lift(r), v)) < 1e-12


def test_physical_units_enter_only_through_kb_h():
    """Dimensional analysis of the discretisation (Section 6 reading): with the
    voxel edge h in metres and k_b = 2 pi eta_m / lambda, the Green's weights
    k_b^2 h^3 e^{j k_b |D| h} / (4 pi |D| h), the equal-volume self term and the
    incident phases depend on k_b h only, so the paper's 50 nm / 406 nm / 1.333
    set-up equals the unit-voxel model with k_b = k_b h."""
    n = 8
    w = synth.small("sim64", n=n, L=2, batch=1)
    kd = synth.illumination_dirs(w)
    x = synth.phantom(w)
    assert x.max() > 0.1                       # strong scattering: (1.43/1.333)^2 - 1
    kbh = w.kb * w.h
    assert abs(kbh - 2 * math.pi * 1.333 * 50 / 406) < 1e-12
    mp = ph.Model(n, kd, model="ls", kb=w.kb, h=w.h, tol=1e-13)
    mu = ph.Model(n, kd, model="ls", kb=kbh, h=1.0, tol=1e-13)
    assert np.allclose(mp.khat, mu.khat, rtol=0, atol=1e-12 * np.abs(mu.khat).max())
    for l in range(2):
        yp, yu = mp.forward(x, l), mu.forward(x, l)
        assert np.max(np.abs(yp - yu)) <= 1e-10 * np.max(np.abs(yu))


def test_remote_detector_propagation_pins():
    """Angular-spectrum remote detector: identity at zero distance with an open
    pupil; a grid plane wave inside the pupil gains exactly exp(j k_z d) (sign of
    the exp(j <k, r>) convention); two distances compose; D is unitary on the
    pupil band; <D a, b> = <a, D^H b>; the data term's adjoint (lift) is the
    transpose of detect."""
    n, h = 16, 1.0
    kb = ph.kb_default(h)
    rng = np.random.default_rng(5)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    b = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H0 = ph.transfer_function(n, kb, h, 0.0, 100.0)
    assert np.allclose(ph.propagate(a, H0), a, atol=1e-13)
    d = 7.5
    H = ph.transfer_function(n, kb, h, d, 0.9)
    fx, fy = 2, 1                                # grid frequency inside the pupil
    kx, ky = 2 * math.pi * fx / (n * h), 2 * math.pi * fy / (n * h)
    assert kx * kx + ky * ky <= (0.9 * kb) ** 2
    yy, xx = np.meshgrid(np.arange(n) * h, np.arange(n) * h, indexing="ij")
    pw = np.exp(1j * (kx * xx + ky * yy))
    kz = math.sqrt(kb * kb - kx * kx - ky * ky)
    assert np.allclose(ph.propagate(pw, H), np.exp(1j * kz * d) * pw, atol=1e-12)
    # an evanescent grid wave (|k| > k_b, pupil opened past 1) decays by exp(-sqrt(k^2 - k_b^2) d)
    fe = 6
    ke = 2 * math.pi * fe / (n * h)
    assert ke > kb
    ew = np.exp(1j * ke * xx)
    He = ph.transfer_function(n, kb, h, d, 3.0)
    assert np.allclose(ph.propagate(ew, He), math.exp(-math.sqrt(ke * ke - kb * kb) * d) * ew, atol=1e-12)
    H1, H2 = ph.transfer_function(n, kb, h, 3.0, 0.9), ph.transfer_function(n, kb, h, 4.5, 0.9)
    assert np.allclose(ph.propagate(ph.propagate(a, H1), H2), ph.propagate(a, H), atol=1e-12)
    band = ph.propagate(a, ph.transfer_function(n, kb, h, 0.0, 0.9))   # pupil-limited field
    assert abs(np.linalg.norm(ph.propagate(band, H)) - np.linalg.norm(band)) < 1e-12 * np.linalg.norm(band)
    lhs = np.vdot(b, ph.propagate(a, H))
    rhs = np.vdot(ph.propagate(b, H, adjoint=True), a)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    kd = np.array([[0.0, 0.0, 1.0]])
    m = ph.Model(n, kd, "born", det_distance=d, det_na=0.9)
    v = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    r = rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n)
    assert abs(np.vdot(r, m.detect(v)) - np.vdot(m.lift(r), v)) < 1e-12 * np.linalg.norm(r) * np.linalg.norm(v)


# ------------------------------------------------------------ truncated kernel
def _ft_by_quadrature(s, kb, R):
    """(1/s) int_0^R exp(j kb r) sin(s r) dr (s > 0), or int_0^R r exp(j kb r) dr (s = 0),
    by adaptive quadrature of the real and imaginary parts."""
    if s == 0:
        re = integrate.quad(lambda r: r * math.cos(kb * r), 0, R, limit=4000, epsabs=0, epsrel=1e-13)[0]
        im = integrate.quad(lambda r: r * math.sin(kb * r), 0, R, limit=4000, epsabs=0, epsrel=1e-13)[0]
        return re + 1j * im
    re = integrate.quad(lambda r: math.cos(kb * r) * math.sin(s * r), 0, R, limit=4000, epsabs=0, epsrel=1e-13)[0]
    im = integrate.quad(lambda r: math.sin(kb * r) * math.sin(s * r), 0, R, limit=4000, epsabs=0, epsrel=1e-13)[0]
    return (re + 1j * im) / s


def test_truncated_kernel_transform_pins():
    """The transform of the truncated Green's function against (i) quadrature of
    its radial integral at generic frequencies, s = 0 and both sides of s = kb,
    and (ii) the closed form of its s -> kb limit,
    exp(j kb R)(R sin kb R + j (kb R cos kb R - sin kb R)/kb) / (2 kb),
    obtained by l'Hopital's rule from [-1 + exp(j kb R)(cos sR - j kb sin(sR)/s)]/(kb^2 - s^2)."""
    kb, R = math.pi / 2, math.sqrt(3.0) * 24
    for s in (0.0, 0.2 * kb, 0.9 * kb, kb * (1 - 1e-7), kb, kb * (1 + 1e-7), 1.7 * kb, 4.1 * kb):
        got = complex(ph.truncated_green_ft(s, kb, R))
        ref = _ft_by_quadrature(s, kb, R)
        assert abs(got - ref) <= 1e-9 * abs(ref), (s, got, ref)
    lim = np.exp(1j * kb * R) * (R * math.sin(kb * R) + 1j * (kb * R * math.cos(kb * R) - math.sin(kb * R)) / kb) / (2 * kb)
    assert abs(complex(ph.truncated_green_ft(kb, kb, R)) - lim) <= 1e-12 * abs(lim)
    # the rational closed form away from s = kb (independent algebra)
    for s in (0.4 * kb, 2.3 * kb):
        cf = (-1 + np.exp(1j * kb * R) * (math.cos(s * R) - 1j * kb * math.sin(s * R) / s)) / (kb * kb - s * s)
        assert abs(complex(ph.truncated_green_ft(s, kb, R)) - cf) <= 1e-12 * abs(cf)


def _gaussian_potential(r, kb, sig):
    """k_b^2 (g * rho)(r) for rho(t) = exp(-t^2 / (2 sig^2)): the shell formula
    int_{|r'| = t} g(r - r') dS' = (t / (2 r)) (exp(j kb (r + t)) - exp(j kb |r - t|)) / (j kb),
    integrated over t by quadrature."""
    def part(t, which):
        v = math.exp(-t * t / (2 * sig * sig)) * t / (2 * r) * (
            (np.exp(1j * kb * (r + t)) - np.exp(1j * kb * abs(r - t))) / (1j * kb))
        return v.real if which == 0 else v.imag
    tot = 0j
    for a, b in ((0.0, r), (r, 12 * sig + r)):
        tot += integrate.quad(part, a, b, args=(0,), limit=400, epsabs=0, epsrel=1e-12)[0]
        tot += 1j * integrate.quad(part, a, b, args=(1,), limit=400, epsabs=0, epsrel=1e-12)[0]
    return kb * kb * tot


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
def test_truncated_kernel_converges_to_the_continuous_convolution():
    """On a smooth source (a Gaussian, sigma = 2.5 voxels, well inside a 32^3
    grid; band-limited to ~1e-13 at the grid's Nyquist frequency) G v with the
    truncated kernel equals the continuous convolution k_b^2 (g * rho) at the
    voxels to the accuracy of the quadrature, while the sampled kernel with the
    sphere self term is off by percents at four voxels per wavelength."""
    n, kb, sig = 32, math.pi / 2, 2.5
    c = np.array([n / 2 - 0.5, n / 2 - 0.2, n / 2 - 0.7])   # centre (z, y, x), off the grid
    i = np.arange(n, dtype=np.float64)
    r2 = (i[:, None, None] - c[0]) ** 2 + (i[None, :, None] - c[1]) ** 2 + (i[None, None, :] - c[2]) ** 2
    v = np.exp(-r2 / (2 * sig * sig)).astype(np.complex128)
    g_tr = ph.green_apply(v, ph.green_hat(n, kb, 1.0, "truncated"))
    g_sa = ph.green_apply(v, ph.green_hat(n, kb, 1.0, "sampled"))
    rng = np.random.default_rng(32)
    err_tr = err_sa = scale = 0.0
    for p in rng.integers(0, n, size=(10, 3)):
        r = math.sqrt(float(np.sum((p - c) ** 2)))
        ref = _gaussian_potential(r, kb, sig)
        err_tr = max(err_tr, abs(g_tr[tuple(p)] - ref))
        err_sa = max(err_sa, abs(g_sa[tuple(p)] - ref))
        scale = max(scale, abs(ref))
    assert err_tr <= 1e-6 * scale, err_tr / scale
    assert err_sa >= 1e-2 * scale


def test_truncated_kernel_is_even_and_symmetric():
    """The truncated kernel's spectrum is even in every axis (g_R is radial) and
    its operator complex symmetric, like the sampled one: <G a, b> = <a, G^H b>."""
    n = 8
    K = ph.green_hat(n, math.pi / 2, 1.0, "truncated")
    P = 2 * n
    m = (-np.arange(P)) % P
    assert np.allclose(K, K[m][:, m][:, :, m], rtol=0, atol=1e-12 * np.abs(K).max())
    assert np.allclose(K, np.transpose(K, (2, 1, 0)), rtol=0, atol=1e-12 * np.abs(K).max())
    rng = np.random.default_rng(8)
    a = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    b = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    lhs = np.vdot(b, ph.green_apply(a, K))
    rhs = np.vdot(ph.green_apply(b, K, adjoint=True), a)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)



# ------------------------------------------------------------ box-shaped grids
@pytest.mark.parametrize("shape", [(3, 4, 5), (5, 3, 4), (2, 6, 3)])
def test_green_fft_equals_direct_sum_on_boxes(shape):
    """G v on nz x ny x nx grids (periods 2 nz, 2 ny, 2 nx) against the pairwise sum."""
    rng = np.random.default_rng(sum(shape))
    v = rand_c(rng, shape)
    Gd = direct_green_matrix(shape, KB)
    kh = ph.green_hat(shape, KB)
    assert kh.shape == tuple(2 * m for m in shape)
    for adj, M in ((False, Gd), (True, Gd.conj().T)):
        ref = (M @ v.reshape(-1)).reshape(shape)
        out = ph.green_apply(v, kh, adjoint=adj)
        assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) < 1e-12


def test_box_incident_field_and_detector_layout():
    """The incident field steps by exp(j kb k_d h) along each axis of a box and
    is 1 at the centre (n_d/2 per axis); the detector is the last z-slice
    (ny x nx) and the lift its adjoint."""
    shape = (6, 4, 8)
    kd = np.array([0.3, -0.4, math.sqrt(1 - 0.25)])
    u = ph.incident_field(shape, kd, KB)
    assert u.shape == shape
    assert abs(u[3, 2, 4] - 1.0) < 1e-15
    for ax, d in ((2, 0), (1, 1), (0, 2)):
        ratio = np.take(u, range(1, shape[ax]), axis=ax) / np.take(u, range(0, shape[ax] - 1), axis=ax)
        assert np.allclose(ratio, np.exp(1j * KB * kd[d]), atol=1e-13)
    m = ph.Model(shape, kd[None, :], "born")
    rng = np.random.default_rng(3)
    vol, r = rand_c(rng, shape), rand_c(rng, (4 * 8,))
    assert np.array_equal(m.detect(vol), vol[-1].reshape(-1))
    assert abs(np.vdot(m.detect(vol), r) - np.vdot(vol, m.lift(r))) < 1e-12 * abs(np.vdot(vol, m.lift(r)))


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
def test_truncated_kernel_on_an_elongated_box():
    """An elongated box needs periods beyond 4 n_d on its short axes (T_d h >=
    n_d h + R with R the box diagonal); with them the truncated kernel's G v of
    a smooth source matches the continuous convolution, as on the cube."""
    shape, kb, sig = (128, 32, 32), math.pi / 2, 2.5
    R, T = ph.truncated_periods(shape)
    assert T[0] == 512 and T[1] > 128 and T[2] > 128
    assert all(t >= n + R for t, n in zip(T, shape))
    c = np.array([63.6, 15.3, 15.8])
    i = [np.arange(m, dtype=np.float64) for m in shape]
    r2 = (i[0][:, None, None] - c[0]) ** 2 + (i[1][None, :, None] - c[1]) ** 2 + (i[2][None, None, :] - c[2]) ** 2
    v = np.exp(-r2 / (2 * sig * sig)).astype(np.complex128)
    g_tr = ph.green_apply(v, ph.green_hat(shape, kb, 1.0, "truncated"))
    rng = np.random.default_rng(40)
    err = scale = 0.0
    for p in zip(rng.integers(0, 128, 8), rng.integers(0, 32, 8), rng.integers(0, 32, 8)):
        rr = math.sqrt(float(np.sum((np.array(p) - c) ** 2)))
        ref = _gaussian_potential(rr, kb, sig)
        err = max(err, abs(g_tr[p] - ref))
        scale = max(scale, abs(ref))
    assert err <= 1e-6 * scale, err / scale
