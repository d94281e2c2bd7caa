"""The one-plane applies against the full apply on the same GPU, at grids whose
launch shapes differ (wide threads per line at P = 192, 320, 384):

* plane output (first-Born data S G(x u_in)): the detector plane of a full
  G(x u_in) from `green_apply`;
* plane input (the adjoint right-hand side G^H S^T r inside the Born gradient):
  Re(conj(u_in) G^H S^T r) with G^H S^T r from a full adjoint `green_apply` of
  the lifted residual.

The oracle pins both transforms elsewhere; here the two GPU routes must agree
to FP32 rounding.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from oracle import physics  # noqa: E402
from paper_2307_02043_gb300 import binding  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
KB = math.pi / 2


def cone(L, deg=40.0):
    t = math.radians(deg)
    return np.array([[math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)]
                     for p in 2 * math.pi * np.arange(L) / L])


@pytest.mark.parametrize("n,tile", [(24, -1), (96, -1), (160, -1), (192, -1), (128, 15), (64, 8)])
def test_plane_applies_equal_full_applies(n, tile):
    rng = np.random.default_rng(900 + n)
    L = 2
    kd = cone(L)
    h = binding.MQNPM(n, kd, [0, 0], [1.0], model="born", max_batch=2, tile=tile)
    x = np.zeros((n, n, n))
    c = n // 2
    x[c - n // 4:c + n // 4, c - n // 4:c + n // 4, 2:n - 2] = 0.02 * rng.random((2 * (n // 4), 2 * (n // 4), n - 4))
    xd = torch.from_numpy(x.astype(np.float32).reshape(-1)).to(DEV)
    uin = np.stack([physics.incident_field(n, kd[l], KB) for l in range(L)])
    v = torch.from_numpy((x[None] * uin).astype(np.complex64).reshape(-1)).to(DEV)
    full = h.green_apply(v).cpu().numpy().reshape(L, n, n, n)
    y, _ = h.forward(xd, [0, 1])
    y = y.cpu().numpy().reshape(L, n, n)
    for b in range(L):
        ref = full[b, n - 1]
        assert np.max(np.abs(y[b] - ref)) <= 1e-5 * np.max(np.abs(ref)), (n, b)
    # Born gradient: its adjoint right-hand side goes through the plane-input apply
    ym = (y + 0.1 * np.max(np.abs(y)) * (rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape))
          ).astype(np.complex64)
    h.set_measurements(torch.from_numpy(ym.reshape(-1)).to(DEV))
    g, loss, _ = h.grad_batch(xd, [0, 1], 0.5)
    g = g.cpu().numpy().astype(np.float64).reshape(n, n, n)
    lift = np.zeros((L, n, n, n), dtype=np.complex64)
    lift[:, n - 1] = (y - ym)
    z = h.green_apply(torch.from_numpy(lift.reshape(-1)).to(DEV), adjoint=True).cpu().numpy().reshape(L, n, n, n)
    ref = 0.5 * sum(np.real(np.conj(uin[b]) * z[b]) for b in range(L))
    assert np.linalg.norm(g - ref) <= 1e-5 * np.linalg.norm(ref), n
    r = (y - ym).astype(np.complex128)
    assert abs(loss - 0.5 * 0.5 * float(np.vdot(r, r).real)) <= 1e-5 * loss
    h.close()
