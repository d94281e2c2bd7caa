"""GPU parity of the truncated Green's kernel (Vico, Greengard and Ferrando;
the optional discretisation of the Section 6 forward model) against the FP64
oracle, which builds it by a full inverse FFT of the sampled transform while
the library uses three even cosine passes in FP64 on the device.

Tolerances as in the other parity tests: Green's apply 2e-6 relative
(max-norm, the complex64 transform floor); forward data 2e-5; gradient 1e-4
norm-wise and loss 1e-5 with Krylov tolerance 1e-6.
"""
import math

import numpy as np
import pytest

import synth
from oracle import physics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2307_02043_gb300 import binding  # noqa: E402

DEV = torch.device("cuda:0")
KB = math.pi / 2


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n", [8, 12, 16, 32, 64])
@pytest.mark.parametrize("adjoint", [False, True])
def test_truncated_apply_matches_oracle(n, adjoint):
    rng = np.random.default_rng(700 + n + adjoint)
    v = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    h = binding.MQNPM(n, [[0.0, 0.0, 1.0]], [0], [1.0], max_batch=1, green_kernel="truncated")
    out = h.green_apply(torch.from_numpy(v.astype(np.complex64)).to(DEV).reshape(-1), adjoint=adjoint)
    ref = physics.green_apply(v, physics.green_hat(n, KB, 1.0, "truncated"), adjoint=adjoint)
    assert relmax(out.cpu().numpy().reshape(n, n, n), ref) < 2e-6
    h.close()


def test_truncated_apply_physical_units():
    """The geometry of the simulated experiment (50 nm voxels, 406 nm vacuum
    wavelength in a 1.333 medium): the kernel depends on kb and h separately
    through R = sqrt(3) n h and the frequency grid."""
    w = synth.workload("sim64")
    n = 32
    rng = np.random.default_rng(701)
    v = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    h = binding.MQNPM(n, [[0.0, 0.0, 1.0]], [0], [1.0], max_batch=1, h=w.h, kb=w.kb, green_kernel="truncated")
    out = h.green_apply(torch.from_numpy(v.astype(np.complex64)).to(DEV).reshape(-1))
    ref = physics.green_apply(v, physics.green_hat(n, w.kb, w.h, "truncated"))
    assert relmax(out.cpu().numpy().reshape(n, n, n), ref) < 2e-6
    h.close()


@pytest.mark.parametrize("model", ["ls", "born"])
def test_truncated_forward_and_gradient_match_oracle(model):
    n = 16
    w = synth.small("ls32", n=n, L=6, batch=3, model=model).with_(contrast_max=0.05)
    kd = synth.illumination_dirs(w)
    xt = synth.phantom(w)
    om = physics.Model(n, kd, model, tol=1e-12, kernel="truncated")
    ys = physics.simulate(om, xt, synth.noise_draws(w), w.snr_db)
    subs = synth.subsets(w)
    so = np.zeros(w.L, dtype=np.int32)
    for s, ii in enumerate(subs):
        so[ii] = s
    h = binding.MQNPM(n, kd, so, [1.0] * w.S, model=model, krylov_tol=1e-6, max_batch=3, green_kernel="truncated")
    xg = torch.from_numpy(xt.astype(np.float32)).to(DEV).reshape(-1)
    y, _ = h.forward(xg, [0, 1, 4])
    for b, l in enumerate([0, 1, 4]):
        assert rel(y[b].cpu().numpy(), om.forward(xt, l)) < 2e-5
    h.set_measurements(torch.from_numpy(ys.astype(np.complex64)).to(DEV).reshape(-1))
    x = 0.7 * xt
    scale = w.S / w.L
    g, loss, its = h.grad_batch(torch.from_numpy(x.astype(np.float32)).to(DEV).reshape(-1), [0, 1, 2], scale)
    lo, go = om.batch_loss_grad(x, [0, 1, 2], ys, scale)
    assert rel(g.cpu().numpy().reshape(go.shape), go) < 1e-4
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    h.close()
