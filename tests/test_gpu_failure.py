"""Failure detection on the GPU without a GPU fault: a bounded device-side
wait is made to run out on purpose and the host reads the error status.

The weighted proximal mapping is one cooperative kernel whose phases are
separated by grid barriers; every block's wait at a barrier is bounded by the
handle's wait limit (SM clock cycles).  With a limit of a few cycles the first
block that has to wait gives up, raises the device error flag, the other
blocks see the flag and leave, and mqnpm_wprox returns MQNPM_ERR_TIMEOUT.  The
same handle, with the default limit restored, then computes the proximal map
exactly as before (the kernel's reductions run in a fixed order) and as the
FP64 oracle does (1e-5 norm-wise, the proximal-map tolerance of the parity
tests).  No kernel is broken, no wait is unbounded and the context stays
usable throughout.
"""
import math

import numpy as np
import pytest

from oracle import wprox as owprox

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2307_02043_gb300 import binding  # noqa: E402

DEV = torch.device("cuda:0")
TIMEOUT = 6


def f32(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.float32)).to(DEV)


@pytest.mark.parametrize("S_eff", [0, 3])
def test_prox_barrier_wait_runs_out_then_recovers(S_eff):
    n, J, tau, c = 24, 12, 1.5, 2e-3
    rng = np.random.default_rng(600 + S_eff)
    v = rng.uniform(-0.02, 0.07, (n, n, n))
    U = rng.standard_normal((S_eff, n, n, n)) * 0.05 if S_eff else None
    P0 = rng.uniform(-0.5, 0.5, (3, n, n, n))
    kd = [[0.0, 0.0, 1.0], [math.sin(0.5), 0.0, math.cos(0.5)]]
    h = binding.MQNPM(n, kd, [0, 0], [1.0], tv="iso", box=(0.0, 0.05), dual_iters=J, newton_tol=1e-6,
                      max_batch=1)
    Ug = None if U is None else f32(U).reshape(-1)

    def run():
        Pw = f32(P0).reshape(-1).clone()
        return h.wprox(f32(v).reshape(-1), tau, Ug, c, P_warm=Pw), Pw

    x_ref, P_ref = run()
    x_ref, P_ref = x_ref.clone(), P_ref.clone()
    h.set_wait_limit(8)                       # far shorter than any barrier takes
    with pytest.raises(binding.MQNPMError) as err:
        run()
    assert err.value.code == TIMEOUT
    h.set_wait_limit(0)                       # the default limit again
    x2, P2 = run()
    assert torch.equal(x2, x_ref) and torch.equal(P2, P_ref)
    xo, _, _ = owprox.wprox(v, tau, U, c, 0.0, 0.05, "iso", J, P0=P0, newton_tol=1e-6)
    got = x2.cpu().numpy().reshape(n, n, n)
    assert np.linalg.norm(got - xo) <= 1e-5 * np.linalg.norm(xo)
    with pytest.raises(binding.MQNPMError) as bad:
        h.set_wait_limit(-1)
    assert bad.value.code == 1
    h.close()


def test_wait_limit_at_create():
    """The limit set in the configuration acts like the setter's."""
    n = 16
    rng = np.random.default_rng(601)
    v = rng.uniform(-0.02, 0.07, (n, n, n))
    kd = [[0.0, 0.0, 1.0]]
    h = binding.MQNPM(n, kd, [0], [1.0], box=(0.0, 0.05), dual_iters=4, max_batch=1, barrier_wait_cycles=8)
    with pytest.raises(binding.MQNPMError) as err:
        h.wprox(f32(v).reshape(-1), 1.0, None, 1e-3)
    assert err.value.code == TIMEOUT
    h.set_wait_limit(0)
    out = h.wprox(f32(v).reshape(-1), 1.0, None, 1e-3)
    assert torch.isfinite(out).all()
    h.close()
