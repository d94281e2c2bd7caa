"""Guard bands around every workspace buffer (the out-of-bounds check that
stands in for compute-sanitizer, which this pool does not offer): after the
public calls of the path on grids with ragged tiles, no band may have been
written; a band overwritten on purpose must be reported."""
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2307_02043_gb300 import binding  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def f32(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.float32)).to(DEV)


@pytest.mark.parametrize("model,n,tile,remote", [("ls", 12, 0, False), ("ls", 24, 15, True),
                                                 ("born", 16, 7, False), ("ls", 48, -1, False)])
def test_no_call_writes_outside_its_buffers(model, n, tile, remote):
    w = synth.small("ls32", n=n, L=5, batch=2, model=model)
    kd = synth.illumination_dirs(w)
    so = np.zeros(w.L, dtype=np.int32)
    for s_, ii in enumerate(synth.subsets(w)):
        so[ii] = s_
    extra = dict(det_distance=4.0, det_na=0.7) if remote else {}
    h = binding.MQNPM(n, kd, so, [1.0] * w.S, model=model, lam=w.lam, box=w.box, krylov_tol=1e-6,
                      max_batch=2, tile=tile, warm_start=(model == "ls"), guard_bytes=4096, **extra)
    assert h.check_guards() == 0
    rng = np.random.default_rng(n)
    y = torch.from_numpy((0.01 * (rng.standard_normal((w.L, n * n)) + 1j * rng.standard_normal((w.L, n * n))))
                         .astype(np.complex64)).to(DEV)
    h.set_measurements(y.reshape(-1))
    x = f32(synth.phantom(w)).reshape(-1)
    v = torch.randn(2 * n ** 3, dtype=torch.complex64, device=DEV)
    h.green_apply(v)
    h.green_apply(v[: n ** 3], adjoint=True)
    h.forward(x, [0, 1])
    h.grad_batch(x, [0, 1, 2, 4], 0.5)              # two chunks, the second ragged
    h.loss_batch(x, [3, 4], 0.5)
    h.grad_fields(x, [3, 4], 0.5)
    U = 0.01 * torch.randn(3 * n ** 3, device=DEV)
    h.wprox(x, 2.0, U, 1e-3, P_warm=torch.zeros(3 * n ** 3, device=DEV))
    h.lipschitz([0, 2], 0.5, f32(synth.power_start(w)).reshape(-1), iters=2)
    xs = torch.zeros(n ** 3, device=DEV)
    for _ in range(w.S + 2):
        info = h.step(xs, allow_not_converged=True)
    h.diagnostics(x, info["subset"], xs)
    assert h.check_guards() == 0
    h.close()


def test_a_written_band_is_reported():
    h = binding.MQNPM(8, [[0.0, 0.0, 1.0], [0.0, 0.6, 0.8]], [0, 0], [1.0], max_batch=1, guard_bytes=256)
    assert h.check_guards() == 0
    assert h.lib.mqnpm_debug_poke_guard(h._h, 3) == 0
    assert h.lib.mqnpm_debug_poke_guard(h._h, 10 ** 6) == 1    # no such band
    assert h.check_guards() == 1
    h.close()
    h = binding.MQNPM(8, [[0.0, 0.0, 1.0]], [0], [1.0], max_batch=1)   # no guards: nothing to report
    assert h.check_guards() == 0
    h.close()
