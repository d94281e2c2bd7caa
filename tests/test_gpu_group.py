"""GPU: shared launches for several reconstructions of one grid (a group of
handles).  Two volumes with different phantoms, illumination counts, subsets
and TV weights step together; every Green's pass and BiCGSTAB iteration of
their subset gradients is one launch over the slots of both.  Each slot's
solve reads only its own volume's data and keeps its own scalars, so when each
member's subset lies in one chunk the group reproduces separate handles bit
for bit; when a chunk boundary splits a member's subset its gradient is summed
in two pieces (held to 1e-5, the batching tolerance of the other tests)."""
import numpy as np
import pytest

import synth
from oracle import physics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2307_02043_gb300 import binding  # noqa: E402

DEV = torch.device("cuda:0")


def volume(config_id, L, batch, lam):
    w = synth.small("ls32", n=16, L=L, batch=batch).with_(config_id=config_id, lam=lam, contrast_max=0.05)
    kd = synth.illumination_dirs(w)
    om = physics.Model(w.n, kd, "ls", tol=1e-12)
    ys = physics.simulate(om, synth.phantom(w), synth.noise_draws(w), w.snr_db)
    so = np.zeros(w.L, dtype=np.int32)
    for s, ii in enumerate(synth.subsets(w)):
        so[ii] = s
    alpha = [om.lipschitz(q, w.S / w.L, synth.power_start(w), 10) for q in synth.subsets(w)]
    return w, kd, so, alpha, torch.from_numpy(ys.astype(np.complex64)).to(DEV).reshape(-1)


def make(v, warm, max_batch):
    w, kd, so, alpha, y = v
    h = binding.MQNPM(w.n, kd, so, alpha, tv=w.tv, lam=w.lam, box=(0.0, 0.06), krylov_tol=1e-6,
                      dual_iters=w.dual_iters, max_batch=max_batch, warm_start=warm, tile=0)
    h.set_measurements(y)
    return h


@pytest.mark.parametrize("warm", [False, True])
@pytest.mark.parametrize("max_slots,exact", [(5, True), (2, False)])
def test_group_equals_separate_handles(warm, max_slots, exact):
    vols = [volume(11, 6, 3, 1e-3), volume(12, 4, 2, 3e-3)]       # subsets of 3 and 2 illuminations
    alone = [make(v, warm, 3) for v in vols]
    members = [make(v, warm, 1) for v in vols]
    group = binding.Group(members, max_slots=max_slots)
    xa = [torch.zeros(16 ** 3, dtype=torch.float32, device=DEV) for _ in vols]
    xg = [torch.zeros_like(x) for x in xa]
    for k in range(1, 7):
        ia = [h.step(x) for h, x in zip(alone, xa)]
        ig = group.step(xg)
        for a, b, x1, x2 in zip(ia, ig, xa, xg):
            assert a["k"] == b["k"] == k and a["subset"] == b["subset"] and a["n_illum"] == b["n_illum"]
            if exact:
                assert a["loss"] == b["loss"] and a["tau_star"] == b["tau_star"]
                assert a["krylov_iters_total"] == b["krylov_iters_total"]
                assert torch.equal(x1, x2), k
            else:
                assert abs(a["loss"] - b["loss"]) <= 1e-5 * abs(a["loss"])
                assert float((x1 - x2).norm() / x1.norm()) < 1e-5, k
    assert group.workspace_bytes > 0
    group.close()
    for h in alone + members:
        h.close()


def test_group_rejects_mismatched_members():
    v16 = volume(11, 6, 3, 1e-3)
    a = make(v16, False, 1)
    w = synth.small("ls32", n=24, L=4, batch=2)
    b = binding.MQNPM(24, synth.illumination_dirs(w), [0, 1, 0, 1], [1.0, 1.0], max_batch=1)
    with pytest.raises(binding.MQNPMError) as err:
        binding.Group([a, b], max_slots=4)
    assert err.value.code == 1                       # different grids
    c = binding.MQNPM(16, synth.illumination_dirs(w), [0, 1, 0, 1], [1.0, 1.0], model="born", max_batch=1,
                      krylov_tol=1e-6, tile=0)
    with pytest.raises(binding.MQNPMError) as err:
        binding.Group([a, c], max_slots=4)
    assert err.value.code == 7                       # first-Born members are not grouped
    with pytest.raises(binding.MQNPMError):
        binding.Group([a, a], max_slots=4)            # a member once
    for h in (a, b, c):
        h.close()
