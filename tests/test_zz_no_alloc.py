"""GPU: the allocation-free Green's apply against the handle's Green's apply.

Both run the same five transform passes in complex64 on the same kernel
spectrum construction, so they are held to the Green's-apply tolerance of the
parity tests (2e-6 relative, max-norm), on two calls in a row.  This file is
collected last so that it also runs after every other GPU test in one process.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2307_02043_gb300 import binding  # noqa: E402

DEV = torch.device("cuda:0")
KB = math.pi / 2


def relmax(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def volume(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    return torch.from_numpy(v.astype(np.complex64)).to(DEV).reshape(-1)


@pytest.mark.parametrize("n", [8, 16, 32])
@pytest.mark.parametrize("adjoint", [False, True])
def test_noalloc_matches_handle_two_calls(n, adjoint):
    h = binding.MQNPM(n, [[0.0, 0.0, 1.0]], [0], [1.0], max_batch=1, kb=KB)
    try:
        for call, seed in enumerate((11 * n, 11 * n + 1)):
            v = volume(n, seed)
            ref = h.green_apply(v, adjoint=adjoint).cpu().numpy()
            out = torch.empty_like(v)
            binding.green_apply_noalloc(n, 1.0, KB, v, out, adjoint=adjoint)
            torch.cuda.synchronize()
            err = relmax(out.cpu().numpy(), ref)
            assert err < 2e-6, (n, adjoint, call, err)
    finally:
        h.close()


def test_noalloc_switches_grid_and_holds_no_new_memory():
    """Changing n rebuilds the spectrum in the static scratch; repeated calls
    leave the device's free memory unchanged."""
    outs = {}
    for n in (16, 8, 16):
        v = volume(n, 5)
        out = torch.empty_like(v)
        binding.green_apply_noalloc(n, 1.0, KB, v, out)
        torch.cuda.synchronize()
        outs.setdefault(n, []).append(out.cpu().numpy())
    assert np.array_equal(outs[16][0], outs[16][1])
    v = volume(16, 6)
    out = torch.empty_like(v)
    binding.green_apply_noalloc(16, 1.0, KB, v, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(DEV)[0]
    for _ in range(3):
        binding.green_apply_noalloc(16, 1.0, KB, v, out, adjoint=True)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(DEV)[0] == free0


def test_noalloc_rebuilds_the_spectrum_for_new_h_and_kb():
    """Same n, new voxel size and wavenumber (the physical units of a 1.333
    medium at four voxels per vacuum wavelength): the second call must rebuild
    the spectrum held in the scratch array.  Checked against the FP64 oracle's
    G v at that (h, kb), since the handle's apply shares the spectrum
    construction with this entry point."""
    from oracle import physics

    n = 16
    v = volume(n, 21)
    first = torch.empty_like(v)
    binding.green_apply_noalloc(n, 1.0, KB, v, first)
    h2, kb2 = 0.25, 2.0 * math.pi * 1.333
    out = torch.empty_like(v)
    for _ in range(2):
        binding.green_apply_noalloc(n, h2, kb2, v, out)
        torch.cuda.synchronize()
        vn = v.cpu().numpy().astype(np.complex128).reshape(n, n, n)
        ref = physics.green_apply(vn, physics.green_hat(n, kb2, h2))
        assert relmax(out.cpu().numpy().reshape(n, n, n), ref) < 2e-6
    assert relmax(first.cpu().numpy(), out.cpu().numpy()) > 1e-2


def test_noalloc_rejects_sizes_beyond_scratch():
    lib = binding.load()
    v = torch.zeros(48 ** 3, dtype=torch.complex64, device=DEV)
    out = torch.empty_like(v)
    for n in (48, 20, 0):
        rc = lib.mqnpm_green_apply_noalloc(n, 1.0, KB, binding._ptr(v), binding._ptr(out), 0, None)
        assert rc == 1, (n, rc)   # MQNPM_ERR_INVALID_ARG
    rc = lib.mqnpm_green_apply_noalloc(16, 1.0, KB, binding._ptr(v), binding._ptr(v), 0, None)
    assert rc == 1
