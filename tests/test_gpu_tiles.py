"""Launch-shape variants of the Green's apply and the autotuner that picks one.

Every tile runs the same arithmetic per line and per column (only the number
of lines or columns per CTA, the pass-3 exchange scheme, or the fusion of the
x and y passes into one cluster kernel change), so a plain Green's apply must
be bit-identical across the tiles at every transform length; reductions inside the Krylov solves regroup with the row shape, so
gradients agree to rounding and against the oracle.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import synth  # noqa: E402
from oracle import physics  # noqa: E402
from paper_2307_02043_gb300 import binding  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
KB = math.pi / 2
TILES = range(32)


def cone(L, deg=30.0):
    t = math.radians(deg)
    return np.array([[math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)]
                     for p in 2 * math.pi * np.arange(L) / L])


def c64(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).to(DEV)


@pytest.mark.parametrize("n", [8, 12, 16, 24, 32, 48, 64, 96, 128, 160, 192])
@pytest.mark.parametrize("adjoint", [False, True])
def test_every_tile_gives_the_same_apply(n, adjoint):
    rng = np.random.default_rng(500 + n)
    nb = 2 if n >= 128 else 3
    v = c64(rng.standard_normal((nb, n, n, n)) + 1j * rng.standard_normal((nb, n, n, n))).reshape(-1)
    ref = None
    skipped = []
    for t in TILES:
        try:
            h = binding.MQNPM(n, cone(2), [0, 0], [1.0], max_batch=nb, tile=t)
        except binding.MQNPMError as err:   # the tile's shared memory exceeds the device's
            assert err.code == 1
            skipped.append(t)
            continue
        info = h.tile_info()
        assert info["tile"] == t and info["tuned_ms"] == [None] * 32
        out = h.green_apply(v, adjoint=adjoint).cpu()
        h.close()
        if ref is None:
            ref = out
        else:
            assert torch.equal(out, ref), (n, t)
    # only the two-buffer z pass with the alternative shape can outgrow shared memory (P = 320);
    # the fused x/y passes (bit 4) run on square planes of edge 64 or 128 with bits 0, 1 clear
    fused_ok = n in (64, 128)
    assert all(t & 12 == 12 or (t & 16 and (t & 3 or not fused_ok)) for t in skipped), skipped
    if fused_ok:
        assert not any(t in skipped for t in (16, 20, 24, 28)), skipped
    if n <= 32:
        vh = v.cpu().numpy().reshape(nb, n, n, n)
        kh = physics.green_hat(n, KB)
        got = ref.numpy().reshape(nb, n, n, n)
        for b in range(nb):
            want = physics.green_apply(vh[b], kh, adjoint=adjoint)
            assert np.max(np.abs(got[b] - want)) / np.max(np.abs(want)) < 2e-6


@pytest.mark.parametrize("n", [128, 160])
def test_shapes_reported_per_tile(n):
    """Bits 0, 1, 2 switch the x-, y- and z-pass shapes, bit 3 the z-pass
    exchange scheme.  At n = 128 the alternatives halve the lines or columns
    per CTA; at n = 160 (P = 320 = 20 x 16, four threads per line by default)
    they give every line and column 20 threads."""
    shape = {}
    for t in TILES:
        try:
            h = binding.MQNPM(n, cone(2), [0, 0], [1.0], max_batch=1, tile=t)
        except binding.MQNPMError:
            continue
        info = h.tile_info()
        h.close()
        shape[t] = (info["x"], info["y"], info["z"])
    for t in shape:
        assert shape[t][0] == shape[t & 1][0] and shape[t][1] == shape[t & 2][1]
        assert {k: v for k, v in shape[t][2].items() if k != "exchange_buffers"} == \
               {k: v for k, v in shape[t & 4][2].items() if k != "exchange_buffers"}
        assert shape[t][2]["exchange_buffers"] == (2 if t & 8 else 1)
    assert shape[0][0] != shape[1][0] and shape[0][1] != shape[2][1]
    assert shape[0][2]["columns_per_cta"] != shape[4][2]["columns_per_cta"] or \
        shape[0][2]["threads_per_column"] != shape[4][2]["threads_per_column"]
    if n == 160:
        assert shape[0][0]["threads_per_line"] == 4 and shape[1][0]["threads_per_line"] == 20
        assert shape[2][1]["threads_per_column"] == 20 and shape[4][2]["threads_per_column"] == 20


def test_autotuner_picks_the_fastest_and_caches():
    n, nb = 64, 4
    h1 = binding.MQNPM(n, cone(2), [0, 0], [1.0], max_batch=nb)
    a = h1.tile_info()
    ms = a["tuned_ms"]
    # every unfused tile fits at n = 64; the fused x/y passes run with bits 0 and 1 clear
    timed = [t for t, m in enumerate(ms) if m is not None]
    assert timed == list(range(16)) + [16, 20, 24, 28], timed
    assert all(ms[t] > 0 for t in timed), ms
    assert a["tile"] == min(timed, key=lambda t: ms[t])
    h2 = binding.MQNPM(n, cone(2), [0, 0], [1.0], max_batch=nb)
    assert h2.tile_info() == a          # same (device, n, slots): cached, not re-timed
    h1.close()
    h2.close()


def test_invalid_tile_is_rejected():
    for t in (-2, 16, 32):   # 16: the fused x/y passes need square planes of edge 64 or 128
        with pytest.raises(binding.MQNPMError):
            binding.MQNPM(16, cone(2), [0, 0], [1.0], tile=t)


@pytest.mark.parametrize("model", ["ls", "born"])
def test_gradient_agrees_across_tiles_and_with_oracle(model):
    """Row shapes regroup the per-CTA partial sums of the Krylov inner
    products: the gradients agree to rounding, and with the oracle."""
    n = 16
    w = synth.small("ls32", n=n, L=6, batch=3, model=model)
    kd = synth.illumination_dirs(w)
    xt = synth.phantom(w)
    om = physics.Model(n, kd, model, tol=1e-12)
    ys = physics.simulate(om, xt, synth.noise_draws(w), w.snr_db)
    so = np.zeros(w.L, dtype=np.int32)
    for s_, ii in enumerate(synth.subsets(w)):
        so[ii] = s_
    x = 0.7 * xt
    illum = [0, 1, 2]
    scale = w.S / w.L
    lo, go = om.batch_loss_grad(x, illum, ys, scale)
    xd = torch.from_numpy(np.ascontiguousarray(x).astype(np.float32).reshape(-1)).to(DEV)
    grads = []
    for t in (0, 1, 6, 15):
        h = binding.MQNPM(n, kd, so, [1.0] * w.S, model=model, krylov_tol=1e-6, max_batch=2, tile=t)
        h.set_measurements(c64(ys).reshape(-1))
        g, loss, _ = h.grad_batch(xd, illum, scale)
        h.close()
        g = g.cpu().numpy().astype(np.float64).reshape(go.shape)
        assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go), (model, t)
        assert abs(loss - lo) <= 1e-5 * abs(lo), (model, t)
        grads.append(g)
    for g in grads[1:]:
        assert np.linalg.norm(g - grads[0]) <= 1e-5 * np.linalg.norm(grads[0]), model


@pytest.mark.parametrize("shape", [(64, 64, 64), (48, 64, 64), (128, 128, 128)])
@pytest.mark.parametrize("model", ["ls", "born"])
def test_fused_xy_passes_equal_the_unfused_ones_bit_for_bit(shape, model):
    """Tile bit 4 replaces passes 1+2 and 4+5 by cluster kernels that keep a
    z-plane in shared memory and run the same register DFTs, and form the
    prologue and epilogue partial sums per group of the unfused row pass's
    lines in its order.  Plain applies, Krylov solves (iteration counts,
    losses) and gradients equal the unfused tile 0's bit for bit."""
    nz, ny, nx = shape
    L, nb = 4, 4 if nx == 64 else 2
    kd = cone(L)
    so = [0] * L
    rng = np.random.default_rng(900 + nz)
    x = (0.02 * rng.random(nz * ny * nx)).astype(np.float32)
    xd = torch.from_numpy(x).to(DEV)
    M = ny * nx
    y = c64(rng.standard_normal((L, M)) + 1j * rng.standard_normal((L, M))).reshape(-1)
    v = c64(rng.standard_normal((nb, nz, ny, nx)) + 1j * rng.standard_normal((nb, nz, ny, nx))).reshape(-1)
    out = []
    for t in (0, 16):
        h = binding.MQNPM(shape, kd, so, [1.0], model=model, krylov_tol=1e-6, max_batch=nb, tile=t)
        assert h.tile_info()["fused_xy"] == bool(t & 16)
        h.set_measurements(y)
        a_f = h.green_apply(v, adjoint=False).cpu()
        a_a = h.green_apply(v, adjoint=True).cpu()
        g, loss, its = h.grad_batch(xd, list(range(nb)), 0.5)
        out.append((a_f, a_a, g.cpu(), loss, list(its)))
        h.close()
    (f0, b0, g0, l0, i0), (f1, b1, g1, l1, i1) = out

    def rel(a, b):
        return float((a - b).abs().max() / b.abs().max())
    d = {"apply": rel(f1, f0), "adjoint": rel(b1, b0), "grad": rel(g1, g0), "loss": abs(l1 - l0) / abs(l0)}
    print(shape, model, d, i0, i1)
    assert i0 == i1 and l0 == l1, (d, i0, i1)
    assert torch.equal(f0, f1) and torch.equal(b0, b1) and torch.equal(g0, g1), d
