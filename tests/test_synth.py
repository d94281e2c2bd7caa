"""CPU: the seeded input generators (geometry and random draws only) give the
same bytes on every call, respect the stated recipe (margin, contrast range,
cone, interleaved subsets, SNR scaling inputs), and cover every named workload."""
import math

import numpy as np
import pytest

import synth


@pytest.mark.parametrize("name", ["ls32", "born128", "ls128", "ls192", "sim64", "yeast96"])
def test_workload_recipe(name):
    w = synth.workload(name)
    assert w.S == math.ceil(w.L / w.batch)
    subs = synth.subsets(w)
    assert sorted(int(i) for s in subs for i in s) == list(range(w.L))       # a partition
    assert all(len(s) <= w.batch for s in subs)
    for s, idx in enumerate(subs):
        assert all(int(i) % w.S == s for i in idx)                           # interleaved
    kd = synth.illumination_dirs(w)
    assert kd.shape == (w.L, 3)
    assert np.allclose(np.linalg.norm(kd, axis=1), 1.0)
    assert np.allclose(kd[:, 2], math.cos(math.radians(w.cone_deg)))          # on the cone boundary
    assert w.kb * w.h > 0


@pytest.mark.parametrize("name,n", [("ls32", 32), ("ls128", 48), ("sim64", 32), ("born128", 40)])
def test_phantom_is_seeded_and_inside_the_recipe(name, n):
    w = synth.small(name, n=n)
    a, b = synth.phantom(w), synth.phantom(w)
    assert np.array_equal(a, b)
    assert a.shape == (n, n, n)
    assert a.min() >= 0.0
    assert a.max() <= w.contrast_max + (w.background[0] if w.background[0] > 0 else 0.0) + 1e-12
    m = w.margin
    if w.background[0] == 0.0:                                               # objects keep the margin
        assert not a[:m].any() and not a[-m:].any()
        assert not a[:, :m].any() and not a[:, -m:].any()
        assert not a[:, :, :m].any() and not a[:, :, -m:].any()


def test_random_draws_are_seeded_per_workload():
    w1, w2 = synth.small("ls32", n=16, L=4, batch=2), synth.small("ls32", n=16, L=4, batch=2)
    assert np.array_equal(synth.noise_draws(w1), synth.noise_draws(w2))
    assert np.array_equal(synth.power_start(w1), synth.power_start(w2))
    d = synth.strategy2_draws(w1, 20)
    assert d.min() >= 0 and d.max() < w1.S and np.array_equal(d, synth.strategy2_draws(w2, 20))
    w3 = synth.small("ls128", n=16, L=4, batch=2)
    assert not np.array_equal(synth.noise_draws(w1), synth.noise_draws(w3))   # config-specific seeds


def test_uneven_mix_matches_its_recipe():
    reqs = synth.uneven_requests()
    assert len(reqs) == 16
    assert {w.n for w in reqs} <= {64, 96, 128, 160}
    assert all(w.L in (24, 48, 60) and 4 <= w.batch <= 8 for w in reqs)
