"""CPU-side checks of the C ABI: the library builds, loads, and exports every
entry point declared in include/mqnpm.h with the signatures the binding uses.
No compute call is made (no GPU here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "mqnpm.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mqnpm_\w+)\s*\(", text)))


def test_header_lists_the_boundary():
    names = declared_functions()
    for required in ("mqnpm_create", "mqnpm_grad_batch", "mqnpm_wprox", "mqnpm_step", "mqnpm_destroy",
                     "mqnpm_set_measurements", "mqnpm_save_state", "mqnpm_load_state"):
        assert required in names


def test_library_loads_and_exports_every_symbol():
    from paper_2307_02043_gb300 import binding

    lib = binding.load(build_if_missing=True)
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in binding.SIGNATURES, "binding lacks a signature for " + name


def test_config_struct_layout_matches_header():
    """The ctypes mirror of mqnpm_config has the header's field order."""
    from paper_2307_02043_gb300 import binding

    with open(os.path.join(ROOT, "include", "mqnpm.h")) as f:
        text = f.read()
    body = text[text.index("typedef struct mqnpm_config"):text.index("} mqnpm_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(?:long long|int|double|size_t|void\*|const \w+\*)\s+([\w, ]+);", body)
    names = [f.strip() for group in fields for f in group.split(",")]
    mirror = [f for f, _ in binding.Config._fields_]
    mirror = ["lambda" if f == "lam" else f for f in mirror]
    assert names == mirror


def test_no_cpu_fallback_when_library_missing(tmp_path, monkeypatch):
    from paper_2307_02043_gb300 import binding, build

    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(binding, "_LIB", None)
    with pytest.raises(ImportError):
        binding.load(build_if_missing=False)


def _config(**kw):
    """A valid ls32-like configuration as the ctypes struct (arrays kept alive
    in the returned tuple)."""
    import ctypes

    import numpy as np

    from paper_2307_02043_gb300 import binding

    L = kw.pop("L", 4)
    S = kw.pop("S", 2)
    kd = np.ascontiguousarray(np.tile([0.0, 0.0, 1.0], (L, 1)), dtype=np.float64)
    so = np.ascontiguousarray(np.arange(L) % max(S, 1), dtype=np.int32)
    al = np.ascontiguousarray(np.ones(S), dtype=np.float64)
    cfg = binding.Config()
    cfg.nx = cfg.ny = cfg.nz = 16
    cfg.h, cfg.kb, cfg.model, cfg.L = 1.0, 1.5707963, 1, L
    cfg.kdir = kd.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cfg.S = S
    cfg.subset_of = so.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    cfg.alpha = al.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cfg.step, cfg.strategy, cfg.tv, cfg.lam = 1.0, 1, 0, 1e-3
    cfg.box_lo, cfg.box_hi, cfg.gamma = 0.0, 0.05, 0.8
    cfg.krylov_tol, cfg.krylov_maxit, cfg.dual_iters = 1e-6, 100, 20
    cfg.newton_tol, cfg.newton_maxit, cfg.max_batch = 1e-6, 50, 2
    cfg.tile = 0
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg, (kd, so, al)


@pytest.mark.parametrize("field,value", [
    ("nx", 3), ("nz", 2), ("L", 0), ("S", 0), ("S", 17), ("max_batch", 0), ("max_batch", 65), ("gamma", 0.0),
    ("gamma", 1.5), ("h", 0.0), ("kb", -1.0), ("lam", -1.0), ("box_lo", 1.0), ("step", 0.0),
    ("krylov_tol", 0.0), ("krylov_maxit", 0), ("dual_iters", -1), ("model", 7), ("tv", 5),
    ("strategy", 3), ("tile", -2), ("tile", 32), ("det_na", -0.5), ("det_na", float("inf")),
    ("det_distance", float("nan")), ("barrier_wait_cycles", -1), ("green_kernel", 2), ("green_kernel", -1), ("adjoint_start", 2), ("adjoint_start", -1),
    ("forward_start", 2), ("forward_start", -1)])
def test_create_rejects_invalid_configurations(field, value):
    """Host-side validation of mqnpm_create runs before any CUDA call: every
    out-of-range option returns MQNPM_ERR_INVALID_ARG and no handle."""
    import ctypes

    from paper_2307_02043_gb300 import binding

    lib = binding.load(build_if_missing=True)
    kw = {"S": 2} if field != "S" else {}
    if field in ("L", "S"):
        kw = {field: value}
        if field == "S" and value > 4:
            kw["L"] = value
    cfg, keep = _config(**kw)
    if field not in ("L", "S"):
        setattr(cfg, field, value)
    out = ctypes.c_void_p()
    rc = lib.mqnpm_create(ctypes.byref(cfg), ctypes.byref(out))
    assert rc == 1, (field, value, rc)
    assert not out.value
    del keep


def test_create_rejects_a_nonfinite_spectrum_and_unsupported_grids():
    import ctypes

    import numpy as np

    from paper_2307_02043_gb300 import binding

    lib = binding.load(build_if_missing=True)
    gh = np.zeros(17 ** 3, dtype=np.complex64)
    gh[5] = np.nan
    cfg, keep = _config()
    cfg.green_hat = gh.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    out = ctypes.c_void_p()
    assert lib.mqnpm_create(ctypes.byref(cfg), ctypes.byref(out)) == 1
    cfg2, keep2 = _config(ny=20)                # P = 40: no compiled transform plan
    assert lib.mqnpm_create(ctypes.byref(cfg2), ctypes.byref(out)) == 7   # MQNPM_ERR_UNSUPPORTED
    assert not out.value
    del keep, keep2
