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
    fields = re.findall(r"(?:int|double|size_t|void\*|const \w+\*)\s+([\w, ]+);", body)
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
