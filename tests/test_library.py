"""CPU-side checks of the C ABI: the library builds, loads, and exports every
symbol declared in include/gcfvmc.h (no compute calls: no GPU here)."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gcfvmc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gcf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2503_20566_gb300 import build

    if not os.path.exists(build.LIB):
        try:
            build.build()
        except RuntimeError as e:  # no nvcc in this environment
            pytest.skip(str(e))
    return build.LIB


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["gcf_init_peps", "gcf_sample_batch", "gcf_amplitude", "gcf_local_energy", "gcf_log_grad",
              "gcf_sr_step", "gcf_destroy", "gcf_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gcf_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches(lib_path):
    import ctypes

    import paper_2503_20566_gb300 as G

    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n)
    assert set(G.exported_symbols()) <= set(declared_functions())
    G.load_library(lib_path)


def test_binding_refuses_missing_library(tmp_path):
    from paper_2503_20566_gb300 import binding

    with pytest.raises(RuntimeError):
        binding._lib = None
        binding.load_library(str(tmp_path / "nope.so"))
    binding._lib = None
