"""Host logic of bench.py that needs no GPU.

* The source hash that keys the committed ncu capture covers exactly the files
  the FP32 sampling kernel is compiled from: its translation unit and the
  closure of its quoted includes.
* The DRAM traffic from the capture is reported only for the captured kernel
  form (kernel and shared-memory level), scaled by the samples per launch.
"""

import os
import re

import pytest

import bench

CSRC = os.path.join(os.path.dirname(bench.__file__), "paper_2503_20566_gb300", "csrc")


def _include_closure(name, seen=None):
    seen = set() if seen is None else seen
    if name in seen:
        return seen
    seen.add(name)
    with open(os.path.join(CSRC, name)) as f:
        for inc in re.findall(r'^\s*#include\s+"([^"]+)"', f.read(), flags=re.M):
            _include_closure(inc, seen)
    return seen


def test_kernel_sources_are_the_include_closure_of_the_fp32_kernel():
    assert _include_closure("vmc_f32.cu") == set(bench.KERNEL_SOURCES)
    assert len(bench.source_hash()) == 16


def test_traffic_only_for_the_captured_form():
    txt = open(bench.PROFILE).read()
    kernel, level = re.search(r"kernel_form: (\S+) level (\d+)", txt).groups()
    per_sample = float(re.search(r"traffic_bytes_per_sample: ([0-9.eE+]+)", txt).group(1))
    if re.search(r"source_sha256: ([0-9a-f]+)", txt).group(1) != bench.source_hash():
        pytest.skip("kernel sources changed since the capture (traffic is then null by design)")
    assert bench.profiled_traffic(1000, kernel, int(level)) == pytest.approx(1000 * per_sample)
    assert bench.profiled_traffic(1000, kernel, int(level) + 1) is None
    assert bench.profiled_traffic(1000, "gcf::vmc_kernel<float>", int(level)) is None


def test_err_vs_fp64_compares_the_two_forms(monkeypatch):
    torch = pytest.importorskip("torch")
    import numpy as np

    import paper_2503_20566_gb300 as G

    class Form:
        """Stands in for a Context: constant amplitudes / energies per form."""

        def __init__(self, *args, precision="fp32", **kwargs):
            self.precision, self.closed, self.params = precision, False, None

        def get_tensors(self):
            return np.ones(3)

        def set_tensors(self, values):
            self.params = values

        def amplitude(self, configs):
            n = configs.shape[0]
            la = torch.full((n,), 2.0, dtype=torch.float64) + (1e-5 if self.precision == "fp32" else 0.0)
            return la, torch.zeros(n, dtype=torch.float64)

        def local_energy(self, configs):
            e = torch.full((configs.shape[0],), 10.0 + 0j, dtype=torch.complex128)
            return e + (1e-3 if self.precision == "fp32" else 0.0)

        def close(self):
            self.closed = True

    monkeypatch.setattr(G, "Context", Form)
    out = bench.err_vs_fp64(Form(), torch.zeros((100, 5), dtype=torch.int8), bench.WORKLOAD, n_check=64)
    assert out["configs"] == 64
    assert out["amp_max"] == pytest.approx(1e-5, rel=1e-3) and out["amp_median"] == pytest.approx(1e-5, rel=1e-3)
    assert out["eloc_max"] == pytest.approx(1e-4, rel=1e-3)
