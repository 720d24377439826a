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


def test_traffic_only_for_the_captured_form(tmp_path):
    """A capture counts for its own workload, kernel form and sources only."""
    kernel, level, wl = "gcf::vmc_kernel_multi<float>", 0, "some_workload"
    (tmp_path / "k.md").write_text(f"workload: {wl}\nsource_sha256: {bench.source_hash()}\n"
                                   f"kernel_form: {kernel} level {level}\ntraffic_bytes_per_sample: 2.5e4\n")
    assert bench.profiled_traffic(1000, kernel, level, wl, str(tmp_path)) == pytest.approx(2.5e7)
    assert bench.profiled_traffic(1000, kernel, level + 1, wl, str(tmp_path)) is None
    assert bench.profiled_traffic(1000, "gcf::vmc_kernel<float>", level, wl, str(tmp_path)) is None
    assert bench.profiled_traffic(1000, kernel, level, "other_workload", str(tmp_path)) is None
    (tmp_path / "k.md").write_text(f"workload: {wl}\nsource_sha256: 0000000000000000\n"
                                   f"kernel_form: {kernel} level {level}\ntraffic_bytes_per_sample: 2.5e4\n")
    assert bench.profiled_traffic(1000, kernel, level, wl, str(tmp_path)) is None


def test_traffic_fields_in_markdown_code_spans(tmp_path):
    """The profiles write their fields as Markdown code spans: the closing
    backtick is not part of the workload name."""
    kernel, level, wl = "gcf::vmc_kernel_multi4<float>", 0, "z2_a+b_D4"
    (tmp_path / "k.md").write_text(f"`workload: {wl}`\n`source_sha256: {bench.source_hash()}`\n"
                                   f"`kernel_form: {kernel} level {level}`\n`traffic_bytes_per_sample: 1.5e8`\n")
    assert bench.profiled_traffic(10, kernel, level, wl, str(tmp_path)) == pytest.approx(1.5e9)


def test_committed_profiles_name_bench_workloads():
    """Every committed profile with a workload line names a bench workload
    and carries the other three fields."""
    pdir = os.path.join(os.path.dirname(CSRC), "..", "profiles")
    names = {w["workload"] for w in bench.WORKLOADS.values()}
    seen = 0
    for name in sorted(os.listdir(pdir)):
        txt = open(os.path.join(pdir, name)).read()
        m = re.search(r"workload: ([^\s`]+)", txt)
        if not m:
            continue
        seen += 1
        assert m.group(1) in names, (name, m.group(1))
        for field in (r"source_sha256: [0-9a-f]{16}", r"kernel_form: \S+ level \d+",
                      r"traffic_bytes_per_sample: [0-9.eE+]+"):
            assert re.search(field, txt), (name, field)
    assert seen >= 1


def test_workloads_follow_the_stated_configurations():
    """The default workload is the mixed-size Z2 + bosons one: 16384 chains
    over 16x16 / 24x24 / 32x32, D = 4, chi = 24, half filling."""
    w = bench.WORKLOADS[bench.DEFAULT_CONFIG]
    assert sum(l["chains"] for l in w["lattices"]) == 16384
    assert [l["Lx"] for l in w["lattices"]] == [16, 24, 32]
    assert all(l["D"] == 4 and l["chi"] == 24 and l["matter"] and l["N"] == 2 for l in w["lattices"])
    assert bench.flops_per_sample(32, 32, 2, 24) == pytest.approx(1.1e9, rel=0.05)


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
    lat = bench.WORKLOADS["z2_8x8"]["lattices"][0]
    out = bench.err_vs_fp64([Form()], [torch.zeros((100, 5), dtype=torch.int8)], [lat], n_check=64)
    assert out["configs"] == 64
    assert out["amp_max"] == pytest.approx(1e-5, rel=1e-3) and out["amp_median"] == pytest.approx(1e-5, rel=1e-3)
    assert out["eloc_max"] == pytest.approx(1e-4, rel=1e-3)
