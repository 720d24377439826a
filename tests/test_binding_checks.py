"""The binding checks every buffer it hands to the C ABI as a raw pointer
(the library cannot see sizes or placement): wrong shapes, dtypes, layouts,
host tensors where device memory is read, and too-small outputs are refused
with ValueError before any library call.  A Context without a library stands
in, so nothing here needs a GPU: a check that did not fire would reach the
missing library and fail differently."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2503_20566_gb300 import binding as B  # noqa: E402


def fake_ctx():
    ctx = B.Context.__new__(B.Context)
    ctx._torch = torch
    ctx.lib, ctx.ctx = None, None
    ctx.N, ctx.Lx, ctx.Ly, ctx.D, ctx.chi, ctx.Dk = 2, 4, 3, 4, 4, 2
    ctx.n_s, ctx.n_plaq, ctx.cfg_len = 12, 6, 29
    ctx.o_dtype, ctx.complex = torch.float32, False
    ctx.device = 0
    ctx._dev = torch.device("cuda", 0)
    return ctx


class _OtherGpuTensor:
    """Stands in for a CUDA tensor on another GPU (cuda:1): right dtype, size
    and layout, wrong device."""

    def __init__(self, dtype, n):
        self.dtype, self._n = dtype, n
        self.is_cuda = True
        self.device = torch.device("cuda", 1)

    def data_ptr(self):
        return 0

    def numel(self):
        return self._n

    def is_contiguous(self):
        return True


def test_buffers_on_another_gpu_are_refused():
    """A buffer on another GPU than the context's would be dereferenced by a
    kernel on the context's GPU: refused before any pointer is passed."""
    buf = _OtherGpuTensor(torch.float64, 100)
    with pytest.raises(ValueError, match="cuda:1, the context lives on cuda:0"):
        B._check_device_buffers([(buf, torch.float64, 10, "out['log_abs']")], 0)
    B._check_device_buffers([(buf, torch.float64, 10, "out['log_abs']")], 1)  # same device: accepted
    with pytest.raises(ValueError, match="cuda:1"):
        B._check_samples({"e_loc": buf}, 4, 2, 12, 16, torch.float32, "sample_batch", 0)


def test_sample_batch_refuses_bad_configs():
    ctx = fake_ctx()
    with pytest.raises(ValueError, match=r"\(n_chains, 29\)"):
        ctx.sample_batch(torch.zeros((4, 28), dtype=torch.int8), 1, seed=0)
    with pytest.raises(ValueError, match="int8"):
        ctx.sample_batch(torch.zeros((4, 29), dtype=torch.int64), 1, seed=0)
    with pytest.raises(ValueError, match="contiguous"):
        ctx.sample_batch(torch.zeros((29, 4), dtype=torch.int8).t(), 1, seed=0)
    with pytest.raises(ValueError, match="GPU"):  # a host pointer never reaches the kernel
        ctx.sample_batch(torch.zeros((4, 29), dtype=torch.int8), 1, seed=0, out={})


def test_outputs_must_hold_what_the_call_writes():
    ctx = fake_ctx()
    out = {"log_abs": torch.zeros(8, dtype=torch.float64), "O": torch.zeros(8 * 12 * 16 - 1)}
    with pytest.raises(ValueError, match="out\\['O'\\] holds"):
        B._check_samples(out, 4, 2, ctx.n_s, 16, torch.float32, "sample_batch")
    out = {"block_ids": torch.zeros(8 * 12, dtype=torch.int64)}
    with pytest.raises(ValueError, match="int32"):
        B._check_samples(out, 4, 2, ctx.n_s, 16, torch.float32, "sample_batch")
    out = {"accepted": torch.zeros(3, dtype=torch.int32)}
    with pytest.raises(ValueError, match="holds 3"):
        B._check_samples(out, 4, 2, ctx.n_s, 16, torch.float32, "sample_batch")


def test_sr_step_refuses_mismatched_samples():
    ctx = fake_ctx()
    ns = 6
    good = {"e_loc": torch.zeros(2 * ns, dtype=torch.float64), "block_ids": torch.zeros((ns, 12), dtype=torch.int32),
            "O": torch.zeros((ns, 12, 16), dtype=torch.float32)}
    for key, bad in [("block_ids", torch.zeros((ns, 11), dtype=torch.int32)),
                     ("O", torch.zeros((ns, 12, 16), dtype=torch.float64)),
                     ("e_loc", torch.zeros(2 * ns, dtype=torch.float32))]:
        with pytest.raises(ValueError, match=key):
            ctx.sr_step(dict(good, **{key: bad}), n_chains=ns)
    with pytest.raises(ValueError, match="GPU"):
        ctx.sr_step(good, n_chains=ns)


def test_host_and_fixed_configuration_calls_refuse_bad_shapes():
    ctx = fake_ctx()
    with pytest.raises(ValueError, match=r"\(n_chains, 29\)"):
        ctx.vmc_step_host(np.zeros((4, 30), dtype=np.int8), 1, seed=0)
    ro = np.zeros((4, 29), dtype=np.int8)
    ro.flags.writeable = False
    with pytest.raises(ValueError, match="writeable"):
        ctx.vmc_step_host(ro, 1, seed=0)
    with pytest.raises(ValueError, match=r"\(n, 29\)"):
        ctx.amplitude(np.zeros((3, 27), dtype=np.int8))
    with pytest.raises(ValueError, match="powers"):
        ctx.init_configs(4, powers=torch.zeros((4, 5), dtype=torch.int8))
    with pytest.raises(ValueError, match="occupations"):
        ctx.init_configs(4, occupations=torch.zeros((4, 11), dtype=torch.int8))


def test_background_charges_must_cover_the_lattice():
    with pytest.raises(ValueError, match="12 background charges"):
        B.Context(2, 4, 3, 4, 4, Q=[1, 0, 0, 1])
