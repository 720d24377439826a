"""gcf_autotune: every fitting kernel form is timed, the fastest is kept, the
caller's configurations are left unchanged, and results stay those of the
oracle."""

import numpy as np
import pytest

from oracle import vmc

from gpu_helpers import TOL, amp_err, configs_for, setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("case", [(8, 8, 2, 4, 16, False), (4, 3, 3, 6, 4, True)], ids=["z2-8x8", "z3-4x3-c"])
def test_autotune_keeps_fastest_form_and_parity(case):
    Lx, Ly, N, D, chi, cplx = case
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=101, complex_=cplx, precision="fp32")
    cfgs, _, _ = configs_for(lat, 64, seed=102)
    dev = torch.from_numpy(cfgs).cuda()
    ms = ctx.autotune(dev, n_sweeps=1)
    assert len(ms) >= 2
    assert any(t < 1e299 for t in ms)
    assert torch.equal(dev.cpu(), torch.from_numpy(cfgs))
    assert ctx.kernel_name in ("gcf::vmc_kernel", "gcf::vmc_kernel_grouped")
    assert 0 <= ctx.smem_level <= 3
    la, ph = ctx.amplitude(dev[:4])
    la, ph = la.cpu().numpy(), ph.cpu().numpy()
    for i in range(4):
        ola, oph = vmc.amplitude(pe, cfgs[i], chi)
        assert amp_err(la[i], ph[i], ola, oph) < TOL["fp32"]
