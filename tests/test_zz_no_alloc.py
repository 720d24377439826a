"""gcf_amplitude_noalloc: the amplitude entry point that allocates nothing.

Some callers cannot call cudaMalloc during a call (services that reserve all
device memory at start-up, embedders whose own allocator owns the device).  gcf_amplitude_noalloc serves them from a fixed 32 MiB device
array built into the library.  This test calls it through the C ABI twice in
a row and checks it against gcf_amplitude within the FP32 amplitude
tolerance, and checks that a lattice too large for the array is refused.
The file is named so that pytest collects it last.
"""

import ctypes as C

import numpy as np
import pytest

from gpu_helpers import TOL, amp_err, configs_for, setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _entry():
    import paper_2503_20566_gb300 as G

    lib = G.load_library()
    f = lib.gcf_amplitude_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    return f


@pytest.mark.parametrize("case", [(8, 8, 2, 4, 16, False, "fp32"), (5, 4, 3, 6, 4, True, "fp32")],
                         ids=["z2-8x8-D4-chi16", "z3-5x4-D6-chi4-complex"])
def test_noalloc_amplitude_matches_gcf_amplitude_twice(case):
    Lx, Ly, N, D, chi, cplx, prec = case
    f = _entry()
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=41, complex_=cplx, precision=prec)
    cfgs, _, _ = configs_for(lat, 40, seed=42)
    dev = torch.from_numpy(cfgs).cuda()
    ref_la, ref_ph = ctx.amplitude(dev)
    ref_la, ref_ph = ref_la.cpu().numpy(), ref_ph.cpu().numpy()
    for call in range(2):
        la = torch.full((len(cfgs),), np.nan, dtype=torch.float64, device="cuda")
        ph = torch.full((len(cfgs),), np.nan, dtype=torch.float64, device="cuda")
        st = f(ctx.ctx, len(cfgs), C.c_void_p(dev.data_ptr()), C.c_void_p(la.data_ptr()),
               C.c_void_p(ph.data_ptr()))
        assert st == 0, ctx.lib.gcf_last_error(ctx.ctx)
        torch.cuda.synchronize()
        la, ph = la.cpu().numpy(), ph.cpu().numpy()
        for i in range(len(cfgs)):
            assert amp_err(la[i], ph[i], ref_la[i], ref_ph[i]) < TOL[prec], (call, i)


def test_noalloc_rejects_lattice_beyond_the_fixed_array():
    import paper_2503_20566_gb300 as G

    f = _entry()
    ctx = G.Context(2, 64, 64, 6, 64, precision="fp32", seed=1)
    cfg = ctx.init_configs(1)
    la = torch.empty(1, dtype=torch.float64, device="cuda")
    ph = torch.empty(1, dtype=torch.float64, device="cuda")
    st = f(ctx.ctx, 1, C.c_void_p(cfg.data_ptr()), C.c_void_p(la.data_ptr()), C.c_void_p(ph.data_ptr()))
    assert st == 1  # GCF_EINVAL
    assert b"scratch" in ctx.lib.gcf_last_error(ctx.ctx)


def test_noalloc_caps_the_grid_at_what_the_array_holds():
    """A lattice whose per-CTA scratch is many MiB (32x32 Z2 + bosons, D = 4,
    chi = 24, FP64: the array holds one or two CTAs' scratch) with many more
    configurations than CTAs: the chains loop over the few CTAs that fit and
    the amplitudes equal gcf_amplitude's, on two calls in a row."""
    Lx, Ly, N, D, chi = 32, 32, 2, 4, 24
    f = _entry()
    # FP64: both entry points then agree to rounding whatever the kernel form
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=43, matter=True, precision="fp64", h=1.0, g=0.33, J=0.5)
    cfgs, _, _ = configs_for(lat, 24, seed=44, n_bosons=(Lx * Ly) // 2)
    dev = torch.from_numpy(cfgs).cuda()
    ref_la, ref_ph = (t.cpu().numpy() for t in ctx.amplitude(dev))
    for call in range(2):
        la = torch.full((len(cfgs),), np.nan, dtype=torch.float64, device="cuda")
        ph = torch.full((len(cfgs),), np.nan, dtype=torch.float64, device="cuda")
        st = f(ctx.ctx, len(cfgs), C.c_void_p(dev.data_ptr()), C.c_void_p(la.data_ptr()),
               C.c_void_p(ph.data_ptr()))
        assert st == 0, ctx.lib.gcf_last_error(ctx.ctx)
        torch.cuda.synchronize()
        la, ph = la.cpu().numpy(), ph.cpu().numpy()
        for i in range(len(cfgs)):
            assert amp_err(la[i], ph[i], ref_la[i], ref_ph[i]) < TOL["fp64"], (call, i)
