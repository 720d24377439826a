"""The hand-written adjoint behind torch.autograd.

gcf_log_grad_vjp gives sum_s w_s d ln psi(s)/d theta; LogAbsPsi wraps
gcf_amplitude (forward) and it (backward).  Checked against the FP64 oracle's
dense O(s) and, independently of the oracle, against central finite
differences of the library's own FP64 amplitudes.
"""

import numpy as np
import pytest

from oracle import vmc

from gpu_helpers import configs_for, setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [
    (6, 5, 2, 4, 4, False, False, "fp64"),   # truncated chi
    (8, 8, 2, 4, 16, False, False, "fp32"),  # the 8x8 workload shape
    (4, 3, 2, 4, 4, False, True, "fp64"),    # with matter
    (3, 4, 3, 6, 4, True, False, "fp64"),    # Z3 complex (C ABI only)
]
TOL = {"fp64": 1e-9, "fp32": 1e-4}


def _ids(c):
    return "{}x{}-Z{}-D{}-chi{}{}{}-{}".format(c[0], c[1], c[2], c[3], c[4], "-c" if c[5] else "",
                                             "-m" if c[6] else "", c[7])


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_vjp_matches_oracle(case):
    Lx, Ly, N, D, chi, cplx, matter, prec = case
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=81, complex_=cplx, matter=matter, precision=prec)
    nb = (Lx * Ly) // 2 if matter else 0
    cfgs, _, _ = configs_for(lat, 5, seed=82, n_bosons=nb)
    rng = np.random.default_rng(83)
    w = rng.normal(size=len(cfgs)) + (1j * rng.normal(size=len(cfgs)) if cplx else 0.0)
    got = ctx.log_grad_vjp(torch.from_numpy(cfgs), torch.from_numpy(np.asarray(w))).cpu().numpy()
    ref = sum(w[i] * vmc.log_grad_dense(pe, c, chi) for i, c in enumerate(cfgs))
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(got - ref).max() <= TOL[prec] * 10 * scale


def test_autograd_backward_is_the_vjp_and_matches_finite_differences():
    from paper_2503_20566_gb300.autograd import log_abs_psi

    Lx, Ly, N, D, chi = 5, 4, 2, 4, 4
    lat, pe, ctx = setup(Lx, Ly, N, D, chi, seed=84, precision="fp64")
    cfgs, _, _ = configs_for(lat, 4, seed=85)
    dev = torch.from_numpy(cfgs).cuda()
    theta = torch.tensor(ctx.get_tensors(), dtype=torch.float64, requires_grad=True)
    w = torch.tensor([0.7, -1.3, 0.4, 2.0], dtype=torch.float64)
    loss = (w * log_abs_psi(theta, ctx, dev)).sum()
    loss.backward()
    g = theta.grad.numpy()
    assert g.shape == (ctx.n_params,)
    # oracle
    ref = sum(float(w[i]) * vmc.log_grad_dense(pe, c, chi) for i, c in enumerate(cfgs))
    assert np.abs(g - ref).max() <= 1e-8 * max(1.0, np.abs(ref).max())
    # central differences of the library's FP64 amplitudes on entries the samples use
    base = theta.detach().numpy().copy()
    idx = np.flatnonzero(np.abs(ref) > 1e-3)[:6]
    assert len(idx) > 0
    h = 1e-6
    for j in idx:
        vals = []
        for sgn in (1.0, -1.0):
            p = base.copy()
            p[j] += sgn * h
            ctx.set_tensors(p)
            la, _ = ctx.amplitude(dev)
            vals.append(float((w * la.cpu()).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[j]) <= 1e-5 * max(1.0, abs(g[j])), (j, fd, g[j])
    ctx.set_tensors(base)
