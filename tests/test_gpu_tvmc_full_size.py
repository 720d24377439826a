"""A tVMC stage at the full size of the real-time workload against the oracle
(Eqs. S6-S8).

Pure Z2 gauge theory on 10x10, D = 6 (D_k = 3), chi = 36, complex tensors
(45,000 parameters), g = 0.2, 8 fixed configurations: the library's FP64
complex form computes E_loc and O and takes the first stage of the two-stage
scheme (gcf_sr_step with TDVP_STAGE1: alpha <- alpha + c_1 dt alpha_dot,
alpha_dot = -i (S + lambda)^{-1} F).  The oracle computes E_loc and the dense
O(s) of the same configurations and solves the same system by its own
conjugate gradient, with S applied as O^H (w * (O v)) - Obar^* (Obar . v),
never formed.  The parameter change agrees to the solver tolerance.
"""

import numpy as np
import pytest

from oracle import vmc

from gpu_helpers import configs_for, oracle_net

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_tdvp_stage_at_full_size_matches_the_oracle():
    import paper_2503_20566_gb300 as G

    L, N, D, chi, h, g, n, shift, dt = 10, 2, 6, 36, 1.0, 0.2, 8, 1e-4, 0.01
    lat, pe, vals = oracle_net(L, L, N, D, 5, complex_=True, precision="fp64")
    ctx = G.Context(N, L, L, D, chi, h=h, g=g, complex_=True, precision="fp64", seed=5)
    ctx.set_tensors(vals)
    cfgs, _, _ = configs_for(lat, n, seed=9)
    dev = torch.from_numpy(cfgs).cuda()
    e = ctx.local_energy(dev)
    bid, O = ctx.log_grad(dev)
    samples = {"e_loc": torch.view_as_real(e).reshape(-1).contiguous(), "block_ids": bid, "O": O}
    p0 = ctx.get_tensors()
    stats = ctx.sr_step(samples, n_chains=n, diag_shift=shift, mode=G.TDVP_STAGE1, dt=dt, max_iter=2000, tol=1e-12)
    dp = ctx.get_tensors() - p0

    model = vmc.Model(h=h, g=g)
    Ed = np.array([vmc.local_energy(pe, model, c, chi) for c in cfgs])
    Od = np.array([vmc.log_grad_dense(pe, c, chi) for c in cfgs])
    w = np.full(n, 1.0 / n)
    Obar, Ebar = w @ Od, w @ Ed
    F = Od.conj().T @ (w * Ed) - Obar.conj() * Ebar

    def matvec(v):
        return Od.conj().T @ (w * (Od @ v)) - Obar.conj() * (Obar @ v) + shift * v

    x, it = vmc.cg_solve(matvec, F, tol=1e-13, maxiter=5000)
    ref = vmc.TDVP_C1 * dt * (-1j * x)
    rel = np.linalg.norm(dp - ref) / np.linalg.norm(ref)
    print(f"10x10 tVMC stage, {ctx.n_params} complex parameters, {n} samples: <E> {stats[0]:.10f} "
          f"(oracle {Ebar.real:.10f}), CG {int(stats[3])} iterations (oracle {it}), "
          f"update relative deviation {rel:.1e}")
    assert ctx.n_params == Od.shape[1]
    assert abs(stats[0] - Ebar.real) < 1e-10 * max(1.0, abs(Ebar))
    assert rel <= 1e-7, rel
