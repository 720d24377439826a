"""The SR update at full size against the oracle (Eqs. S3 and S7).

Z2 gauge field + hard-core bosons at half filling on 16x16, D = 4, chi = 24
(53,824 parameters), 16 fixed configurations: the library's FP64 form
computes E_loc and O and takes one SR step (gcf_sr_step: FP64 reductions and
CG on (S + lambda) x = F, then alpha <- alpha - lr x).  The oracle computes
E_loc and the dense O(s) of the same configurations and solves the same
system by its own conjugate gradient with S applied as
O^T (w * (O v)) - Obar (Obar . v), never formed (53,824^2 entries).  The
sample mean energy and the update agree to the solver tolerance.
"""

import numpy as np
import pytest

from oracle import vmc

from gpu_helpers import configs_for, oracle_net

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_sr_step_at_full_size_matches_the_oracle():
    import paper_2503_20566_gb300 as G

    L, chi, h, g, J, n, shift, lr = 16, 24, 1.0, 0.33, 0.5, 16, 1e-3, 0.1
    lat, pe, vals = oracle_net(L, L, 2, 4, 5, matter=True, precision="fp64")
    ctx = G.Context(2, L, L, 4, chi, matter=True, h=h, g=g, J=J, precision="fp64", seed=5)
    ctx.set_tensors(vals)
    cfgs, _, _ = configs_for(lat, n, seed=8, n_bosons=L * L // 2)
    dev = torch.from_numpy(cfgs).cuda()
    e = ctx.local_energy(dev)
    bid, O = ctx.log_grad(dev)
    samples = {"e_loc": torch.view_as_real(e).reshape(-1).contiguous(), "block_ids": bid, "O": O}
    p0 = ctx.get_tensors()
    stats = ctx.sr_step(samples, n_chains=n, diag_shift=shift, lr=lr, max_iter=2000, tol=1e-12)
    dp = ctx.get_tensors() - p0

    model = vmc.Model(h=h, g=g, J=J)
    Ed = np.array([vmc.local_energy(pe, model, c, chi) for c in cfgs]).real
    Od = np.array([vmc.log_grad_dense(pe, c, chi) for c in cfgs])
    w = np.full(n, 1.0 / n)
    Obar, Ebar = w @ Od, w @ Ed
    F = Od.T @ (w * Ed) - Obar * Ebar

    def matvec(v):
        return Od.T @ (w * (Od @ v)) - Obar * (Obar @ v) + shift * v

    x, it = vmc.cg_solve(matvec, F, tol=1e-13, maxiter=5000)
    ref = -lr * x
    rel = np.linalg.norm(dp - ref) / np.linalg.norm(ref)
    print(f"16x16 SR step, {ctx.n_params} parameters, {n} samples: <E> {stats[0]:.10f} (oracle {Ebar:.10f}), "
          f"CG {int(stats[3])} iterations (oracle {it}), update relative deviation {rel:.1e}")
    assert ctx.n_params == Od.shape[1]
    assert abs(stats[0] - Ebar) < 1e-10 * max(1.0, abs(Ebar))
    assert rel <= 1e-7, rel
