"""A tVMC trajectory run through the library against exact dynamics (Eqs. S6-S8).

The vison initial state (sigma_z on the bottom-left vertical link, applied to
a random complex GCF PEPS by the product's exact block-store transform) on the
3x3 Z2 lattice (16 physical configurations) is evolved with the two-stage
scheme: each stage samples the chains with gcf_sample_batch and updates the
tensors with gcf_sr_step (TDVP_STAGE1 / TDVP_STAGE2), driven by
drivers.tvmc_evolve.  After every step the library's tensors are read back and
the state they define is contracted exactly by the oracle on the full basis,
so what is compared is the trajectory itself, not a further estimate:

* <P + P^dag> on every plaquette tracks exp(-iHt) psi(0) (oracle/dynamics.py)
  within the sampling error of the stages;
* the final state is closer to exp(-iHt) psi(0) than to exp(+iHt) psi(0);
* the energy drift |<H>(T) - <H>(0)| / |<H>(0)| is printed beside the paper's
  bound for its long runs (below 0.2 % over 7200 steps).
"""

import numpy as np
import pytest

import synth
from oracle import dynamics as dyn
from oracle import peps as P
from oracle.lattice import Lattice

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _psi(lat, Dk, params, basis):
    pe = P.GIPEPS(lat, Dk, params)
    v = np.array([P.contract_exact(pe.sampled_network(b)) for b in basis])
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tvmc_trajectory_follows_exact_dynamics(precision):
    import paper_2503_20566_gb300 as G
    from paper_2503_20566_gb300 import drivers, states

    lat, Dk, h, g, chi = Lattice(3, 3, 2), 2, 1.0, 0.1, 4
    _, n = P.layout(lat, Dk)
    params0 = states.vison(synth.tensor_entries(71, n, True), 2, 3, 3, Dk)
    ctx = G.Context(2, 3, 3, 2 * Dk, chi, h=h, g=g, complex_=True, precision=precision, seed=71)
    ctx.set_tensors(params0)
    basis = lat.physical_basis()
    psi0 = _psi(lat, Dk, ctx.get_tensors(), basis)
    H = lat.hamiltonian_matrix(basis, h, g)
    plaqs = [dyn.plaquette_matrix(lat, basis, x, y) for y in range(2) for x in range(2)]
    n_chains, n_sweeps, dt, n_steps = 4096, 4, 0.02, 10
    powers = synth.plaquette_powers(72, n_chains, lat.n_plaquettes, 2)
    configs = ctx.init_configs(n_chains, powers=torch.from_numpy(powers))
    track = []

    def on_step(rec):
        psi = _psi(lat, Dk, ctx.get_tensors(), basis)
        track.append(([dyn.expectation(psi, M).real for M in plaqs], dyn.expectation(psi, H).real))

    drivers.tvmc_evolve(ctx, configs, n_steps=n_steps, dt=dt, n_sweeps=n_sweeps, seed=73, diag_shift=1e-4,
                        max_iter=200, tol=1e-10, on_step=on_step)
    times = dt * np.arange(1, n_steps + 1)
    exact = dyn.evolve(H, psi0, times)
    worst = 0.0
    for (pl, _), ps in zip(track, exact):
        ref = [dyn.expectation(ps, M).real for M in plaqs]
        worst = max(worst, max(abs(a - b) for a, b in zip(pl, ref)))
    psi_T = _psi(lat, Dk, ctx.get_tensors(), basis)
    f_fwd = abs(np.vdot(exact[-1], psi_T))
    f_bwd = abs(np.vdot(dyn.evolve(-H, psi0, [times[-1]])[0], psi_T))
    e0 = dyn.expectation(psi0, H).real
    drift = abs(track[-1][1] - e0) / abs(e0)
    p_change = max(abs(a - b) for a, b in zip(track[-1][0], [dyn.expectation(psi0, M).real for M in plaqs]))
    print(f"{precision}: T = {times[-1]:.2f}, plaquette error max {worst:.2e} (exact change {p_change:.2e}), "
          f"fidelity forward {f_fwd:.6f} backward {f_bwd:.6f}, energy drift {100 * drift:.3f} % "
          f"(paper: < 0.2 % over 7200 steps)")
    assert f_fwd > 0.999 and f_fwd > f_bwd + 0.05, (f_fwd, f_bwd)
    assert worst < 0.1 * p_change + 5e-3, (worst, p_change)
    assert drift < 5e-3, drift
