"""The tVMC driver against exact dynamics (NEXT-1 pipeline, CPU).

A stand-in context implements gcf_sr_step as the header documents it, with
exact expectations over the complete basis from the oracle (S, F of Eq. S7;
x = (S + lambda)^-1 F; stage k: A <- A + c_k dt (-i x), c_{1,2} = (1 +- i)/2).
The product's vison transform prepares the initial state and the product's
tvmc_evolve drives the stages.  The resulting state must follow
exp(-iHt) psi(0) (and not exp(+iHt)), and the vison's plaquette value must
track the exact one.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import dynamics as dyn  # noqa: E402
from oracle import peps as P  # noqa: E402
from oracle import vmc  # noqa: E402
from oracle.lattice import Lattice  # noqa: E402
from paper_2503_20566_gb300 import drivers, states  # noqa: E402
from paper_2503_20566_gb300.binding import SR, TDVP_STAGE1, TDVP_STAGE2  # noqa: E402


class ExactContext:
    """gcf_sr_step semantics with exact expectations (no sampling noise)."""

    def __init__(self, lat, Dk, params, h, g, chi):
        self.lat, self.Dk, self.params, self.chi = lat, Dk, np.array(params, dtype=np.complex128), chi
        self.N, self.Lx, self.Ly, self.D = lat.N, lat.Lx, lat.Ly, lat.N * Dk
        self.matter, self.complex, self.precision = False, True, "fp64"
        self.h, self.g, self.J, self.m, self.Q = h, g, 0.0, 0.0, None
        self.n_params, self.cfg_len = len(self.params), lat.cfg_len
        self.model = vmc.Model(h=h, g=g)
        self.basis = lat.physical_basis()

    def get_tensors(self):
        return self.params.copy()

    def set_tensors(self, v):
        self.params = np.array(v, dtype=np.complex128)

    def alloc_samples(self, n_chains, n_sweeps, grad=True):
        return {"accepted": torch.zeros(n_chains, dtype=torch.int32),
                "proposed": torch.ones(n_chains, dtype=torch.int32)}

    def sample_batch(self, configs, n_sweeps, seed, out=None):
        return out

    def sr_step(self, samples, n_chains, diag_shift=1e-4, lr=0.01, mode=SR, dt=0.0, max_iter=100, tol=1e-10):
        pe = P.GIPEPS(self.lat, self.Dk, self.params)
        w = vmc.exact_weights(pe, self.basis, self.chi)
        E = np.array([vmc.local_energy(pe, self.model, b, self.chi) for b in self.basis])
        O = np.array([vmc.log_grad_dense(pe, b, self.chi) for b in self.basis])
        S, F, eb = vmc.sr_matrices(O, E, w)
        x = np.linalg.solve(S + diag_shift * np.eye(len(F)), F)
        if mode == SR:
            self.params = self.params - lr * x
        else:
            c = (1 + 1j) / 2 if mode == TDVP_STAGE1 else (1 - 1j) / 2
            self.params = self.params + c * dt * (-1j * x)
        return [eb.real, eb.imag, 0.0, 1.0, 0.0, 1.0, 1.0, 0.0]


def _psi(lat, Dk, params, basis):
    pe = P.GIPEPS(lat, Dk, params)
    v = np.array([P.contract_exact(pe.sampled_network(b)) for b in basis])
    return v / np.linalg.norm(v)


def test_tvmc_driver_follows_exact_vison_dynamics():
    lat, Dk, h, g, chi = Lattice(3, 3, 2), 2, 1.0, 0.1, 2
    _, n = P.layout(lat, Dk)
    params = states.vison(synth.tensor_entries(71, n, True), 2, 3, 3, Dk)
    ctx = ExactContext(lat, Dk, params, h, g, chi)
    basis = ctx.basis
    psi0 = _psi(lat, Dk, ctx.params, basis)
    dt, n_steps = 0.02, 5
    configs = torch.zeros((2, lat.cfg_len), dtype=torch.int8)
    plaq = dyn.plaquette_matrix(lat, basis, 0, 0)
    seen = []
    drivers.tvmc_evolve(ctx, configs, n_steps=n_steps, dt=dt, n_sweeps=1, diag_shift=1e-8,
                        on_step=lambda rec: seen.append(dyn.expectation(_psi(lat, Dk, ctx.params, basis), plaq).real))
    H = lat.hamiltonian_matrix(basis, h, g)
    t = dt * n_steps
    fwd = dyn.evolve(H, psi0, [t])[0]
    bwd = dyn.evolve(-H, psi0, [t])[0]
    psi_t = _psi(lat, Dk, ctx.params, basis)
    f_fwd, f_bwd = abs(np.vdot(fwd, psi_t)), abs(np.vdot(bwd, psi_t))
    print("fidelity forward %.8f backward %.8f" % (f_fwd, f_bwd))
    assert f_fwd > 0.99999 and f_fwd > f_bwd + 0.1, (f_fwd, f_bwd)
    exact = [dyn.expectation(p, plaq).real for p in dyn.evolve(H, psi0, dt * np.arange(1, n_steps + 1))]
    assert np.allclose(seen, exact, atol=1e-3), (seen, exact)


def test_sr_driver_lowers_the_exact_energy_towards_the_ground_state():
    """SR steps with exact statistics: the energy falls step by step and stays
    above the exact ground-state energy (variational bound)."""
    lat, Dk, h, g, chi = Lattice(3, 3, 2), 2, 1.0, 0.3, 2
    _, n = P.layout(lat, Dk)
    ctx = ExactContext(lat, Dk, synth.tensor_entries(73, n, False), h, g, chi)
    e0, _ = dyn.ground_state(lat.hamiltonian_matrix(ctx.basis, h, g))
    _, recs = drivers.sr_optimize(ctx, torch.zeros((2, lat.cfg_len), dtype=torch.int8), n_steps=15, n_sweeps=1,
                                  lr=0.05, diag_shift=1e-3)
    energies = [r["e_mean"] for r in recs]
    assert all(b < a for a, b in zip(energies, energies[1:])), energies
    assert energies[-1] >= e0 - 1e-9 and energies[-1] < energies[0] - 0.1 * (energies[0] - e0)
