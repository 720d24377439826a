"""The exact-statistics SR campaign (oracle): on a tiny lattice the energy
falls and stays above the exact ground-state energy (variational bound)."""

import numpy as np

import synth
from oracle import campaign
from oracle import peps as P
from oracle import vmc
from oracle.lattice import Lattice


def test_exact_sr_lowers_the_energy_above_the_ground_state():
    lat = Lattice(3, 2, 2, matter=True)
    model = vmc.Model(h=1.0, g=0.33, J=0.5)
    basis = lat.physical_basis(n_bosons=2)
    e0 = np.linalg.eigvalsh(lat.hamiltonian_matrix(basis, model.h, model.g, model.J))[0]
    _, n = P.layout(lat, 2)
    params, energies, e_final = campaign.sr_exact(lat, model, 2, 2, 0.5 * synth.tensor_entries(3, n, False), 12,
                                                  lr=0.1, basis=basis)
    assert all(b < a + 1e-12 for a, b in zip(energies, energies[1:]))
    assert e0 - 1e-9 <= e_final < energies[0]


def test_exact_tvmc_follows_the_exact_evolution():
    from oracle import dynamics as dyn

    lat = Lattice(3, 3, 2)
    model = vmc.Model(h=1.0, g=0.2)
    basis = lat.physical_basis()
    _, n = P.layout(lat, 2)
    params = synth.tensor_entries(9, n, True)
    psi0 = campaign.psi_vector(lat, 2, params, basis)
    out = campaign.tvmc_exact(lat, model, 2, 2, params, 0.02, 3, shift=1e-8, basis=basis)
    H = lat.hamiltonian_matrix(basis, model.h, model.g)
    fwd = dyn.evolve(H, psi0, [0.06])[0]
    bwd = dyn.evolve(-H, psi0, [0.06])[0]
    psi = campaign.psi_vector(lat, 2, out, basis)
    assert abs(np.vdot(fwd, psi)) > 0.99999 and abs(np.vdot(fwd, psi)) > abs(np.vdot(bwd, psi)) + 0.01
