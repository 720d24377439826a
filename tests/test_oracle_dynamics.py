"""Pins of the oracle's exact real-time evolution.

* The single-plaquette 2x2 Z2 lattice is a two-level system: the population
  of the flipped state follows the closed-form Rabi formula.
* exp(-iHt) by eigendecomposition equals scipy's matrix exponential.
* Norm and energy are conserved; <P_x + P_x^dag> is real.
* The vison (sigma_z on the bottom-left vertical link of the ground state)
  flips <P + P^dag> of its plaquette and leaves the others; its energy lies
  above the ground state.
"""

import numpy as np
import pytest

from oracle import dynamics as dyn
from oracle.lattice import Lattice


def test_single_plaquette_is_a_rabi_oscillation():
    h, g = 0.7, 0.3
    lat = Lattice(2, 2, 2)
    basis = lat.physical_basis()
    H = lat.hamiltonian_matrix(basis, h, g)
    i0 = [i for i, b in enumerate(basis) if not np.any(b)][0]
    psi0 = np.zeros(len(basis))
    psi0[i0] = 1.0
    # two levels: energies 0 and 16 g (four links at n = 1), coupling -2h
    a, c, b = 0.0, 16.0 * g, -2.0 * h
    omega = np.sqrt((c - a) ** 2 + 4 * b ** 2)
    times = np.linspace(0.0, 3.0, 13)
    psi = dyn.evolve(H, psi0, times)
    p1 = np.abs(psi[:, 1 - i0]) ** 2
    assert np.allclose(p1, 4 * b ** 2 / omega ** 2 * np.sin(omega * times / 2) ** 2, atol=1e-12)


def test_evolution_matches_the_matrix_exponential_and_conserves():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    lat = Lattice(3, 3, 3)
    basis = lat.physical_basis()
    H = lat.hamiltonian_matrix(basis, 1.0, 0.4)
    g = np.random.default_rng(1)
    psi0 = g.standard_normal(len(basis)) + 1j * g.standard_normal(len(basis))
    psi0 /= np.linalg.norm(psi0)
    t = 0.37
    got = dyn.evolve(H, psi0, [t])[0]
    ref = scipy_linalg.expm(-1j * H * t) @ psi0
    assert np.linalg.norm(got - ref) < 1e-10
    traj = dyn.evolve(H, psi0, np.linspace(0, 2, 5))
    e0 = dyn.expectation(psi0, H).real
    for psi in traj:
        assert abs(np.linalg.norm(psi) - 1.0) < 1e-12
        assert abs(dyn.expectation(psi, H) - e0) < 1e-10
        assert abs(dyn.expectation(psi, dyn.plaquette_matrix(lat, basis, 1, 0)).imag) < 1e-12


def test_vison_flips_its_plaquette_in_the_ground_state():
    lat = Lattice(3, 3, 2)
    basis = lat.physical_basis()
    H = lat.hamiltonian_matrix(basis, 1.0, 0.1)
    e0, gs = dyn.ground_state(H)
    v = dyn.vison(lat, basis, gs)
    for y in range(lat.Ly - 1):
        for x in range(lat.Lx - 1):
            M = dyn.plaquette_matrix(lat, basis, x, y)
            before, after = dyn.expectation(gs, M).real, dyn.expectation(v, M).real
            assert abs(after - (-before if (x, y) == (0, 0) else before)) < 1e-12
    assert dyn.expectation(v, H).real > e0 + 1.0
