"""Exact real-time evolution on small lattices (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The reference for tVMC trajectories (Sec. S-3, Eqs. S6-S8) and for the vison
dynamics of the real-time study: on a complete physical basis,
psi(t) = exp(-i H t) psi(0) from the eigendecomposition of the Hermitian H
(`Lattice.hamiltonian_matrix`), and expectation values
<psi|M|psi> / <psi|psi> of operators written as matrices on that basis.

The vison (real-time study): the Pauli sigma_z in the electric basis,
|n> -> (-1)^n |n>, on the bottom-left vertical link, applied to the ground
state; for Z_N the clock operator |n> -> omega^n |n> generalises it.
"""

from __future__ import annotations

import numpy as np

from .lattice import Lattice


def evolve(H, psi0, times):
    """psi(t) for every t in `times`: rows of a (len(times), dim) array."""
    evals, evecs = np.linalg.eigh(H)
    c = evecs.conj().T @ np.asarray(psi0, dtype=np.complex128)
    return np.array([evecs @ (np.exp(-1j * evals * t) * c) for t in times])


def expectation(psi, M):
    """<psi|M|psi> / <psi|psi>."""
    psi = np.asarray(psi)
    return (psi.conj() @ (M @ psi)) / (psi.conj() @ psi)


def _index(basis):
    return {tuple(int(v) for v in b): i for i, b in enumerate(basis)}


def plaquette_matrix(lat: Lattice, basis, x, y):
    """P_x + P_x^dag on the basis (P_x raises the bottom and right links of
    the plaquette with lower-left corner (x, y), Eq. 4)."""
    idx = _index(basis)
    M = np.zeros((len(basis), len(basis)))
    for j, b in enumerate(basis):
        M[idx[tuple(int(v) for v in lat.plaquette(b, x, y, 1))], j] += 1.0
        M[idx[tuple(int(v) for v in lat.plaquette(b, x, y, lat.N - 1))], j] += 1.0
    return M


def clock_matrix(lat: Lattice, basis, x, y, axis):
    """Diagonal |n> -> omega^n |n> on link (x, y, axis) (sigma_z for N = 2)."""
    li = lat.hi(x, y) if axis == 1 else lat.vi(x, y)
    n = np.array([int(b[li]) for b in basis])
    return np.diag(np.exp(2j * np.pi * n / lat.N))


def ground_state(H):
    evals, evecs = np.linalg.eigh(H)
    return evals[0], evecs[:, 0]


def vison(lat: Lattice, basis, psi):
    """sigma_z (clock operator) on the bottom-left vertical link applied to psi."""
    return clock_matrix(lat, basis, 0, 0, 2) @ psi
