"""Pins of the (1+1)D Schwinger-model oracle (End Matter; NEXT-4).

Exact diagonalisation of the stated Hamiltonian, pinned by:
* g = 0: free fermions, E_0 = sum of the n_f lowest single-particle levels
  of diag(m_x) + J (nearest-neighbour hopping);
* J = 0: the minimum of the diagonal over all occupations, by brute force;
* the phase of J does not change the spectrum (a gauge choice on a chain).
The GCF time evolution (U(1)-symmetric MPS whose bond charges are the
electric fields, hopping of the globally symmetric model, exp(-tau g E^2) on
the charges, split at fixed site charge) is pinned against that ED:
imaginary time reaches the ground energy, real time follows exp(-iHt) (and
not exp(+iHt)), the state never leaves its fermion-number sector, and a
truncated bond gives a variational energy above the exact one.
(The printed 16-site value is not reproduced by the stated Hamiltonian; see
the Schwinger-model reading.)
"""

import itertools

import numpy as np
import pytest

from oracle import schwinger as S


def test_free_fermions_fill_the_lowest_levels():
    L, m, J, nf = 8, 0.3, 0.7 - 0.4j, 4
    H, _ = S.hamiltonian(L, m, J, 0.0, nf)
    h1 = np.diag(S.masses(L, m)).astype(complex)
    for x in range(L - 1):
        h1[x, x + 1] = J
        h1[x + 1, x] = np.conj(J)
    assert abs(np.linalg.eigvalsh(H)[0] - np.sort(np.linalg.eigvalsh(h1))[:nf].sum()) < 1e-10


def test_static_limit_is_the_brute_force_minimum():
    L, m, g, nf = 8, 0.4, 0.9, 4
    H, _ = S.hamiltonian(L, m, 0.0, g, nf)
    Q = [(1 + (-1) ** x) // 2 for x in range(L)]
    best = np.inf
    for occ in itertools.product((0, 1), repeat=L):
        if sum(occ) != nf:
            continue
        e, E = 0.0, 0
        for x in range(L):
            e += ((-1) ** x) * m * occ[x]
            E += occ[x] - Q[x]
            if x < L - 1:
                e += g * E * E
        best = min(best, e)
    assert abs(np.linalg.eigvalsh(H)[0] - best) < 1e-12


def test_phase_of_the_hopping_is_a_gauge_choice():
    e = [np.linalg.eigvalsh(S.hamiltonian(8, 0.2, J, 0.3, 4)[0])[:3] for J in (2.0, -2.0j, 2.0 * np.exp(0.7j))]
    assert np.allclose(e[0], e[1]) and np.allclose(e[0], e[2])


@pytest.fixture(scope="module")
def chain():
    L, m, J, g = 8, 0.2, 1.0, 0.5
    H, B = S.hamiltonian(L, m, J, g, 4)
    return L, m, J, g, H, B, tuple(S.charges(L))


def _energy(mps, H, B):
    v = mps.dense(B)
    return (v.conj() @ H @ v).real / np.vdot(v, v).real


def test_imaginary_time_reaches_the_ground_energy(chain):
    L, m, J, g, H, B, vac = chain
    mps = S.ChargedMPS(vac)
    S.evolve(mps, L, m, J, g, 0.05, 200, chi=16)
    S.evolve(mps, L, m, J, g, 0.01, 100, chi=16)
    e0 = np.linalg.eigvalsh(H)[0]
    assert abs(_energy(mps, H, B) - e0) < 1e-6
    # nothing outside the four-fermion sector
    assert np.abs(mps.dense(S.basis(L, 3))).max() < 1e-12 and np.abs(mps.dense(S.basis(L, 5))).max() < 1e-12
    # a truncated bond stays above the exact energy (variational) and is worse than chi = 16
    small = S.ChargedMPS(vac)
    S.evolve(small, L, m, J, g, 0.05, 200, chi=2)
    assert e0 < _energy(small, H, B) and _energy(small, H, B) - e0 > 1e-3


def test_real_time_follows_the_exact_evolution(chain):
    L, m, J, g, H, B, vac = chain
    mps = S.ChargedMPS(vac)
    dt, n = 0.01, 100
    S.evolve(mps, L, m, J, g, 1j * dt, n, chi=32)
    v = mps.dense(B)
    w, U = np.linalg.eigh(H)
    p0 = np.zeros(len(B), dtype=complex)
    p0[B.index(vac)] = 1.0
    fwd = U @ (np.exp(-1j * w * dt * n) * (U.conj().T @ p0))
    bwd = U @ (np.exp(+1j * w * dt * n) * (U.conj().T @ p0))
    f, b = abs(np.vdot(fwd, v)) / np.linalg.norm(v), abs(np.vdot(bwd, v)) / np.linalg.norm(v)
    assert f > 0.99999 and b < 0.9, (f, b)


def test_sparse_and_dense_hamiltonians_agree():
    Hd, B = S.hamiltonian(8, 0.2, -5j, 0.05, 4)
    Hs, B2 = S.hamiltonian(8, 0.2, -5j, 0.05, 4, sparse=True)
    assert B == B2 and np.allclose(Hs.toarray(), Hd) and np.allclose(Hd, Hd.conj().T)
