"""Pins of the oracle's lattice model: Gauss law, moves, basis, Hamiltonian.

These tests fix the oracle against facts outside itself: the paper's printed
exact-diagonalisation energy, brute-force enumeration, and the published
SplitMix64 test vector.
"""

import os

import numpy as np
import pytest

import synth
from oracle import rng
from oracle.lattice import Lattice

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (s.strip() for s in line.split("=", 1))
                vals[k] = float(v) if "." in v or "e" in v else int(v)
    return vals


def test_ed_pin_z2_hardcore_bosons_3x3():
    """The paper's ED energy/site for Z2 + 2 hard-core bosons on 3x3."""
    gd = read_golden("ed_z2_hardcore_bosons_3x3.txt")
    lat = Lattice(gd["Lx"], gd["Ly"], gd["N"], matter=True)
    basis = lat.physical_basis(n_bosons=gd["n_bosons"])
    H = lat.hamiltonian_matrix(basis, gd["h"], gd["g"], gd["J"])
    assert np.allclose(H, H.T)
    e0 = np.linalg.eigvalsh(H)[0] / (gd["Lx"] * gd["Ly"])
    assert abs(e0 - gd["energy_per_site"]) < 0.6 * 10.0 ** -gd["digits"]


def test_ed_pin_rejects_single_counted_z2_plaquette():
    """Without the factor 2 on the Z2 plaquette (P = P^dag counted once) the
    printed ED value is not reproduced: the pin really fixes the convention."""
    gd = read_golden("ed_z2_hardcore_bosons_3x3.txt")
    lat = Lattice(3, 3, 2, matter=True)
    basis = lat.physical_basis(n_bosons=2)
    H = lat.hamiltonian_matrix(basis, gd["h"] / 2.0, gd["g"], gd["J"])
    e0 = np.linalg.eigvalsh(H)[0] / 9
    assert abs(e0 - gd["energy_per_site"]) > 1e-2


@pytest.mark.parametrize("Lx,Ly,N,matter,Q", [(2, 2, 2, False, None), (3, 2, 3, False, None),
                                              (3, 3, 2, False, None), (2, 2, 4, False, None),
                                              (3, 2, 2, True, None), (2, 2, 3, True, None),
                                              (3, 2, 3, False, [[1, 0, 0], [0, 0, 2]]),
                                              (3, 2, 2, True, [[0, 1, 0], [0, 0, 0]])])
def test_physical_basis_equals_brute_force(Lx, Ly, N, matter, Q):
    # the last two carry static background charges Q_x (Eq. 1)
    lat = Lattice(Lx, Ly, N, matter=matter, Q=Q)
    a = lat.physical_basis()
    b = lat.brute_force_physical()
    assert len(a) == len(b)
    assert set(map(tuple, a)) == set(map(tuple, b))
    if not matter:
        assert len(a) == N ** lat.n_plaquettes


def test_hilbert_dimension_pin():
    gd = read_golden("hilbert_dimension.txt")
    lat = Lattice(gd["Lx"], gd["Ly"], gd["N"])
    assert lat.n_plaquettes * np.log2(lat.N) == gd["log2_dimension"]
    # plaquette operators are independent: distinct powers give distinct configs
    small = Lattice(4, 3, 2)
    basis = small.physical_basis()
    assert len(set(map(tuple, basis))) == 2 ** small.n_plaquettes


@pytest.mark.parametrize("N", [2, 3, 4])
def test_moves_preserve_gauss_law(N):
    lat = Lattice(4, 3, N, matter=True)
    occ = synth.occupations(5, 1, lat.n_s, 4 if N == 2 else N)[0].reshape(3, 4)
    cfg = lat.config_from_powers(occ, synth.plaquette_powers(6, 1, lat.n_plaquettes, N)[0])
    assert lat.is_physical(cfg)
    for y in range(lat.Ly - 1):
        for x in range(lat.Lx - 1):
            for t in range(1, N):
                assert lat.is_physical(lat.plaquette(cfg, x, y, t))
            assert np.array_equal(lat.plaquette(lat.plaquette(cfg, x, y, 1), x, y, N - 1), cfg)
    for y in range(lat.Ly):
        for x in range(lat.Lx):
            for a in (1, 2):
                if (a == 1 and x == lat.Lx - 1) or (a == 2 and y == lat.Ly - 1):
                    continue
                c2 = lat.hop(cfg, x, y, a)
                if c2 is not None:
                    assert lat.is_physical(c2)
                    assert c2[lat.n_h + lat.n_v:].sum() == cfg[lat.n_h + lat.n_v:].sum()
                    back = lat.hop(c2, x, y, a)
                    assert np.array_equal(back, cfg)


def test_gauss_violation_detected():
    lat = Lattice(3, 3, 3)
    cfg = lat.config_from_powers(np.zeros((3, 3)), [1, 2, 0, 1])
    assert lat.is_physical(cfg)
    bad = cfg.copy()
    bad[lat.hi(0, 0)] = (bad[lat.hi(0, 0)] + 1) % 3
    res = lat.gauss_residual(bad)
    assert res[0, 0] != 0 and res[0, 1] != 0 and res.sum() != 0
    assert not lat.is_physical(bad)


def test_hamiltonian_hermitian_and_electric_term():
    lat = Lattice(3, 3, 3)
    basis = lat.physical_basis()
    H = lat.hamiltonian_matrix(basis, 0.7, 0.4)
    assert np.allclose(H, H.T)
    # g-only: diagonal with 2 - 2cos(2 pi n / 3) = 3 for n = 1, 2
    Hg = lat.hamiltonian_matrix(basis, 0.0, 1.0)
    nz = np.count_nonzero(basis[:, : lat.n_h + lat.n_v], axis=1)
    assert np.allclose(np.diag(Hg), 3.0 * nz)
    # h-only Z2 on one plaquette (2x2): spectrum of -2h X is {-2h, 2h}
    small = Lattice(2, 2, 2)
    Hs = small.hamiltonian_matrix(small.physical_basis(), 1.0, 0.0)
    assert np.allclose(np.linalg.eigvalsh(Hs), [-2.0, 2.0])


def test_splitmix64_reference_vector():
    """Published SplitMix64 outputs for seed 1234567 (the generator's
    reference test sequence); the oracle's chain key / word functions are its
    outputs at counters (c+1) and (k+1)."""
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423,
           4593380528125082431, 16408922859458223821]
    state = 1234567
    for k, r in enumerate(ref):
        assert rng.mix64(state + (k + 1) * rng.GAMMA) == r
        assert int(synth.mix64(np.uint64((state + (k + 1) * rng.GAMMA) & rng.MASK))) == r
    assert rng.chain_key(1234567, 0) == ref[0]
    assert rng.word(7, 3, 4) == rng.mix64(rng.chain_key(7, 3) + 5 * rng.GAMMA)
    assert int(synth.draws(7, 3, [4])[0]) == rng.word(7, 3, 4)


def test_synth_distributions():
    z = synth.normals(11, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    t = synth.plaquette_powers(3, 100, 50, 3)
    assert set(np.unique(t)) == {0, 1, 2}
    occ = synth.occupations(4, 20, 16, 8)
    assert np.all(occ.sum(axis=1) == 8)
