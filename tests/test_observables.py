"""Observable estimators (NEXT-2 analysis layer) against exact expectations.

With amplitudes supplied by the oracle at exact chi, each local estimator
averaged over the complete physical basis with Born weights |psi|^2 / sum |psi|^2
must equal psi^H M psi / psi^H psi, where M is the operator's matrix on that
basis built from the oracle's own moves (plaquette operators composed for the
Wilson loop).  Complex Z3 tensors make W and W^dag differ, so a reversed loop
or a wrong local-estimator direction fails.  The configuration moves are also
checked against the oracle's plaquette and hop moves, and the diagonal
estimators against the oracle's electric term, an explicit staggered sum and
the occupations.
"""

import numpy as np
import pytest

from oracle import peps as P
from oracle import vmc
from paper_2503_20566_gb300 import observables as obs

from test_oracle_peps import make_peps


class OracleAmplitudes:
    """Context stand-in: amplitude() from the oracle at exact chi."""

    def __init__(self, pe, chi):
        self.pe, self.chi = pe, chi

    def amplitude(self, configs):
        out = [vmc.amplitude(self.pe, c.astype(np.int64), self.chi) for c in np.asarray(configs)]
        return np.array([o[0] for o in out]), np.array([o[1] for o in out])


@pytest.fixture(scope="module")
def system():
    pe = make_peps(3, 3, 3, 2, seed=91, complex_=True)
    lat = pe.lat
    basis = lat.physical_basis()
    psi = np.array([P.contract_exact(pe.sampled_network(b)) for b in basis])
    w = np.abs(psi) ** 2 / np.sum(np.abs(psi) ** 2)
    index = {tuple(b): i for i, b in enumerate(basis)}
    return pe, lat, basis, psi, w, index


def _matrix(lat, basis, index, moves):
    """Permutation matrix M[i, j] = 1 iff basis[i] = (composed moves)(basis[j])."""
    M = np.zeros((len(basis), len(basis)))
    for j, b in enumerate(basis):
        c = b.copy()
        for (x, y) in moves:
            c = lat.plaquette(c, x, y, 1)
        M[index[tuple(c)], j] = 1.0
    return M


def _expect(psi, M):
    return (psi.conj() @ M @ psi) / (psi.conj() @ psi)


def test_moves_match_the_oracle(system):
    pe, lat, basis, *_ = system
    cfgs = basis[::7].astype(np.int8)
    for (x, y) in [(0, 0), (1, 0), (0, 1), (1, 1)]:
        for t in (1, lat.N - 1):
            got = obs.shift_block(cfgs, lat.Lx, lat.Ly, lat.N, x, y, 1, 1, t)
            ref = np.array([lat.plaquette(c, x, y, t) for c in cfgs])
            assert np.array_equal(got, ref)
    got = obs.shift_block(cfgs, lat.Lx, lat.Ly, lat.N, 0, 0, 2, 2, 1)
    ref = []
    for c in cfgs:
        for (x, y) in [(0, 0), (1, 0), (0, 1), (1, 1)]:
            c = lat.plaquette(c, x, y, 1)
        ref.append(c)
    assert np.array_equal(got, np.array(ref))
    assert all(lat.is_physical(c) for c in got)
    with pytest.raises(ValueError):
        obs.shift_block(cfgs, lat.Lx, lat.Ly, lat.N, 1, 1, 2, 1, 1)


def test_plaquette_map_is_the_exact_expectation(system):
    pe, lat, basis, psi, w, index = system
    est = obs.plaquette_map(OracleAmplitudes(pe, 2), basis.astype(np.int8), lat.Lx, lat.Ly, lat.N)
    for y in range(lat.Ly - 1):
        for x in range(lat.Lx - 1):
            M = _matrix(lat, basis, index, [(x, y)])
            exact = _expect(psi, M + M.T)
            assert abs(w @ est[:, y, x] - exact) < 1e-10 * max(1.0, abs(exact))


@pytest.mark.parametrize("size", [1, 2])
def test_wilson_loop_is_the_exact_expectation(system, size):
    pe, lat, basis, psi, w, index = system
    est = obs.wilson_loop(OracleAmplitudes(pe, 2), basis.astype(np.int8), lat.Lx, lat.Ly, lat.N, size,
                          origin=(0, 0))
    moves = [(x, y) for y in range(size) for x in range(size)]
    M = _matrix(lat, basis, index, moves)
    exact = _expect(psi, M)
    assert abs(w @ est - exact) < 1e-10 * max(1.0, abs(exact))
    assert abs(exact - _expect(psi, M.T)) > 1e-3  # W and W^dag differ here: direction is pinned


def test_diagonal_estimators(system):
    pe, lat, basis, psi, w, index = system
    cfgs = basis.astype(np.int8)
    he = obs.electric_term(cfgs, lat.Lx, lat.Ly, lat.N)
    assert np.allclose(he, [lat.diagonal_energy(b, 1.0) for b in basis])
    dx, dy = obs.vbs_order(cfgs, lat.Lx, lat.Ly, lat.N)
    e = lambda n: 2.0 - 2.0 * np.cos(2.0 * np.pi * n / lat.N)  # noqa: E731
    for k, b in enumerate(basis[:20]):
        rx = sum((-1) ** x * e(b[lat.hi(x, y)]) for y in range(lat.Ly) for x in range(lat.Lx - 1)) / lat.n_h
        ry = sum((-1) ** y * e(b[lat.vi(x, y)]) for y in range(lat.Ly - 1) for x in range(lat.Lx)) / lat.n_v
        assert abs(dx[k] - rx) < 1e-12 and abs(dy[k] - ry) < 1e-12


def test_mean_and_error_over_chains():
    v = np.arange(12.0)
    m, err = obs.mean_and_error(v, 3)
    means = v.reshape(3, 4).mean(axis=1)
    assert m == pytest.approx(means.mean()) and err == pytest.approx(means.std(ddof=1) / np.sqrt(3))


def test_matter_observables_are_exact_expectations():
    pe = make_peps(3, 2, 2, 2, seed=93, matter=True, complex_=True)
    lat = pe.lat
    basis = np.concatenate([lat.physical_basis(n_bosons=k) for k in (0, 2, 4, 6)])
    psi = np.array([P.contract_exact(pe.sampled_network(b)) for b in basis])
    w = np.abs(psi) ** 2 / np.sum(np.abs(psi) ** 2)
    index = {tuple(b): i for i, b in enumerate(basis)}
    cfgs = basis.astype(np.int8)
    dens = obs.boson_density(cfgs, lat.Lx, lat.Ly)
    assert np.allclose(dens.reshape(len(basis), -1), basis[:, lat.n_h + lat.n_v:])
    hh, hv = obs.hop_map(OracleAmplitudes(pe, 2), cfgs, lat.Lx, lat.Ly, lat.N)
    for axis, est, ny, nx in ((1, hh, lat.Ly, lat.Lx - 1), (2, hv, lat.Ly - 1, lat.Lx)):
        for y in range(ny):
            for x in range(nx):
                M = np.zeros((len(basis), len(basis)))
                for j, b in enumerate(basis):
                    c2 = lat.hop(b, x, y, axis)
                    if c2 is not None:
                        M[index[tuple(c2)], j] = 1.0
                exact = (psi.conj() @ M @ psi) / (psi.conj() @ psi)
                assert abs(w @ est[:, y, x] - exact) < 1e-10 * max(1.0, abs(exact))
                moved, mask = obs.hop_configs(cfgs, lat.Lx, lat.Ly, lat.N, x, y, axis)
                for k in np.nonzero(mask)[0]:
                    assert np.array_equal(moved[k], lat.hop(basis[k], x, y, axis))
