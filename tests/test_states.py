"""State preparation by exact parameter transforms (NEXT-1 initial state).

* The product's block layout and block decoding agree with the oracle's
  (the layout is an interface both sides implement).
* Z^power on one link multiplies every amplitude by omega^(power n_link(s))
  (exact contraction, full physical basis; Z2 real, Z3 complex, with matter
  and background charges).
* The vison (sigma_z on the bottom-left vertical link) flips <P + P^dag> on
  the one plaquette that contains the link and leaves every other plaquette's
  value unchanged (sigma_z anticommutes with the first, commutes with the rest).
"""

import itertools

import numpy as np
import pytest

import synth
from oracle import peps as P
from oracle.lattice import Lattice
from paper_2503_20566_gb300 import states

CASES = [(3, 3, 2, 2, False, False, None), (3, 3, 3, 2, False, True, None), (3, 2, 2, 2, True, False, None),
         (3, 2, 3, 1, True, True, [[1, 0, 0], [0, 0, 0]])]


def _ids(c):
    return "{}x{}-Z{}-Dk{}{}{}{}".format(c[0], c[1], c[2], c[3], "-m" if c[4] else "", "-c" if c[5] else "",
                                        "-Q" if c[6] else "")


def _peps(Lx, Ly, N, Dk, matter, cplx, Q, seed=5):
    lat = Lattice(Lx, Ly, N, matter=matter, Q=Q)
    _, n = P.layout(lat, Dk)
    return lat, P.GIPEPS(lat, Dk, synth.tensor_entries(seed, n, cplx))


def _basis(lat):
    if not lat.matter:
        return lat.physical_basis()
    return np.concatenate([lat.physical_basis(n_bosons=nb) for nb in range(lat.n_s + 1)
                           if (nb - lat.Q.sum()) % lat.N == 0])


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_layout_and_block_decoding_match_the_oracle(case):
    Lx, Ly, N, Dk, matter, cplx, Q = case
    lat, pe = _peps(*case)
    lay = states.vertex_layout(N, Lx, Ly, Dk, matter)
    for v, (off, nb, bs, legs) in enumerate(lay):
        vl = pe.verts[v]
        assert (off, nb, bs, legs) == (vl.offset, vl.n_blocks, vl.block_size, vl.legs)
        x, y = v % Lx, v // Lx
        q = int(lat.Q[y, x])
        for p in range(2 if matter else 1):
            for ch in itertools.product(range(N), repeat=4):
                bid = P.block_id(lat, vl, x, y, p, ch)
                if bid < 0:
                    continue
                p2, got = states.block_charges(N, bid, legs, q)
                assert p2 == p and all(got[i] == ch[i] for i in legs)


@pytest.mark.parametrize("case", CASES, ids=_ids)
@pytest.mark.parametrize("link", [(0, 0, 2, 1), (1, 0, 1, 1), (1, 1, 2, 2)])
def test_link_phase_multiplies_every_amplitude(case, link):
    Lx, Ly, N, Dk, matter, cplx, Q = case
    x, y, axis, power = link
    if (axis == 2 and y >= Ly - 1) or (axis == 1 and x >= Lx - 1):
        pytest.skip("no such link")
    lat, pe = _peps(*case)
    new = states.link_phase(pe.params, N, Lx, Ly, Dk, x, y, axis, power, matter, Q)
    pe2 = P.GIPEPS(lat, Dk, new)
    li = lat.hi(x, y) if axis == 1 else lat.vi(x, y)
    for s in _basis(lat):
        a = P.contract_exact(pe.sampled_network(s))
        b = P.contract_exact(pe2.sampled_network(s))
        f = np.exp(2j * np.pi * power * s[li] / N)
        assert abs(b - f * a) <= 1e-12 * max(1.0, abs(a))
    if N == 2 and not cplx:
        assert not np.iscomplexobj(new)


def test_vison_flips_its_plaquette_only():
    lat, pe = _peps(3, 3, 2, 2, False, False, None, seed=8)
    basis = lat.physical_basis()
    index = {tuple(b): i for i, b in enumerate(basis)}
    psi = np.array([P.contract_exact(pe.sampled_network(b)) for b in basis])
    pe2 = P.GIPEPS(lat, 2, states.vison(pe.params, 2, 3, 3, 2))
    psi2 = np.array([P.contract_exact(pe2.sampled_network(b)) for b in basis])
    for y in range(lat.Ly - 1):
        for x in range(lat.Lx - 1):
            M = np.zeros((len(basis), len(basis)))
            for j, b in enumerate(basis):
                M[index[tuple(lat.plaquette(b, x, y, 1))], j] = 1.0
            op = M + M.T
            before = (psi @ op @ psi) / (psi @ psi)
            after = (psi2 @ op @ psi2) / (psi2 @ psi2)
            want = -before if (x, y) == (0, 0) else before
            assert abs(after - want) < 1e-10 * max(1.0, abs(before))
            if (x, y) == (0, 0):
                assert abs(before) > 1e-3


def test_link_phase_refuses_missing_links():
    with pytest.raises(ValueError):
        states.link_phase(np.zeros(10), 2, 3, 3, 2, 2, 0, 1)
    with pytest.raises(ValueError):
        states.link_phase(np.zeros(10), 2, 3, 3, 2, 0, 2, 2)


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_product_and_oracle_link_operators_agree(case):
    """The product's transform and the oracle's own (written separately)
    give the same parameters on every link."""
    Lx, Ly, N, Dk, matter, cplx, Q = case
    lat, pe = _peps(*case)
    for x, y, axis in [(0, 0, 2), (1, 0, 1), (Lx - 2, Ly - 1, 1), (Lx - 1, Ly - 2, 2)]:
        for power in (1, N - 1):
            a = states.link_phase(pe.params, N, Lx, Ly, Dk, x, y, axis, power, matter, Q)
            b = P.link_clock_params(pe, x, y, axis, power)
            assert np.allclose(a, b, atol=0, rtol=1e-15)
