"""Pins of the oracle's PEPS layer: block sparsity, GCF, contraction.

* Definition-level: the full GI-PEPS with explicit link tensors (Eqs. 6-7)
  vanishes on every Gauss-violating configuration and equals the sampled
  single-layer network (Eq. S5) on every physical one (exhaustive, 3x3).
* GCF (Eqs. 8-9): the gauge transformation with random general B blocks
  leaves every amplitude unchanged.
* Contraction: D_k = 1 gives a product of scalars; the row-by-row contraction
  equals an explicit sum over all bond indices; the boundary MPS is exact when
  chi >= D_k^floor(Lx/2) and converges to it as chi grows; the two-site SVD
  compression is the Eckart-Young best rank-chi approximation.
"""

import itertools

import numpy as np
import pytest

import synth
from oracle import peps as P
from oracle import vmc
from oracle.lattice import Lattice


def make_peps(Lx, Ly, N, Dk, seed, matter=False, complex_=False):
    lat = Lattice(Lx, Ly, N, matter=matter)
    _, n = P.layout(lat, Dk)
    return P.GIPEPS(lat, Dk, synth.tensor_entries(seed, n, complex_))


def random_physical(lat, seed, n_bosons=0):
    occ = synth.occupations(seed, 1, lat.n_s, n_bosons)[0] if lat.matter else np.zeros(lat.n_s)
    return lat.config_from_powers(occ.reshape(lat.Ly, lat.Lx),
                                  synth.plaquette_powers(seed, 1, lat.n_plaquettes, lat.N)[0])


def brute_force_amplitude(rows):
    """Explicit sum over every bond index assignment (tiny networks only)."""
    Ly, Lx = len(rows), len(rows[0])
    hb = [(x, y) for y in range(Ly) for x in range(Lx - 1)]
    vb = [(x, y) for y in range(Ly - 1) for x in range(Lx)]
    Dk = rows[0][0].shape[1]
    tot = 0.0
    for hv in itertools.product(range(Dk), repeat=len(hb)):
        H = dict(zip(hb, hv))
        for vv in itertools.product(range(Dk), repeat=len(vb)):
            V = dict(zip(vb, vv))
            pr = 1.0
            for y in range(Ly):
                for x in range(Lx):
                    pr *= rows[y][x][H.get((x - 1, y), 0), H.get((x, y), 0),
                                     V.get((x, y - 1), 0), V.get((x, y), 0)]
            tot += pr
    return tot


def test_parameter_count_matches_block_counting():
    # 8x8 Z2 with D_k = 2: 36 bulk (8 blocks x 16) + 24 edge (4 x 8) + 4 corner (2 x 4)
    lat = Lattice(8, 8, 2)
    assert P.layout(lat, 2)[1] == 36 * 128 + 24 * 32 + 4 * 8
    # Z4 16x16 D_k = 2: bulk 4^3 blocks of 2^4
    lat = Lattice(16, 16, 4)
    assert P.layout(lat, 2)[1] == 14 * 14 * 64 * 16 + 4 * 14 * 16 * 8 + 4 * 4 * 4


@pytest.mark.parametrize("N,Dk,matter,Lx,Ly", [(2, 2, False, 3, 3), (3, 1, False, 3, 2), (2, 1, True, 3, 2),
                                                (3, 1, True, 2, 2), (3, (2, 1, 1), False, 3, 2),
                                                (2, (2, 1), True, 2, 2)])
def test_gi_peps_vanishes_off_gauss_and_matches_sampled_network(N, Dk, matter, Lx, Ly):
    # Z3 with matter fixes the sign of the matter charge against the leg sum
    # (for Z2 both signs agree, and without matter the sum's overall sign is free).
    pe = make_peps(Lx, Ly, N, Dk, seed=1, matter=matter)
    lat = pe.lat
    A = [[pe.dense_A(x, y) for x in range(Lx)] for y in range(Ly)]
    Bg = P.gcf_link_tensor(N, Dk)
    Bh = [[Bg] * (Lx - 1) for _ in range(Ly)]
    Bv = [[Bg] * Lx for _ in range(Ly - 1)]
    occs = list(itertools.product((0, 1), repeat=lat.n_s)) if matter else [(0,) * lat.n_s]
    n_phys = 0
    for occ in occs:
        for links in itertools.product(range(N), repeat=lat.n_h + lat.n_v):
            cfg = np.array(links + tuple(occ))
            full = P.full_amplitude(lat, A, Bh, Bv, cfg)
            rows = pe.sampled_network(cfg)
            if lat.is_physical(cfg):
                n_phys += 1
                assert rows is not None
                ref = P.contract_exact(rows)
                assert abs(full - ref) <= 1e-12 * max(1.0, abs(ref))
                assert abs(ref) > 0
            else:
                assert rows is None
                assert full == 0.0
    assert n_phys == len(lat.brute_force_physical())


def test_gauge_canonical_form_leaves_amplitudes_unchanged():
    N, Dk, Lx, Ly = 2, 2, 3, 3
    pe = make_peps(Lx, Ly, N, Dk, seed=3)
    lat = pe.lat
    A = [[pe.dense_A(x, y).copy() for x in range(Lx)] for y in range(Ly)]
    g = np.random.default_rng(0)
    Bh, Bv = [], []
    A_gcf = [[a.copy() for a in row] for row in A]
    for y in range(Ly):
        row = []
        for x in range(Lx - 1):
            blocks = [g.normal(size=(Dk, Dk)) + 2 * np.eye(Dk) for _ in range(N)]
            row.append(P.general_link_tensor(blocks, N, Dk))
            X = np.zeros((N * Dk, N * Dk))
            for k in range(N):
                X[k * Dk:(k + 1) * Dk, k * Dk:(k + 1) * Dk] = blocks[k]
            # A -> A X on the right leg of the tensor left of the link
            A_gcf[y][x] = np.einsum("plrdu,rs->plsdu", A_gcf[y][x], X)
        Bh.append(row)
    for y in range(Ly - 1):
        row = []
        for x in range(Lx):
            blocks = [g.normal(size=(Dk, Dk)) + 2 * np.eye(Dk) for _ in range(N)]
            row.append(P.general_link_tensor(blocks, N, Dk))
            X = np.zeros((N * Dk, N * Dk))
            for k in range(N):
                X[k * Dk:(k + 1) * Dk, k * Dk:(k + 1) * Dk] = blocks[k]
            A_gcf[y][x] = np.einsum("plrdu,us->plrds", A_gcf[y][x], X)
        Bv.append(row)
    Bg = P.gcf_link_tensor(N, Dk)
    Bh_g = [[Bg] * (Lx - 1) for _ in range(Ly)]
    Bv_g = [[Bg] * Lx for _ in range(Ly - 1)]
    for cfg in lat.physical_basis():
        a = P.full_amplitude(lat, A, Bh, Bv, cfg)
        b = P.full_amplitude(lat, A_gcf, Bh_g, Bv_g, cfg)
        assert abs(a - b) <= 1e-10 * max(1.0, abs(a))
    # and the transformed A keeps the block structure of Eq. (6)
    for y in range(Ly):
        for x in range(Lx):
            assert np.all(A_gcf[y][x][~_allowed_mask(pe, x, y)] == 0)


def _allowed_mask(pe, x, y):
    lat, Dk = pe.lat, pe.Dk
    A = pe.dense_A(x, y)
    mask = np.zeros(A.shape, dtype=bool)
    vl = pe.vertex(x, y)
    for p in range(A.shape[0]):
        for ch in itertools.product(*[range(lat.N) if i in vl.legs else range(1) for i in range(4)]):
            if P.block_id(lat, vl, x, y, p, ch) >= 0:
                sl = tuple(slice(ch[i] * Dk, (ch[i] + 1) * Dk) if i in vl.legs else slice(0, 1) for i in range(4))
                mask[(p,) + sl] = True
    return mask


def test_dk1_amplitude_is_product_of_scalars():
    pe = make_peps(5, 4, 3, 1, seed=7)
    cfg = random_physical(pe.lat, 8)
    rows = pe.sampled_network(cfg)
    prod = np.prod([rows[y][x].reshape(()) for y in range(4) for x in range(5)])
    assert abs(P.contract_exact(rows) - prod) <= 1e-12 * abs(prod)
    la, ph = vmc.amplitude(pe, cfg, chi=1)
    assert abs(np.exp(la) * np.cos(ph) - prod) <= 1e-12 * abs(prod)


def test_exact_contraction_equals_explicit_index_sum():
    pe = make_peps(3, 3, 2, 2, seed=9)
    for seed in range(3):
        rows = pe.sampled_network(random_physical(pe.lat, seed))
        a, b = P.contract_exact(rows), brute_force_amplitude(rows)
        assert abs(a - b) <= 1e-11 * abs(b)


@pytest.mark.parametrize("Lx,Ly,N,Dk,complex_", [(6, 5, 2, 2, False), (5, 4, 3, 2, True), (4, 4, 2, 3, False)])
def test_boundary_mps_exact_when_chi_reaches_bound(Lx, Ly, N, Dk, complex_):
    pe = make_peps(Lx, Ly, N, Dk, seed=2, complex_=complex_)
    cfg = random_physical(pe.lat, 3)
    ex = P.contract_exact(pe.sampled_network(cfg))
    chi_exact = Dk ** (Lx // 2)
    la, ph = vmc.amplitude(pe, cfg, chi_exact)
    val = np.exp(la + 1j * ph)
    assert abs(val - ex) <= 1e-10 * abs(ex)


def test_boundary_mps_converges_with_chi():
    pe = make_peps(8, 6, 2, 2, seed=5)
    cfg = random_physical(pe.lat, 6)
    ex = P.contract_exact(pe.sampled_network(cfg))
    errs = []
    for chi in (2, 4, 8, 16):
        la, ph = vmc.amplitude(pe, cfg, chi)
        errs.append(abs(np.exp(la) * np.cos(ph) - ex) / abs(ex))
    assert errs[-1] < 1e-10
    assert errs[0] > errs[-1] and errs[1] > errs[-1] and errs[2] < 0.1


def test_two_site_compression_is_eckart_young():
    g = np.random.default_rng(1)
    A = g.normal(size=(1, 6, 5))
    B = g.normal(size=(5, 7, 1))
    M = np.einsum("adb,bec->de", A, B)
    for chi in (1, 2, 3, 5):
        out, ls = P.compress([A, B], chi)
        approx = np.einsum("adb,bec->de", out[0], out[1]) * np.exp(ls)
        U, S, Vh = np.linalg.svd(M)
        best = (U[:, :chi] * S[:chi]) @ Vh[:chi]
        assert np.allclose(approx, best, atol=1e-10)


def test_compress_without_truncation_preserves_state():
    pe = make_peps(5, 3, 3, 2, seed=4, complex_=True)
    cfg = random_physical(pe.lat, 2)
    rows = pe.sampled_network(cfg)
    mps = P.absorb(P.absorb(P.trivial_mps(5, np.complex128), rows[0]), rows[1])

    def dense(m):
        v = np.ones((1, 1))
        for s in m:
            v = np.einsum("xa,adb->xdb", v, s).reshape(-1, s.shape[2])
        return v.reshape(-1)

    out, ls = P.compress(mps, chi=1000)
    assert np.allclose(dense(out) * np.exp(ls), dense(mps), atol=1e-10)
    assert abs(np.linalg.norm(dense(out)) - 1.0) < 1e-12


def _random_mps(seed, L, d, D, cplx=False):
    g = np.random.default_rng(seed)
    dims = [1] + [D] * (L - 1) + [1]
    out = []
    for i in range(L):
        t = g.standard_normal((dims[i], d, dims[i + 1]))
        out.append(t + 1j * g.standard_normal(t.shape) if cplx else t)
    return out


def _dense(mps, log_norm=0.0):
    v = np.ones((1, 1))
    for s in mps:
        v = np.einsum("xa,adb->xdb", v, s).reshape(-1, s.shape[2])
    return v.reshape(-1) * np.exp(log_norm)


def test_variational_compression_of_one_bond_is_the_eckart_young_optimum():
    """Two sites: the best rank-chi approximation is the SVD truncation, and
    its error is the root of the discarded squared singular values."""
    for chi, cplx in [(1, False), (2, True), (3, False)]:
        A = _random_mps(3, 2, 4, 5, cplx)
        v = _dense(A)
        out, ls = P.compress_variational(A, chi, sweeps=3)
        s = np.linalg.svd(v.reshape(4, 4), compute_uv=False)
        err = np.linalg.norm(v - _dense(out, ls))
        assert abs(err - np.sqrt(np.sum(s[chi:] ** 2))) <= 1e-10 * np.linalg.norm(v)


def test_variational_compression_is_exact_without_truncation():
    A = _random_mps(4, 6, 2, 8, True)
    v = _dense(A)
    out, ls = P.compress_variational(A, chi=16, sweeps=2)
    assert np.linalg.norm(v - _dense(out, ls)) <= 1e-10 * np.linalg.norm(v)


@pytest.mark.parametrize("L,d,D,chi,cplx", [(6, 2, 8, 3, True), (5, 3, 9, 4, False), (7, 2, 6, 2, False)])
def test_variational_compression_improves_on_svd_and_never_gets_worse(L, d, D, chi, cplx):
    """With several truncated bonds the SVD sweep is not the optimum: the fit
    must end below it, and no sweep may raise the error."""
    A = _random_mps(10 + L, L, d, D, cplx)
    v = _dense(A)
    s, ls = P.compress(A, chi)
    e_svd = np.linalg.norm(v - _dense(s, ls))
    hist = []
    out, lv = P.compress_variational(A, chi, sweeps=5, history=hist)
    e_var = np.linalg.norm(v - _dense(out, lv))
    assert e_var < e_svd * (1 - 1e-4)
    assert abs(hist[-1] - e_var ** 2) <= 1e-8 * np.linalg.norm(v) ** 2
    assert all(b <= a + 1e-9 * hist[0] for a, b in zip(hist, hist[1:]))
    assert max(m.shape[2] for m in out[:-1]) <= chi



# ---- uneven charge sectors (a different degeneracy per charge) -------------

def test_uneven_sector_parameter_count():
    """Every block's size is the product of its legs' sector degeneracies:
    count them by enumerating the Gauss-allowed charges of every vertex."""
    lat = Lattice(3, 3, 3, matter=True)
    dq = (2, 1, 3)
    total = 0
    for y in range(lat.Ly):
        for x in range(lat.Lx):
            has = lat.has_legs(x, y)
            for p in (0, 1):
                for ch in itertools.product(*[range(3) if has[i] else (0,) for i in range(4)]):
                    tot = p + ch[0] - ch[1] + ch[2] - ch[3]
                    if tot % 3 == 0:
                        total += int(np.prod([dq[ch[i]] for i in range(4) if has[i]]))
    assert P.layout(lat, dq)[1] == total


def test_uneven_sector_gauge_transformation_leaves_amplitudes_unchanged():
    N, dq, Lx, Ly = 3, (2, 1, 1), 3, 2
    pe = make_peps(Lx, Ly, N, dq, seed=13)
    lat = pe.lat
    g = np.random.default_rng(4)
    start = np.concatenate([[0], np.cumsum(dq)])
    A = [[pe.dense_A(x, y) for x in range(Lx)] for y in range(Ly)]
    A2 = [[a.copy() for a in row] for row in A]

    def xblocks():
        return [g.normal(size=(d, d)) + 2 * np.eye(d) for d in dq]

    def bd(blocks):
        X = np.zeros((start[-1], start[-1]))
        for n, b in enumerate(blocks):
            X[start[n]:start[n + 1], start[n]:start[n + 1]] = b
        return X

    Bh, Bv = [], []
    for y in range(Ly):
        row = []
        for x in range(Lx - 1):
            b = xblocks()
            row.append(P.general_link_tensor(b, N, dq))
            A2[y][x] = np.einsum("plrdu,rs->plsdu", A2[y][x], bd(b))
        Bh.append(row)
    for y in range(Ly - 1):
        row = []
        for x in range(Lx):
            b = xblocks()
            row.append(P.general_link_tensor(b, N, dq))
            A2[y][x] = np.einsum("plrdu,us->plrds", A2[y][x], bd(b))
        Bv.append(row)
    Bg = P.gcf_link_tensor(N, dq)
    for cfg in lat.physical_basis():
        a = P.full_amplitude(lat, A, Bh, Bv, cfg)
        b = P.full_amplitude(lat, A2, [[Bg] * (Lx - 1)] * Ly, [[Bg] * Lx] * (Ly - 1), cfg)
        assert abs(a - b) <= 1e-10 * max(1.0, abs(a))


def test_uneven_sector_boundary_mps_is_exact_at_the_bound():
    pe = make_peps(5, 4, 3, (2, 1, 1), seed=15, complex_=True)
    for seed in range(3):
        cfg = random_physical(pe.lat, 20 + seed)
        ex = P.contract_exact(pe.sampled_network(cfg))
        la, ph = vmc.amplitude(pe, cfg, chi=4)   # max degeneracy 2, floor(5/2) = 2 cuts deep
        assert abs(np.exp(la + 1j * ph) - ex) <= 1e-10 * abs(ex)



@pytest.mark.parametrize("N,Dk,cplx,link", [(2, 2, False, (0, 0, 2)), (3, (2, 1, 1), True, (1, 0, 1)),
                                            (3, 1, True, (1, 1, 2))])
def test_link_clock_multiplies_every_amplitude(N, Dk, cplx, link):
    """Z on one link: psi'(s) = omega^(n_link(s)) psi(s) on every physical s."""
    pe = make_peps(3, 3, N, Dk, seed=19, complex_=cplx)
    lat = pe.lat
    x, y, axis = link
    pe2 = P.GIPEPS(lat, Dk, P.link_clock_params(pe, x, y, axis))
    li = lat.hi(x, y) if axis == 1 else lat.vi(x, y)
    for s in lat.physical_basis():
        a = P.contract_exact(pe.sampled_network(s))
        b = P.contract_exact(pe2.sampled_network(s))
        assert abs(b - np.exp(2j * np.pi * s[li] / N) * a) <= 1e-12 * max(1.0, abs(a))


def test_pairwise_chain_equals_one_einsum():
    """The exact contractions sum over the same indices as one np.einsum of
    all operands; the chain of pairwise contractions only changes the order
    of evaluation (strip, row and open-row specs, complex operands)."""
    rng = np.random.default_rng(5)

    def rnd(*shape):
        return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)

    E, Bs, W1, W2, Ts = rnd(3, 2, 2, 4), rnd(3, 2, 5), rnd(2, 3, 2, 2), rnd(2, 3, 2, 2), rnd(4, 2, 6)
    for spec, ops in [("aijb,adA,iIdm,jJmu,buB->AIJB", (E, Bs, W1, W2, Ts)),
                      ("alb,adA,lrdu,buB->ArB", (E[:, :, 0, :], Bs, W1, Ts)),
                      ("ArB,buB,lrdu,adA->alb", (rnd(5, 3, 6), Ts, W1, Bs)),
                      ("alb,adA,ArB,buB->lrdu", (E[:, :, 0, :], Bs, rnd(5, 3, 6), Ts))]:
        ref = np.einsum(spec, *ops)
        np.testing.assert_allclose(P._chain(spec, *ops), ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_compress_reports_the_spectrum_of_every_cut():
    """The diagnostic `spectra` of `compress` records, for each bond the sweep
    cuts, the singular values of that bond; on a two-site MPS the one bond's
    values are those of the contracted two-site matrix (Eckart-Young setting),
    and recording them changes nothing in the result."""
    rng = np.random.default_rng(6)
    A = rng.standard_normal((1, 6, 5))
    B = rng.standard_normal((5, 7, 1))
    chi = 3
    sp = []
    m1, s1 = P.compress([A, B], chi, sp)
    m0, s0 = P.compress([A, B], chi)
    assert len(sp) == 1 and sp[0][0] == 1
    ref = np.linalg.svd((A.reshape(6, 5) @ B.reshape(5, 7)), compute_uv=False)
    np.testing.assert_allclose(sp[0][1], ref[:len(sp[0][1])], rtol=1e-12)
    assert s0 == s1 and all(np.array_equal(x, y) for x, y in zip(m0, m1))
    # no cut is recorded when chi covers every bond
    sp2 = []
    P.compress([A, B], 5, sp2)
    assert sp2 == []
