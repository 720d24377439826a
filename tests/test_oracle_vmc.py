"""Pins of the oracle's VMC layer.

* E_loc(s) equals (H psi)(s) / psi(s) computed from the exact-diagonalisation
  matrix and the exactly contracted amplitudes, per configuration (Eq. S2).
* Zero-variance principle (Sec. S-1): at the toric-code point (D_k = 1, all
  entries 1, g = 0) E_loc is the same for every configuration.
* O = d ln psi / d A~ equals central finite differences, both of the row value
  with fixed environments and of the full exact amplitude.
* The Metropolis sweep samples |psi|^2 (histograms on 3x3 and 3x4 Z2 and 3x2
  Z3, and with two hard-core bosons on 3x2 and 2x3 Z2, where the horizontal
  and the vertical hops move them); at exact chi every ratio it forms from its carried environments equals
  the exact amplitude ratio (plaquette and both hop passes); it conserves the
  Gauss law and the boson number.
* SR: CG equals the dense solve; an SR step lowers the exact energy.
* tVMC: the two-stage update with alpha_dot = -i (S+lambda)^{-1} F follows
  exact Schroedinger evolution exp(-iHt) (and not exp(+iHt)).
"""

import numpy as np
import pytest

import synth
from oracle import peps as P
from oracle import vmc
from oracle.lattice import Lattice

from test_oracle_peps import make_peps, random_physical


def exact_psi(pe, basis):
    return np.array([P.contract_exact(pe.sampled_network(b)) for b in basis])


@pytest.mark.parametrize("Lx,Ly,N,Dk,complex_,n_cfg", [(4, 4, 2, 2, False, 24), (3, 3, 3, 2, True, 81),
                                                       (4, 3, 4, 1, True, 30)])
def test_local_energy_equals_H_psi_over_psi(Lx, Ly, N, Dk, complex_, n_cfg):
    pe = make_peps(Lx, Ly, N, Dk, seed=12, complex_=complex_)
    lat = pe.lat
    model = vmc.Model(h=1.0, g=0.37)
    basis = lat.physical_basis()
    psi = exact_psi(pe, basis)
    H = lat.hamiltonian_matrix(basis, model.h, model.g)
    Hpsi = H @ psi
    chi = Dk ** (Lx // 2)
    sel = np.random.default_rng(0).choice(len(basis), size=min(n_cfg, len(basis)), replace=False)
    for i in sel:
        e = vmc.local_energy(pe, model, basis[i], chi)
        ref = Hpsi[i] / psi[i]
        assert abs(e - ref) <= 1e-9 * max(1.0, abs(ref))


def test_local_energy_with_matter_hops():
    pe = make_peps(3, 3, 2, 2, seed=21, matter=True)
    lat = pe.lat
    model = vmc.Model(h=1.0, g=0.33, J=0.5)
    basis = lat.physical_basis(n_bosons=2)
    psi = exact_psi(pe, basis)
    H = lat.hamiltonian_matrix(basis, model.h, model.g, model.J)
    Hpsi = H @ psi
    for i in np.random.default_rng(1).choice(len(basis), size=25, replace=False):
        e = vmc.local_energy(pe, model, basis[i], 2)
        assert abs(e - Hpsi[i] / psi[i]) <= 1e-9 * max(1.0, abs(Hpsi[i] / psi[i]))


def test_expectation_value_and_variational_bound():
    pe = make_peps(3, 3, 3, 2, seed=13)
    lat = pe.lat
    model = vmc.Model(h=1.0, g=0.375)
    basis = lat.physical_basis()
    psi = exact_psi(pe, basis)
    H = lat.hamiltonian_matrix(basis, model.h, model.g)
    # the oracle's Born weights (boundary-MPS amplitudes) against the Rayleigh
    # quotient of the exactly contracted state
    w = vmc.exact_weights(pe, basis, 2)
    e_mc = sum(w[i] * vmc.local_energy(pe, model, b, 2) for i, b in enumerate(basis))
    e_ed = (psi.conj() @ H @ psi) / (psi.conj() @ psi)
    assert abs(e_mc - e_ed) < 1e-10 * abs(e_ed)
    assert e_ed.real >= np.linalg.eigvalsh(H)[0] - 1e-12


@pytest.mark.parametrize("N", [2, 3])
def test_zero_variance_at_toric_code_point(N):
    lat = Lattice(4, 4, N)
    _, n = P.layout(lat, 1)
    pe = P.GIPEPS(lat, 1, np.ones(n))
    model = vmc.Model(h=0.8, g=0.0)
    for seed in range(6):
        cfg = random_physical(lat, seed)
        e = vmc.local_energy(pe, model, cfg, chi=1)
        assert abs(e - (-2.0 * model.h * lat.n_plaquettes)) < 1e-12


@pytest.mark.parametrize("complex_", [False, True])
def test_log_grad_matches_finite_differences(complex_):
    pe = make_peps(4, 4, 2, 2, seed=31, complex_=complex_)
    lat = pe.lat
    cfg = random_physical(lat, 4)
    chi = 4  # exact for Lx = 4, D_k = 2
    O = vmc.log_grad(pe, cfg, chi)
    la0, ph0 = vmc.amplitude(pe, cfg, chi)
    psi0 = np.exp(la0 + 1j * ph0)
    rng = np.random.default_rng(2)
    for v in rng.choice(lat.n_s, size=6, replace=False):
        x, y = v % lat.Lx, v // lat.Lx
        bid, blk = O[v]
        vl = pe.verts[v]
        for e in rng.choice(vl.block_size, size=3, replace=False):
            k = vl.offset + bid * vl.block_size + e
            eps = 1e-6
            pp, pm = pe.params.copy(), pe.params.copy()
            pp[k] += eps
            pm[k] -= eps
            ap = vmc.amplitude(P.GIPEPS(lat, 2, pp), cfg, chi)
            am = vmc.amplitude(P.GIPEPS(lat, 2, pm), cfg, chi)
            d = (np.exp(ap[0] + 1j * ap[1]) - np.exp(am[0] + 1j * am[1])) / (2 * eps) / psi0
            assert abs(blk.reshape(-1)[e] - d) <= 1e-6 * max(1.0, abs(d))


def test_log_grad_fixed_environment_finite_difference_truncated():
    """With chi below the exact bound, O is the derivative of the row value
    at fixed environments (the definition used on the GPU as well)."""
    pe = make_peps(6, 4, 2, 2, seed=33)
    lat = pe.lat
    cfg = random_physical(lat, 5)
    chi = 2
    rows, Benv, Tenv = vmc.environments(pe, cfg, chi)
    O = vmc.log_grad(pe, cfg, chi)
    r, x = 2, 3
    Bm, Tm = Benv[r - 1][0], Tenv[r + 1][0]
    val = P.contract_row(Bm, rows[r], Tm)
    bid, blk = O[r * lat.Lx + x]
    for idx in np.ndindex(*rows[r][x].shape):
        eps = 1e-6
        rp = [w.copy() for w in rows[r]]
        rm = [w.copy() for w in rows[r]]
        rp[x][idx] += eps
        rm[x][idx] -= eps
        d = (P.contract_row(Bm, rp, Tm) - P.contract_row(Bm, rm, Tm)) / (2 * eps) / val
        assert abs(blk[idx] - d) <= 1e-7 * max(1.0, abs(d))


@pytest.mark.parametrize("Lx,Ly,N,tv_max", [(3, 3, 2, 0.05), (3, 2, 3, 0.05), (3, 4, 2, 0.1)])
def test_sampler_histogram_matches_born_weights(Lx, Ly, N, tv_max):
    # Z3 also fixes the proposal: P^t with t uniform in [1, N-1] is symmetric
    # (P^t and its inverse P^(N-t) equally likely), P alone is not.  Four rows
    # (three row pairs, 64 states, hence the wider bound) fix the bottom
    # environment that the sweep carries from one row pair to the next.
    pe = make_peps(Lx, Ly, N, 2, seed=41)
    lat = pe.lat
    basis = lat.physical_basis()
    psi = exact_psi(pe, basis)
    target = np.abs(psi) ** 2 / np.sum(np.abs(psi) ** 2)
    index = {tuple(b): i for i, b in enumerate(basis)}
    counts = np.zeros(len(basis))
    n_chains, n_sweeps = 16, 150
    for c in range(n_chains):
        cfg = random_physical(lat, 100 + c)
        for w in range(n_sweeps):
            cfg, _, _ = vmc.sweep(pe, cfg, 2, seed=77, chain=c, w=w)
            if w >= 10:
                counts[index[tuple(cfg)]] += 1
    freq = counts / counts.sum()
    tv = 0.5 * np.abs(freq - target).sum()
    assert tv < tv_max, (tv, freq, target)


@pytest.mark.parametrize("Lx,Ly", [(3, 2), (2, 3)])
def test_sampler_histogram_matches_born_weights_with_matter(Lx, Ly, n_sweeps=150):
    # Two bosons in the 2-boson sector (60 physical states).  On 3x2 a boson
    # crosses between columns only by the horizontal hops (row values), on
    # 2x3 between rows only by the vertical hops (strip values); a hop
    # proposed in one direction only, or accepted with the wrong ratio,
    # leaves the histogram far from |psi|^2.  The bound is about twice the
    # total variation that 2240 independent draws from 60 states reach (the
    # planted-mistake test runs the pin with fewer sweeps: the mistakes miss
    # it by far more).
    pe = make_peps(Lx, Ly, 2, 2, seed=41, matter=True)
    lat = pe.lat
    basis = lat.physical_basis(n_bosons=2)
    psi = exact_psi(pe, basis)
    target = np.abs(psi) ** 2 / np.sum(np.abs(psi) ** 2)
    index = {tuple(b): i for i, b in enumerate(basis)}
    counts = np.zeros(len(basis))
    n_chains = 16
    for c in range(n_chains):
        cfg = random_physical(lat, 100 + c, n_bosons=2)
        for w in range(n_sweeps):
            cfg, _, _ = vmc.sweep(pe, cfg, 4, seed=77, chain=c, w=w)
            if w >= 10:
                counts[index[tuple(cfg)]] += 1
    freq = counts / counts.sum()
    tv = 0.5 * np.abs(freq - target).sum()
    assert tv < 0.08, (tv, freq, target)


@pytest.mark.parametrize("Lx,Ly,N,matter", [(4, 4, 3, False), (4, 4, 2, True), (3, 4, 3, True)])
def test_sweep_ratios_equal_exact_amplitude_ratios(Lx, Ly, N, matter, monkeypatch):
    """At exact chi every Metropolis ratio the sweep forms from its carried
    environments (plaquette pass, horizontal and vertical hop passes) equals
    psi(s') / psi(s) of the exactly contracted network.  The proposed s' is
    recorded from the move functions, the ratio from the acceptance rule."""
    pe = make_peps(Lx, Ly, N, 2, seed=45, matter=matter)
    lat = pe.lat
    nb = (4 if N == 2 else 3) if matter else 0  # the open lattice holds sum(p) = 0 mod N
    cfg = random_physical(lat, 7, n_bosons=nb)
    last, checked = {}, []
    plaquette, hop, accept = Lattice.plaquette, Lattice.hop, vmc._accept

    def rec_plaquette(self, c, x, y, t=1):
        out = plaquette(self, c, x, y, t)
        last["move"] = (np.array(c), out)
        return out

    def rec_hop(self, c, x, y, a):
        out = hop(self, c, x, y, a)
        last["move"] = (np.array(c), out)
        return out

    def rec_accept(u, num, den):
        s0, s1 = last.pop("move")
        ref = P.contract_exact(pe.sampled_network(s1)) / P.contract_exact(pe.sampled_network(s0))
        checked.append(abs(num / den - ref) / max(1.0, abs(ref)))
        return accept(u, num, den)

    monkeypatch.setattr(Lattice, "plaquette", rec_plaquette)
    monkeypatch.setattr(Lattice, "hop", rec_hop)
    monkeypatch.setattr(vmc, "_accept", rec_accept)
    chi = 2 ** (Lx // 2)
    n_acc = 0
    for w in range(2):
        cfg, acc, prop = vmc.sweep(pe, cfg, chi, seed=5, chain=0, w=w)
        n_acc += acc
    assert len(checked) >= 2 * lat.n_plaquettes and n_acc > 0
    assert max(checked) < 1e-9, max(checked)


def test_matter_sweep_conserves_gauss_and_boson_number():
    pe = make_peps(4, 3, 2, 2, seed=51, matter=True)
    lat = pe.lat
    cfg = random_physical(lat, 3, n_bosons=6)
    acc_tot = 0
    for w in range(4):
        cfg, acc, prop = vmc.sweep(pe, cfg, 4, seed=9, chain=0, w=w)
        acc_tot += acc
        assert lat.is_physical(cfg)
        assert cfg[lat.n_h + lat.n_v:].sum() == 6
        assert prop >= lat.n_plaquettes
    assert acc_tot > 0


def test_cg_equals_dense_solve_and_residual():
    g = np.random.default_rng(3)
    Ns, Np = 60, 25
    O = g.normal(size=(Ns, Np)) + 1j * g.normal(size=(Ns, Np))
    E = g.normal(size=Ns) + 0.1j * g.normal(size=Ns)
    w = np.full(Ns, 1.0 / Ns)
    S, F, _ = vmc.sr_matrices(O, E, w)
    assert np.allclose(S, S.conj().T)
    assert np.linalg.eigvalsh(S).min() > -1e-12
    x = vmc.sr_solve(S, F, 1e-4)
    assert np.linalg.norm((S + 1e-4 * np.eye(Np)) @ x - F) / np.linalg.norm(F) < 1e-10
    xc, it = vmc.cg_solve(lambda v: S @ v + 1e-4 * v, F, tol=1e-13)
    assert np.linalg.norm(xc - x) / np.linalg.norm(x) < 1e-9


def _exact_stats(pe, model, basis, chi):
    w = vmc.exact_weights(pe, basis, chi)
    E = np.array([vmc.local_energy(pe, model, b, chi) for b in basis])
    O = np.array([vmc.log_grad_dense(pe, b, chi) for b in basis])
    return w, E, O


def test_sr_step_lowers_exact_energy():
    pe = make_peps(3, 3, 2, 2, seed=61)
    lat = pe.lat
    model = vmc.Model(h=1.0, g=0.3)
    basis = lat.physical_basis()
    w, E, O = _exact_stats(pe, model, basis, 2)
    S, F, e0 = vmc.sr_matrices(O, E, w)
    x = vmc.sr_solve(S, F, 1e-4)
    pe2 = P.GIPEPS(lat, 2, vmc.sr_update(pe.params, x.real, 0.05))
    w2, E2, _ = _exact_stats(pe2, model, basis, 2)
    assert (w2 @ E2).real < e0.real - 1e-4


def test_tvmc_two_stage_follows_exact_evolution():
    """Reading of Eqs. (S6, S8): alpha_dot = -i (S+lambda)^-1 F and the two
    stages alpha += c dt alpha_dot with c = (1+i)/2 then (1-i)/2."""
    pe = make_peps(3, 3, 2, 2, seed=71, complex_=True)
    lat = pe.lat
    model = vmc.Model(h=1.0, g=0.4)
    basis = lat.physical_basis()
    H = lat.hamiltonian_matrix(basis, model.h, model.g)
    evals, evecs = np.linalg.eigh(H)
    psi0 = exact_psi(pe, basis)
    psi0 = psi0 / np.linalg.norm(psi0)
    dt, n_steps, shift = 0.02, 5, 1e-8
    params = pe.params.copy()
    for _ in range(n_steps):
        for c in (vmc.TDVP_C1, vmc.TDVP_C2):
            cur = P.GIPEPS(lat, 2, params)
            w, E, O = _exact_stats(cur, model, basis, 2)
            S, F, _ = vmc.sr_matrices(O, E, w)
            params = params + c * dt * vmc.tdvp_velocity(S, F, shift)
    psi_t = exact_psi(P.GIPEPS(lat, 2, params), basis)
    psi_t /= np.linalg.norm(psi_t)
    t = dt * n_steps
    fwd = evecs @ (np.exp(-1j * evals * t) * (evecs.conj().T @ psi0))
    bwd = evecs @ (np.exp(+1j * evals * t) * (evecs.conj().T @ psi0))
    f_fwd = abs(np.vdot(fwd, psi_t))
    f_bwd = abs(np.vdot(bwd, psi_t))
    assert f_fwd > 1 - 1e-5, f_fwd
    assert f_bwd < f_fwd - 1e-3


@pytest.mark.parametrize("complex_", [False, True])
def test_gradient_through_truncation_equals_o_at_exact_chi(complex_):
    """With chi at the exact bound nothing is truncated: the derivative with
    moving environments is the fixed-environment O."""
    pe = make_peps(4, 3, 2, 2, seed=35, complex_=complex_)
    cfg = random_physical(pe.lat, 6)
    full = vmc.log_grad_through_truncation(pe, cfg, chi=4)
    fixed = vmc.log_grad_dense(pe, cfg, chi=4)
    assert np.linalg.norm(full - fixed) <= 1e-6 * np.linalg.norm(fixed)


def test_gradient_through_truncation_differs_below_exact_chi():
    """Below the exact bound the environments depend on the parameters through
    the truncation, so the full derivative is not O; it is stable in the step."""
    pe = make_peps(6, 4, 2, 2, seed=37)
    cfg = random_physical(pe.lat, 7)
    full = vmc.log_grad_through_truncation(pe, cfg, chi=2, eps=1e-6)
    full2 = vmc.log_grad_through_truncation(pe, cfg, chi=2, eps=1e-5)
    fixed = vmc.log_grad_dense(pe, cfg, chi=2)
    assert np.linalg.norm(full - full2) <= 1e-5 * np.linalg.norm(full)
    assert np.linalg.norm(full - fixed) >= 1e-3 * np.linalg.norm(fixed)


def test_odd_z2_theory():
    """The odd-Z2 gauge theory (Q_x = 1 on every vertex; an even number of
    vertices on the open lattice): its physical basis is the brute-force
    filter, and E_loc equals (H psi)(s) / psi(s) there."""
    Lx, Ly = 4, 2
    lat = Lattice(Lx, Ly, 2, Q=np.ones((Ly, Lx), dtype=int))
    basis = lat.physical_basis()
    assert set(map(tuple, basis)) == set(map(tuple, lat.brute_force_physical()))
    assert len(basis) == 2 ** lat.n_plaquettes
    _, n = P.layout(lat, 2)
    pe = P.GIPEPS(lat, 2, synth.tensor_entries(47, n, False))
    model = vmc.Model(h=1.0, g=0.6)
    psi = exact_psi(pe, basis)
    Hpsi = lat.hamiltonian_matrix(basis, model.h, model.g) @ psi
    for i in range(len(basis)):
        e = vmc.local_energy(pe, model, basis[i], chi=4)
        assert abs(e - Hpsi[i] / psi[i]) <= 1e-9 * max(1.0, abs(Hpsi[i] / psi[i]))



def test_uneven_sectors_local_energy_and_log_grad():
    """Uneven charge sectors (degeneracies 2, 1, 1 for Z3): E_loc equals
    (H psi)(s) / psi(s), and O equals central differences of the amplitude."""
    pe = make_peps(3, 3, 3, (2, 1, 1), seed=17, complex_=True)
    lat = pe.lat
    model = vmc.Model(h=1.0, g=0.45)
    basis = lat.physical_basis()
    psi = exact_psi(pe, basis)
    Hpsi = lat.hamiltonian_matrix(basis, model.h, model.g) @ psi
    for i in range(0, len(basis), 5):
        e = vmc.local_energy(pe, model, basis[i], chi=2)
        assert abs(e - Hpsi[i] / psi[i]) <= 1e-9 * max(1.0, abs(Hpsi[i] / psi[i]))
    cfg = basis[7]
    O = vmc.log_grad_dense(pe, cfg, 2)
    la0, ph0 = vmc.amplitude(pe, cfg, 2)
    psi0 = np.exp(la0 + 1j * ph0)
    for k in np.nonzero(O)[0][::3]:
        pp, pm = pe.params.copy(), pe.params.copy()
        pp[k] += 1e-6
        pm[k] -= 1e-6
        ap = vmc.amplitude(P.GIPEPS(lat, pe.Dk, pp), cfg, 2)
        am = vmc.amplitude(P.GIPEPS(lat, pe.Dk, pm), cfg, 2)
        d = (np.exp(ap[0] + 1j * ap[1]) - np.exp(am[0] + 1j * am[1])) / 2e-6 / psi0
        assert abs(O[k] - d) <= 1e-6 * max(1.0, abs(d))


def test_amplitude_in_single_precision_follows_the_same_steps():
    """`amplitude(..., dtype=float32)` runs the oracle's steps in single
    precision: at exact chi it agrees with the FP64 amplitude to single
    precision rounding (and not to double), and the singular spectra it
    reports are those of the FP64 run to the same accuracy."""
    import synth

    lat = Lattice(4, 4, 2)
    _, n = P.layout(lat, 2)
    pe = P.GIPEPS(lat, 2, synth.round_to(synth.tensor_entries(17, n, False), "f32"))
    cfg = lat.config_from_powers(np.zeros((4, 4)), synth.plaquette_powers(18, 1, lat.n_plaquettes, 2)[0])
    la64, ph64 = vmc.amplitude(pe, cfg, 4)
    la32, ph32 = vmc.amplitude(pe, cfg, 4, dtype=np.float32)
    d = abs(np.exp((la32 - la64) + 1j * (ph32 - ph64)) - 1)
    assert 1e-12 < d < 1e-5
    sp64, sp32 = [], []
    vmc.amplitude(pe, cfg, 2, spectra=sp64)
    vmc.amplitude(pe, cfg, 2, spectra=sp32, dtype=np.float32)
    assert len(sp64) == len(sp32) > 0
    for (r, b, s64), (r2, b2, s32) in zip(sp64, sp32):
        assert (r, b) == (r2, b2) and s32.dtype == np.float32
        np.testing.assert_allclose(s32, s64, rtol=1e-4, atol=1e-5 * s64[0])
