"""Variational Monte Carlo estimators for the GCF PEPS (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows Sec. S-1 (Eqs. S1-S3), Sec. S-2 (sampling) and Sec. S-3 (Eqs. S6-S8).

Environments.  For a configuration s with sampled rows W_0..W_{Ly-1}
(``peps.GIPEPS.sampled_network``), B[r] is the boundary MPS of rows 0..r
absorbed bottom-up and T[r] that of rows r..Ly-1 absorbed top-down, each
compressed to chi (``peps.compress``).

* amplitude       psi(s) = <B[Ly-2] | W_{Ly-1}>, contracted exactly.
* plaquette ratio for the plaquette with lower-left corner (x, r) uses the
  strip value  psi_r(s) = <B[r-1] | W_r W_{r+1} | T[r+2]>  with the same
  environments (those of s) in numerator and denominator.
* hop ratio: a horizontal hop in row r uses <B[r-1] | W_r | T[r+1]>, a
  vertical hop between rows r and r+1 uses the strip value above.
* log-derivative O_x = (d psi_r / d A~_x) / psi_r with psi_r the row value
  <B[r-1] | W_r | T[r+1]> (exact for fixed environments).

Local energy, Eq. (S2): E_loc(s) = sum_{s'} <s|H|s'> psi(s')/psi(s), i.e.
    diag(s) - h sum_x [psi(P_x s) + psi(P_x^dag s)] / psi(s)
           + J sum_{hops} psi(s')/psi(s)
(for N = 2 the plaquette term is -2h psi(P_x s)/psi(s)).

Gradient / SR (Eq. S3 is garbled in the source; read as the standard form):
    F_m  = <O_m^* E_loc> - <O_m^*><E_loc>
    S_mn = <O_m^* O_n> - <O_m^*><O_n>                         (Eq. S7)
SR step: alpha <- alpha - lr (S + lambda I)^{-1} F.
tVMC (Eqs. S6, S8): alpha_dot = -i (S + lambda I)^{-1} F;
    alpha_1 = alpha + c_1 dt alpha_dot(alpha),
    alpha(t+dt) = alpha_1 + c_2 dt alpha_dot(alpha_1),  c_{1,2} = (1 +- i)/2.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import peps as P
from . import rng
from .lattice import Lattice


@dataclass
class Model:
    """Couplings of Eqs. (3)-(5) in the paper's form."""
    h: float = 1.0
    g: float = 0.0
    J: float = 0.0
    m: float = 0.0


def _close(mps):
    """Contract an MPS whose physical legs all have dimension 1 to a scalar."""
    v = np.ones((1,))
    for M in mps:
        v = np.tensordot(v, M[:, 0, :], axes=(0, 0))
    return v.reshape(-1)[0]


def environments(peps: P.GIPEPS, cfg, chi):
    rows = peps.sampled_network(cfg)
    if rows is None:
        return None, None, None
    return rows, P.bottom_envs(rows, chi), P.top_envs(rows, chi)


def amplitude(peps: P.GIPEPS, cfg, chi, spectra=None, dtype=None):
    """(log|psi|, arg psi) of the boundary-MPS amplitude; (-inf, 0) if s is
    unphysical (its amplitude is exactly zero, Sec. S-2).  `spectra`, if a
    list, receives the singular values of every cut the bottom environments
    make (diagnostic, see `peps.compress`).  `dtype` (e.g. np.float32 or
    np.complex64), if given, runs the same steps in that type, with NumPy's
    LAPACK routines of that precision: its distance from the FP64 result
    measures how sensitive this amplitude is to rounding at that precision."""
    rows = peps.sampled_network(cfg)
    if rows is None:
        return -np.inf, 0.0
    if dtype is not None:
        rows = [[w.astype(dtype) for w in row] for row in rows]
    Ly = len(rows)
    Benv = P.bottom_envs(rows[:-1], chi, spectra)
    Bm, s = Benv[Ly - 2]
    val = _close(P.absorb(Bm, rows[Ly - 1]))
    if val == 0:
        return -np.inf, 0.0
    return s + float(np.log(abs(val))), float(np.angle(val))


def _strip_value(peps, cfg, r, Bm, Tm):
    lat = peps.lat
    b1 = [peps.selected_block(cfg, x, r)[1] for x in range(lat.Lx)]
    b2 = [peps.selected_block(cfg, x, r + 1)[1] for x in range(lat.Lx)]
    return P.contract_strip(Bm, b1, b2, Tm)


def _row_value(peps, cfg, r, Bm, Tm):
    row = [peps.selected_block(cfg, x, r)[1] for x in range(peps.lat.Lx)]
    return P.contract_row(Bm, row, Tm)


def local_energy(peps: P.GIPEPS, model: Model, cfg, chi):
    """E_loc(s), Eq. (S2), with strip/row ratios on the environments of s."""
    lat = peps.lat
    rows, Benv, Tenv = environments(peps, cfg, chi)
    if rows is None:
        raise ValueError("configuration violates the Gauss law")
    e = complex(lat.diagonal_energy(cfg, model.g, model.m))
    for r in range(lat.Ly - 1):
        Bm, Tm = Benv[r - 1][0], Tenv[r + 2][0]
        den = P.contract_strip(Bm, rows[r], rows[r + 1], Tm)
        for x in range(lat.Lx - 1):
            powers = (1,) if lat.N == 2 else (1, lat.N - 1)
            amp = -2.0 * model.h if lat.N == 2 else -model.h
            for t in powers:
                c2 = lat.plaquette(cfg, x, r, t)
                e += amp * _strip_value(peps, c2, r, Bm, Tm) / den
        if lat.matter and model.J != 0.0:
            for x in range(lat.Lx):
                c2 = lat.hop(cfg, x, r, 2)
                if c2 is not None:
                    e += model.J * _strip_value(peps, c2, r, Bm, Tm) / den
    if lat.matter and model.J != 0.0:
        for r in range(lat.Ly):
            Bm, Tm = Benv[r - 1][0], Tenv[r + 1][0]
            den = P.contract_row(Bm, rows[r], Tm)
            for x in range(lat.Lx - 1):
                c2 = lat.hop(cfg, x, r, 1)
                if c2 is not None:
                    e += model.J * _row_value(peps, c2, r, Bm, Tm) / den
    return e


def log_grad(peps: P.GIPEPS, cfg, chi):
    """Per vertex (row-major): (block id, O_x) with O_x = d ln psi_r / d A~_x."""
    lat = peps.lat
    rows, Benv, Tenv = environments(peps, cfg, chi)
    if rows is None:
        raise ValueError("configuration violates the Gauss law")
    out = []
    for r in range(lat.Ly):
        Bm, Tm = Benv[r - 1][0], Tenv[r + 1][0]
        val = P.contract_row(Bm, rows[r], Tm)
        for x in range(lat.Lx):
            bid, _ = peps.selected_block(cfg, x, r)
            out.append((bid, P.row_site_environment(Bm, rows[r], Tm, x) / val))
    return out


def log_grad_dense(peps: P.GIPEPS, cfg, chi):
    """O(s) as a dense vector over all parameters (zeros off the selected blocks)."""
    vec = np.zeros(peps.n_params, dtype=np.complex128)
    for v, (bid, blk) in enumerate(log_grad(peps, cfg, chi)):
        a = peps.verts[v].block_offsets[bid]
        vec[a:a + blk.size] = blk.reshape(-1)
    return vec if np.iscomplexobj(peps.params) else vec.real


def log_grad_through_truncation(peps: P.GIPEPS, cfg, chi, eps=1e-6):
    """d ln psi_chi(s) / d theta for the selected blocks, where psi_chi is the
    boundary-MPS amplitude with its chi truncations: the environments move
    with the parameters too (the adjoint *through* the truncation).  The
    definition written out: central differences of ln psi_chi in every
    selected parameter (real and imaginary parts for complex tensors),
    ln psi = log|psi| + i arg psi.  Dense over all parameters, zeros
    elsewhere.  Slow: two amplitudes per parameter; small lattices only."""
    base = log_grad_dense(peps, cfg, chi)
    sel = np.nonzero(base)[0]
    cplx = np.iscomplexobj(peps.params)
    out = np.zeros(peps.n_params, dtype=np.complex128)

    def lnpsi(params):
        la, ph = amplitude(P.GIPEPS(peps.lat, peps.Dk, params), cfg, chi)
        return la + 1j * ph

    for k in sel:
        d = []
        for step in ((eps, 1j * eps) if cplx else (eps,)):
            pp, pm = peps.params.copy(), peps.params.copy()
            pp[k] += step
            pm[k] -= step
            diff = lnpsi(pp) - lnpsi(pm)
            diff = diff.real + 1j * np.angle(np.exp(1j * diff.imag))  # phase difference modulo 2 pi
            d.append(diff / (2 * eps))
        # holomorphic derivative: d/dtheta = (d/dRe) for a real step; for complex
        # tensors the imaginary step gives i d/dtheta, so average the two
        out[k] = d[0] if not cplx else 0.5 * (d[0] - 1j * d[1])
    return out if cplx else out.real


# ---------------------------------------------------------------------------
# Sequential Metropolis sweep (Sec. S-1 acceptance rule, Sec. S-2 moves/order)
# ---------------------------------------------------------------------------

def n_slots(lat: Lattice):
    return 2 * lat.n_plaquettes + ((lat.n_h + lat.n_v) if lat.matter else 0)


def _accept(u, num, den):
    """Metropolis: accept iff u < |psi(s1)|^2 / |psi(s0)|^2 (division-free)."""
    return u * abs(den) ** 2 < abs(num) ** 2


def sweep(peps: P.GIPEPS, cfg, chi, seed, chain, w):
    """One Monte Carlo sweep of chain ``chain``, sweep index ``w``.

    Plaquettes: row pairs bottom to top, plaquettes left to right, P^t with
    t drawn in [1, N-1]; bottom environment advanced after each row pair; top
    environments from the configuration at the start of the pass.
    Matter: then horizontal links (rows top to bottom, links left to right)
    with 3-layer row values, then vertical links (row pairs bottom to top,
    columns left to right) with strip values.
    Returns (new cfg, accepted moves, proposed moves).
    """
    lat = peps.lat
    Lx, Ly, N = lat.Lx, lat.Ly, lat.N
    base = w * n_slots(lat)
    cfg = np.array(cfg, dtype=np.int64)
    acc = prop = 0

    rows = peps.sampled_network(cfg)
    Tenv = P.top_envs(rows, chi)
    Bm = P.trivial_mps(Lx, peps.params.dtype)
    for r in range(Ly - 1):
        Tm = Tenv[r + 2][0]
        for x in range(Lx - 1):
            j = r * (Lx - 1) + x
            t = rng.power(seed, chain, base + 2 * j, N)
            u = rng.uniform(seed, chain, base + 2 * j + 1)
            c2 = lat.plaquette(cfg, x, r, t)
            num = _strip_value(peps, c2, r, Bm, Tm)
            den = _strip_value(peps, cfg, r, Bm, Tm)
            prop += 1
            if _accept(u, num, den):
                cfg, acc = c2, acc + 1
        rows = peps.sampled_network(cfg)
        Bm, _ = P.compress(P.absorb(Bm, rows[r]), chi)

    if lat.matter:
        rows = peps.sampled_network(cfg)
        Benv = P.bottom_envs(rows, chi)
        Tm = P.trivial_mps(Lx, peps.params.dtype)
        for r in range(Ly - 1, -1, -1):
            Bm = Benv[r - 1][0]
            for x in range(Lx - 1):
                u = rng.uniform(seed, chain, base + 2 * lat.n_plaquettes + r * (Lx - 1) + x)
                c2 = lat.hop(cfg, x, r, 1)
                if c2 is None:
                    continue
                prop += 1
                if _accept(u, _row_value(peps, c2, r, Bm, Tm), _row_value(peps, cfg, r, Bm, Tm)):
                    cfg, acc = c2, acc + 1
            rows = peps.sampled_network(cfg)
            Tm, _ = P.compress(P.absorb(Tm, P.flip_row(rows[r])), chi)

        rows = peps.sampled_network(cfg)
        Tenv = P.top_envs(rows, chi)
        Bm = P.trivial_mps(Lx, peps.params.dtype)
        for r in range(Ly - 1):
            Tm = Tenv[r + 2][0]
            for x in range(Lx):
                u = rng.uniform(seed, chain, base + 2 * lat.n_plaquettes + lat.n_h + r * Lx + x)
                c2 = lat.hop(cfg, x, r, 2)
                if c2 is None:
                    continue
                prop += 1
                if _accept(u, _strip_value(peps, c2, r, Bm, Tm), _strip_value(peps, cfg, r, Bm, Tm)):
                    cfg, acc = c2, acc + 1
            rows = peps.sampled_network(cfg)
            Bm, _ = P.compress(P.absorb(Bm, rows[r]), chi)
    return cfg, acc, prop


def run_chain(peps: P.GIPEPS, model: Model, cfg, chi, seed, chain, n_sweeps, measure=True):
    """n_sweeps sweeps; after each, measure (log|psi|, arg psi, E_loc, O)."""
    out = []
    for w in range(n_sweeps):
        cfg, a, p = sweep(peps, cfg, chi, seed, chain, w)
        rec = {"cfg": cfg.copy(), "accepted": a, "proposed": p}
        if measure:
            rec["log_abs"], rec["phase"] = amplitude(peps, cfg, chi)
            rec["e_loc"] = local_energy(peps, model, cfg, chi)
            rec["O"] = log_grad(peps, cfg, chi)
        out.append(rec)
    return out


# ---------------------------------------------------------------------------
# Exact expectations (all configurations enumerated) and SR / tVMC
# ---------------------------------------------------------------------------

def exact_weights(peps: P.GIPEPS, basis, chi):
    """p(s) = |psi(s)|^2 / sum |psi|^2 over a complete physical basis (Eq. S1)."""
    la = np.array([amplitude(peps, b, chi)[0] for b in basis])
    w = np.exp(2.0 * (la - la.max()))
    return w / w.sum()


def sr_matrices(O, E, w):
    """S (Eq. S7) and F (Eq. S3, standard reading) from per-sample O (Ns x Np),
    E_loc (Ns) and weights w (Ns, summing to 1)."""
    O = np.asarray(O)
    E = np.asarray(E)
    w = np.asarray(w, dtype=np.float64)
    Obar = w @ O
    Ebar = w @ E
    S = (O.conj().T * w) @ O - np.outer(Obar.conj(), Obar)
    F = (O.conj().T * w) @ E - Obar.conj() * Ebar
    return S, F, Ebar


def sr_solve(S, F, diag_shift):
    """x = (S + lambda I)^{-1} F by a dense solve."""
    return np.linalg.solve(S + diag_shift * np.eye(S.shape[0]), F)


def cg_solve(matvec, F, tol=1e-12, maxiter=1000):
    """Conjugate gradient for a Hermitian positive-definite operator (Sec. S-3)."""
    x = np.zeros_like(F)
    r = F - matvec(x)
    p = r.copy()
    rs = np.vdot(r, r).real
    f2 = np.vdot(F, F).real
    it = 0
    while it < maxiter and rs > tol * tol * f2:
        Ap = matvec(p)
        alpha = rs / np.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rs_new = np.vdot(r, r).real
        p = r + (rs_new / rs) * p
        rs = rs_new
        it += 1
    return x, it


def sr_update(params, x, lr):
    return params - lr * x


TDVP_C1 = (1.0 + 1.0j) / 2.0
TDVP_C2 = (1.0 - 1.0j) / 2.0


def tdvp_velocity(S, F, diag_shift):
    """alpha_dot = -i (S + lambda I)^{-1} F  (Eq. S6 with F the gradient)."""
    return -1j * sr_solve(S, F, diag_shift)
