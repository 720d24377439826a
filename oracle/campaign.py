"""SR optimisation with exact statistics on small lattices (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The ground-state workflow of Sec. S-3 with the Monte Carlo averages replaced
by exact ones over the complete physical basis: at every step the Born
weights, E_loc and O of every configuration (``vmc``), S and F (Eq. S7), the
shifted solve and the update alpha <- alpha - lr x.  On a lattice small
enough to enumerate, this tests what the ansatz can reach free of sampling
noise, e.g. the paper's 3x3 Z2 + 2 hard-core bosons check (D = 6 against the
exact-diagonalisation energy).

    python -m oracle.campaign            # 3x3 Z2 + 2 bosons, D = 6, (h, g, J) = (1, 0.33, 0.5)
    python -m oracle.campaign vison      # 4x4 Z2, g = 0.1, D = 4: vison dynamics vs exact evolution
"""

from __future__ import annotations

import argparse
import json
import time

import numpy as np

import synth

from . import peps as P
from . import vmc
from .lattice import Lattice


def sr_exact(lat: Lattice, model: vmc.Model, Dk, chi, params, n_steps, lr=0.1, shift=1e-4, basis=None,
             on_step=None):
    """n_steps SR updates with exact expectations.  Returns (params, energies
    per step, the energy of the returned parameters)."""
    basis = lat.physical_basis() if basis is None else basis
    energies = []
    for step in range(n_steps):
        pe = P.GIPEPS(lat, Dk, params)
        w = vmc.exact_weights(pe, basis, chi)
        E = np.array([vmc.local_energy(pe, model, b, chi) for b in basis])
        O = np.array([vmc.log_grad_dense(pe, b, chi) for b in basis])
        S, F, eb = vmc.sr_matrices(O, E, w)
        energies.append(eb.real)
        if on_step:
            on_step(step, eb.real)
        x = vmc.sr_solve(S, F, shift)
        params = vmc.sr_update(params, x.real if not np.iscomplexobj(params) else x, lr)
    pe = P.GIPEPS(lat, Dk, params)
    w = vmc.exact_weights(pe, basis, chi)
    E = np.array([vmc.local_energy(pe, model, b, chi) for b in basis])
    return params, energies, float(np.real(w @ E))


def tvmc_exact(lat: Lattice, model: vmc.Model, Dk, chi, params, dt, n_steps, shift=1e-6, basis=None,
               on_step=None):
    """n_steps two-stage tVMC steps (Eqs. S6-S8) with exact expectations:
    alpha_dot = -i (S + shift)^-1 F, then alpha += c_1 dt alpha_dot and, at
    the new parameters, alpha += c_2 dt alpha_dot.  on_step(step, params)
    after every time step.  Returns the parameters (complex)."""
    basis = lat.physical_basis() if basis is None else basis
    params = np.asarray(params, dtype=np.complex128)
    for step in range(n_steps):
        for c in (vmc.TDVP_C1, vmc.TDVP_C2):
            pe = P.GIPEPS(lat, Dk, params)
            w = vmc.exact_weights(pe, basis, chi)
            E = np.array([vmc.local_energy(pe, model, b, chi) for b in basis])
            O = np.array([vmc.log_grad_dense(pe, b, chi) for b in basis])
            S, F, _ = vmc.sr_matrices(O, E, w)
            params = params + c * dt * vmc.tdvp_velocity(S, F, shift)
        if on_step:
            on_step(step, params)
    return params


def psi_vector(lat: Lattice, Dk, params, basis):
    """Normalised exact amplitudes of the PEPS on the basis."""
    pe = P.GIPEPS(lat, Dk, params)
    v = np.array([P.contract_exact(pe.sampled_network(b)) for b in basis], dtype=np.complex128)
    return v / np.linalg.norm(v)


def vison_run(L=4, g=0.1, Dk=2, gs_steps=200, dt=0.01, n_steps=100, seed=7, plaquettes=((0, 0), (1, 1), (2, 2))):
    """The vison check of the real-time study at L x L: an SR ground state
    (exact statistics), sigma_z on the bottom-left vertical link, exact-
    statistics tVMC, and <P + P^dag> on `plaquettes` against the exact
    evolution of the same initial state.  Prints one JSON line per step."""
    from . import dynamics as dyn

    lat = Lattice(L, L, 2)
    model = vmc.Model(h=1.0, g=g)
    chi = Dk ** (L // 2)
    basis = lat.physical_basis()
    H = lat.hamiltonian_matrix(basis, model.h, model.g)
    e_ed = np.linalg.eigvalsh(H)[0] / lat.n_s
    _, n = P.layout(lat, Dk)
    gs, _, e = sr_exact(lat, model, Dk, chi, 0.5 * synth.tensor_entries(seed, n, False), gs_steps, basis=basis)
    print(json.dumps({"ground_state_e_site": e / lat.n_s, "ed_e_site": e_ed}), flush=True)
    v = P.link_clock_params(P.GIPEPS(lat, Dk, gs), 0, 0, 2)
    psi0 = psi_vector(lat, Dk, v, basis)
    mats = [dyn.plaquette_matrix(lat, basis, x, y) for (x, y) in plaquettes]
    worst = [0.0]

    def report(step, params):
        t = (step + 1) * dt
        psi = psi_vector(lat, Dk, params, basis)
        ex = dyn.evolve(H, psi0, [t])[0]
        a = [float(dyn.expectation(psi, M).real) for M in mats]
        b = [float(dyn.expectation(ex, M).real) for M in mats]
        worst[0] = max(worst[0], max(abs(p - q) for p, q in zip(a, b)))
        print(json.dumps({"t": round(t, 6), "tvmc": a, "exact": b, "fidelity": float(abs(np.vdot(ex, psi)))}),
              flush=True)

    tvmc_exact(lat, model, Dk, chi, v, dt, n_steps, basis=basis, on_step=report)
    print(json.dumps({"max_abs_deviation": worst[0]}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("mode", nargs="?", default="boson", choices=["boson", "vison"])
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--lr", type=float, default=0.1)
    ap.add_argument("--seed", type=int, default=5)
    args = ap.parse_args()
    if args.mode == "vison":
        vison_run()
        return
    lat = Lattice(3, 3, 2, matter=True)
    model = vmc.Model(h=1.0, g=0.33, J=0.5)
    Dk, chi = 3, 3
    basis = lat.physical_basis(n_bosons=2)
    e_ed = np.linalg.eigvalsh(lat.hamiltonian_matrix(basis, model.h, model.g, model.J))[0] / lat.n_s
    _, n = P.layout(lat, Dk)
    t0 = time.time()

    def report(step, e):
        if step % 50 == 0:
            print(json.dumps({"step": step, "e_site": e / lat.n_s, "err": e / lat.n_s - e_ed,
                              "seconds": round(time.time() - t0, 1)}), flush=True)

    _, _, e = sr_exact(lat, model, Dk, chi, 0.5 * synth.tensor_entries(args.seed, n, False), args.steps,
                       lr=args.lr, basis=basis, on_step=report)
    print(json.dumps({"final_e_site": e / lat.n_s, "ed_e_site": e_ed, "err": e / lat.n_s - e_ed}))


if __name__ == "__main__":
    main()
