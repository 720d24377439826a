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


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--lr", type=float, default=0.1)
    ap.add_argument("--seed", type=int, default=5)
    args = ap.parse_args()
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
