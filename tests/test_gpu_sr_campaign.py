"""A ground-state SR optimisation run through the library (Sec. S-3), checked
against the paper's exact-diagonalisation energy.

The paper's small-lattice check of the matter-coupled theory: Z2 gauge field +
2 hard-core bosons on the 3x3 open lattice, (h, g, J) = (1, 0.33, 0.5),
D = 6 (D_k = 3), where its optimised PEPS reaches -0.470713502(3) per site
against the ED energy -0.4707135061 (main text, paragraph on Z2 gauge theory
coupled to hard-core bosons; `tests/golden/ed_z2_hardcore_bosons_3x3.txt`).
chi = 3 is exact on three rows.

drivers.sr_optimize samples the chains with gcf_sample_batch (sampling in the
2-boson sector) and updates the tensors with gcf_sr_step, from the same start
as the oracle's exact-statistics campaign (`oracle/campaign.py`: 0.5 x the
seed-5 entries, lr = 0.1, diagonal shift 1e-4).  After the run the library's
tensors are read back and the state they define is contracted exactly by the
oracle on all 576 physical configurations, so the energy compared is the
variational energy of the optimised state, free of sampling error:

* it lies above the ED energy (variational principle);
* it is within 1e-3 per site of it, from 1.38 per site above at the start;
* the last step's sampled <E> is within 1e-4 per site of that exact energy.

The precision reached is printed beside the paper's.  The sampled
optimisation does not always reach it: in nine runs (FP64 and FP32, 4 or 8
sweeps per step, several seeds) five came within 1e-9 per site of the ED
energy, one 7.8e-7 above it, and three stopped 2.0e-4 to 3.7e-4 above it.
The three that stopped
show the signature of a sign structure the samples cannot move (the
fixed-node situation of real-valued VMC): the sampled <E> lies about 8e-6 per
site below the state's exact energy with an error bar near 1e-7, because the
configurations next to the state's nodes, where E_loc is large, have so small
a weight that a step's samples almost never hold one, so the sampled force
does not see them.  The oracle's exact-statistics SR from the same start
(`python -m oracle.campaign`) passes that level by step 100.  The FP32 form
is the one the throughput benchmark runs.
"""

import os

import numpy as np
import pytest

import synth
from oracle import peps as P
from oracle.lattice import Lattice

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PRECISION = "fp32"
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ed_z2_hardcore_bosons_3x3.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (s.strip() for s in line.split("=", 1))
                vals[k] = float(v) if "." in v or "e" in v else int(v)
    return vals


def _exact_energy(lat, Dk, params, basis, H):
    pe = P.GIPEPS(lat, Dk, params)
    v = np.array([P.contract_exact(pe.sampled_network(b)) for b in basis])
    return float(np.real(np.vdot(v, H @ v) / np.vdot(v, v)))


def test_sr_reaches_the_printed_ed_energy():
    import paper_2503_20566_gb300 as G
    from paper_2503_20566_gb300 import drivers

    gd = _golden()
    lat = Lattice(gd["Lx"], gd["Ly"], gd["N"], matter=True)
    Dk, chi, n_b = 3, 3, gd["n_bosons"]
    basis = lat.physical_basis(n_bosons=n_b)
    H = lat.hamiltonian_matrix(basis, gd["h"], gd["g"], gd["J"])
    e_ed = gd["energy_per_site"]
    _, n = P.layout(lat, Dk)
    params0 = 0.5 * synth.tensor_entries(5, n, False)
    ctx = G.Context(gd["N"], lat.Lx, lat.Ly, gd["N"] * Dk, chi, matter=True, h=gd["h"], g=gd["g"], J=gd["J"],
                    precision=PRECISION, seed=5)
    ctx.set_tensors(params0)
    e_start = _exact_energy(lat, Dk, ctx.get_tensors(), basis, H) / lat.n_s

    n_chains, n_sweeps, n_steps = 2048, 4, 600
    powers = synth.plaquette_powers(6, n_chains, lat.n_plaquettes, gd["N"])
    occ = synth.occupations(6, n_chains, lat.n_s, n_b)
    configs = ctx.init_configs(n_chains, occupations=torch.from_numpy(occ), powers=torch.from_numpy(powers))
    _, recs = drivers.sr_optimize(ctx, configs, n_steps=n_steps, n_sweeps=n_sweeps, seed=7, diag_shift=1e-4,
                                  lr=0.1, max_iter=200, tol=1e-10)
    e_final = _exact_energy(lat, Dk, ctx.get_tensors(), basis, H) / lat.n_s
    trace = {r["step"]: r["e_mean"] / lat.n_s for r in recs if r["step"] % 100 == 0 or r["step"] == n_steps - 1}
    tail = recs[-50:]
    e_tail = np.mean([r["e_mean"] for r in tail]) / lat.n_s
    err_tail = np.sqrt(np.mean([r["e_err"] ** 2 for r in tail]) / len(tail)) / lat.n_s
    print(f"{PRECISION}: start {e_start:.10f}, sampled <E>/site by step {trace}")
    print(f"{PRECISION}: optimised state, exact energy/site {e_final:.10f}; ED {e_ed:.10f}; "
          f"above ED by {e_final - e_ed:.3e} (paper's D=6 PEPS: -0.470713502(3)); "
          f"last 50 steps sampled {e_tail:.10f} +- {err_tail:.1e}; "
          f"seconds per step {np.mean([r['seconds'] for r in recs[10:]]):.4f}")
    assert e_final > e_ed - 1e-9, (e_final, e_ed)
    assert e_final - e_ed < 1e-3, (e_final, e_ed)
    assert abs(recs[-1]["e_mean"] / lat.n_s - e_final) < 1e-4, (recs[-1]["e_mean"] / lat.n_s, e_final)
