"""Planted mistakes: each plausible error in the oracle fails at least one pin.

Each case rewrites one expression of one oracle function, installs the
altered function with monkeypatch (on the CPU, in this process only) and runs
a pin from the oracle's own test modules, which must then fail.  The text to
replace must occur exactly once in the function's source, so a refactor of
the oracle makes this test fail loudly instead of checking nothing.  The
unaltered oracle passes the same pins in test_oracle_model.py,
test_oracle_peps.py and test_oracle_vmc.py.
"""

import inspect
import textwrap

import pytest

from oracle import dynamics as DY
from oracle import lattice as L
from oracle import peps as P
from oracle import rng
from oracle import schwinger as SW
from oracle import vmc

import test_oracle_dynamics as TD
import test_oracle_model as TM
import test_oracle_peps as TP
import test_oracle_schwinger as TS
import test_oracle_vmc as TV


def plant(monkeypatch, owner, name, old, new):
    """Replace ``owner.name`` by a copy of it whose source has ``old`` -> ``new``."""
    fn = getattr(owner, name)
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, f"{name}: expected exactly one {old!r}"
    ns = dict(vars(inspect.getmodule(fn)))
    exec(compile(src.replace(old, new), f"<{name} with a planted mistake>", "exec"), ns)
    monkeypatch.setattr(owner, name, ns[name])


def _schwinger_chain():
    L, m, J, g = 8, 0.2, 1.0, 0.5
    H, B = SW.hamiltonian(L, m, J, g, 4)
    return L, m, J, g, H, B, tuple(SW.charges(L))


# (case id, owner, function, original text, planted text, pin that must fail;
#  each pin is called with the monkeypatch fixture)
CASES = [
    # Hamiltonian, Eqs. (2-5)
    ("z2-plaquette-counted-once", L.Lattice, "off_diagonal", "-2.0 * h", "-h",
     lambda mp: TM.test_ed_pin_z2_hardcore_bosons_3x3()),
    ("electric-term-halved", L.Lattice, "diagonal_energy", "2.0 - 2.0 * np.cos", "1.0 - np.cos",
     lambda mp: TM.test_ed_pin_z2_hardcore_bosons_3x3()),
    # Gauss law, Eq. (1), and the moves that preserve it
    ("gauss-law-signs", L.Lattice, "gauss_residual", "p + nl + nd - nr - nu", "p + nl - nd - nr + nu",
     lambda mp: TM.test_physical_basis_equals_brute_force(3, 2, 3, False, None)),
    ("gauss-law-ignores-background-charge", L.Lattice, "gauss_residual", " - self.Q[y, x]) % self.N", ") % self.N",
     lambda mp: TM.test_physical_basis_equals_brute_force(3, 2, 3, False, [[1, 0, 0], [0, 0, 2]])),
    ("plaquette-orientation", L.Lattice, "plaquette", "c[self.hi(x, y + 1)] - t", "c[self.hi(x, y + 1)] + t",
     lambda mp: TM.test_moves_preserve_gauss_law(3)),
    ("hop-lowers-instead-of-raising", L.Lattice, "hop", "c[li] = (c[li] + 1) % self.N",
     "c[li] = (c[li] - 1) % self.N", lambda mp: TM.test_moves_preserve_gauss_law(3)),
    ("block-selection-leg-signs", P, "block_id", "tot = p + sum(", "tot = p - sum(",
     lambda mp: TP.test_gi_peps_vanishes_off_gauss_and_matches_sampled_network(3, 1, True, 2, 2)),
    ("leg-values-up-down-swapped", L.Lattice, "leg_values", "return nl, nr, nd, nu", "return nl, nr, nu, nd",
     lambda mp: TM.test_physical_basis_equals_brute_force(3, 2, 3, False, None)),
    ("uneven-sectors-sized-by-one-degeneracy", P, "layout", "d = tuple(dq[ch[i]] if has[i] else 1 for i in range(4))",
     "d = tuple(dq[0] if has[i] else 1 for i in range(4))", lambda mp: TP.test_uneven_sector_parameter_count()),
    # counter-based generator
    ("splitmix-shift", rng, "mix64", "z ^ (z >> 30)", "z ^ (z >> 31)", lambda mp: TM.test_splitmix64_reference_vector()),
    # boundary MPS (Sec. S-2)
    ("absorb-transposed-bond", P, "absorb", '"adb,lrdu->alubr"', '"adb,lrdu->laubr"',
     lambda mp: TP.test_boundary_mps_exact_when_chi_reaches_bound(6, 5, 2, 2, False)),
    ("compress-drops-a-singular-value", P, "compress", "k = min(chi, len(S))",
     "k = max(1, min(chi, len(S)) - 1)",
     lambda mp: TP.test_boundary_mps_exact_when_chi_reaches_bound(6, 5, 2, 2, False)),
    ("compress-drops-singular-weights", P, "compress", "U[:, :k] * S[:k]", "U[:, :k]",
     lambda mp: TP.test_two_site_compression_is_eckart_young()),
    ("strip-rows-swapped", P, "contract_strip", '"aijb,adA,iIdm,jJmu,buB->AIJB"', '"aijb,adA,iIdm,jJmu,buB->AJIB"',
     lambda mp: TV.test_local_energy_equals_H_psi_over_psi(4, 4, 2, 2, False, 24)),
    ("compress-log-norm-halved", P, "compress", "return mps, float(np.log(nrm))", "return mps, float(np.log(nrm)) / 2",
     lambda mp: TP.test_boundary_mps_exact_when_chi_reaches_bound(6, 5, 2, 2, False)),
    ("amplitude-drops-environment-scale", vmc, "amplitude", "return s + float(np.log(abs(val)))",
     "return float(np.log(abs(val)))", lambda mp: TP.test_boundary_mps_exact_when_chi_reaches_bound(6, 5, 2, 2, False)),
    ("variational-right-env-without-conjugate", P, "compress_variational",
     'np.einsum("bdc,ade,ce->ba", B[i].conj(), A[i], env_next)', 'np.einsum("bdc,ade,ce->ba", B[i], A[i], env_next)',
     lambda mp: TP.test_variational_compression_improves_on_svd_and_never_gets_worse(6, 2, 8, 3, True)),
    ("variational-lq-factor-untransposed", P, "compress_variational",
     "B[i] = Q.T.reshape(Q.shape[1], d, c)", "B[i] = Q.reshape(Q.shape[1], d, c)",
     lambda mp: TP.test_variational_compression_is_exact_without_truncation()),
    ("exact-evolution-time-reversed", DY, "evolve", "np.exp(-1j * evals * t)", "np.exp(1j * evals * t)",
     lambda mp: TD.test_evolution_matches_the_matrix_exponential_and_conserves()),
    # (1+1)D Schwinger model (End Matter)
    ("schwinger-electric-term-not-squared", SW, "hamiltonian", "g * np.sum(fields(s, Q) ** 2)",
     "g * np.sum(fields(s, Q))", lambda mp: TS.test_static_limit_is_the_brute_force_minimum()),
    ("schwinger-step-not-halved", SW, "evolve", "half = tau / 2.0", "half = tau",
     lambda mp: TS.test_real_time_follows_the_exact_evolution(_schwinger_chain())),
    ("schwinger-last-mass-dropped", SW, "_bond_gate", "(mx[x + 1] * n2 if x + 1 == L - 1 else 0.0)", "0.0",
     lambda mp: TS.test_imaginary_time_reaches_the_ground_energy(_schwinger_chain())),
    # E_loc, Eq. (S2)
    ("eloc-z2-factor", vmc, "local_energy", "amp = -2.0 * model.h if", "amp = -1.0 * model.h if",
     lambda mp: TV.test_local_energy_equals_H_psi_over_psi(4, 4, 2, 2, False, 24)),
    ("eloc-missing-plaquette-dagger", vmc, "local_energy", "powers = (1,) if lat.N == 2 else (1, lat.N - 1)",
     "powers = (1,)", lambda mp: TV.test_local_energy_equals_H_psi_over_psi(3, 3, 3, 2, True, 81)),
    ("eloc-hop-sign", vmc, "local_energy", "e += model.J * _strip_value", "e -= model.J * _strip_value",
     lambda mp: TV.test_local_energy_with_matter_hops()),
    ("eloc-horizontal-hop-sign", vmc, "local_energy", "e += model.J * _row_value", "e -= model.J * _row_value",
     lambda mp: TV.test_local_energy_with_matter_hops()),
    # O = d ln psi / d A (Eq. S3)
    ("log-grad-not-divided-by-psi", vmc, "log_grad", "P.row_site_environment(Bm, rows[r], Tm, x) / val",
     "P.row_site_environment(Bm, rows[r], Tm, x)", lambda mp: TV.test_log_grad_matches_finite_differences(False)),
    ("log-grad-conjugated", vmc, "log_grad", "P.row_site_environment(Bm, rows[r], Tm, x) / val",
     "np.conj(P.row_site_environment(Bm, rows[r], Tm, x) / val)",
     lambda mp: TV.test_log_grad_matches_finite_differences(True)),
    # Metropolis rule (Sec. S-1)
    ("metropolis-ratio-not-squared", vmc, "_accept", "abs(den) ** 2 < abs(num) ** 2", "abs(den) < abs(num)",
     lambda mp: TV.test_sampler_histogram_matches_born_weights(3, 3, 2, 0.05)),
    ("proposal-without-inverse-power", rng, "power", "return 1 + word(seed, chain, counter) % (N - 1)",
     "return 1", lambda mp: TV.test_sampler_histogram_matches_born_weights(3, 2, 3, 0.05)),
    ("plaquette-pass-environment-from-stale-rows", vmc, "sweep",
     "        rows = peps.sampled_network(cfg)\n        Bm, _ = P.compress(P.absorb(Bm, rows[r]), chi)",
     "        Bm, _ = P.compress(P.absorb(Bm, rows[r]), chi)",
     lambda mp: TV.test_sampler_histogram_matches_born_weights(3, 4, 2, 0.1)),
    ("plaquette-pass-environment-from-stale-rows-ratios", vmc, "sweep",
     "        rows = peps.sampled_network(cfg)\n        Bm, _ = P.compress(P.absorb(Bm, rows[r]), chi)",
     "        Bm, _ = P.compress(P.absorb(Bm, rows[r]), chi)",
     lambda mp: TV.test_sweep_ratios_equal_exact_amplitude_ratios(4, 4, 3, False, mp)),
    ("horizontal-hop-pass-environment-from-stale-rows", vmc, "sweep",
     "            rows = peps.sampled_network(cfg)\n            Tm, _ = P.compress(",
     "            Tm, _ = P.compress(",
     lambda mp: TV.test_sweep_ratios_equal_exact_amplitude_ratios(4, 4, 2, True, mp)),
    ("vertical-hop-pass-environment-from-stale-rows", vmc, "sweep",
     "            rows = peps.sampled_network(cfg)\n            Bm, _ = P.compress(P.absorb(Bm, rows[r]), chi)",
     "            Bm, _ = P.compress(P.absorb(Bm, rows[r]), chi)",
     lambda mp: TV.test_sweep_ratios_equal_exact_amplitude_ratios(4, 4, 2, True, mp)),
    ("hop-pass-row-value-on-wrong-row", vmc, "sweep",
     "_row_value(peps, c2, r, Bm, Tm), _row_value(peps, cfg, r, Bm, Tm)",
     "_row_value(peps, c2, r, Bm, Tm), _row_value(peps, c2, r, Bm, Tm)",
     lambda mp: TV.test_sweep_ratios_equal_exact_amplitude_ratios(3, 4, 3, True, mp)),
    # SR / tVMC (Eqs. S3, S6-S8)
    ("horizontal-hop-ratio-inverted", vmc, "sweep",
     "_accept(u, _row_value(peps, c2, r, Bm, Tm), _row_value(peps, cfg, r, Bm, Tm))",
     "_accept(u, _row_value(peps, cfg, r, Bm, Tm), _row_value(peps, c2, r, Bm, Tm))",
     lambda mp: TV.test_sampler_histogram_matches_born_weights_with_matter(3, 2, n_sweeps=60)),
    ("vertical-hops-never-proposed", vmc, "sweep", "c2 = lat.hop(cfg, x, r, 2)", "c2 = None",
     lambda mp: TV.test_sampler_histogram_matches_born_weights_with_matter(2, 3, n_sweeps=60)),
    ("sr-matrix-missing-conjugate", vmc, "sr_matrices", "(O.conj().T * w) @ O", "(O.T * w) @ O",
     lambda mp: TV.test_cg_equals_dense_solve_and_residual()),
    ("cg-direction-update", vmc, "cg_solve", "(rs_new / rs) * p", "(rs / rs_new) * p",
     lambda mp: TV.test_cg_equals_dense_solve_and_residual()),
    ("sr-force-without-mean-subtraction", vmc, "sr_matrices", " - Obar.conj() * Ebar", "",
     lambda mp: TV.test_tvmc_two_stage_follows_exact_evolution()),
    ("sr-update-ascends", vmc, "sr_update", "params - lr * x", "params + lr * x",
     lambda mp: TV.test_sr_step_lowers_exact_energy()),
    ("cg-step-length", vmc, "cg_solve", "alpha = rs / np.vdot(p, Ap).real", "alpha = rs / np.vdot(Ap, Ap).real",
     lambda mp: TV.test_cg_equals_dense_solve_and_residual()),
    ("born-weights-not-squared", vmc, "exact_weights", "np.exp(2.0 * (la - la.max()))", "np.exp(la - la.max())",
     lambda mp: TV.test_expectation_value_and_variational_bound()),
    ("tdvp-time-direction", vmc, "tdvp_velocity", "-1j * sr_solve", "1j * sr_solve",
     lambda mp: TV.test_tvmc_two_stage_follows_exact_evolution()),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(case, monkeypatch):
    _, owner, name, old, new, pin = case
    plant(monkeypatch, owner, name, old, new)
    with pytest.raises(AssertionError):
        pin(monkeypatch)
