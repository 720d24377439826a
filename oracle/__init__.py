"""Plain FP64 CPU oracle for the GCF-PEPS variational Monte Carlo hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it, and it never calls the CUDA library:
the two share no code.  Only the raw random numbers of ``synth`` feed both.

Everything here is written for a reader checking it against the paper
(Wu & Liu, "Accurate gauge-invariant tensor network simulations for Abelian
lattice gauge theory in (2+1)D"): slow, FP64 / complex128, NumPy only, with no
blocking, fusion or reordering beyond what the definitions state.

Modules
-------
lattice  Z_N lattice gauge theory: Gauss law (Eq. 1), Hamiltonian
         H = H_M + H_B + H_E (Eqs. 3-5), moves, enumeration, exact
         diagonalisation.
peps     Gauge-invariant PEPS (Eqs. 6-7), gauge canonical form (Eq. 9), the
         sampled single-layer network (Sec. S-2, Eq. S5), exact contraction and
         the boundary-MPS contraction with SVD truncation to chi; variational
         compression (Sec. S-2) as the alternative.
vmc      VMC estimators (Sec. S-1, Eqs. S1-S3), sequential Metropolis sweep
         (Sec. S-2), stochastic reconfiguration and the two-stage tVMC update
         (Sec. S-3, Eqs. S6-S8); the gradient of the truncated amplitude
         through the truncation (finite differences, small lattices).
dynamics Exact real-time evolution exp(-iHt) on small complete bases, plaquette
         and clock-operator matrices, the vison state (reference for tVMC).
schwinger (1+1)D Schwinger model (End Matter): exact diagonalisation and the GCF
         time evolution on a U(1)-symmetric MPS whose bond charges are the
         electric fields.
campaign SR optimisation with exact statistics on enumerable lattices (the
         ground-state workflow of Sec. S-3 free of sampling noise).
rng      The counter-based SplitMix64 generator used for the Metropolis draws
         (the oracle's own implementation of the published definition).

Parity pins: every function is pinned by tests in ``tests/test_oracle_*.py``
against closed forms, brute force or numbers printed in the paper, and
``tests/test_oracle_planted.py`` checks that planted mistakes fail them;
functions without such a pin say "parity unpinned" in their docstring.
"""
