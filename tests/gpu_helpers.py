"""Shared helpers of the GPU parity tests (oracle on one side, C ABI on the other)."""

import numpy as np

import synth
from oracle import peps as P
from oracle import vmc
from oracle.lattice import Lattice

# Tolerances.  The FP32 bound is the stated one for FP32 amplitudes (relative
# error 1e-4, compared as |delta log|psi|| + |delta phase|); FP64 runs are
# held to 1e-9.
TOL = {"fp32": 1e-4, "fp64": 1e-9}


def oracle_net(Lx, Ly, N, D, seed, complex_=False, matter=False, precision="fp32", Q=None):
    """Lattice, oracle PEPS and the parameter vector, the tensors rounded to
    the storage type of `precision` (no GPU needed)."""
    lat = Lattice(Lx, Ly, N, matter=matter, Q=Q)
    Dk = D // N
    _, n = P.layout(lat, Dk)
    raw = synth.tensor_entries(seed, n, complex_)
    store = ("c64" if complex_ else "f32") if precision != "fp64" else ("c128" if complex_ else "f64")
    vals = synth.round_to(raw, store)
    return lat, P.GIPEPS(lat, Dk, vals), vals


def setup(Lx, Ly, N, D, chi, seed, complex_=False, matter=False, precision="fp32", h=1.0, g=0.5, J=0.0,
          Q=None):
    """Oracle PEPS + GPU context on the same rounded tensors."""
    import paper_2503_20566_gb300 as G

    lat, pe, vals = oracle_net(Lx, Ly, N, D, seed, complex_, matter, precision, Q)
    n = pe.n_params
    ctx = G.Context(N, Lx, Ly, D, chi, matter=matter, Q=Q, h=h, g=g, J=J, complex_=complex_,
                    precision=precision, seed=seed)
    assert ctx.n_params == n
    ctx.set_tensors(vals)
    return lat, pe, ctx


def configs_for(lat, n, seed, n_bosons=0):
    powers = synth.plaquette_powers(seed, n, lat.n_plaquettes, lat.N)
    occ = synth.occupations(seed, n, lat.n_s, n_bosons) if lat.matter else np.zeros((n, lat.n_s), np.int8)
    cfgs = np.array([lat.config_from_powers(occ[i].reshape(lat.Ly, lat.Lx), powers[i]) for i in range(n)],
                    dtype=np.int8)
    return cfgs, occ, powers


def amp_err(la_a, ph_a, la_b, ph_b):
    """|exp(delta log + i delta phase) - 1| (relative amplitude error)."""
    return abs(np.exp((la_a - la_b) + 1j * (ph_a - ph_b)) - 1.0)
