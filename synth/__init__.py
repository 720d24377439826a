"""Seeded synthetic inputs shared by the oracle-side tests and the GPU path.

This module holds *raw random numbers only*: no lattice geometry, Gauss law,
tensor layout or contraction arithmetic lives here.  Everything is derived from
one counter-based generator, SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), so that any stream element can
be recomputed independently from ``(seed, stream, counter)``:

    mix64(z)      = SplitMix64 output finaliser (shift-xor-multiply, 3 rounds)
    key(seed, s)  = mix64(seed + (s + 1) * GAMMA)            (stream key)
    draw(seed, s, k) = mix64(key(seed, s) + (k + 1) * GAMMA)  (k-th 64-bit word)

with GAMMA = 0x9E3779B97F4A7C15 and all arithmetic modulo 2**64.

Derived quantities:

* uniform double in [0, 1): ``(draw >> 11) * 2**-53``;
* standard normal: Box-Muller, cosine branch, from two consecutive uniforms
  ``z = sqrt(-2 ln(1 - u0)) * cos(2 pi u1)`` (one normal per pair of words);
* complex normal: real part = normal 2j, imaginary part = normal 2j + 1.

The synthetic workloads follow the paper's setting: i.i.d. N(0,1) entries for
every symmetry-allowed block of the PEPS tensors, plaquette powers uniform in
Z_N for the initial gauge configurations, and a uniformly random set of
occupied sites (fixed boson number) for the matter field.
"""

from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream ids used by the generators below (documented so other components can
# reproduce a stream from its definition).
STREAM_TENSORS = 0
STREAM_PLAQUETTE_POWERS = 1
STREAM_OCCUPATIONS = 2


def mix64(z):
    """SplitMix64 finaliser on a uint64 numpy array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed: int, stream: int):
    with np.errstate(over="ignore"):
        return mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + np.uint64(stream + 1) * GAMMA)


def draws(seed: int, stream: int, counters) -> np.ndarray:
    """64-bit words ``draw(seed, stream, k)`` for every k in ``counters``."""
    k = np.asarray(counters, dtype=np.uint64)
    key = stream_key(seed, stream)
    with np.errstate(over="ignore"):
        return mix64(key + (k + np.uint64(1)) * GAMMA)


def uniforms(seed: int, stream: int, counters) -> np.ndarray:
    w = draws(seed, stream, counters)
    return (w >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normals(seed: int, n: int, stream: int = STREAM_TENSORS, offset: int = 0) -> np.ndarray:
    """``n`` standard normals; normal j uses words 2j and 2j+1 of the stream."""
    j = np.arange(offset, offset + n, dtype=np.uint64)
    u0 = uniforms(seed, stream, 2 * j)
    u1 = uniforms(seed, stream, 2 * j + 1)
    return np.sqrt(-2.0 * np.log1p(-u0)) * np.cos(2.0 * np.pi * u1)


def tensor_entries(seed: int, n_params: int, complex_: bool) -> np.ndarray:
    """Flat parameter vector of length ``n_params`` (float64 or complex128).

    Real: entry k is normal k.  Complex: entry k is normal 2k + i * normal 2k+1.
    """
    if not complex_:
        return normals(seed, n_params)
    z = normals(seed, 2 * n_params)
    return z[0::2] + 1j * z[1::2]


def plaquette_powers(seed: int, n_chains: int, n_plaquettes: int, N: int) -> np.ndarray:
    """int8 array (n_chains, n_plaquettes), entries uniform in [0, N)."""
    k = np.arange(n_chains * n_plaquettes, dtype=np.uint64)
    w = draws(seed, STREAM_PLAQUETTE_POWERS, k)
    return (w % np.uint64(N)).astype(np.int8).reshape(n_chains, n_plaquettes)


def occupations(seed: int, n_chains: int, n_sites: int, n_bosons: int) -> np.ndarray:
    """int8 array (n_chains, n_sites) of 0/1 with exactly ``n_bosons`` ones per row.

    The occupied set of chain c is the ``n_bosons`` sites with the smallest
    keys ``draw(seed, 2, c * n_sites + site)`` (a uniformly random subset).
    """
    if not 0 <= n_bosons <= n_sites:
        raise ValueError("n_bosons out of range")
    k = np.arange(n_chains * n_sites, dtype=np.uint64)
    w = draws(seed, STREAM_OCCUPATIONS, k).reshape(n_chains, n_sites)
    order = np.argsort(w, axis=1, kind="stable")
    occ = np.zeros((n_chains, n_sites), dtype=np.int8)
    rows = np.arange(n_chains)[:, None]
    occ[rows, order[:, :n_bosons]] = 1
    return occ


def round_to(values: np.ndarray, dtype: str) -> np.ndarray:
    """Round FP64 values to a storage dtype and return them promoted back.

    ``dtype`` is one of 'f64', 'f32', 'c64', 'c128'.  Both sides of a parity
    check consume the rounded values, so storage rounding is not counted as
    arithmetic error.
    """
    if dtype == "f64":
        return np.asarray(values, dtype=np.float64)
    if dtype == "f32":
        return np.asarray(values, dtype=np.float32).astype(np.float64)
    if dtype == "c64":
        return np.asarray(values, dtype=np.complex64).astype(np.complex128)
    if dtype == "c128":
        return np.asarray(values, dtype=np.complex128)
    raise ValueError(dtype)
