"""Counter-based SplitMix64 generator for the Metropolis draws (oracle copy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper does not specify a generator.  Both the oracle and the CUDA sampler
implement SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) in counter form so a
chain can be replayed draw by draw:

    mix64(z)          = SplitMix64 finaliser
    key(seed, c)      = mix64(seed + (c + 1) * GAMMA)       chain key
    word(seed, c, k)  = mix64(key(seed, c) + (k + 1) * GAMMA)
    uniform           = (word >> 11) * 2**-53               in [0, 1)

Counter layout inside one sample-batch call, for sweep ``w`` of chain ``c``
(slot numbers are fixed per sweep, whether or not the move exists):

    k = w * n_slots + slot
    plaquette j = y*(Lx-1) + x : slot 2j   -> power t = 1 + word % (N-1)
                                  slot 2j+1 -> Metropolis uniform
    horizontal link j (matter)  : slot 2*Np + j          -> uniform
    vertical link j (matter)    : slot 2*Np + n_h + j    -> uniform
    n_slots = 2*Np + (n_h + n_v if matter else 0)
"""

from __future__ import annotations

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def mix64(z: int) -> int:
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def chain_key(seed: int, chain: int) -> int:
    return mix64(seed + (chain + 1) * GAMMA)


def word(seed: int, chain: int, counter: int) -> int:
    return mix64(chain_key(seed, chain) + (counter + 1) * GAMMA)


def uniform(seed: int, chain: int, counter: int) -> float:
    return (word(seed, chain, counter) >> 11) * (2.0 ** -53)


def power(seed: int, chain: int, counter: int, N: int) -> int:
    """Plaquette power t uniform in [1, N-1] (Sec. S-2)."""
    if N == 2:
        return 1
    return 1 + word(seed, chain, counter) % (N - 1)
