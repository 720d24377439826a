"""Exact transformations of GCF-PEPS parameters that prepare states.

The parameter vector follows the library's documented block layout (Eqs. 6
and 9): vertices in row-major order; at a vertex with existing legs
legs[0..k-1] (in the order l, r, d, u) there are P * N^(k-1) blocks (P = 2
with matter, else 1) of D_k^k entries, block index = mixed radix
(p, n_legs[0], ..., n_legs[k-2]) with p most significant, and the last leg's
charge fixed by the Gauss law p + n_l + n_d - n_r - n_u = Q_x (mod N).

In a GCF PEPS the charge on a leg equals the electric value n of the link it
belongs to, for every configuration the block is selected by.  A diagonal
operator on one link, |n> -> f(n) |n>, is therefore exact on the ansatz:
multiply each block of one adjacent vertex by f(charge of that leg).  The
vison initial state of the real-time study (the Pauli sigma_z, |n> ->
(-1)^n |n>, on the bottom-left vertical link of the ground state) is the case
N = 2, f(n) = (-1)^n; for Z_N the clock operator |n> -> omega^n |n>,
omega = exp(2 pi i / N), generalises it.
"""

from __future__ import annotations

import numpy as np

LEG_SIGNS = (1, -1, 1, -1)  # l, r, d, u in the Gauss law


def vertex_layout(N, Lx, Ly, Dk, matter=False):
    """Per vertex (row-major): (offset, n_blocks, block_size, existing legs)."""
    P = 2 if matter else 1
    out, off = [], 0
    for y in range(Ly):
        for x in range(Lx):
            legs = tuple(i for i, has in enumerate((x > 0, x < Lx - 1, y > 0, y < Ly - 1)) if has)
            k = len(legs)
            nb, bs = P * N ** (k - 1), Dk ** k
            out.append((off, nb, bs, legs))
            off += nb * bs
    return out


def block_charges(N, b, legs, Q=0):
    """(p, {leg: charge}) of block b at a vertex with existing `legs` and
    background charge Q."""
    k = len(legs)
    digits = []
    for _ in range(k - 1):
        digits.append(b % N)
        b //= N
    p = b
    ch = dict(zip(legs[:-1], reversed(digits)))
    rest = (Q - p - sum(LEG_SIGNS[i] * c for i, c in ch.items())) % N
    ch[legs[-1]] = (LEG_SIGNS[legs[-1]] * rest) % N
    return p, ch


def link_phase(params, N, Lx, Ly, Dk, x, y, axis, power=1, matter=False, Q=None):
    """Parameters of Z^power psi, Z the clock operator |n> -> omega^n |n> on
    link (x, y, axis) (axis 1: to (x+1, y); axis 2: to (x, y+1)), applied to
    the blocks of vertex (x, y) through its r (axis 1) or u (axis 2) leg.
    For N = 2 and power 1 this is sigma_z and keeps real parameters real."""
    if axis == 1 and not (0 <= x < Lx - 1 and 0 <= y < Ly):
        raise ValueError("no horizontal link there")
    if axis == 2 and not (0 <= x < Lx and 0 <= y < Ly - 1):
        raise ValueError("no vertical link there")
    lay = vertex_layout(N, Lx, Ly, Dk, matter)
    if len(params) != lay[-1][0] + lay[-1][1] * lay[-1][2]:
        raise ValueError("parameter count does not match the layout")
    off, nb, bs, legs = lay[y * Lx + x]
    leg = 1 if axis == 1 else 3
    q = 0 if Q is None else int(np.asarray(Q).reshape(-1)[y * Lx + x]) % N
    real = N == 2 and not np.iscomplexobj(params)
    out = np.array(params, dtype=np.float64 if real else np.complex128, copy=True)
    for b in range(nb):
        _, ch = block_charges(N, b, legs, q)
        n = (power * ch[leg]) % N
        f = (-1.0) ** n if real else np.exp(2j * np.pi * n / N)
        out[off + b * bs: off + (b + 1) * bs] *= f
    return out


def vison(params, N, Lx, Ly, Dk, matter=False, Q=None):
    """The vison initial state: sigma_z (clock operator for Z_N) on the
    bottom-left vertical link, (0, 0) -> (0, 1)."""
    return link_phase(params, N, Lx, Ly, Dk, 0, 0, 2, 1, matter, Q)
