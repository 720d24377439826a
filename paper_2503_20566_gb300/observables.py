"""Observables of the paper's analysis as Monte Carlo estimators over samples.

For an operator O and a sample s drawn from |psi|^2 the local estimator is
O_loc(s) = sum_s' <s|O|s'> psi(s') / psi(s); its mean over samples estimates
<psi|O|psi> / <psi|psi>.  Diagonal operators need only the configurations;
the others need amplitudes of moved configurations, which come from the
library (Context.amplitude), so the contraction work stays on the GPU.  The
configuration moves are index shifts on the host.

* Electric term (Eq. 5): H_E / g = sum_links (2 - 2 cos(2 pi n / N)); its mean
  is d<H>/dg (the first derivative of the energy used to locate transitions).
* Plaquette operator P_x + P_x^dag with P_x = U_(x,1) U_(x+e1,2) U^dag_(x+e2,1)
  U^dag_(x,2) (Eq. 4): local value [psi(P^dag s) + psi(P s)] / psi(s).
* VBS order parameter D_alpha = (1 / n_alpha) sum_x (-1)^{x_alpha} Ebar^alpha_x
  with Ebar = 2 - 2 cos(2 pi n / N) on the alpha-links and n_alpha their number
  (L(L-1) on an L x L lattice).
* With matter: the boson density n_x, and the gauge-dressed hop
  c^dag_x U c_{x'} + h.c. on every link (Eq. 3), local value psi(s') / psi(s)
  for the configuration s' the hop reaches.
* Wilson loop W around a w x h block of plaquettes (U on its bottom and right
  edges, U^dag on its top and left edges): W is the product of the block's
  plaquette operators, so W s shifts only the boundary links; local value
  psi(W^dag s) / psi(s).

Configurations use the library's layout: [h: Ly x (Lx-1)][v: (Ly-1) x Lx]
[p: Ly x Lx] int8, link values in [0, N).  A link value n is raised by U.
"""

from __future__ import annotations

import numpy as np


def _np(x):
    return x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)


def _links(configs, Lx, Ly):
    c = _np(configs).astype(np.int64)
    n_h, n_v = Ly * (Lx - 1), (Ly - 1) * Lx
    return c[:, :n_h].reshape(-1, Ly, Lx - 1), c[:, n_h:n_h + n_v].reshape(-1, Ly - 1, Lx)


def electric_field(configs, Lx, Ly, N):
    """Ebar = 2 - 2 cos(2 pi n / N) per link: (horizontal (n, Ly, Lx-1),
    vertical (n, Ly-1, Lx))."""
    h, v = _links(configs, Lx, Ly)
    f = lambda n: 2.0 - 2.0 * np.cos(2.0 * np.pi * n / N)  # noqa: E731
    return f(h), f(v)


def electric_term(configs, Lx, Ly, N):
    """Per-sample H_E / g = sum over links of Ebar (its mean is d<H>/dg)."""
    eh, ev = electric_field(configs, Lx, Ly, N)
    return eh.sum(axis=(1, 2)) + ev.sum(axis=(1, 2))


def vbs_order(configs, Lx, Ly, N):
    """Per-sample (D_x, D_y): the staggered means of Ebar over the horizontal
    links (sign (-1)^x) and the vertical links (sign (-1)^y)."""
    eh, ev = electric_field(configs, Lx, Ly, N)
    sx = (-1.0) ** np.arange(Lx - 1)
    sy = (-1.0) ** np.arange(Ly - 1)
    dx = (eh * sx[None, None, :]).sum(axis=(1, 2)) / eh[0].size
    dy = (ev * sy[None, :, None]).sum(axis=(1, 2)) / ev[0].size
    return dx, dy


def shift_block(configs, Lx, Ly, N, x0, y0, w, h, t):
    """Apply (P^t) to every plaquette of the w x h block whose lower-left
    plaquette is (x0, y0): the block's bottom and right boundary links are
    raised by t, its top and left boundary links lowered by t (interior
    links cancel).  Returns new int8 configurations."""
    if not (0 <= x0 and x0 + w <= Lx - 1 and 0 <= y0 and y0 + h <= Ly - 1 and w >= 1 and h >= 1):
        raise ValueError("block outside the lattice's plaquettes")
    c = _np(configs).astype(np.int64).copy()
    n_h = Ly * (Lx - 1)
    hi = lambda x, y: y * (Lx - 1) + x  # noqa: E731
    vi = lambda x, y: n_h + y * Lx + x  # noqa: E731
    for x in range(x0, x0 + w):
        c[:, hi(x, y0)] += t          # bottom edge: U
        c[:, hi(x, y0 + h)] -= t      # top edge: U^dag
    for y in range(y0, y0 + h):
        c[:, vi(x0 + w, y)] += t      # right edge: U
        c[:, vi(x0, y)] -= t          # left edge: U^dag
    nl = n_h + (Ly - 1) * Lx
    c[:, :nl] %= N
    return c.astype(np.int8)


def _ratio(ctx, moved, la, ph):
    la2, ph2 = ctx.amplitude(moved)
    return np.exp((_np(la2) - la) + 1j * (_np(ph2) - ph))


def _amps(ctx, configs, la, ph):
    if la is None or ph is None:
        la, ph = ctx.amplitude(configs)
    return _np(la).astype(np.float64), _np(ph).astype(np.float64)


def plaquette_map(ctx, configs, Lx, Ly, N, la=None, ph=None):
    """Per-sample local values of P_x + P_x^dag for every plaquette:
    complex array (n, Ly-1, Lx-1).  la, ph: log|psi| and arg psi of
    `configs` (computed if not given)."""
    la, ph = _amps(ctx, configs, la, ph)
    out = np.zeros((la.shape[0], Ly - 1, Lx - 1), dtype=np.complex128)
    for y in range(Ly - 1):
        for x in range(Lx - 1):
            up = _ratio(ctx, shift_block(configs, Lx, Ly, N, x, y, 1, 1, 1), la, ph)
            dn = up if N == 2 else _ratio(ctx, shift_block(configs, Lx, Ly, N, x, y, 1, 1, N - 1), la, ph)
            out[:, y, x] = up + dn
    return out


def wilson_loop(ctx, configs, Lx, Ly, N, w, h=None, origin=None, la=None, ph=None):
    """Per-sample local values of the Wilson loop around a w x h block of
    plaquettes (default h = w, block centred): psi(W^dag s) / psi(s)."""
    h = w if h is None else h
    if origin is None:
        origin = ((Lx - 1 - w) // 2, (Ly - 1 - h) // 2)
    la, ph = _amps(ctx, configs, la, ph)
    return _ratio(ctx, shift_block(configs, Lx, Ly, N, origin[0], origin[1], w, h, N - 1), la, ph)


def boson_density(configs, Lx, Ly):
    """Per-sample occupations n_x: (n, Ly, Lx) (hard-core bosons)."""
    c = _np(configs).astype(np.int64)
    n_l = Ly * (Lx - 1) + (Ly - 1) * Lx
    return c[:, n_l:n_l + Lx * Ly].reshape(-1, Ly, Lx).astype(np.float64)


def hop_configs(configs, Lx, Ly, N, x, y, axis):
    """The configurations reached by the gauge-dressed hop on link (x, y,
    axis) (Eq. 3): a boson moves from the far end to (x, y) raising the link,
    or from (x, y) to the far end lowering it.  Rows where neither applies
    (hard-core) come back unchanged with mask False.  Returns (moved int8
    configurations, mask)."""
    c = _np(configs).astype(np.int64).copy()
    n_h = Ly * (Lx - 1)
    n_l = n_h + (Ly - 1) * Lx
    x2, y2 = (x + 1, y) if axis == 1 else (x, y + 1)
    li = y * (Lx - 1) + x if axis == 1 else n_h + y * Lx + x
    s1, s2 = n_l + y * Lx + x, n_l + y2 * Lx + x2
    fwd = (c[:, s1] == 0) & (c[:, s2] == 1)
    bwd = (c[:, s1] == 1) & (c[:, s2] == 0)
    c[fwd, s1], c[fwd, s2] = 1, 0
    c[fwd, li] = (c[fwd, li] + 1) % N
    c[bwd, s1], c[bwd, s2] = 0, 1
    c[bwd, li] = (c[bwd, li] - 1) % N
    return c.astype(np.int8), fwd | bwd


def hop_map(ctx, configs, Lx, Ly, N, la=None, ph=None):
    """Per-sample local values of c^dag_x U c_{x'} + h.c. on every link:
    (horizontal (n, Ly, Lx-1), vertical (n, Ly-1, Lx)), psi(s')/psi(s) where
    the hop applies and 0 elsewhere."""
    la, ph = _amps(ctx, configs, la, ph)
    n = la.shape[0]
    hh = np.zeros((n, Ly, Lx - 1), dtype=np.complex128)
    hv = np.zeros((n, Ly - 1, Lx), dtype=np.complex128)
    for axis, out, ny, nx in ((1, hh, Ly, Lx - 1), (2, hv, Ly - 1, Lx)):
        for y in range(ny):
            for x in range(nx):
                moved, mask = hop_configs(configs, Lx, Ly, N, x, y, axis)
                if mask.any():
                    r = np.zeros(n, dtype=np.complex128)
                    r[mask] = _ratio(ctx, moved[mask], la[mask], ph[mask])
                    out[:, y, x] = r
    return hh, hv


def mean_and_error(values, n_chains):
    """Mean and standard error over chain means; values chain-major
    (n_chains x samples per chain)."""
    v = np.asarray(values).reshape(n_chains, -1).mean(axis=1)
    err = v.std(ddof=1) / np.sqrt(n_chains) if n_chains > 1 else float("nan")
    return v.mean(), err
