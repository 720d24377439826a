"""Gauge-invariant PEPS in gauge canonical form and its contraction (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Ansatz (main text, "Gauge-invariant TNS", Eqs. 6-7): every vertex carries a
matter tensor A^p_{l r d u}; virtual index j on a leg has charge q(j) in Z_N,
and A is non-zero only where p + q(l) + q(d) - q(r) - q(u) = Q_x (mod N).
Gauge tensors B^n_{l r} on the links are non-zero only for n = q(l) = q(r).
Bond dimension D = sum_q D_q over the charge sectors; `Dk` is either one
degeneracy for every sector (the layout shared with the CUDA library) or one
per charge (uneven sectors: block sizes then differ within a vertex).

Gauge canonical form (Eqs. 8-9): after A -> A X, B -> X^{-1} B with
X = (+)_k B^[k], every B becomes delta_{lr} delta_{n,q(l)} delta_{n,q(r)}; only
the A tensors carry parameters.

Sampled network (Sec. S-2, Eq. S5): a physical configuration s = (n, p)
selects, at every vertex, the single block of A whose leg charges are the
electric fields on the four adjacent links; B is absent, and every bond of the
resulting single-layer network has dimension D_k.  Open-boundary legs have
dimension 1 and charge 0.

Parameter layout (interface shared with the CUDA library; float64/complex128
here).  Vertices in row-major order v = y*Lx + x.  At a vertex the existing
legs, in the order (l, r, d, u), are legs[0..k-1].  The block index is the
mixed-radix number (p, n_legs[0], ..., n_legs[k-2]) with p most significant
and radix N for charges (P = 2 for matter, 1 without); the last existing leg's
charge is fixed by Eq. (1).  A block holds prod_legs D_(charge of the leg)
entries (D_k^k for uniform sectors) ordered [i_l][i_r][i_d][i_u] over existing
legs (row-major).  Blocks of a vertex are
contiguous; vertices follow one another.

Boundary-MPS contraction (Sec. S-2: "SVD or variational compression"; main
text, cost paragraph: cutoff chi).  Reading used here (the paper gives no more
detail): rows are absorbed bottom-up into an MPS; after each row the MPS is
left-canonicalised by QR (left to right), then swept right to left with an SVD
on every bond keeping the chi largest singular values, and normalised with the
norm accumulated in a log-scale.  Top environments are built the same way
from the top row downward.
`compress_variational` gives the other option the paper names: the
bond-chi MPS closest to the input, fitted by one-site alternating least
squares from the SVD truncation.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .lattice import Lattice

LEG_SIGN = (+1, -1, +1, -1)  # l, r, d, u in Eq. (1)


@dataclass
class VertexLayout:
    legs: tuple          # indices into (l, r, d, u) of the existing legs
    dims: tuple          # (Dl, Dr, Dd, Du) with 1 for missing legs (uniform sectors; else None)
    n_blocks: int
    block_size: int      # D_k^k (uniform sectors; else None)
    offset: int
    block_offsets: tuple = ()   # start of every block in the parameter vector
    block_dims: tuple = ()      # (Dl, Dr, Dd, Du) of every block


def sector_dims(N, Dk):
    """Degeneracy of every charge sector: D_k for all N charges (an int), or
    one entry per charge (uneven sectors)."""
    if np.ndim(Dk) == 0:
        return (int(Dk),) * N
    dq = tuple(int(d) for d in Dk)
    if len(dq) != N or min(dq) < 1:
        raise ValueError("one degeneracy >= 1 per charge sector")
    return dq


def _block_leg_charges(lat: Lattice, legs, x, y, bid):
    """Leg charges (n_l, n_r, n_d, n_u) of block bid: the mixed-radix digits
    of the first k-1 existing legs, the last leg's charge from Eq. (1)."""
    N, k = lat.N, len(legs)
    ch = [0, 0, 0, 0]
    b = bid
    for i in reversed(legs[:-1]):
        ch[i] = b % N
        b //= N
    p = b
    rest = (int(lat.Q[y, x]) - p - sum(LEG_SIGN[i] * ch[i] for i in legs[:-1])) % N
    ch[legs[-1]] = (LEG_SIGN[legs[-1]] * rest) % N
    return p, tuple(ch)


def layout(lat: Lattice, Dk):
    """Per-vertex block layout and the total parameter count.  Dk: the
    degeneracy of every charge sector (an int), or one per charge; a block's
    leg has the degeneracy of the charge it carries, so with uneven sectors
    the blocks of a vertex differ in size."""
    P = 2 if lat.matter else 1
    dq = sector_dims(lat.N, Dk)
    uniform = len(set(dq)) == 1
    verts = []
    off = 0
    for y in range(lat.Ly):
        for x in range(lat.Lx):
            has = lat.has_legs(x, y)
            legs = tuple(i for i in range(4) if has[i])
            k = len(legs)
            nb = P * lat.N ** (k - 1)
            offs, bdims = [], []
            start = off
            for bid in range(nb):
                _, ch = _block_leg_charges(lat, legs, x, y, bid)
                d = tuple(dq[ch[i]] if has[i] else 1 for i in range(4))
                offs.append(off)
                bdims.append(d)
                off += int(np.prod(d))
            dims = tuple(dq[0] if has[i] else 1 for i in range(4)) if uniform else None
            bs = dq[0] ** k if uniform else None
            verts.append(VertexLayout(legs, dims, nb, bs, start, tuple(offs), tuple(bdims)))
    return verts, off


def block_id(lat: Lattice, vl: VertexLayout, x, y, p, charges):
    """Block index for matter value p and leg charges (n_l, n_r, n_d, n_u).

    Returns -1 when the charges violate Eq. (1) at this vertex (or a missing
    leg carries a non-zero charge), i.e. when A has no such block.
    """
    for i in range(4):
        if i not in vl.legs and charges[i] != 0:
            return -1
    tot = p + sum(LEG_SIGN[i] * charges[i] for i in range(4))
    if (tot - lat.Q[y, x]) % lat.N:
        return -1
    bid = p
    for i in vl.legs[:-1]:
        bid = bid * lat.N + charges[i] % lat.N
    return bid


class GIPEPS:
    """A GCF gauge-invariant PEPS: the flat parameter vector plus its layout."""

    def __init__(self, lat: Lattice, Dk: int, params: np.ndarray):
        self.lat = lat
        self.Dk = Dk
        self.verts, self.n_params = layout(lat, Dk)
        params = np.asarray(params)
        if params.shape != (self.n_params,):
            raise ValueError(f"expected {self.n_params} parameters, got {params.shape}")
        self.params = params.astype(np.complex128 if np.iscomplexobj(params) else np.float64)

    def vertex(self, x, y) -> VertexLayout:
        return self.verts[y * self.lat.Lx + x]

    def block(self, x, y, bid):
        vl = self.vertex(x, y)
        a, d = vl.block_offsets[bid], vl.block_dims[bid]
        return self.params[a:a + int(np.prod(d))].reshape(d)

    def selected_block(self, cfg, x, y):
        """(block id, tensor A~_x) selected by configuration cfg (Eq. S5).

        Returns (-1, None) if the configuration violates Eq. (1) at (x, y).
        """
        lat = self.lat
        p = int(cfg[lat.pi(x, y)])
        if p not in ((0, 1) if lat.matter else (0,)):
            return -1, None
        ch = lat.leg_values(cfg, x, y)
        bid = block_id(lat, self.vertex(x, y), x, y, p, ch)
        if bid < 0:
            return -1, None
        return bid, self.block(x, y, bid)

    def sampled_network(self, cfg):
        """tensors[y][x] = A~_x with shape (Dl, Dr, Dd, Du), or None if unphysical."""
        rows = []
        for y in range(self.lat.Ly):
            row = []
            for x in range(self.lat.Lx):
                bid, t = self.selected_block(cfg, x, y)
                if bid < 0:
                    return None
                row.append(t)
            rows.append(row)
        return rows

    # ---- dense (non-sampled) tensors for definition-level checks --------
    def dense_A(self, x, y):
        """Full A^p_{lrdu}: shape (P, Dl', Dr', Dd', Du') with D' = sum of the
        sector degeneracies on existing legs (charge q occupies indices
        start(q) .. start(q) + D_q - 1, sectors in charge order) and 1 on
        missing legs."""
        lat = self.lat
        dq = sector_dims(lat.N, self.Dk)
        start = np.concatenate([[0], np.cumsum(dq)])
        vl = self.vertex(x, y)
        P = 2 if lat.matter else 1
        full = tuple(int(start[-1]) if i in vl.legs else 1 for i in range(4))
        A = np.zeros((P,) + full, dtype=self.params.dtype)
        ranges = [range(lat.N) if i in vl.legs else range(1) for i in range(4)]
        for p in range(P):
            for ch in np.ndindex(*[len(r) for r in ranges]):
                bid = block_id(lat, vl, x, y, p, ch)
                if bid < 0:
                    continue
                sl = tuple(slice(int(start[ch[i]]), int(start[ch[i] + 1])) if i in vl.legs else slice(0, 1)
                           for i in range(4))
                A[(p,) + sl] = self.block(x, y, bid)
        return A


def link_clock_params(pe: "GIPEPS", x, y, axis, power=1):
    """Parameters of Z^power psi for the clock operator Z |n> = omega^n |n>
    (sigma_z for N = 2) on link (x, y, axis): in the GCF the charge on a leg
    is the electric value of its link, so every block of vertex (x, y) is
    multiplied by omega^(power * charge on its r leg (axis 1) or u leg
    (axis 2)).  Real parameters stay real for N = 2."""
    lat = pe.lat
    leg = 1 if axis == 1 else 3
    vl = pe.vertex(x, y)
    if leg not in vl.legs:
        raise ValueError("no such link")
    real = lat.N == 2 and not np.iscomplexobj(pe.params)
    out = pe.params.astype(np.float64 if real else np.complex128)
    for bid in range(vl.n_blocks):
        _, ch = _block_leg_charges(lat, vl.legs, x, y, bid)
        n = (power * ch[leg]) % lat.N
        a, d = vl.block_offsets[bid], vl.block_dims[bid]
        out[a:a + int(np.prod(d))] *= (-1.0) ** n if real else np.exp(2j * np.pi * n / lat.N)
    return out


# ---------------------------------------------------------------------------
# Full (double-index) network with explicit B tensors: the definition of the
# amplitude <s|Psi> before the GCF / sampling simplifications.
# ---------------------------------------------------------------------------

def gcf_link_tensor(N, Dk):
    """B^n_{lr} in gauge canonical form, Eq. (9): shape (N, D, D), D the sum
    of the sector degeneracies; the identity on sector n."""
    dq = sector_dims(N, Dk)
    start = np.concatenate([[0], np.cumsum(dq)])
    B = np.zeros((N, int(start[-1]), int(start[-1])))
    for n in range(N):
        for i in range(int(start[n]), int(start[n + 1])):
            B[n, i, i] = 1.0
    return B


def general_link_tensor(blocks, N, Dk):
    """B^n_{lr} = calB^n_{lr} delta_{n,q(l)} delta_{n,q(r)}, Eq. (7), from
    blocks[n] of shape (D_n, D_n)."""
    dq = sector_dims(N, Dk)
    start = np.concatenate([[0], np.cumsum(dq)])
    D = int(start[-1])
    B = np.zeros((N, D, D), dtype=np.result_type(*blocks))
    for n in range(N):
        a, b = int(start[n]), int(start[n + 1])
        B[n, a:b, a:b] = blocks[n]
    return B


def full_amplitude(lat: Lattice, A, Bh, Bv, cfg):
    """<s|Psi> of the GI-PEPS with matter tensors A[y][x] (dense, shape
    (P, l, r, d, u)) and link tensors Bh[y][x], Bv[y][x] (shape (N, D, D)),
    by direct contraction of every virtual index.  Defined for any integer
    configuration, physical or not."""
    Lx, Ly = lat.Lx, lat.Ly
    # Build the projected single-layer network with double-size bonds: link
    # tensor matrices are absorbed into the tensor on their left / below.
    T = []
    for y in range(Ly):
        row = []
        for x in range(Lx):
            p = int(cfg[lat.pi(x, y)])
            t = A[y][x][p]
            if x < Lx - 1:
                n = int(cfg[lat.hi(x, y)])
                t = np.einsum("lrdu,rs->lsdu", t, Bh[y][x][n])
            if y < Ly - 1:
                n = int(cfg[lat.vi(x, y)])
                t = np.einsum("lrdu,uv->lrdv", t, Bv[y][x][n])
            row.append(t)
        T.append(row)
    return contract_exact(T)


# ---------------------------------------------------------------------------
# Exact contraction of a single-layer network (the plain definition).
# ---------------------------------------------------------------------------

def contract_exact(T):
    """Sum over all virtual indices of prod_x T[y][x][l, r, d, u].

    Row by row on the full vector over the up-legs of the rows absorbed so far
    (no truncation).  Exponential in Lx: small lattices only.
    """
    Ly, Lx = len(T), len(T[0])
    vec = np.ones((1,) * Lx)  # down-legs of row 0 all have dimension 1
    for y in range(Ly):
        # carry t with axes (h, u_0..u_{x-1}, d_x..d_{Lx-1})
        t = vec[None, ...]
        for x in range(Lx):
            W = T[y][x]
            # contract h (axis 0) and d_x (axis 1 + x) with W[l, r, d, u]
            t = np.tensordot(t, W, axes=([0, 1 + x], [0, 2]))
            # now axes: (u_0..u_{x-1}, d_{x+1}..d_{Lx-1}, r, u_x)
            nd = t.ndim
            order = [nd - 2] + list(range(x)) + [nd - 1] + list(range(x, nd - 2))
            t = np.transpose(t, order)
        vec = t[0]  # right-most horizontal leg has dimension 1
    return complex(vec.reshape(-1)[0]) if np.iscomplexobj(vec) else float(vec.reshape(-1)[0])


# ---------------------------------------------------------------------------
# Boundary MPS (Sec. S-2; cutoff chi from the main-text cost paragraph).
# MPS site tensors have shape (left bond, physical, right bond).
# ---------------------------------------------------------------------------

def trivial_mps(Lx, dtype=np.float64):
    return [np.ones((1, 1, 1), dtype=dtype) for _ in range(Lx)]


def absorb(mps, row):
    """Apply one PEPS row (tensors W[l, r, d, u]) to an MPS whose physical legs
    are the d legs: M'[(a,l), u, (b,r)] = sum_d M[a, d, b] W[l, r, d, u]."""
    out = []
    for M, W in zip(mps, row):
        a, _, b = M.shape
        l, r, _, u = W.shape
        X = np.einsum("adb,lrdu->alubr", M, W)
        out.append(X.reshape(a * l, u, b * r))
    return out


def flip_row(row):
    """Swap the d and u legs so a row can be absorbed from above."""
    return [np.transpose(W, (0, 1, 3, 2)) for W in row]


def compress(mps, chi, spectra=None):
    """SVD compression of an MPS to bond dimension <= chi, normalised.

    1. QR left to right (left-canonical sites 0..L-2);
    2. right to left: SVD of each site as (left bond) x (phys, right bond),
       keep the chi largest singular values, push U S into the left
       neighbour;
    3. divide the first site by the state norm.
    Returns (mps, log_norm); the input state equals exp(log_norm) * output
    (up to the discarded weight).
    `spectra`, if a list, receives (bond i, all singular values of that
    bond) for every bond the sweep cuts (more than chi values); it is a
    diagnostic and changes nothing in the result.  The kept subspace at a cut
    is well defined only when sigma_chi > sigma_chi+1, and a small gap there
    makes the truncated state sensitive to rounding in its input.
    """
    mps = [m.copy() for m in mps]
    L = len(mps)
    for i in range(L - 1):
        a, d, b = mps[i].shape
        Qm, R = np.linalg.qr(mps[i].reshape(a * d, b))
        k = Qm.shape[1]
        mps[i] = Qm.reshape(a, d, k)
        mps[i + 1] = np.tensordot(R, mps[i + 1], axes=(1, 0))
    for i in range(L - 1, 0, -1):
        a, d, b = mps[i].shape
        U, S, Vh = np.linalg.svd(mps[i].reshape(a, d * b), full_matrices=False)
        k = min(chi, len(S))
        if spectra is not None and len(S) > chi:
            spectra.append((i, S.copy()))
        mps[i] = Vh[:k].reshape(k, d, b)
        mps[i - 1] = np.tensordot(mps[i - 1], U[:, :k] * S[:k], axes=(2, 0))
    nrm = np.linalg.norm(mps[0])
    if nrm == 0.0:
        return mps, -np.inf
    mps[0] = mps[0] / nrm
    return mps, float(np.log(nrm))


def compress_variational(mps, chi, sweeps=4, history=None):
    """Variational compression (Sec. S-2, the alternative to SVD truncation):
    the MPS phi of bond dimension <= chi that minimises ||psi - phi||, by
    alternating least squares on one site at a time.

    phi starts as the SVD truncation (`compress`), which is right-canonical
    with its centre at site 0.  With every other site of phi orthonormal
    towards the centre i, the best site tensor is the projection of psi,
    B_i[b, d, b'] = sum L_i[b, a] A_i[a, d, a'] R_{i+1}[b', a'], where L and R
    are the overlaps <phi|psi> of the sites left and right of i.  A sweep
    updates left to right (QR moves the centre right) and back (LQ moves it
    left).  Then ||psi - phi||^2 = ||psi||^2 - ||B_centre||^2, which never
    grows from one update to the next; `history`, if a list, receives it
    after the initial truncation and after every sweep.  Returns
    (mps, log_norm) as `compress` does.
    """
    A = [np.asarray(m) for m in mps]
    L = len(A)
    B, _ = compress(A, chi)
    B = [b.astype(np.result_type(b, *A)) for b in B]
    psi2 = None
    if history is not None:
        # ||psi||^2 by the exact overlap <psi|psi>
        E = np.ones((1, 1))
        for a in A:
            E = np.einsum("xy,xdb,yde->be", E, a.conj(), a)
        psi2 = float(np.real(E.reshape(-1)[0]))

    def right_env(i, env_next):
        # R_i[b, a] = sum conj(B_i[b, d, b']) A_i[a, d, a'] R_{i+1}[b', a']
        return np.einsum("bdc,ade,ce->ba", B[i].conj(), A[i], env_next)

    def left_env(i, env_prev):
        # L_{i+1}[b', a'] = sum L_i[b, a] conj(B_i[b, d, b']) A_i[a, d, a']
        return np.einsum("ba,bdc,ade->ce", env_prev, B[i].conj(), A[i])

    def optimal(i, Lenv, Renv):
        return np.einsum("ba,ade,ce->bdc", Lenv, A[i], Renv)

    R = [None] * (L + 1)
    R[L] = np.ones((1, 1))
    for i in range(L - 1, 0, -1):
        R[i] = right_env(i, R[i + 1])
    if history is not None:
        c = optimal(0, np.ones((1, 1)), R[1])
        history.append(max(psi2 - float(np.sum(np.abs(c) ** 2)), 0.0))
    Lenv = [None] * (L + 1)
    Lenv[0] = np.ones((1, 1))
    for _ in range(sweeps):
        for i in range(L - 1):                      # left to right
            X = optimal(i, Lenv[i], R[i + 1])
            b, d, c = X.shape
            Q, _r = np.linalg.qr(X.reshape(b * d, c))
            B[i] = Q.reshape(b, d, Q.shape[1])
            Lenv[i + 1] = left_env(i, Lenv[i])
        for i in range(L - 1, 0, -1):               # right to left
            X = optimal(i, Lenv[i], R[i + 1])
            b, d, c = X.shape
            Q, _r = np.linalg.qr(X.reshape(b, d * c).T)   # X^T = Q r, so X = r^T Q^T (LQ)
            B[i] = Q.T.reshape(Q.shape[1], d, c)
            R[i] = right_env(i, R[i + 1])
        B[0] = optimal(0, Lenv[0], R[1])
        if history is not None:
            history.append(max(psi2 - float(np.sum(np.abs(B[0]) ** 2)), 0.0))
    nrm = np.linalg.norm(B[0])
    if nrm == 0.0:
        return B, -np.inf
    B[0] = B[0] / nrm
    return B, float(np.log(nrm))


def bottom_envs(rows, chi, spectra=None):
    """B[r] (r = -1 .. Ly-1) as (mps, log_scale): rows 0..r absorbed bottom-up.

    Returned as a dict keyed by r; B[-1] is the trivial MPS with log-scale 0.
    `spectra`, if a list, receives (r, bond, singular values) of every cut
    (see `compress`).
    """
    Lx = len(rows[0])
    dt = np.result_type(*[w.dtype for w in rows[0]])
    env = {-1: (trivial_mps(Lx, dt), 0.0)}
    for r in range(len(rows)):
        m, s = env[r - 1]
        cuts = [] if spectra is not None else None
        m2, ds = compress(absorb(m, rows[r]), chi, cuts)
        if spectra is not None:
            spectra.extend((r, i, S) for i, S in cuts)
        env[r] = (m2, s + ds)
    return env


def top_envs(rows, chi, spectra=None):
    """T[r] (r = Ly .. 0): rows r..Ly-1 absorbed top-down; physical legs are
    the down legs of row r.  T[Ly] is trivial.  `spectra` as in
    `bottom_envs`."""
    Ly, Lx = len(rows), len(rows[0])
    dt = np.result_type(*[w.dtype for w in rows[0]])
    env = {Ly: (trivial_mps(Lx, dt), 0.0)}
    for r in range(Ly - 1, -1, -1):
        m, s = env[r + 1]
        cuts = [] if spectra is not None else None
        m2, ds = compress(absorb(m, flip_row(rows[r])), chi, cuts)
        if spectra is not None:
            spectra.extend((r, i, S) for i, S in cuts)
        env[r] = (m2, s + ds)
    return env


def _chain(spec, *ops):
    """np.einsum(spec, *ops) evaluated as a left-to-right chain of two-operand
    contractions: each step sums the indices that no later operand and not the
    output carries.  The same sum as the single einsum, reached through
    pairwise products (BLAS) instead of one loop over every index at once."""
    ins, out = spec.split("->")
    ins = ins.split(",")
    cur, cur_idx = ops[0], ins[0]
    for k in range(1, len(ops)):
        rest = "".join(ins[k + 1:]) + out
        keep = "".join(ch for ch in dict.fromkeys(cur_idx + ins[k]) if ch in rest)
        cur = np.einsum(f"{cur_idx},{ins[k]}->{keep}", cur, ops[k], optimize=True)
        cur_idx = keep
    return np.einsum(f"{cur_idx}->{out}", cur)


def contract_row(Bm, row, Tm):
    """<B| row |T> for one PEPS row between two MPS (3 layers), exact."""
    E = np.ones((1, 1, 1))
    for Bs, W, Ts in zip(Bm, row, Tm):
        # E[a, l, b] Bs[a, d, a'] W[l, r, d, u] Ts[b, u, b']
        E = _chain("alb,adA,lrdu,buB->ArB", E, Bs, W, Ts)
    return E.reshape(-1)[0]


def contract_strip(Bm, row1, row2, Tm):
    """<B| row1 row2 |T> for two adjacent rows between two MPS (4 layers), exact."""
    E = np.ones((1, 1, 1, 1))
    for Bs, W1, W2, Ts in zip(Bm, row1, row2, Tm):
        # E[a,i,j,b] Bs[a,d,A] W1[i,I,d,m] W2[j,J,m,u] Ts[b,u,B] -> E[A,I,J,B]
        E = _chain("aijb,adA,iIdm,jJmu,buB->AIJB", E, Bs, W1, W2, Ts)
    return E.reshape(-1)[0]


def row_site_environment(Bm, row, Tm, x):
    """d<B|row|T>/dW_x: the open tensor of shape W_x.shape (Dl, Dr, Dd, Du)."""
    L = np.ones((1, 1, 1))
    for c in range(x):
        L = _chain("alb,adA,lrdu,buB->ArB", L, Bm[c], row[c], Tm[c])
    R = np.ones((1, 1, 1))
    for c in range(len(row) - 1, x, -1):
        R = _chain("ArB,buB,lrdu,adA->alb", R, Tm[c], row[c], Bm[c])
    return _chain("alb,adA,ArB,buB->lrdu", L, Bm[x], R, Tm[x])


def mps_bond_dims(mps):
    return [m.shape[2] for m in mps[:-1]]
