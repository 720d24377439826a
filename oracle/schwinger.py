"""(1+1)D Schwinger model and its GCF time evolution (End Matter), oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Model (End Matter): a U(1) gauge field on the links of an open chain of L
sites with staggered fermions, static charges Q_x = (1 + (-1)^x) / 2 and
masses m_x = (-1)^x m,

    H = sum_x m_x n_x + sum_x (J c^dag_x U_x c_{x+1} + h.c.) + g sum_x E_x^2,

with Gauss's law E_x - E_{x-1} = n_x - Q_x and E_{-1} = 0 (E_x lives on the
link between x and x+1).  On an open chain the gauge field is fixed by the
fermions, E_x = sum_{y <= x} (n_y - Q_y), so the states are fermion
occupations; U_x raises E_x, which is what moving a fermion from x+1 to x does
to that sum.  Nearest-neighbour hopping on a chain carries no fermionic sign.

GCF time evolution (End Matter, Fact 1 and the two rules that follow it): an
MPS of A tensors only, U(1) symmetric, whose bond charges are the electric
fields: the bond right of site x carries E_x.  A two-site gate exp(-tau h) on
sites (x, x+1) acts with the hopping of the globally symmetric model (the
charge-neutral c^dag_x c_{x+1}), the masses, and exp(-tau g E^2) on the
virtual charges; the two-site tensor is split keeping the charge of A_x at
Q_x, so the new middle bond charge is E_{x-1} + n_x - Q_x, i.e. a hop raises
E_x by one exactly as c^dag_x U_x c_{x+1} does.  The split is an SVD per
charge sector, truncated to chi at the canonical centre; sweeps left to right
and back with tau / 2 each give a second-order step.

Readings (the End Matter gives no more): bonds carry E only, E_{-1} = 0 at the
left end; the mass of site x is applied in the gate of bond x (the last site's
in the last bond's gate); the electric term of link x in the gate of bond x.
"""

from __future__ import annotations

import itertools

import numpy as np


def charges(L):
    return np.array([(1 + (-1) ** x) // 2 for x in range(L)])


def masses(L, m):
    return np.array([((-1) ** x) * m for x in range(L)], dtype=np.float64)


def basis(L, n_f):
    """Occupation tuples with n_f fermions, in a fixed order."""
    return [s for s in itertools.product((0, 1), repeat=L) if sum(s) == n_f]


def fields(occ, Q):
    """E_x for x = 0..L-2 (Gauss's law from the left end)."""
    return np.cumsum(np.asarray(occ) - Q)[:-1]


def hamiltonian(L, m, J, g, n_f, sparse=False):
    """H on the n_f-fermion sector, in `basis` order: dense, or a scipy
    sparse matrix when `sparse` (for 16 sites and beyond)."""
    B = basis(L, n_f)
    index = {s: i for i, s in enumerate(B)}
    Q, mx = charges(L), masses(L, m)
    rows, cols, vals = [], [], []
    for i, s in enumerate(B):
        rows.append(i)
        cols.append(i)
        vals.append(mx @ np.asarray(s) + g * np.sum(fields(s, Q) ** 2))
        for x in range(L - 1):
            if s[x] == 0 and s[x + 1] == 1:          # c^dag_x U_x c_{x+1}: fermion x+1 -> x
                t = list(s)
                t[x], t[x + 1] = 1, 0
                j = index[tuple(t)]
                rows += [j, i]
                cols += [i, j]
                vals += [J, np.conj(J)]
    if sparse:
        import scipy.sparse as sp

        return sp.csr_matrix((np.array(vals, dtype=np.complex128), (rows, cols)), shape=(len(B), len(B))), B
    H = np.zeros((len(B), len(B)), dtype=np.complex128)
    np.add.at(H, (rows, cols), vals)
    return H, B


# ---------------------------------------------------------------------------
# GCF time evolution on a U(1)-symmetric MPS
# ---------------------------------------------------------------------------

class ChargedMPS:
    """Site tensors A[x] (left bond, occupation, right bond) and the charge
    (electric field) of every bond state; bond x+1 sits right of site x,
    bond 0 is the left end (E = 0)."""

    def __init__(self, occ):
        occ = list(occ)
        L = len(occ)
        Q = charges(L)
        self.L, self.Q = L, Q
        self.A = []
        for n in occ:
            t = np.zeros((1, 2, 1), dtype=np.complex128)
            t[0, n, 0] = 1.0
            self.A.append(t)
        e = np.concatenate([[0], np.cumsum(np.asarray(occ) - Q)])
        self.q = [np.array([int(v)]) for v in e]   # q[b]: charges of bond b's states

    def dense(self, B):
        """Amplitudes on the basis list B (occupation tuples)."""
        out = np.zeros(len(B), dtype=np.complex128)
        for i, s in enumerate(B):
            v = np.ones(1, dtype=np.complex128)
            for x, n in enumerate(s):
                v = v @ self.A[x][:, n, :]
            out[i] = v.sum()
        return out


def _bond_gate(qa, x, L, m, J, g, tau, Q):
    """exp(-tau h) on (n_x, n_{x+1}) for left-bond charge qa: h holds the
    hopping J c^dag_x c_{x+1} + h.c., m_x n_x (and m_{x+1} n_{x+1} on the last
    bond) and g E_x^2 with E_x = qa + n_x - Q_x.  Basis index n_x * 2 + n_{x+1}."""
    mx = masses(L, m)
    h = np.zeros((4, 4), dtype=np.complex128)
    for n1 in (0, 1):
        for n2 in (0, 1):
            k = 2 * n1 + n2
            E = qa + n1 - Q[x]
            h[k, k] = mx[x] * n1 + g * E * E + (mx[x + 1] * n2 if x + 1 == L - 1 else 0.0)
    h[2, 1] += J                # |n_x = 1, n_{x+1} = 0> <- |0, 1>
    h[1, 2] += np.conj(J)
    w, v = np.linalg.eigh(h)
    return (v * np.exp(-tau * w)) @ v.conj().T


def _update(mps, x, gates, chi, move_right):
    """Apply the gates of bond (x, x+1) and split per middle charge."""
    A1, A2 = mps.A[x], mps.A[x + 1]
    qa, qb = mps.q[x], mps.q[x + 2]
    th = np.einsum("asc,ctb->astb", A1, A2)
    out = np.zeros_like(th)
    for a in range(th.shape[0]):
        G = gates[int(qa[a])]
        out[a] = np.einsum("kl,lb->kb", G, th[a].reshape(4, -1)).reshape(2, 2, -1)
    th = out
    Dl, Dr = th.shape[0], th.shape[3]
    Qx = mps.Q[x]
    rows = {}
    for a in range(Dl):
        for s in (0, 1):
            rows.setdefault(int(qa[a]) + s - Qx, []).append((a, s))
    cols = {}
    Qy = mps.Q[x + 1]
    for b in range(Dr):
        for t in (0, 1):
            cols.setdefault(int(qb[b]) - t + Qy, []).append((t, b))
    blocks = []
    for c in sorted(set(rows) & set(cols)):
        R, C = rows[c], cols[c]
        M = np.array([[th[a, s, t, b] for (t, b) in C] for (a, s) in R])
        U, S, Vh = np.linalg.svd(M, full_matrices=False)
        for k in range(len(S)):
            blocks.append((S[k], c, R, C, U[:, k], Vh[k]))
    blocks.sort(key=lambda z: -z[0])
    blocks = [z for z in blocks[:chi] if z[0] > 1e-14 * blocks[0][0]] if blocks else []
    norm = np.sqrt(sum(z[0] ** 2 for z in blocks))
    k = len(blocks)
    N1 = np.zeros((Dl, 2, k), dtype=np.complex128)
    N2 = np.zeros((k, 2, Dr), dtype=np.complex128)
    for j, (s_, c, R, C, u, vh) in enumerate(blocks):
        sv = s_ / norm
        for r, (a, s) in enumerate(R):
            N1[a, s, j] = u[r] * (sv if not move_right else 1.0)
        for cc, (t, b) in enumerate(C):
            N2[j, t, b] = vh[cc] * (sv if move_right else 1.0)
    mps.A[x], mps.A[x + 1] = N1, N2
    mps.q[x + 1] = np.array([z[1] for z in blocks])


def evolve(mps, L, m, J, g, tau, n_steps, chi):
    """n_steps second-order steps of exp(-tau H): a left-to-right sweep of
    the bond gates with tau / 2 and a right-to-left sweep with tau / 2.
    tau real: imaginary time (normalised); tau = i dt: real time."""
    Q = charges(L)
    half = tau / 2.0
    for _ in range(n_steps):
        for direction in (1, -1):
            order = range(L - 1) if direction == 1 else range(L - 2, -1, -1)
            for x in order:
                qs = set(int(v) for v in mps.q[x])
                gates = {qa: _bond_gate(qa, x, L, m, J, g, half, Q) for qa in qs}
                _update(mps, x, gates, chi, move_right=(direction == 1))
    return mps
