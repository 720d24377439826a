"""Z_N lattice gauge theory on an open Lx x Ly square lattice (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Conventions (main text, "Hamiltonian" paragraph):

* vertex (x, y), x in [0, Lx) to the right (e_1), y in [0, Ly) up (e_2);
* link (x, 1) joins (x, y) and (x+1, y) ("horizontal", value h[y][x]);
  link (x, 2) joins (x, y) and (x, y+1) ("vertical",   value v[y][x]);
* electric field E|n> = n|n>, n in Z_N; raising operator U|n> = |n+1 mod N>;
* hard-core boson occupation p in {0, 1} per vertex (matter models only).

Flat configuration layout (the interface shared with the CUDA library, int8):
``[h (Ly x (Lx-1)) row-major][v ((Ly-1) x Lx) row-major][p (Ly x Lx) row-major]``.

Gauss law, Eq. (1) and Eq. (S4): at every vertex
    p + n_l + n_d - n_r - n_u = Q_x  (mod N)
with n_l the link to the left, n_d below, n_r to the right, n_u above; a link
that does not exist on the open boundary counts as n = 0.

Hamiltonian, Eqs. (2)-(5):
    H_M = sum_x m p_x + sum_{x,a} (J c_x^dag U_(x,a) c_(x+e_a) + h.c.)
    H_B = -h sum_x (P_x + P_x^dag),  P_x = U_(x,1) U_(x+e1,2) U_(x+e2,1)^dag U_(x,2)^dag
    H_E = g sum_links (2 - 2 cos(2 pi n / N))
For N = 2, P_x = P_x^dag, so the magnetic term is -2h P_x; this factor 2 is what
reproduces the paper's printed exact-diagonalisation energy (tests).
"""

from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Lattice:
    Lx: int
    Ly: int
    N: int
    matter: bool = False
    Q: np.ndarray | None = None  # (Ly, Lx) background charges, default 0
    n_h: int = field(init=False)
    n_v: int = field(init=False)
    n_s: int = field(init=False)
    cfg_len: int = field(init=False)

    def __post_init__(self):
        if self.Lx < 2 or self.Ly < 2 or self.N < 2:
            raise ValueError("need Lx, Ly >= 2 and N >= 2")
        self.n_h = self.Ly * (self.Lx - 1)
        self.n_v = (self.Ly - 1) * self.Lx
        self.n_s = self.Lx * self.Ly
        self.cfg_len = self.n_h + self.n_v + self.n_s
        if self.Q is None:
            self.Q = np.zeros((self.Ly, self.Lx), dtype=np.int64)
        self.Q = np.asarray(self.Q, dtype=np.int64).reshape(self.Ly, self.Lx) % self.N

    # ---- flat indices -------------------------------------------------
    def hi(self, x, y):
        return y * (self.Lx - 1) + x

    def vi(self, x, y):
        return self.n_h + y * self.Lx + x

    def pi(self, x, y):
        return self.n_h + self.n_v + y * self.Lx + x

    @property
    def n_plaquettes(self):
        return (self.Lx - 1) * (self.Ly - 1)

    # ---- legs ---------------------------------------------------------
    def has_legs(self, x, y):
        """(has_l, has_r, has_d, has_u) on the open lattice."""
        return (x > 0, x < self.Lx - 1, y > 0, y < self.Ly - 1)

    def leg_values(self, cfg, x, y):
        """Electric fields (n_l, n_r, n_d, n_u) at vertex (x, y); 0 if absent."""
        nl = int(cfg[self.hi(x - 1, y)]) if x > 0 else 0
        nr = int(cfg[self.hi(x, y)]) if x < self.Lx - 1 else 0
        nd = int(cfg[self.vi(x, y - 1)]) if y > 0 else 0
        nu = int(cfg[self.vi(x, y)]) if y < self.Ly - 1 else 0
        return nl, nr, nd, nu

    def gauss_residual(self, cfg):
        """(Ly, Lx) array of p + n_l + n_d - n_r - n_u - Q mod N (0 = physical)."""
        res = np.zeros((self.Ly, self.Lx), dtype=np.int64)
        for y in range(self.Ly):
            for x in range(self.Lx):
                nl, nr, nd, nu = self.leg_values(cfg, x, y)
                p = int(cfg[self.pi(x, y)])
                res[y, x] = (p + nl + nd - nr - nu - self.Q[y, x]) % self.N
        return res

    def is_physical(self, cfg):
        if self.matter:
            if np.any((np.asarray(cfg[self.n_h + self.n_v:]) < 0) | (np.asarray(cfg[self.n_h + self.n_v:]) > 1)):
                return False
        elif np.any(np.asarray(cfg[self.n_h + self.n_v:]) != 0):
            return False
        return not np.any(self.gauss_residual(cfg))

    # ---- moves (Sec. S-2) ---------------------------------------------
    def plaquette(self, cfg, x, y, t=1):
        """P_x^t on the plaquette with lower-left corner (x, y), Eq. (4)."""
        c = np.array(cfg, dtype=np.int64)
        N = self.N
        c[self.hi(x, y)] = (c[self.hi(x, y)] + t) % N          # U_(x,1)
        c[self.vi(x + 1, y)] = (c[self.vi(x + 1, y)] + t) % N  # U_(x+e1,2)
        c[self.hi(x, y + 1)] = (c[self.hi(x, y + 1)] - t) % N  # U_(x+e2,1)^dag
        c[self.vi(x, y)] = (c[self.vi(x, y)] - t) % N          # U_(x,2)^dag
        return c

    def link_index(self, x, y, a):
        return self.hi(x, y) if a == 1 else self.vi(x, y)

    def hop(self, cfg, x, y, a):
        """The single gauge-dressed hop across link (x, a), or None.

        c_x^dag U_(x,a) c_(x+e_a) moves a boson from x+e_a to x and raises the
        link; its conjugate moves it from x to x+e_a and lowers the link
        (Eq. 3).  On a hard-core lattice at most one of the two applies.
        """
        x2, y2 = (x + 1, y) if a == 1 else (x, y + 1)
        c = np.array(cfg, dtype=np.int64)
        s1, s2, li = self.pi(x, y), self.pi(x2, y2), self.link_index(x, y, a)
        if c[s1] == 0 and c[s2] == 1:
            c[s1], c[s2] = 1, 0
            c[li] = (c[li] + 1) % self.N
            return c
        if c[s1] == 1 and c[s2] == 0:
            c[s1], c[s2] = 0, 1
            c[li] = (c[li] - 1) % self.N
            return c
        return None

    # ---- Hamiltonian (Eqs. 2-5) ----------------------------------------
    def diagonal_energy(self, cfg, g, m=0.0):
        n = np.asarray(cfg[: self.n_h + self.n_v], dtype=np.float64)
        e = g * np.sum(2.0 - 2.0 * np.cos(2.0 * np.pi * n / self.N))
        if self.matter:
            e += m * float(np.sum(cfg[self.n_h + self.n_v:]))
        return float(e)

    def off_diagonal(self, cfg, h, J=0.0):
        """All (cfg', <cfg'|H|cfg>) with cfg' != cfg reached by one term of H.

        H_B: -h for P_x and -h for P_x^dag; for N = 2 they coincide (-2h).
        H_M hopping: J for either direction (J real).
        """
        out = []
        for y in range(self.Ly - 1):
            for x in range(self.Lx - 1):
                if self.N == 2:
                    out.append((self.plaquette(cfg, x, y, 1), -2.0 * h))
                else:
                    out.append((self.plaquette(cfg, x, y, 1), -h))
                    out.append((self.plaquette(cfg, x, y, self.N - 1), -h))
        if self.matter and J != 0.0:
            for y in range(self.Ly):
                for x in range(self.Lx):
                    for a in (1, 2):
                        if (a == 1 and x == self.Lx - 1) or (a == 2 and y == self.Ly - 1):
                            continue
                        c2 = self.hop(cfg, x, y, a)
                        if c2 is not None:
                            out.append((c2, J))
        return out

    # ---- physical basis ------------------------------------------------
    def gauge_fixed_base(self, occ):
        """A physical link configuration for occupations ``occ`` (Ly, Lx).

        Links off the comb tree (vertical links in columns x >= 1) are 0; the
        tree links (all horizontal links, vertical links in column 0) are
        fixed leaf-first so that every vertex satisfies Eq. (1).  Requires
        sum(p) = sum(Q) mod N (the global constraint of an open lattice).
        """
        occ = np.asarray(occ, dtype=np.int64).reshape(self.Ly, self.Lx)
        N, Lx, Ly = self.N, self.Lx, self.Ly
        if (occ.sum() - self.Q.sum()) % N:
            raise ValueError("sum of occupations must equal sum of charges mod N")
        c = np.zeros(self.cfg_len, dtype=np.int64)
        c[self.n_h + self.n_v:] = occ.reshape(-1)
        for y in range(Ly):
            # Along the row from the right: p + n_l - n_r = Q at (x, y), x >= 1.
            nr = 0
            for x in range(Lx - 1, 0, -1):
                nl = (self.Q[y, x] - occ[y, x] + nr) % N
                c[self.hi(x - 1, y)] = nl
                nr = nl
        nu = 0
        for y in range(Ly - 1, 0, -1):
            # Column 0: p + n_d - n_r - n_u = Q at (0, y).
            nr = c[self.hi(0, y)]
            nd = (self.Q[y, 0] - occ[y, 0] + nr + nu) % N
            c[self.vi(0, y - 1)] = nd
            nu = nd
        return c

    def config_from_powers(self, occ, powers):
        """gauge_fixed_base(occ) followed by P_j^{t_j} for every plaquette j."""
        c = self.gauge_fixed_base(occ)
        powers = np.asarray(powers, dtype=np.int64).reshape(self.Ly - 1, self.Lx - 1)
        for y in range(self.Ly - 1):
            for x in range(self.Lx - 1):
                if powers[y, x] % self.N:
                    c = self.plaquette(c, x, y, int(powers[y, x]))
        return c

    def occupation_patterns(self, n_bosons=None):
        """All matter configurations allowed by the global Gauss constraint."""
        if not self.matter:
            return [np.zeros((self.Ly, self.Lx), dtype=np.int64)]
        pats = []
        for bits in itertools.product((0, 1), repeat=self.n_s):
            b = np.array(bits, dtype=np.int64).reshape(self.Ly, self.Lx)
            if n_bosons is not None and b.sum() != n_bosons:
                continue
            if (b.sum() - self.Q.sum()) % self.N == 0:
                pats.append(b)
        return pats

    def physical_basis(self, n_bosons=None):
        """All physical configurations: base(occ) times every plaquette power set."""
        basis = []
        for occ in self.occupation_patterns(n_bosons):
            for t in itertools.product(range(self.N), repeat=self.n_plaquettes):
                basis.append(self.config_from_powers(occ, t))
        return np.array(basis, dtype=np.int64)

    def brute_force_physical(self):
        """Physical configurations by filtering every link/matter assignment."""
        out = []
        occs = itertools.product((0, 1), repeat=self.n_s) if self.matter else [(0,) * self.n_s]
        for occ in occs:
            for links in itertools.product(range(self.N), repeat=self.n_h + self.n_v):
                c = np.array(links + tuple(occ), dtype=np.int64)
                if not np.any(self.gauss_residual(c)):
                    out.append(c)
        return np.array(out, dtype=np.int64)

    def hamiltonian_matrix(self, basis, h, g, J=0.0, m=0.0):
        """Dense H[i, j] = <b_i|H|b_j> on a closed basis (exact diagonalisation)."""
        index = {tuple(b): i for i, b in enumerate(basis)}
        n = len(basis)
        H = np.zeros((n, n))
        for j, b in enumerate(basis):
            H[j, j] += self.diagonal_energy(b, g, m)
            for b2, amp in self.off_diagonal(b, h, J):
                H[index[tuple(b2)], j] += amp
        return H
