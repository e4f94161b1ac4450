"""Exact-arithmetic lattice Boltzmann stepper (test helper, pure Python ``fractions``).

An independent restatement of one step of the method for tiny lattices, used to pin the
FP64 oracle.  It differs from the oracle in every place where a mistake could hide:

* velocity sets are enumerated with ``itertools`` (no literal table) and matched to the
  oracle's order by velocity vector;
* streaming is written in PUSH form (each post-collision population travels along c_i and
  reflects off what it meets), whereas the oracle pulls; the outflow slots left empty by
  the push are filled afterwards from the upstream neighbour;
* all arithmetic is exact rational; the one square root (Smagorinsky) is taken with 80
  significant decimal digits.

Physics (Sec. 2, Eq. LBCollision / Eq. LBStreaming of arXiv 2305.09910, with the TRT,
Guo-forcing, Smagorinsky and boundary readings stated in the oracle's header).
"""
from __future__ import annotations

import itertools
from decimal import Decimal, getcontext
from fractions import Fraction as Fr

getcontext().prec = 80


def velocity_set(q):
    vs = []
    for c in itertools.product((-1, 0, 1), repeat=3):
        n = sum(abs(a) for a in c)
        if q == 19 and n == 3:
            continue
        vs.append(c)
    if q == 19:
        wt = {0: Fr(1, 3), 1: Fr(1, 18), 2: Fr(1, 36)}
    else:
        wt = {0: Fr(8, 27), 1: Fr(2, 27), 2: Fr(1, 54), 3: Fr(1, 216)}
    return {c: wt[sum(abs(a) for a in c)] for c in vs}


def neg(c):
    return tuple(-a for a in c)


def dot(a, b):
    return sum(x * y for x, y in zip(a, b))


def sqrt_fr(v: Fr) -> Fr:
    if v == 0:
        return Fr(0)
    d = (Decimal(v.numerator) / Decimal(v.denominator)).sqrt()
    return Fr(d)


class ExactLattice:
    """cells: dict (x,y,z) -> dict velocity -> Fraction (pre-collision populations)."""

    RANK = {"wall": 4, "inflow": 3, "outflow": 2, "freeslip": 1, "periodic": 1}

    def __init__(self, n, q, tau, lam, force=(0, 0, 0), cs=None, faces=("periodic",) * 6,
                 solid=(), inflow_cells=(), u_w=(0, 0, 0), rho_w=1):
        self.n = tuple(n)
        self.W = velocity_set(q)
        self.tau = Fr(tau)
        self.lam = Fr(lam)
        self.F = tuple(Fr(a) for a in force)
        self.cs = None if cs is None else Fr(cs)
        self.faces = faces
        self.solid = set(map(tuple, solid))
        self.inflow_cells = set(map(tuple, inflow_cells))
        self.u_w = tuple(Fr(a) for a in u_w)
        self.rho_w = Fr(rho_w)
        self.f = {}

    def fluid(self, p):
        return p not in self.solid and p not in self.inflow_cells

    def cells(self):
        nx, ny, nz = self.n
        return [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]

    def moments(self, fc):
        rho = sum(fc.values())
        m = [sum(c[a] * v for c, v in fc.items()) for a in range(3)]
        u = tuple((m[a] + self.F[a] / 2) / rho for a in range(3))
        return rho, u

    def feq(self, rho, u):
        usq = dot(u, u)
        return {c: w * rho * (1 + 3 * dot(c, u) + Fr(9, 2) * dot(c, u) ** 2 - Fr(3, 2) * usq)
                for c, w in self.W.items()}

    def collide(self, fc):
        rho, u = self.moments(fc)
        eq = self.feq(rho, u)
        tau = self.tau
        if self.cs is not None:
            pi = [[sum(c[a] * c[b] * (fc[c] - eq[c]) for c in self.W) for b in range(3)]
                  for a in range(3)]
            qn = sum(pi[a][b] ** 2 for a in range(3) for b in range(3))
            disc = tau ** 2 + 18 * sqrt_fr(Fr(2)) * self.cs ** 2 * sqrt_fr(qn) / rho
            tau = (tau + sqrt_fr(disc)) / 2
        wp = 1 / tau
        wm = 1 / (self.lam / (tau - Fr(1, 2)) + Fr(1, 2))
        forcing = {c: w * (3 * dot(tuple(c[a] - u[a] for a in range(3)), self.F)
                           + 9 * dot(c, u) * dot(c, self.F)) for c, w in self.W.items()}
        out = {}
        for c in self.W:
            o = neg(c)
            fp, fm = (fc[c] + fc[o]) / 2, (fc[c] - fc[o]) / 2
            ep, em = (eq[c] + eq[o]) / 2, (eq[c] - eq[o]) / 2
            Fp, Fm = (forcing[c] + forcing[o]) / 2, (forcing[c] - forcing[o]) / 2
            out[c] = (fc[c] - wp * (fp - ep) - wm * (fm - em) + (1 - wp / 2) * Fp
                      + (1 - wm / 2) * Fm)
        return out

    def _moving_wall(self, c):
        # population arriving with velocity c after bouncing off a wall moving at u_w
        return 6 * self.W[c] * self.rho_w * dot(c, self.u_w)

    def step(self):
        post = {p: self.collide(self.f[p]) for p in self.cells() if self.fluid(p)}
        new = {p: {} for p in post}
        for p, fc in post.items():
            for c, v in fc.items():
                d = [p[a] + c[a] for a in range(3)]
                crossed = []
                for a in range(3):
                    if d[a] < 0:
                        crossed.append((a, self.faces[2 * a]))
                    elif d[a] >= self.n[a]:
                        crossed.append((a, self.faces[2 * a + 1]))
                rank = max([self.RANK[t] for _, t in crossed], default=0)
                back = neg(c)
                if rank == 4:
                    new[p][back] = v
                    continue
                if rank == 3:
                    new[p][back] = v + self._moving_wall(back)
                    continue
                if rank == 2:
                    continue  # leaves through the outflow face
                cv = list(c)
                for a, t in crossed:
                    if t == "periodic":
                        d[a] %= self.n[a]
                    else:  # free-slip: stays in its plane, normal velocity reversed
                        d[a] = p[a]
                        cv[a] = -cv[a]
                d = tuple(d)
                if d in self.solid:
                    new[p][back] = v
                elif d in self.inflow_cells:
                    new[p][back] = v + self._moving_wall(back)
                else:
                    new[d][tuple(cv)] = v
        # outflow slots: copy what the upstream neighbour received, or bounce back
        for p in new:
            for c in self.W:
                if c in new[p]:
                    continue
                up = (p[0] - 1, p[1], p[2])
                assert p[0] == self.n[0] - 1 and c[0] == -1 and self.faces[1] == "outflow"
                if up in new:
                    new[p][c] = new[up][c]
                else:
                    new[p][c] = post[p][neg(c)]
        self.f = new
