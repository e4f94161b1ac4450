"""FP64 oracle of 2:1 static grid refinement across z planes (two levels).

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/``, only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.  It shares no
code with the CUDA path.

What the paper fixes (Sec. 3, Fig. 2 and Sec. 5.2): the domain is a forest of blocks refined
2:1, and besides the stream-collide kernel the code runs interpolation kernels for the
coarse-to-fine and fine-to-coarse transitions; it does not define them.  The reading taken
here is the volumetric, mass-conserving transfer of Rohde, Kandhai, Derksen and van den
Akker (Int. J. Numer. Meth. Fluids 51, 2006), the scheme of waLBerla's refinement
(Schornbaum and Ruede, SIAM J. Sci. Comput. 38, 2016):

* acoustic scaling: dx_f = dx_c / 2 and dt_f = dt_c / 2, so a velocity has the same value in
  the lattice units of both levels, the lattice viscosity doubles,
  tau_f - 1/2 = 2 (tau_c - 1/2), and a body-force density halves, F_f = F_c / 2;
* a coarse cell is the volume of 2 x 2 x 2 fine cells; the refined slab covers the coarse
  planes z0 .. z1-1, and its fine lattice has two ghost planes on each z side, which lie in
  the volume of the first coarse plane outside the slab (the coarse interface cells);
* one coarse step: (1) collide the coarse cells; (2) explosion: every fine ghost cell takes
  the post-collision populations of the coarse interface cell whose volume it lies in,
  unchanged; (3) two fine steps, each a collision of the fine interior cells followed by
  streaming of all fine cells, ghost cells included (these are streamed, never collided);
  (4) coalescence: the populations of a coarse interface cell that point away from the slab
  are the mean of the values the 8 fine ghost cells in its volume hold after the second
  fine step; (5) stream the coarse cells; a population that would arrive from a covered
  coarse cell is the coalesced one.

Populations are plain (unshifted) pre-collision values, shape (q, nz, ny, nx) per level;
the x and y faces are periodic, the global z faces periodic or no-slip walls (halfway
bounce-back).  Covered coarse cells hold NaN so that any use of them shows.  Streaming is
written here in push form (f_i(x + c_i) = f*_i(x)) on numpy arrays; the collision is the C
oracle's (Eq. LBCollision).
"""
from __future__ import annotations

import numpy as np

from . import Oracle, stencil


def fine_tau(tau_c: float) -> float:
    """Relaxation time of the fine level under acoustic scaling: tau_f - 1/2 = 2 (tau_c - 1/2)."""
    return 0.5 + 2.0 * (tau_c - 0.5)


class RefinedOracle:
    """A coarse nx x ny x nz lattice whose planes z0 .. z1-1 are refined 2:1."""

    def __init__(self, nx, ny, nz, z0, z1, q=19, tau=0.8, lam=3.0 / 16.0, closure="none", cs=0.0,
                 force=(0.0, 0.0, 0.0), walls=False):
        if not (0 <= z0 < z1 <= nz):
            raise ValueError("need 0 <= z0 < z1 <= nz")
        if nz - (z1 - z0) < 2:
            raise ValueError("need at least two coarse planes outside the refined slab")
        if walls and (z0 < 1 or z1 > nz - 1):
            raise ValueError("with walls the refined slab must not touch a wall")
        self.nx, self.ny, self.nz, self.z0, self.z1, self.q = nx, ny, nz, z0, z1, q
        self.walls = walls
        zf = ("wall", "wall") if walls else ("periodic", "periodic")
        force = tuple(float(v) for v in force)
        self.coarse = Oracle(nx, ny, nz, q=q, tau=tau, lam=lam, closure=closure, cs=cs,
                             faces=("periodic",) * 4 + zf, force=force)
        self.nzf = 2 * (z1 - z0)
        self.fine = Oracle(2 * nx, 2 * ny, self.nzf, q=q, tau=fine_tau(tau), lam=lam, closure=closure,
                           cs=cs, faces=("periodic",) * 6, force=tuple(v / 2 for v in force))
        self.c, self.w, self.opp = stencil(q)
        self.lo = (z0 - 1) % nz  # coarse interface planes below and above the slab
        self.hi = z1 % nz
        self.covered = np.zeros(nz, dtype=bool)
        self.covered[z0:z1] = True
        self.fc = self.coarse.f
        self.ff = self.fine.f
        self.fc[:, self.covered] = np.nan

    # ---- state -------------------------------------------------------------------------------
    def init_equilibrium(self, rho_c, u_c, rho_f, u_f):
        self.coarse.init_equilibrium(rho_c, u_c)
        self.fine.init_equilibrium(rho_f, u_f)
        self.fc = self.coarse.f
        self.ff = self.fine.f
        self.fc[:, self.covered] = np.nan

    def set_shifted(self, dfc, dff):
        """Plain populations w + df on both levels (df as a GPU state holds them)."""
        self.fc = self.w[:, None, None, None] + np.asarray(dfc, dtype=np.float64)
        self.fc[:, self.covered] = np.nan
        self.ff = self.w[:, None, None, None] + np.asarray(dff, dtype=np.float64)

    def post_collision(self):
        """(f*_c, f*_f): Eq. LBCollision applied to the current pre-collision state."""
        return self.coarse.collide_all(self.fc), self.fine.collide_all(self.ff)

    def mass(self):
        """Total mass in fine-cell volumes: 8 per coarse cell, 1 per fine cell."""
        return 8.0 * np.nansum(self.fc[:, ~self.covered]) + self.ff.sum()

    def momentum(self):
        c = self.c.astype(np.float64)
        jc = c.T @ self.fc[:, ~self.covered].reshape(self.q, -1).sum(axis=1)
        jf = c.T @ self.ff.reshape(self.q, -1).sum(axis=1)
        return 8.0 * jc + jf

    # ---- the transfer steps ------------------------------------------------------------------
    def explode(self, cstar):
        """Fine array with two ghost planes on each side, shape (q, nzf + 4, 2 ny, 2 nx): the
        ghost planes take the coarse interface cells' post-collision populations (all
        directions, unchanged, 2 x 2 x 2 fine cells per coarse cell); the interior is NaN."""
        ext = np.full((self.q, self.nzf + 4, 2 * self.ny, 2 * self.nx), np.nan)
        for zc, planes in ((self.lo, (0, 1)), (self.hi, (self.nzf + 2, self.nzf + 3))):
            block = np.repeat(np.repeat(cstar[:, zc], 2, axis=1), 2, axis=2)
            for zp in planes:
                ext[:, zp] = block
        return ext

    def fine_stream(self, fstar_ext):
        """Push streaming of every fine cell, ghost planes included: f_i(x + c_i) = f*_i(x),
        periodic in x and y; what leaves the extended array is dropped, and a plane with no
        source keeps NaN."""
        out = np.full_like(fstar_ext, np.nan)
        nz = fstar_ext.shape[1]
        for i in range(self.q):
            cx, cy, cz = (int(v) for v in self.c[i])
            moved = np.roll(fstar_ext[i], (cy, cx), axis=(1, 2))
            src = slice(max(0, -cz), nz - max(0, cz))
            dst = slice(max(0, cz), nz - max(0, -cz))
            out[i, dst] = moved[src]
        return out

    def coalesce(self, ext):
        """{coarse plane: (q, ny, nx) values}: for each interface plane, the mean over the 8 fine
        ghost cells in a coarse cell's volume, for the directions pointing away from the slab
        (c_z = -1 below it, +1 above it); other directions are NaN."""
        out = {}
        for zc, planes, sign in ((self.lo, slice(0, 2), -1), (self.hi, slice(self.nzf + 2, self.nzf + 4), 1)):
            g = ext[:, planes]  # (q, 2, 2 ny, 2 nx)
            mean = g.reshape(self.q, 2, self.ny, 2, self.nx, 2).mean(axis=(1, 3, 5))
            vals = np.full((self.q, self.ny, self.nx), np.nan)
            for i in range(self.q):
                if self.c[i][2] == sign:
                    vals[i] = mean[i]
            out[zc] = vals
        return out

    def coarse_stream(self, cstar, coal):
        """Push streaming of the coarse cells (periodic x, y; z periodic or halfway bounce-back
        at the walls); populations arriving from covered cells are the coalesced ones."""
        out = np.empty_like(cstar)
        nz = self.nz
        for i in range(self.q):
            cx, cy, cz = (int(v) for v in self.c[i])
            if not self.walls:
                out[i] = np.roll(cstar[i], (cz, cy, cx), axis=(0, 1, 2))
                continue
            moved = np.roll(cstar[i], (cy, cx), axis=(1, 2))
            out[i] = np.nan
            src = slice(max(0, -cz), nz - max(0, cz))
            dst = slice(max(0, cz), nz - max(0, -cz))
            out[i, dst] = moved[src]
        if self.walls:  # a population that would cross a wall returns reversed to its cell
            for i in range(self.q):
                cz = int(self.c[i][2])
                if cz == -1:
                    out[self.opp[i], 0] = cstar[i, 0]
                elif cz == 1:
                    out[self.opp[i], nz - 1] = cstar[i, nz - 1]
        for zc, vals in coal.items():
            sign = -1 if zc == self.lo else 1
            for i in range(self.q):
                if self.c[i][2] == sign:
                    out[i, zc] = vals[i]
        out[:, self.covered] = np.nan
        return out

    # ---- one coarse step ---------------------------------------------------------------------
    def step(self, n=1):
        for _ in range(int(n)):
            cstar = self.coarse.collide_all(self.fc)
            ext = self.explode(cstar)
            ext[:, 2:-2] = self.ff
            for _sub in range(2):
                fstar = ext.copy()
                fstar[:, 2:-2] = self.fine.collide_all(np.ascontiguousarray(ext[:, 2:-2]))
                ext = self.fine_stream(fstar)
            self.ff = np.ascontiguousarray(ext[:, 2:-2])
            self.fc = self.coarse_stream(cstar, self.coalesce(ext))
