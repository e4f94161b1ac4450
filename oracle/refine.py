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
* a coarse cell is the volume of 2 x 2 x 2 fine cells; a refined slab covers the coarse
  planes z0 .. z1-1, and its fine lattice has two ghost planes on each z side that meets
  coarse cells, which lie in the volume of the first coarse plane outside the slab (the coarse
  interface cells); a side on a global no-slip wall has no ghost planes;
* one coarse step: (1) collide the coarse cells; (2) explosion: every fine ghost cell takes
  the post-collision populations of the coarse interface cell whose volume it lies in,
  unchanged; (3) two fine steps, each a collision of the fine interior cells followed by
  streaming of all fine cells, ghost cells included (these are streamed, never collided);
  (4) coalescence: the populations of a coarse interface cell that point away from the slab
  are the mean of the values the 8 fine ghost cells in its volume hold after the second
  fine step; (5) stream the coarse cells; a population that would arrive from a covered
  coarse cell is the coalesced one.

Populations are plain (unshifted) pre-collision values, shape (q, nz, ny, nx) per lattice;
the x and y faces are periodic, the global z faces periodic or no-slip walls (halfway
bounce-back, on whichever level meets them).  Covered coarse cells hold NaN so that any use
of them shows.  Streaming is written here in push form (f_i(x + c_i) = f*_i(x)) on numpy
arrays; the collision is the C oracle's (Eq. LBCollision).
"""
from __future__ import annotations

import numpy as np

from . import Oracle, stencil


def fine_tau(tau_c: float) -> float:
    """Relaxation time of the fine level under acoustic scaling: tau_f - 1/2 = 2 (tau_c - 1/2)."""
    return 0.5 + 2.0 * (tau_c - 0.5)


class _Slab:
    """One refined slab: its fine lattice and which of its z sides meet coarse cells."""

    def __init__(self, z0, z1, nz, walls):
        self.z0, self.z1 = z0, z1
        self.nzf = 2 * (z1 - z0)
        self.ghost_lo = not (walls and z0 == 0)
        self.ghost_hi = not (walls and z1 == nz)
        self.lo = (z0 - 1) % nz if self.ghost_lo else None  # coarse interface planes
        self.hi = z1 % nz if self.ghost_hi else None
        self.g0 = 2 if self.ghost_lo else 0  # first interior plane of the extended array


class RefinedOracle:
    """A coarse nx x ny x nz lattice whose planes z0 .. z1-1 are refined 2:1, or several such
    slabs (``slabs=[(z0, z1), ...]``)."""

    def __init__(self, nx, ny, nz, z0=None, z1=None, q=19, tau=0.8, lam=3.0 / 16.0, closure="none", cs=0.0,
                 force=(0.0, 0.0, 0.0), walls=False, slabs=None):
        if slabs is None:
            slabs = [(z0, z1)]
        slabs = sorted((int(a), int(b)) for a, b in slabs)
        for a, b in slabs:
            if not (0 <= a < b <= nz):
                raise ValueError("need 0 <= z0 < z1 <= nz")
        for (a0, b0), (a1, b1) in zip(slabs, slabs[1:]):
            if a1 <= b0:
                raise ValueError("refined slabs must be separated by coarse planes")
        ncov = sum(b - a for a, b in slabs)
        if nz - ncov < 1 or (not walls and len(slabs) == 1 and nz - ncov < 2):
            raise ValueError("too few coarse planes outside the refined slabs")
        if not walls and slabs[0][0] == 0 and slabs[-1][1] == nz:
            raise ValueError("with periodic z faces the first and last slabs would touch")
        self.nx, self.ny, self.nz, self.q = nx, ny, nz, q
        self.walls = walls
        zf = ("wall", "wall") if walls else ("periodic", "periodic")
        force = tuple(float(v) for v in force)
        self.coarse = Oracle(nx, ny, nz, q=q, tau=tau, lam=lam, closure=closure, cs=cs,
                             faces=("periodic",) * 4 + zf, force=force)
        self.slabs = [_Slab(a, b, nz, walls) for a, b in slabs]
        self.fines = [Oracle(2 * nx, 2 * ny, s.nzf, q=q, tau=fine_tau(tau), lam=lam, closure=closure, cs=cs,
                             faces=("periodic",) * 6, force=tuple(v / 2 for v in force)) for s in self.slabs]
        self.c, self.w, self.opp = stencil(q)
        self.covered = np.zeros(nz, dtype=bool)
        for a, b in slabs:
            self.covered[a:b] = True
        self.fc = self.coarse.f
        self.ffs = [o.f for o in self.fines]
        self.fc[:, self.covered] = np.nan

    # ---- the single-slab view (the transfer pins use it) ------------------------------------
    @property
    def fine(self):
        return self.fines[0]

    @fine.setter
    def fine(self, oracle):
        self.fines[0] = oracle

    @property
    def ff(self):
        return self.ffs[0]

    @property
    def nzf(self):
        return self.slabs[0].nzf

    @property
    def lo(self):
        return self.slabs[0].lo

    @property
    def hi(self):
        return self.slabs[0].hi

    # ---- state -------------------------------------------------------------------------------
    def init_equilibrium(self, rho_c, u_c, rho_f, u_f):
        """rho_f, u_f: one value (or field) per slab as a list, or one for a single slab."""
        self.coarse.init_equilibrium(rho_c, u_c)
        if len(self.slabs) == 1 and not isinstance(rho_f, list):
            rho_f, u_f = [rho_f], [u_f]
        for o, r, u in zip(self.fines, rho_f, u_f):
            o.init_equilibrium(r, u)
        self.fc = self.coarse.f
        self.ffs = [o.f for o in self.fines]
        self.fc[:, self.covered] = np.nan

    def set_shifted(self, dfc, dff):
        """Plain populations w + df on both levels (df as a GPU state holds them); dff is one
        array per slab (a list) or one array for a single slab."""
        w = self.w[:, None, None, None]
        self.fc = w + np.asarray(dfc, dtype=np.float64)
        self.fc[:, self.covered] = np.nan
        if len(self.slabs) == 1 and not isinstance(dff, list):
            dff = [dff]
        self.ffs = [w + np.asarray(d, dtype=np.float64) for d in dff]

    def post_collision(self):
        """(f*_c, f*_f): Eq. LBCollision applied to the current pre-collision state (f*_f a list
        with several slabs)."""
        fs = [o.collide_all(f) for o, f in zip(self.fines, self.ffs)]
        return self.coarse.collide_all(self.fc), fs[0] if len(fs) == 1 else fs

    def mass(self):
        """Total mass in fine-cell volumes: 8 per coarse cell, 1 per fine cell."""
        return 8.0 * np.nansum(self.fc[:, ~self.covered]) + sum(f.sum() for f in self.ffs)

    def momentum(self):
        c = self.c.astype(np.float64)
        jc = c.T @ self.fc[:, ~self.covered].reshape(self.q, -1).sum(axis=1)
        jf = sum(c.T @ f.reshape(self.q, -1).sum(axis=1) for f in self.ffs)
        return 8.0 * jc + jf

    # ---- the transfer steps ------------------------------------------------------------------
    def explode(self, cstar, k=0):
        """Fine array of slab k with its ghost planes, shape (q, g + nzf, 2 ny, 2 nx): the ghost
        planes take the coarse interface cells' post-collision populations (all directions,
        unchanged, 2 x 2 x 2 fine cells per coarse cell); the interior is NaN."""
        s = self.slabs[k]
        nze = s.nzf + 2 * s.ghost_lo + 2 * s.ghost_hi
        ext = np.full((self.q, nze, 2 * self.ny, 2 * self.nx), np.nan)
        sides = []
        if s.ghost_lo:
            sides.append((s.lo, (0, 1)))
        if s.ghost_hi:
            sides.append((s.hi, (nze - 2, nze - 1)))
        for zc, planes in sides:
            block = np.repeat(np.repeat(cstar[:, zc], 2, axis=1), 2, axis=2)
            for zp in planes:
                ext[:, zp] = block
        return ext

    def fine_stream(self, fstar_ext, k=0):
        """Push streaming of every fine cell of slab k, ghost planes included:
        f_i(x + c_i) = f*_i(x), periodic in x and y; what leaves the extended array is dropped
        (a plane with no source keeps NaN), except through a global wall, where it returns
        reversed to its cell (halfway bounce-back)."""
        s = self.slabs[k]
        out = np.full_like(fstar_ext, np.nan)
        nz = fstar_ext.shape[1]
        for i in range(self.q):
            cx, cy, cz = (int(v) for v in self.c[i])
            moved = np.roll(fstar_ext[i], (cy, cx), axis=(1, 2))
            src = slice(max(0, -cz), nz - max(0, cz))
            dst = slice(max(0, cz), nz - max(0, -cz))
            out[i, dst] = moved[src]
        for i in range(self.q):
            cz = int(self.c[i][2])
            if cz == -1 and not s.ghost_lo:
                out[self.opp[i], 0] = fstar_ext[i, 0]
            elif cz == 1 and not s.ghost_hi:
                out[self.opp[i], nz - 1] = fstar_ext[i, nz - 1]
        return out

    def coalesce(self, ext, k=0):
        """{(coarse plane, sign): (q, ny, nx) values}: for each interface plane of slab k, the
        mean over the 8 fine ghost cells in a coarse cell's volume, for the directions pointing
        away from the slab (sign = c_z: -1 below it, +1 above it); other directions are NaN.
        With a single slab the planes alone are keys as well."""
        s = self.slabs[k]
        nze = ext.shape[1]
        sides = []
        if s.ghost_lo:
            sides.append((s.lo, slice(0, 2), -1))
        if s.ghost_hi:
            sides.append((s.hi, slice(nze - 2, nze), 1))
        out = {}
        for zc, planes, sign in sides:
            g = ext[:, planes]  # (q, 2, 2 ny, 2 nx)
            mean = g.reshape(self.q, 2, self.ny, 2, self.nx, 2).mean(axis=(1, 3, 5))
            vals = np.full((self.q, self.ny, self.nx), np.nan)
            for i in range(self.q):
                if self.c[i][2] == sign:
                    vals[i] = mean[i]
            out[(zc, sign)] = vals
            if len(self.slabs) == 1:
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
        for key, vals in coal.items():
            if not isinstance(key, tuple):
                continue
            zc, sign = key
            for i in range(self.q):
                if self.c[i][2] == sign:
                    out[i, zc] = vals[i]
        out[:, self.covered] = np.nan
        return out

    # ---- one coarse step ---------------------------------------------------------------------
    def step(self, n=1):
        for _ in range(int(n)):
            cstar = self.coarse.collide_all(self.fc)
            coal = {}
            for k, (s, o) in enumerate(zip(self.slabs, self.fines)):
                ext = self.explode(cstar, k)
                inner = slice(s.g0, s.g0 + s.nzf)
                ext[:, inner] = self.ffs[k]
                for _sub in range(2):
                    fstar = ext.copy()
                    fstar[:, inner] = o.collide_all(np.ascontiguousarray(ext[:, inner]))
                    ext = self.fine_stream(fstar, k)
                self.ffs[k] = np.ascontiguousarray(ext[:, inner])
                coal.update({key: v for key, v in self.coalesce(ext, k).items() if isinstance(key, tuple)})
            self.fc = self.coarse_stream(cstar, coal)
