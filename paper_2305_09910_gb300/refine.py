"""A lattice with one z slab refined 2:1 (Sec. 3, Fig. 2: the block forest refines blocks 2:1
and interpolation kernels carry the populations across coarse-fine transitions; Sec. 5.2
runs them between the levels of the landing-gear case).

A refined slab (coarse planes z0 .. z1-1) is its own fine two-grid pull lattice of
2 nx x 2 ny x 2 (z1 - z0) cells with relaxation time tau_f = 1/2 + 2 (tau_c - 1/2) and body
force F_c / 2 (acoustic scaling: dx and dt halve); the rest of the domain is cut into coarse
lattices, one per run of unrefined planes (with periodic z the run across the faces is one
lattice).  A slab may lie on a global no-slip wall (refinement next to the walls of a
channel), which then bounds its fine lattice.  Facing z faces are halo faces, and the transfer across them
is the volumetric, mass-conserving scheme of Rohde et al. (2006) in pull form, carried out
by the library's ``lbm_refine_explode`` and ``lbm_refine_coalesce``.  x and y are periodic.

Time: ``step(n)`` advances n coarse steps (two fine steps each).  Internally every lattice
holds its post-collision state; after k coarse steps ``get_post_collision`` returns C*(k) and
F*(k), the collision of the pre-collision state at time k of both levels.
"""
from __future__ import annotations

import numpy as np

from . import lbm

FACE_LO, FACE_HI = 4, 5


def fine_tau(tau_c: float) -> float:
    """tau_f - 1/2 = 2 (tau_c - 1/2): the lattice viscosity doubles when dx and dt halve."""
    return 0.5 + 2.0 * (tau_c - 0.5)


def plan(nz: int, slabs, walls: bool):
    """Coarse pieces, fine pieces and interfaces of refined slabs [(z0, z1), ...] in a coarse
    column of nz planes.

    Returns (coarse, fine, interfaces): coarse is a list of (global coarse planes in piece
    order, (face -z, face +z)); fine a list of ((z0, z1), (face -z, face +z)); interfaces a
    list of (coarse piece, coarse face, fine piece, fine face).  Faces are "halo" where a
    coarse and a fine lattice meet, "wall" on a global no-slip face."""
    slabs = sorted((int(a), int(b)) for a, b in slabs)
    if not slabs:
        raise ValueError("no refined slab")
    for a, b in slabs:
        if not (0 <= a < b <= nz):
            raise ValueError("need 0 <= z0 < z1 <= nz")
    for (a0, b0), (a1, b1) in zip(slabs, slabs[1:]):
        if a1 <= b0:
            raise ValueError("refined slabs must be separated by coarse planes")
    covered = [False] * nz
    for a, b in slabs:
        for z in range(a, b):
            covered[z] = True
    ncoarse = nz - sum(covered)
    if ncoarse < 1 or (not walls and len(slabs) == 1 and ncoarse < 2):
        raise ValueError("too few coarse planes outside the refined slabs")
    if not walls and covered[0] and covered[-1]:
        raise ValueError("with periodic z faces the first and last slabs would touch")
    runs, z = [], 0
    while z < nz:  # maximal runs of coarse planes
        if covered[z]:
            z += 1
            continue
        start = z
        while z < nz and not covered[z]:
            z += 1
        runs.append(list(range(start, z)))
    if not walls and len(runs) > 1 and runs[0][0] == 0 and runs[-1][-1] == nz - 1:
        runs[0] = runs.pop() + runs[0]  # periodic z: the run across the faces is one piece
    coarse = []
    for planes in runs:
        flo = "wall" if walls and planes[0] == 0 else "halo"
        fhi = "wall" if walls and planes[-1] == nz - 1 else "halo"
        coarse.append((planes, (flo, fhi)))
    fine = [((a, b), ("wall" if walls and a == 0 else "halo", "wall" if walls and b == nz else "halo"))
            for a, b in slabs]
    first = {planes[0]: k for k, (planes, _) in enumerate(coarse)}
    last = {planes[-1]: k for k, (planes, _) in enumerate(coarse)}
    interfaces = []
    for j, ((a, b), (flo, fhi)) in enumerate(fine):
        if flo == "halo":
            interfaces.append((last[(a - 1) % nz], FACE_HI, j, FACE_LO))
        if fhi == "halo":
            interfaces.append((first[b % nz], FACE_LO, j, FACE_HI))
    return coarse, fine, interfaces


class RefinedSlab:
    """A coarse nx x ny x nz lattice (periodic x, y; periodic or no-slip z faces) whose planes
    z0 .. z1-1 are refined 2:1, or several such slabs (``slabs=[(z0, z1), ...]``; a slab may
    lie on a wall, which then bounds its fine lattice)."""

    def __init__(self, nx, ny, nz, z0=None, z1=None, stencil=19, tau=0.8, walls=False, force=(0.0, 0.0, 0.0),
                 slabs=None, **params):
        params = dict(params)
        params["streaming"] = "pull"
        for k in ("faces", "u_inflow", "rho_inflow"):
            if k in params:
                raise ValueError(f"{k} is fixed by the refined slab")
        if slabs is None:
            slabs = [(z0, z1)]
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.q, self.walls = int(stencil), bool(walls)
        coarse, fine, self.interfaces = plan(self.nz, slabs, self.walls)
        self.planes = [p for p, _ in coarse]
        self.slabs = [zz for zz, _ in fine]
        self.nzfs = [2 * (b - a) for a, b in self.slabs]
        force = tuple(float(v) for v in force)
        self.coarse, self.fines = [], []
        try:
            for planes, (flo, fhi) in coarse:
                lat = lbm.Lattice(self.nx, self.ny, len(planes), stencil=self.q, tau=tau,
                                  faces=("periodic",) * 4 + (flo, fhi), **params)
                self.coarse.append(lat)
                lat.set_force(*force)  # cells are all fluid from creation, ghost planes included
            for nzf, (_, (flo, fhi)) in zip(self.nzfs, fine):
                lat = lbm.Lattice(2 * self.nx, 2 * self.ny, nzf, stencil=self.q, tau=fine_tau(tau),
                                  faces=("periodic",) * 4 + (flo, fhi), **params)
                self.fines.append(lat)
                lat.set_force(*(v / 2 for v in force))
        except Exception:
            self.close()
            raise
        self._primed = False

    @property
    def fine(self):
        """The fine lattice of the first slab."""
        return self.fines[0]

    @property
    def nzf(self):
        return self.nzfs[0]

    # ---- state -------------------------------------------------------------------------------
    def init_equilibrium(self, rho_c=None, u_c=None, rho_f=None, u_f=None):
        """rho_c (nz, ny, nx), u_c (3, nz, ny, nx) on the coarse grid (the covered planes are
        ignored); rho_f, u_f on the fine grid of each slab (nzf, 2 ny, 2 nx), as lists with
        several slabs.  None: rho = 1, u = 0."""
        for lat, planes in zip(self.coarse, self.planes):
            r = None if rho_c is None else np.ascontiguousarray(np.asarray(rho_c, dtype=np.float32)[planes])
            v = None if u_c is None else np.ascontiguousarray(np.asarray(u_c, dtype=np.float32)[:, planes])
            lat.init_equilibrium(r, v)
        rho_f, u_f = self._per_slab(rho_f), self._per_slab(u_f)
        for lat, r, v in zip(self.fines, rho_f, u_f):
            lat.init_equilibrium(r, v)
        self._primed = False

    def _per_slab(self, a):
        """One entry per slab: a list as given, None for every slab, or a single array for a
        single slab."""
        if isinstance(a, (list, tuple)):
            if len(a) != len(self.fines):
                raise ValueError(f"expected {len(self.fines)} fine-level arrays, got {len(a)}")
            return list(a)
        if a is None:
            return [None] * len(self.fines)
        if len(self.fines) != 1:
            raise ValueError("several refined slabs: pass one fine-level array per slab (a list)")
        return [a]

    def set_populations(self, dfc, dff):
        """Shifted populations df = f - w (pre-collision): dfc (q, nz, ny, nx), dff one
        (q, nzf, 2 ny, 2 nx) array per slab (a list with several slabs)."""
        dfc = np.asarray(dfc, dtype=np.float32)
        for lat, planes in zip(self.coarse, self.planes):
            lat.set_populations(np.ascontiguousarray(dfc[:, planes]))
        for lat, d in zip(self.fines, self._per_slab(dff)):
            lat.set_populations(np.ascontiguousarray(d, dtype=np.float32))
        self._primed = False

    def get_post_collision(self):
        """(C*, F*): shifted post-collision populations of both levels; covered coarse planes
        NaN; F* one array, or a list with several slabs."""
        out = np.full((self.q, self.nz, self.ny, self.nx), np.nan, dtype=np.float32)
        for lat, planes in zip(self.coarse, self.planes):
            out[:, planes] = lat.get_post_collision()
        fs = [lat.get_post_collision() for lat in self.fines]
        return out, fs[0] if len(fs) == 1 else fs

    # ---- stepping ----------------------------------------------------------------------------
    def _prime(self):
        """Collision only (the first step after an import gathers from the own cell): both
        levels then hold post-collision states at the same time."""
        for lat in self.coarse + self.fines:
            lat.step(1)
        self._primed = True

    def step(self, n: int = 1):
        if n <= 0:
            return
        if not self._primed:
            self._prime()
        for _ in range(int(n)):
            for k, cf, j, ff in self.interfaces:
                lbm.lbm_refine_explode(self.coarse[k].h, cf, self.fines[j].h, ff, 0)
            for lat in self.fines:
                lbm.lbm_step(lat.h, 1)
            for k, cf, j, ff in self.interfaces:
                lbm.lbm_refine_coalesce(self.fines[j].h, ff, self.coarse[k].h, cf)
            for k, cf, j, ff in self.interfaces:
                lbm.lbm_refine_explode(self.coarse[k].h, cf, self.fines[j].h, ff, 1)
            for lat in self.fines:
                lbm.lbm_step(lat.h, 1)
            for lat in self.coarse:
                lbm.lbm_step(lat.h, 1)

    def sync(self):
        for lat in self.coarse + self.fines:
            lat.sync()

    # ---- diagnostics -------------------------------------------------------------------------
    @property
    def updates_per_step(self) -> int:
        """Cell updates per coarse step: every coarse cell once, every fine cell twice."""
        nc = sum(len(p) for p in self.planes)
        return self.nx * self.ny * nc + 2 * 4 * self.nx * self.ny * sum(self.nzfs)

    def mass(self):
        """Total mass in fine-cell volumes (8 per coarse cell), FP64 from the post-collision
        state (the collision conserves mass)."""
        w = np.asarray(lbm.lbm_stencil(self.q)[1], dtype=np.float64)[:, None, None, None]
        m = 0.0
        for lat in self.coarse:
            m += 8.0 * (lat.get_post_collision().astype(np.float64) + w).sum()
        for lat in self.fines:
            m += (lat.get_post_collision().astype(np.float64) + w).sum()
        return m

    def close(self):
        for lat in getattr(self, "coarse", []) + getattr(self, "fines", []):
            lat.close()
        self.coarse, self.fines = [], []
