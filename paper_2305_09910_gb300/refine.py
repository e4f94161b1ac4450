"""A lattice with one z slab refined 2:1 (Sec. 3, Fig. 2: the block forest refines blocks 2:1
and interpolation kernels carry the populations across coarse-fine transitions; Sec. 5.2
runs them between the levels of the landing-gear case).

The refined slab (coarse planes z0 .. z1-1) is its own fine two-grid pull lattice of
2 nx x 2 ny x 2 (z1 - z0) cells with relaxation time tau_f = 1/2 + 2 (tau_c - 1/2) and body
force F_c / 2 (acoustic scaling: dx and dt halve); the rest of the domain is one coarse
lattice (periodic z: it wraps around from z1 to z0) or two (no-slip walls at the global z
faces: [0, z0) and [z1, nz)).  Facing z faces are halo faces, and the transfer across them
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


def plan(nz: int, z0: int, z1: int, walls: bool):
    """The coarse pieces and interfaces of a refined slab [z0, z1) in a coarse column of nz planes.

    Returns (pieces, interfaces): pieces is a list of (global coarse planes in piece order,
    (face -z, face +z)); interfaces is a list of (piece index, coarse face, fine face)."""
    if not (0 <= z0 < z1 <= nz):
        raise ValueError("need 0 <= z0 < z1 <= nz")
    if nz - (z1 - z0) < 2:
        raise ValueError("need at least two coarse planes outside the refined slab")
    if not walls:
        planes = list(range(z1, nz)) + list(range(0, z0))
        return [(planes, ("halo", "halo"))], [(0, FACE_LO, FACE_HI), (0, FACE_HI, FACE_LO)]
    if z0 < 1 or z1 > nz - 1:
        raise ValueError("with walls the refined slab must not touch a wall")
    pieces = [(list(range(0, z0)), ("wall", "halo")), (list(range(z1, nz)), ("halo", "wall"))]
    return pieces, [(0, FACE_HI, FACE_LO), (1, FACE_LO, FACE_HI)]


class RefinedSlab:
    """A coarse nx x ny x nz lattice (periodic x, y; periodic or no-slip z faces) whose planes
    z0 .. z1-1 are refined 2:1."""

    def __init__(self, nx, ny, nz, z0, z1, stencil=19, tau=0.8, walls=False, force=(0.0, 0.0, 0.0),
                 **params):
        params = dict(params)
        params["streaming"] = "pull"
        for k in ("faces", "u_inflow", "rho_inflow"):
            if k in params:
                raise ValueError(f"{k} is fixed by the refined slab")
        self.nx, self.ny, self.nz, self.z0, self.z1 = int(nx), int(ny), int(nz), int(z0), int(z1)
        self.q, self.walls = int(stencil), bool(walls)
        self.nzf = 2 * (self.z1 - self.z0)
        pieces, self.interfaces = plan(self.nz, self.z0, self.z1, self.walls)
        self.planes = [p for p, _ in pieces]
        force = tuple(float(v) for v in force)
        self.coarse = []
        try:
            for planes, (flo, fhi) in pieces:
                lat = lbm.Lattice(self.nx, self.ny, len(planes), stencil=self.q, tau=tau,
                                  faces=("periodic",) * 4 + (flo, fhi), **params)
                self.coarse.append(lat)
                lat.set_force(*force)  # cells are all fluid from creation, ghost planes included
            self.fine = lbm.Lattice(2 * self.nx, 2 * self.ny, self.nzf, stencil=self.q, tau=fine_tau(tau),
                                    faces=("periodic",) * 4 + ("halo", "halo"), **params)
            self.fine.set_force(*(v / 2 for v in force))
        except Exception:
            self.close()
            raise
        self._primed = False

    # ---- state -------------------------------------------------------------------------------
    def init_equilibrium(self, rho_c=None, u_c=None, rho_f=None, u_f=None):
        """rho_c (nz, ny, nx), u_c (3, nz, ny, nx) on the coarse grid (the covered planes are
        ignored); rho_f, u_f on the fine grid (nzf, 2 ny, 2 nx).  None: rho = 1, u = 0."""
        for lat, planes in zip(self.coarse, self.planes):
            r = None if rho_c is None else np.ascontiguousarray(np.asarray(rho_c, dtype=np.float32)[planes])
            v = None if u_c is None else np.ascontiguousarray(np.asarray(u_c, dtype=np.float32)[:, planes])
            lat.init_equilibrium(r, v)
        self.fine.init_equilibrium(rho_f, u_f)
        self._primed = False

    def set_populations(self, dfc, dff):
        """Shifted populations df = f - w (pre-collision): dfc (q, nz, ny, nx), dff (q, nzf, 2 ny, 2 nx)."""
        dfc = np.asarray(dfc, dtype=np.float32)
        for lat, planes in zip(self.coarse, self.planes):
            lat.set_populations(np.ascontiguousarray(dfc[:, planes]))
        self.fine.set_populations(np.ascontiguousarray(dff, dtype=np.float32))
        self._primed = False

    def get_post_collision(self):
        """(C*, F*): shifted post-collision populations of both levels; covered coarse planes NaN."""
        out = np.full((self.q, self.nz, self.ny, self.nx), np.nan, dtype=np.float32)
        for lat, planes in zip(self.coarse, self.planes):
            out[:, planes] = lat.get_post_collision()
        return out, self.fine.get_post_collision()

    # ---- stepping ----------------------------------------------------------------------------
    def _prime(self):
        """Collision only (the first step after an import gathers from the own cell): both
        levels then hold post-collision states at the same time."""
        for lat in self.coarse:
            lat.step(1)
        self.fine.step(1)
        self._primed = True

    def step(self, n: int = 1):
        if n <= 0:
            return
        if not self._primed:
            self._prime()
        fine = self.fine.h
        for _ in range(int(n)):
            for k, cf, ff in self.interfaces:
                lbm.lbm_refine_explode(self.coarse[k].h, cf, fine, ff, 0)
            lbm.lbm_step(fine, 1)
            for k, cf, ff in self.interfaces:
                lbm.lbm_refine_coalesce(fine, ff, self.coarse[k].h, cf)
            for k, cf, ff in self.interfaces:
                lbm.lbm_refine_explode(self.coarse[k].h, cf, fine, ff, 1)
            lbm.lbm_step(fine, 1)
            for lat in self.coarse:
                lbm.lbm_step(lat.h, 1)

    def sync(self):
        for lat in self.coarse + [self.fine]:
            lat.sync()

    # ---- diagnostics -------------------------------------------------------------------------
    @property
    def updates_per_step(self) -> int:
        """Cell updates per coarse step: every coarse cell once, every fine cell twice."""
        return self.nx * self.ny * (self.nz - (self.z1 - self.z0)) + 2 * 4 * self.nx * self.ny * self.nzf

    def mass(self):
        """Total mass in fine-cell volumes (8 per coarse cell), FP64 from the post-collision
        state (the collision conserves mass)."""
        w = np.asarray(lbm.lbm_stencil(self.q)[1], dtype=np.float64)[:, None, None, None]
        c, f = self.get_post_collision()
        covered = np.zeros(self.nz, dtype=bool)
        covered[self.z0:self.z1] = True
        return 8.0 * (c[:, ~covered].astype(np.float64) + w).sum() + (f.astype(np.float64) + w).sum()

    def close(self):
        for lat in getattr(self, "coarse", []):
            lat.close()
        self.coarse = []
        if getattr(self, "fine", None) is not None:
            self.fine.close()
            self.fine = None
