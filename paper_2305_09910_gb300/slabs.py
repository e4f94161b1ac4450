"""A lattice split along z into slabs that exchange halos (Sec. 3: blocks with communication
kernels that pack and unpack only the populations crossing a face, 5 of 19 or 9 of 27).

Every slab is its own two-grid pull lattice whose inner z faces are ``"halo"`` faces: the
cells beyond such a face are a ghost plane of populations (and flags) that the neighbouring
slab fills after every step with ``lbm_halo_pack`` -> buffer -> ``lbm_halo_unpack``.  A step
of the whole lattice is one step of every slab followed by the exchange, and it gives the
bits of the undivided lattice.

``ZSlabs`` keeps all slabs on one GPU (buffers in device memory, one stream).
``exchange_plan`` and ``dist_exchange`` are the same exchange between ranks that own one slab
each (torch.distributed point-to-point; NCCL for device buffers, gloo for host buffers).
"""
from __future__ import annotations

import numpy as np

from . import lbm

FACE_LO, FACE_HI = 4, 5  # -z, +z


def split(nz: int, nslab: int):
    """[z0, z1) ranges of nslab nearly equal slabs."""
    if not 1 <= nslab <= nz:
        raise ValueError("need 1 <= nslab <= nz")
    edges = [nz * k // nslab for k in range(nslab + 1)]
    return [(edges[k], edges[k + 1]) for k in range(nslab)]


def slab_faces(faces, k: int, nslab: int):
    """Face types of slab k: the global x and y faces; "halo" toward a neighbour slab (and
    across the global z faces when they are periodic), else the global z face."""
    faces = list(faces)
    periodic = faces[FACE_LO] == "periodic"
    lo = "halo" if (k > 0 or periodic) else faces[FACE_LO]
    hi = "halo" if (k < nslab - 1 or periodic) else faces[FACE_HI]
    return tuple(faces[:4]) + (lo, hi)


def exchange_plan(nslab: int, periodic: bool):
    """The transfers of one exchange: (src slab, src face, dst slab, dst face).  The +z face
    of slab k feeds the -z ghost plane of slab k+1 and the -z face of slab k+1 feeds the +z
    ghost plane of slab k; with periodic z the last and first slabs are neighbours too."""
    plan = []
    pairs = [(k, k + 1) for k in range(nslab - 1)]
    if periodic and nslab > 1:
        pairs.append((nslab - 1, 0))
    for a, b in pairs:
        plan.append((a, FACE_HI, b, FACE_LO))
        plan.append((b, FACE_LO, a, FACE_HI))
    if periodic and nslab == 1:  # a single slab is its own neighbour across the periodic faces
        plan.append((0, FACE_HI, 0, FACE_LO))
        plan.append((0, FACE_LO, 0, FACE_HI))
    return plan


def ghost_flags(flags, z0: int, z1: int, periodic: bool):
    """The flags of slab [z0, z1) with one ghost plane on each side (z0-1 .. z1), taken from
    the global (nz, ny, nx) flags; across a non-periodic global face the ghost plane repeats
    the boundary plane (it is never read there)."""
    nz = flags.shape[0]
    idx = np.arange(z0 - 1, z1 + 1)
    idx = np.mod(idx, nz) if periodic else np.clip(idx, 0, nz - 1)
    return np.ascontiguousarray(flags[idx])


class ZSlabs:
    """nslab z slabs of an nx x ny x nz two-grid pull lattice on one GPU."""

    def __init__(self, nx, ny, nz, nslab, stencil=19, tau=0.8, faces=("periodic",) * 6, **params):
        import torch

        params = dict(params)
        params["streaming"] = "pull"
        self.nx, self.ny, self.nz, self.q = int(nx), int(ny), int(nz), int(stencil)
        self.faces = tuple(faces)
        self.periodic = self.faces[FACE_LO] == "periodic"
        self.ranges = split(self.nz, nslab)
        self.slabs = [lbm.Lattice(nx, ny, z1 - z0, stencil=stencil, tau=tau,
                                  faces=slab_faces(self.faces, k, nslab), **params)
                      for k, (z0, z1) in enumerate(self.ranges)]
        self.plan = exchange_plan(nslab, self.periodic)
        self.bufs = [torch.empty(lbm.lbm_halo_bytes(self.slabs[a].h, fa), dtype=torch.uint8, device="cuda")
                     for a, fa, _, _ in self.plan]
        self._flags = np.zeros((self.nz, self.ny, self.nx), dtype=np.uint8)
        for k in range(len(self.slabs)):
            self._set_slab_flags(k)

    def _set_slab_flags(self, k):
        z0, z1 = self.ranges[k]
        lat = self.slabs[k]
        if lat.params.face_bc[FACE_LO] == lbm.FACE["halo"] or lat.params.face_bc[FACE_HI] == lbm.FACE["halo"]:
            lat.set_flags(ghost_flags(self._flags, z0, z1, self.periodic))
        else:
            lat.set_flags(np.ascontiguousarray(self._flags[z0:z1]))

    def set_flags(self, flags):
        self._flags = np.ascontiguousarray(np.asarray(flags, dtype=np.uint8).reshape(self.nz, self.ny, self.nx))
        for k in range(len(self.slabs)):
            self._set_slab_flags(k)

    def set_force(self, fx, fy=0.0, fz=0.0):
        for lat in self.slabs:
            lat.set_force(fx, fy, fz)

    def init_equilibrium(self, rho=None, u=None):
        for lat, (z0, z1) in zip(self.slabs, self.ranges):
            r = None if rho is None else np.ascontiguousarray(np.asarray(rho, dtype=np.float32)[z0:z1])
            v = None if u is None else np.ascontiguousarray(np.asarray(u, dtype=np.float32)[:, z0:z1])
            lat.init_equilibrium(r, v)

    def exchange(self):
        for (a, fa, b, fb), buf in zip(self.plan, self.bufs):
            lbm.lbm_halo_pack(self.slabs[a].h, fa, buf)
            lbm.lbm_halo_unpack(self.slabs[b].h, fb, buf)

    def step(self, n=1):
        for _ in range(int(n)):
            for lat in self.slabs:
                lat.step(1)
            self.exchange()

    def sync(self):
        for lat in self.slabs:
            lat.sync()

    def get_populations(self):
        return np.concatenate([lat.get_populations() for lat in self.slabs], axis=1)

    def moments(self):
        parts = [lat.moments() for lat in self.slabs]
        return np.concatenate([p[0] for p in parts], axis=0), np.concatenate([p[1] for p in parts], axis=1)

    def reduce(self):
        return np.sum([lat.reduce() for lat in self.slabs], axis=0)

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz

    def close(self):
        for lat in self.slabs:
            lat.close()


def dist_exchange(dist, rank: int, world: int, periodic: bool, pack, unpack, make_buf):
    """One halo exchange between ranks that own one slab each (slab k on rank k).

    pack(face) -> buffer to send; unpack(face, buffer) consumes a received one; make_buf(face)
    -> an empty receive buffer for that face.  All receives are posted before the sends and
    every transfer carries its own tag, so the exchange cannot deadlock and the two transfers
    between one pair of ranks (periodic z with two ranks) cannot be confused."""
    plan = exchange_plan(world, periodic)
    recvs, sends, outs = [], [], []
    for t, (a, fa, b, fb) in enumerate(plan):
        if b == rank and a != rank:
            buf = make_buf(fb)
            recvs.append((dist.irecv(buf, src=a, tag=t), fb, buf))
    for t, (a, fa, b, fb) in enumerate(plan):
        if a == rank and b != rank:
            buf = pack(fa)
            outs.append(buf)
            sends.append(dist.isend(buf, dst=b, tag=t))
        elif a == rank and b == rank:
            unpack(fb, pack(fa))
    for req, fb, buf in recvs:
        req.wait()
        unpack(fb, buf)
    for req in sends:
        req.wait()
