"""Host logic of the z-slab halo exchange: the split, the ghost flags, the exchange plan, and
the exchange between two ranks over gloo (world size 2), with slabs stood in for by numpy
arrays that pack and unpack by the contract of lbm_halo_pack / lbm_halo_unpack."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_split_and_faces():
    from paper_2305_09910_gb300 import slabs

    assert slabs.split(21, 3) == [(0, 7), (7, 14), (14, 21)]
    assert slabs.split(5, 2) == [(0, 2), (2, 5)]
    tunnel = ("inflow", "outflow", "freeslip", "freeslip", "freeslip", "freeslip")
    assert slabs.slab_faces(tunnel, 0, 2)[4:] == ("freeslip", "halo")
    assert slabs.slab_faces(tunnel, 1, 2)[4:] == ("halo", "freeslip")
    assert slabs.slab_faces(("periodic",) * 6, 0, 2)[4:] == ("halo", "halo")


def test_exchange_plan_covers_every_interface_both_ways():
    from paper_2305_09910_gb300 import slabs

    assert slabs.exchange_plan(2, False) == [(0, 5, 1, 4), (1, 4, 0, 5)]
    plan = slabs.exchange_plan(3, True)
    assert len(plan) == 6 and (2, 5, 0, 4) in plan and (0, 4, 2, 5) in plan
    assert slabs.exchange_plan(1, True) == [(0, 5, 0, 4), (0, 4, 0, 5)]
    assert slabs.exchange_plan(1, False) == []


def test_ghost_flags():
    from paper_2305_09910_gb300 import slabs

    f = np.arange(5)[:, None, None] * np.ones((1, 2, 3), np.uint8)
    assert list(slabs.ghost_flags(f, 0, 2, True)[:, 0, 0]) == [4, 0, 1, 2]
    assert list(slabs.ghost_flags(f, 3, 5, True)[:, 0, 0]) == [2, 3, 4, 0]
    assert list(slabs.ghost_flags(f, 0, 2, False)[:, 0, 0]) == [0, 0, 1, 2]


# A stand-in slab: populations [q][nz + 2][ny][nxp] with ghost planes at both ends.
CZ19 = [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]


class FakeSlab:
    def __init__(self, rank, nz, ny=3, nxp=4):
        rng = np.random.default_rng(rank)
        self.f = rng.random((19, nz + 2, ny, nxp)).astype(np.float32)
        self.nz = nz

    def dirs(self, sign):
        return [i for i in range(19) if CZ19[i] == sign]

    def pack(self, face):  # leaving directions of the plane next to the face
        z = self.nz if face == 5 else 1
        return np.ascontiguousarray(self.f[self.dirs(1 if face == 5 else -1), z])

    def unpack(self, face, buf):  # entering directions, ghost plane beyond the face
        z = 0 if face == 4 else self.nz + 1
        self.f[self.dirs(1 if face == 4 else -1), z] = buf


def _rank(rank, world, port, periodic, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_2305_09910_gb300 import slabs

    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = FakeSlab(rank, nz=4)
    before = s.f.copy()
    slabs.dist_exchange(dist, rank, world, periodic,
                        pack=lambda face: torch.from_numpy(s.pack(face)),
                        unpack=lambda face, buf: s.unpack(face, buf.numpy()),
                        make_buf=lambda face: torch.empty((5, 3, 4), dtype=torch.float32))
    out[rank] = (before, s.f.copy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("periodic", [False, True])
def test_dist_exchange_two_gloo_ranks(periodic):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, periodic, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    (b0, a0), (b1, a1) = out[0], out[1]
    up = [i for i in range(19) if CZ19[i] == 1]
    dn = [i for i in range(19) if CZ19[i] == -1]
    # rank 1's -z ghost plane holds rank 0's top plane (c_z = +1), rank 0's +z ghost rank 1's bottom
    assert np.array_equal(a1[up, 0], b0[up, 4]) and np.array_equal(a0[dn, 5], b1[dn, 1])
    if periodic:
        assert np.array_equal(a0[up, 0], b1[up, 4]) and np.array_equal(a1[dn, 5], b0[dn, 1])
    else:
        assert np.array_equal(a0[:, 0], b0[:, 0]) and np.array_equal(a1[:, 5], b1[:, 5])
    # interior planes untouched
    assert np.array_equal(a0[:, 1:5], b0[:, 1:5]) and np.array_equal(a1[:, 1:5], b1[:, 1:5])
