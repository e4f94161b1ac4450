"""lbm_reduce_noalloc: FP64 sums without any allocation by the library.

Some callers may not allocate device memory at the point where they need the mass and
momentum of a lattice (for example an analysis hook inside another application's time loop,
on a GPU whose free memory that application's caching allocator owns).  They already hold
the populations, so lbm_reduce_noalloc takes those and works in a static scratch array.
This file checks it against lbm_reduce (the handle-based entry point, itself checked against
the FP64 oracle's sums) on calls in a row, since the scratch keeps the previous call's
contents: two calls on one lattice, then a smaller lattice (fewer partial sums) after a
larger one, and a wind tunnel with moving-wall cells and an outflow face.  It also checks the
size limit of the C call and the binding's size and device checks.  It runs last (file name)
and passes alone or after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FACES_CHANNEL = ("periodic", "periodic", "wall", "wall", "periodic", "periodic")


@pytest.fixture(scope="module", autouse=True)
def _library():
    import torch

    from paper_2305_09910_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


@pytest.mark.parametrize("q", [19, 27])
def test_noalloc_reduce_matches_lbm_reduce_twice(q):
    import torch

    from paper_2305_09910_gb300 import inputs, lbm

    nx, ny, nz = 70, 37, 23
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[5:12, 10:20, 30:41] = 1
    force = (3e-6, 1e-6, 0.0)
    lat = lbm.Lattice(nx, ny, nz, stencil=q, tau=0.6, closure="smag", faces=FACES_CHANNEL)
    lat.set_flags(flags)
    lat.set_force(*force)
    rho, u = inputs.channel_init(nx, ny, nz, u_bulk=0.05, seed=4)
    lat.init_equilibrium(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    fl = torch.from_numpy(flags).cuda()
    df = torch.empty((q, nz, ny, nx), dtype=torch.float32, device="cuda")
    for steps in (3, 4):  # two calls in a row, at both AA parities
        lat.step(steps)
        ref = lat.reduce()
        lbm.lbm_get_populations(lat.h, df)
        got = lbm.lbm_reduce_noalloc(df, fl, nx, ny, nz, q, force)
        assert abs(got[0] - ref[0]) <= 1e-6 * ref[0]
        assert np.abs(got[1:] - ref[1:]).max() <= 1e-6 * ref[0]


FACES_TUNNEL = ("inflow", "outflow", "freeslip", "freeslip", "freeslip", "freeslip")


def _populations(lat, q, nx, ny, nz):
    import torch

    from paper_2305_09910_gb300 import lbm

    df = torch.empty((q, nz, ny, nx), dtype=torch.float32, device="cuda")
    lbm.lbm_get_populations(lat.h, df)
    return df


def test_noalloc_reduce_smaller_lattice_after_larger_and_tunnel():
    """A large lattice (many partial sums) and then smaller ones: a leftover partial of the
    earlier call would show in the later sums.  The tunnel has moving-wall (inflow) cells,
    which are not fluid, and an outflow face, whose incoming populations the export has
    already filled."""
    import torch

    from paper_2305_09910_gb300 import inputs, lbm

    cases = [(19, (300, 96, 80), FACES_CHANNEL, False), (19, (40, 12, 10), FACES_CHANNEL, False),
             (27, (96, 48, 48), FACES_TUNNEL, True), (19, (34, 9, 7), FACES_TUNNEL, True)]
    nblocks = []
    for q, (nx, ny, nz), faces, gear in cases:
        n = nx * ny * nz
        nblocks.append(-(-n // 16384))
        flags = inputs.landing_gear_flags(nx, ny, nz, scale=nx / 768) if gear and nx >= 96 else \
            np.zeros((nz, ny, nx), np.uint8)
        if gear:
            flags[nz // 2, ny // 2, 3] = 2  # a moving-wall cell
            flags[1:3, 1:3, nx // 2:nx // 2 + 2] = 1
        force = (0.0, 0.0, 0.0) if gear else (4e-6, 0.0, 1e-6)
        lat = lbm.Lattice(nx, ny, nz, stencil=q, tau=0.6, closure="smag", faces=faces, u_inflow=(0.05, 0, 0))
        lat.set_flags(flags)
        lat.set_force(*force)
        rho, u = inputs.channel_init(nx, ny, nz, u_bulk=0.05, seed=6)
        lat.init_equilibrium(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
        lat.step(5)
        ref = lat.reduce()
        got = lbm.lbm_reduce_noalloc(_populations(lat, q, nx, ny, nz), torch.from_numpy(flags).cuda(),
                                     nx, ny, nz, q, force)
        assert abs(got[0] - ref[0]) <= 1e-6 * ref[0], (q, nx, got, ref)
        assert np.abs(got[1:] - ref[1:]).max() <= 1e-6 * ref[0], (q, nx, got, ref)
        lat.close()
    assert nblocks[0] > nblocks[1] and nblocks[2] > nblocks[3]


def test_noalloc_reduce_rejects_oversized_lattice():
    """The C call's own limit, reached with a NULL flags pointer and a tiny buffer: the size
    check comes before any launch."""
    import ctypes

    import torch

    from paper_2305_09910_gb300 import lbm

    tiny = torch.zeros(19, dtype=torch.float32, device="cuda")
    out = np.zeros(4)
    st = lbm.load().lbm_reduce_noalloc(ctypes.c_void_p(tiny.data_ptr()), None, 1024, 1024, 512, 19, None,
                                       out.ctypes.data_as(ctypes.c_void_p), None)  # 2^29 cells > 2^28
    assert st == lbm.LBM_EINVAL
    assert "exceed the maximum" in lbm.lbm_last_error(None)


def test_noalloc_binding_checks_sizes_before_the_call():
    import torch

    from paper_2305_09910_gb300 import lbm

    df = torch.zeros((19, 4, 4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        lbm.lbm_reduce_noalloc(df, None, 4, 4, 5, 19)  # 19 * 80 values needed
    with pytest.raises(ValueError):
        lbm.lbm_reduce_noalloc(df, torch.zeros(63, dtype=torch.uint8, device="cuda"), 4, 4, 4, 19)
    with pytest.raises(ValueError):
        lbm.lbm_reduce_noalloc(df, None, 4, 4, 4, 27)
