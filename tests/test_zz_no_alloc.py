"""lbm_reduce_noalloc: FP64 sums without any allocation by the library.

Some callers may not allocate device memory at the point where they need the mass and
momentum of a lattice (for example an analysis hook inside another application's time loop,
on a GPU whose free memory that application's caching allocator owns).  They already hold
the populations, so lbm_reduce_noalloc takes those and works in a static scratch array.
This file checks it against lbm_reduce (the handle-based entry point) on two calls in a row,
since the scratch keeps the previous call's contents, and checks the size limit.  It runs
last (file name) and passes alone or after the other tests.
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


def test_noalloc_reduce_rejects_oversized_lattice():
    import torch

    from paper_2305_09910_gb300 import lbm

    tiny = torch.zeros(19, dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_reduce_noalloc(tiny, None, 1024, 1024, 512, 19)  # 2^29 cells > 2^28
    assert e.value.status == lbm.LBM_EINVAL
    assert "exceed the maximum" in lbm.lbm_last_error(None)
