"""The benchmark's own kernel against the FP64 oracle, element by element.

bench.py times the turbulent channel (Sec. 5.1 shape) as two-grid pull steps, every 10th of
which also samples the plane statistics inside the step kernel (the gather form of the pull
step with the statistics epilogue).  These tests run exactly that kernel:

* the 128 x 64 x 64 sub-case of the channel (above the size up to which several steps share
  one launch, so every step is its own launch of the benchmark kernel), 30 steps through
  lbm_step_stats(every = 10): every population against the oracle (1e-6 absolute per
  population, the single-step bound of turbulent runs) and the FP64 plane statistics of the
  three sampled states against the oracle's (Sec. 5.1's profiles);
* the 512 x 256 x 256 channel itself: one import step, then one sampling step of the gather
  kernel, checked at sampled cells against one oracle step from the exported state, and the
  statistics of four planes against the oracle's moments of those planes.
"""
import numpy as np
import pytest

from tests.cases import FACES_CHANNEL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    import torch

    from paper_2305_09910_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()


def _stats_tolerance(count, umax, samples):
    """Bound on the difference of FP64 plane sums of per-cell float32 values: a velocity off
    by at most 10 populations x 1e-6 (the per-population bound) over rho, plus its float32
    rounding; squares and products off by 2 |u|max times that."""
    eu = 10 * 1e-6 / 0.98 + 2.0 ** -23 * umax
    tol = np.zeros(10)
    tol[1:4] = samples * count * eu
    tol[4:10] = samples * count * eu * 2 * umax
    return tol


def test_bench_kernel_pull_stats_128x64x64_matches_oracle():
    import oracle
    from paper_2305_09910_gb300 import inputs, lbm

    nx, ny, nz = 128, 64, 64
    par = inputs.channel_parameters(ny)
    rho, u = inputs.channel_init(nx, ny, nz)
    lat = lbm.Lattice(nx, ny, nz, stencil=19, tau=par["tau"], closure="smag", cs_smag=0.1,
                      faces=FACES_CHANNEL, streaming="pull")
    nxp, _, _ = lbm.lbm_info(lat.h)
    assert nxp * ny * nz > 2 ** 17  # single launches, as at the benchmark size
    lat.set_force(par["force"])
    lat.init_equilibrium(rho, u)
    ora = oracle.Oracle(nx, ny, nz, q=19, tau=par["tau"], closure="smag", cs=0.1, faces=FACES_CHANNEL,
                        force=(par["force"], 0, 0))
    ora.init_equilibrium(rho.astype(np.float64), u.astype(np.float64))
    lbm.lbm_stats_reset(lat.h)
    lbm.lbm_step_stats(lat.h, 30, 10)
    acc = np.zeros((ny, 10))
    for k in range(30):
        if k % 10 == 0:
            ora.stats_sample(acc)
        ora.step(1)
    lat.sync()
    df = lat.get_populations().astype(np.float64)
    err = float(np.abs(df - ora.shifted()).max())
    print(f"128x64x64 pull + statistics, 30 steps: max |df - oracle| = {err:.2e}")
    assert err <= 1e-6
    st, ns = lbm.lbm_stats_get(lat.h, ny)
    assert ns == 3
    assert np.array_equal(st[:, 0], acc[:, 0])
    _, ur = ora.moments()
    tol = _stats_tolerance(nx * nz, float(np.abs(ur).max()), 3)
    d = np.abs(st - acc).max(axis=0)
    print("plane statistics: max |gpu - oracle| per column", d, "bound", tol)
    assert np.all(d[1:] <= tol[1:])


def test_bench_kernel_full_size_gather_step_sampled():
    """512 x 256 x 256: the sampling gather step checked at sampled cells and planes."""
    import torch

    import oracle
    from paper_2305_09910_gb300 import inputs, lbm

    nx, ny, nz = 512, 256, 256
    par = inputs.channel_parameters(ny)
    rho, u = inputs.channel_init(nx, ny, nz)
    lat = lbm.Lattice(nx, ny, nz, stencil=19, tau=par["tau"], closure="smag", cs_smag=0.1,
                      faces=FACES_CHANNEL, streaming="pull")
    lat.set_force(par["force"])
    lat.init_equilibrium(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    del rho, u
    lat.step(1)  # the import step (own-cell loads); the state is now post-collision, gathered next
    dfa = torch.empty((19, nz, ny, nx), dtype=torch.float32, device="cuda")
    lbm.lbm_get_populations(lat.h, dfa)
    lbm.lbm_stats_reset(lat.h)
    lbm.lbm_step_stats(lat.h, 1, 1)  # the benchmark's sampling step
    dfb = torch.empty_like(dfa)
    lbm.lbm_get_populations(lat.h, dfb)
    lat.sync()
    st, ns = lbm.lbm_stats_get(lat.h, ny)
    assert ns == 1
    cells = inputs.sample_cells(nx * ny * nz, 400, stream=22)
    extra = [0, nx - 1, (ny - 1) * nx, nx * (ny - 1) + 5, nx * ny * (nz - 1) + (ny - 1) * nx + nx - 1,
             nx * ny * 7 + nx * 128 + 300]
    cells = np.unique(np.concatenate([cells, np.array(extra, np.int64)]))
    got = dfb.reshape(19, -1)[:, torch.from_numpy(cells).cuda()].T.cpu().numpy().astype(np.float64)
    del dfb
    ha = dfa.cpu().numpy()
    del dfa
    ora = oracle.Oracle(nx, ny, nz, q=19, tau=par["tau"], closure="smag", cs=0.1, faces=FACES_CHANNEL,
                        force=(par["force"], 0, 0))
    ref = ora.step_sampled_pop(ha, cells) - ora.w[None, :]
    err = float(np.abs(got - ref).max())
    print(f"512x256x256 gather + statistics step at {cells.size} cells: max |df - oracle| = {err:.2e}")
    assert err <= 1e-6
    # plane statistics of the sampled state: the oracle's moments of single planes (the
    # statistics need no neighbours, so a plane is its own lattice of nx x 1 x nz cells)
    for y in (0, 1, 128, 255):
        plane = oracle.Oracle(nx, 1, nz, q=19, tau=par["tau"], force=(par["force"], 0, 0))
        plane.set_shifted(np.ascontiguousarray(ha[:, :, y:y + 1, :]))
        acc = plane.stats_sample()
        _, ur = plane.moments()
        tol = _stats_tolerance(nx * nz, float(np.abs(ur).max()), 1)
        assert st[y, 0] == acc[0, 0]
        assert np.all(np.abs(st[y, 1:] - acc[0, 1:]) <= tol[1:]), (y, st[y], acc[0])
