"""Self-consistency of the turbulent-channel statistics (Sec. 5.1).

The paper's channel assesses the symmetry and regularity of the solution and the shear
stresses along the wall normal.  No DNS data are available here, so the FP64 plane
statistics of a developed turbulent run (Re_tau = 180, 256 x 128 x 128, D3Q19 TRT +
Smagorinsky, two-grid pull with the statistics sampled inside the step kernel, as in the
benchmark; FP32 storage, and FP16-shifted storage through the split half-storage step) are
checked against what the equations themselves fix:

* the flow is turbulent: the streamwise RMS peak lies between 2 and 3.5 u_tau and the wall-
  normal one between 0.5 and 1.3 u_tau (channel-flow values are about 2.7 and 0.9);
* the mean profile is symmetric about the centre plane;
* the total shear stress nu d<u>/dy - <u'v'> is linear in y (momentum balance of a
  statistically steady channel, d tau / dy = -g), with slope -g;
* u_tau from the wall gradient equals sqrt(g delta) (the walls carry the driving force).

Tolerances: the averages cover 100k steps (10 eddy turnovers delta / u_tau, 10,000 samples
of 32,768-cell planes).  Over 20k-step windows the same quantities fluctuated by symmetry
2-6 %, stress-line residual 5-14 % of g delta, slope 0.87-1.02 g and wall u_tau 0.90-0.95
sqrt(g delta); over the 100k steps FP32 gave 0.016 / 0.073 / 0.949 / 0.938 and FP16
0.022 / 0.080 / 0.931 / 0.933 (the unresolved Smagorinsky stress, about 8 % of the wall stress at this
resolution, is not in the statistics).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_turbulent_channel_statistics_are_self_consistent(precision):
    import torch

    from paper_2305_09910_gb300 import build, closure, inputs, lbm

    assert torch.cuda.is_available()
    build.build()
    nx, ny, nz, ub = 256, 128, 128, 0.1
    par = inputs.channel_parameters(ny, u_bulk=ub)
    nu, g, delta, utau = (par["tau"] - 0.5) / 3, par["force"], par["delta"], par["u_tau"]
    lat = closure.channel(nx, ny, nz, closure="smag", cs0=0.1, u_bulk=ub, amp=0.5, streaming="pull",
                          precision=precision)
    lat.step(60000)
    lbm.lbm_stats_reset(lat.h)
    lbm.lbm_step_stats(lat.h, 100000, 10)
    lat.sync()
    st, ns = lbm.lbm_stats_get(lat.h, ny)
    assert ns == 10000 and np.all(st[:, 0] == ns * nx * nz)
    mean = st[:, 1:4] / st[:, :1]
    var = st[:, 4:7] / st[:, :1] - mean ** 2
    uv = st[:, 7] / st[:, 0] - mean[:, 0] * mean[:, 1]
    u = mean[:, 0]
    rms = np.sqrt(np.maximum(var, 0.0)).max(axis=0) / utau
    sym = float(np.abs(u - u[::-1]).max() / u.max())
    # total stress at the interior planes (central differences), its straight-line fit
    y = np.arange(1, ny - 1, dtype=np.float64)
    tau_t = nu * (u[2:] - u[:-2]) / 2 - uv[1:-1]
    A = np.vstack([np.ones_like(y), y]).T
    coef = np.linalg.lstsq(A, tau_t, rcond=None)[0]
    resid = float(np.abs(tau_t - A @ coef).max() / (g * delta))
    slope = float(-coef[1] / g)
    # wall gradient: quadratic through u = 0 at the wall (half a cell below plane 0) and the
    # first two planes (distances 0.5 and 1.5), both walls averaged
    def grad(u0, u1):
        return (2.25 * u0 - 0.25 * u1) / 0.75

    utau_wall = float(np.sqrt(nu * 0.5 * (grad(u[0], u[1]) + grad(u[-1], u[-2]))) / np.sqrt(g * delta))
    print(f"channel statistics ({precision}): u'/u_tau {rms.round(3).tolist()}, symmetry {sym:.3f}, stress-line residual "
          f"{resid:.3f} g delta, slope {slope:.3f} g, wall u_tau {utau_wall:.3f} sqrt(g delta), "
          f"bulk velocity {u.mean():.4f}")
    assert 2.0 <= rms[0] <= 3.5 and 0.5 <= rms[1] <= 1.3
    assert sym <= 0.05
    assert resid <= 0.12
    assert abs(slope - 1.0) <= 0.2
    assert abs(utau_wall - 1.0) <= 0.1
