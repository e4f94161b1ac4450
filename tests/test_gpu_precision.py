"""Precision forms against the FP64 oracle and the FP32 run (the 128 x 64 x 64 sub-case).

The perturbed channel (Re_tau ~ 180, walls at the y faces, Smagorinsky C_s = 0.1) is run
for 300 steps from the same initial fields by the FP64 oracle and by the GPU with float32,
float16-shifted and bfloat16-shifted populations (float32 arithmetic in every case).  For
each form the test states (prints) and bounds:
  * the largest population error against the oracle,
  * the relative errors of the mean u_x and RMS velocity profiles (x-z plane statistics),
  * the relative drift of the total mass (FP64 sums on the GPU).
"""
import numpy as np
import pytest

from tests.cases import FACES_CHANNEL

pytestmark = pytest.mark.gpu

STEPS = 300
# Ceilings, not targets: FP32 holds the 1e-6 per-population parity bound; the half forms
# store every population with a relative rounding of 2^-11 (FP16) or 2^-8 (BF16) per step,
# and these ceilings sit a few times above the errors measured for them (values measured on
# GB300 after 300 steps: FP16 6e-4 / 1.5e-5 / 4.4e-4 / 2e-8, BF16 4.7e-3 / 6e-4 / 1.5e-2 / 3e-6).
BOUNDS = {  # pop error, mean-profile error, rms-profile error, mass drift
    "f32": (1e-6, 1e-5, 1e-4, 1e-7),
    "f16": (3e-3, 2e-4, 5e-3, 1e-6),
    "bf16": (3e-2, 5e-3, 0.1, 3e-5),
}


def _profiles(u):
    mean = u.mean(axis=(1, 3))                     # (3, ny)
    rms = np.sqrt(np.maximum((u * u).mean(axis=(1, 3)) - mean ** 2, 0.0))
    return mean[0], rms


def test_precision_forms_against_oracle():
    import torch

    import oracle
    from paper_2305_09910_gb300 import build, inputs, lbm

    assert torch.cuda.is_available()
    build.build()
    nx, ny, nz = 128, 64, 64
    par = inputs.channel_parameters(ny)
    rho, u = inputs.channel_init(nx, ny, nz)
    ora = oracle.Oracle(nx, ny, nz, q=19, tau=par["tau"], closure="smag", cs=0.1, faces=FACES_CHANNEL,
                        force=(par["force"], 0, 0))
    ora.init_equilibrium(rho.astype(np.float64), u.astype(np.float64))
    m0 = ora.mass_momentum()[0]
    ora.step(STEPS)
    _, ur = ora.moments()
    ref_mean, ref_rms = _profiles(ur)
    ref_df = ora.shifted()
    report = {}
    for prec, (b_pop, b_mean, b_rms, b_mass) in BOUNDS.items():
        lat = lbm.Lattice(nx, ny, nz, stencil=19, tau=par["tau"], precision=prec, closure="smag",
                          cs_smag=0.1, faces=FACES_CHANNEL)
        lat.set_force(par["force"])
        lat.init_equilibrium(rho, u)
        g0 = lat.reduce()[0]
        lat.step(STEPS)
        lat.sync()
        _, ug = lat.moments()
        mean, rms = _profiles(ug.astype(np.float64))
        pop = float(np.abs(lat.get_populations() - ref_df).max())
        e_mean = float(np.linalg.norm(mean - ref_mean) / np.linalg.norm(ref_mean))
        e_rms = float(np.linalg.norm(rms - ref_rms) / np.linalg.norm(ref_rms))
        drift = float(abs(lat.reduce()[0] - g0) / g0)
        report[prec] = {"pop_err": pop, "mean_profile_err": e_mean, "rms_profile_err": e_rms,
                        "mass_drift": drift}
        lat.close()
    report["oracle_mass_drift"] = float(abs(ora.mass_momentum()[0] - m0) / m0)
    print("precision forms vs FP64 oracle after", STEPS, "steps:", report)
    for prec, (b_pop, b_mean, b_rms, b_mass) in BOUNDS.items():
        r = report[prec]
        assert r["pop_err"] <= b_pop, (prec, r)
        assert r["mean_profile_err"] <= b_mean, (prec, r)
        assert r["rms_profile_err"] <= b_rms, (prec, r)
        assert r["mass_drift"] <= b_mass, (prec, r)
