"""Precision forms against the FP64 oracle and the FP32 run (the 128 x 64 x 64 sub-case).

The perturbed channel (Re_tau ~ 180, walls at the y faces, Smagorinsky C_s = 0.1) is run
for 300 steps from the same initial fields by the FP64 oracle and by the GPU with float32,
float16-shifted and bfloat16-shifted populations (float32 arithmetic in every case), each in
AA and in two-grid pull streaming.  For each form the test states (prints) and bounds:
  * the largest population error against the oracle,
  * the relative errors of the mean u_x and RMS velocity profiles (x-z plane statistics),
  * the relative drift of the total mass (FP64 sums on the GPU).
"""
import os

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
    # AA in place (one-cell kernel / x-pairs) and two-grid pull (the half forms: the split step,
    # x-pairs with the wall rows and periodic z planes as listed cells)
    for streaming in ("aa", "pull"):
        for prec in BOUNDS:
            lat = lbm.Lattice(nx, ny, nz, stencil=19, tau=par["tau"], precision=prec, closure="smag",
                              cs_smag=0.1, faces=FACES_CHANNEL, streaming=streaming)
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
            report[f"{prec}/{streaming}"] = {"pop_err": pop, "mean_profile_err": e_mean, "rms_profile_err": e_rms,
                                             "mass_drift": drift}
            lat.close()
    report["oracle_mass_drift"] = float(abs(ora.mass_momentum()[0] - m0) / m0)
    print("precision forms vs FP64 oracle after", STEPS, "steps:", report)
    for key, r in report.items():
        if "/" not in key:
            continue
        b_pop, b_mean, b_rms, b_mass = BOUNDS[key.split("/")[0]]
        assert r["pop_err"] <= b_pop, (key, r)
        assert r["mean_profile_err"] <= b_mean, (key, r)
        assert r["rms_profile_err"] <= b_rms, (key, r)
        assert r["mass_drift"] <= b_mass, (key, r)


# Bluff-body sub-case: D3Q27, 96 x 48 x 48 with the landing-gear geometry scaled by 1/8, inflow
# 0.05, outflow, free-slip sides, 100 steps from the uniform inflow state.  Ceilings 3-8 times
# above the errors measured on GB300 (f32 1.2e-7 / 1.6e-7 / 2.4e-9, f16 2.5e-4 / 5.2e-4 / 3.3e-5,
# bf16 1.7e-3 / 3.9e-3 / 5.7e-5).  With inflow and outflow the mass is not conserved: the
# half forms round the boundary fluxes, so their mass departs from the oracle's by ~1e-5 per
# hundred steps, against 2e-8 in the closed channel.
BLUFF_BOUNDS = {  # pop error, velocity-field relative error, mass difference vs the oracle
    "f32": (1e-6, 1e-6, 1e-8),
    "f16": (1e-3, 2e-3, 1.5e-4),
    "bf16": (1e-2, 2e-2, 3e-4),
}


def test_bluff_body_precision_forms_against_oracle():
    import torch

    import oracle
    from paper_2305_09910_gb300 import build, inputs, lbm

    assert torch.cuda.is_available()
    build.build()
    nx, ny, nz, steps = 96, 48, 48, 100
    flags = inputs.landing_gear_flags(nx, ny, nz, scale=1 / 8)
    tau = 0.5 + 3 * 0.05 * 10 / 1e4
    faces = ("inflow", "outflow", "freeslip", "freeslip", "freeslip", "freeslip")
    ora = oracle.Oracle(nx, ny, nz, q=27, tau=tau, closure="smag", cs=0.1, faces=faces,
                        u_w=(0.05, 0, 0), flags=flags)
    u0 = np.zeros((3, nz, ny, nx))
    u0[0] = 0.05
    ora.init_equilibrium(1.0, u0)
    ora.step(steps, threads=os.cpu_count() or 1)
    _, ur = ora.moments()
    ref_df = ora.shifted()
    m_ref = ora.mass_momentum()[0]
    report = {}
    # AA (one-cell kernel) and two-grid pull (the half forms: the split step, x-pairs and the
    # listed boundary cells read through their source table)
    for streaming in ("aa", "pull"):
        for prec in BLUFF_BOUNDS:
            lat = lbm.Lattice(nx, ny, nz, stencil=27, tau=tau, precision=prec, closure="smag", cs_smag=0.1,
                              faces=faces, u_inflow=(0.05, 0, 0), streaming=streaming)
            lat.set_flags(flags)
            lat.init_equilibrium(None, u0.astype(np.float32))
            lat.step(steps)
            lat.sync()
            _, ug = lat.moments()
            report[f"{prec}/{streaming}"] = {
                "pop_err": float(np.abs(lat.get_populations() - ref_df).max()),
                "u_rel_err": float(np.linalg.norm(ug - ur) / np.linalg.norm(ur)),
                "mass_rel_diff": float(abs(lat.reduce()[0] - m_ref) / m_ref),
            }
            lat.close()
    print("bluff-body precision forms vs FP64 oracle after", steps, "steps:", report)
    for key, r in report.items():
        b_pop, b_u, b_m = BLUFF_BOUNDS[key.split("/")[0]]
        assert r["pop_err"] <= b_pop, (key, r)
        assert r["u_rel_err"] <= b_u, (key, r)
        assert r["mass_rel_diff"] <= b_m, (key, r)
