"""Helpers shared by the GPU parity tests: one configuration, built twice.

``make_pair`` creates the CUDA lattice (through the C ABI binding) and the FP64 oracle
with the same sizes, stencil, relaxation, closure, faces, flags and force.  Neither side
sees the other's code; only the input arrays are shared.
"""
from __future__ import annotations

import numpy as np

FACES_CHANNEL = ("periodic", "periodic", "wall", "wall", "periodic", "periodic")
FACES_TUNNEL = ("inflow", "outflow", "freeslip", "freeslip", "freeslip", "freeslip")


def make_pair(nx, ny, nz, q=19, tau=0.8, lam=3.0 / 16.0, closure="none", cs=0.1,
              faces=("periodic",) * 6, u_w=(0.0, 0.0, 0.0), rho_w=1.0, force=(0.0, 0.0, 0.0),
              flags=None, precision="f32", mlp=None, mlp_scale=(1.0, 1.0), pipeline="direct",
              collision="trt", mrt_s=(1.19, 1.4, 1.2, 1.4, 1.98), streaming="aa"):
    import oracle
    from paper_2305_09910_gb300 import lbm

    lat = lbm.Lattice(nx, ny, nz, stencil=q, tau=tau, precision=precision, closure=closure,
                      magic_lambda=lam, cs_smag=cs, faces=faces, u_inflow=u_w, rho_inflow=rho_w,
                      pipeline=pipeline, collision=collision, mrt_rates=mrt_s, streaming=streaming)
    if flags is not None:
        lat.set_flags(np.ascontiguousarray(flags, dtype=np.uint8))
    lat.set_force(*force)
    ora = oracle.Oracle(nx, ny, nz, q=q, tau=tau, lam=lam, closure=closure, cs=cs, faces=faces,
                        u_w=u_w, rho_w=rho_w, force=force, flags=flags, mlp=mlp,
                        mlp_scale=mlp_scale, collision=collision, mrt_s=mrt_s)
    return lat, ora


def developed_state(ora, rho, u, steps, noise_seed=None, noise=0.0):
    """Runs the ORACLE from f^eq(rho, u) for ``steps`` steps and returns its state as the
    float32 shifted populations both sides will start from (solid cells zero)."""
    ora.init_equilibrium(rho, u)
    if noise:
        from paper_2305_09910_gb300 import inputs

        eps = inputs.uniform_field(noise_seed, 30, ora.f.shape, -noise, noise)
        ora.f += eps * ora.w[:, None, None, None]
    if steps:
        ora.step(steps)
    df = ora.shifted().astype(np.float32)
    df[:, ora.flags != 0] = 0.0
    return df


def max_abs_pop_error(lat, ora):
    """max |f_gpu - f_oracle| over fluid cells and directions (on f, i.e. on shifted df)."""
    df = lat.get_populations().astype(np.float64)
    ref = ora.shifted()
    fluid = ora.flags == 0
    return float(np.abs(df - ref)[:, fluid].max())
