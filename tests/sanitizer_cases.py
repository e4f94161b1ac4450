"""Tiny lattices through every step, export and exchange kernel with every boundary type:
D3Q19/D3Q27, FP32/FP16/BF16, AA and two-grid pull, TRT/MRT/Smagorinsky/learned closure,
statistics sampled in the step, moments, sums, population export/import, z slabs with halo
exchange, graph replays, a boundary list long enough for its own launch and the
allocation-free sums.  Run against the bounds-checked library
(``LBM_LIBRARY=.../liblbm_check.so python -m tests.sanitizer_cases``), every global access of
these kernels is checked against its array and lbm_sync fails on any skipped access.  Not a
pytest module (no test_ prefix): tests/test_gpu_bounds.py runs it."""
import hashlib
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2305_09910_gb300 import build, inputs, lbm, slabs  # noqa: E402

CHANNEL = ("periodic", "periodic", "wall", "wall", "periodic", "periodic")
TUNNEL = ("inflow", "outflow", "freeslip", "freeslip", "freeslip", "freeslip")


def run():
    build.build()
    nx, ny, nz = 40, 12, 10
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[3:6, 4:7, 10:14] = 1       # a solid block
    flags[7, 2, 20] = 2              # a moving-wall cell
    rho, u = inputs.channel_init(nx, ny, nz, u_bulk=0.05, seed=3)
    n = 0
    digest = hashlib.sha256()
    for q in (19, 27):
        for prec in ("f32", "f16", "bf16"):
            for streaming in ("aa", "pull"):
                for faces, fl in ((CHANNEL, None), (TUNNEL, flags)):
                    for coll in (("trt", "mrt", "reg") if q == 19 else ("trt", "reg")):
                        lat = lbm.Lattice(nx, ny, nz, stencil=q, tau=0.6, precision=prec, closure="smag",
                                          cs_smag=0.12, faces=faces, u_inflow=(0.04, 0, 0), streaming=streaming,
                                          collision=coll)
                        if fl is not None:
                            lat.set_flags(fl)
                        lat.set_force(1e-5)
                        lat.init_equilibrium(rho, u)
                        lat.step(3)
                        lbm.lbm_step_stats(lat.h, 4, 2)
                        lat.step(18)  # graph replays
                        lat.moments()
                        lat.reduce()
                        df = lat.get_populations()
                        lat.set_populations(df)
                        lat.step(1)
                        lat.sync()
                        digest.update(lat.get_populations().tobytes())
                        lat.close()
                        n += 1
    W = np.random.default_rng(5).normal(0, 0.2, 1345).astype(np.float32)
    for prec, streaming in (("f32", "aa"), ("f16", "pull")):  # learned closure (tensor-core kernel)
        lat = lbm.Lattice(nx, ny, nz, stencil=19, tau=0.6, precision=prec, closure="mlp", cs_smag=0.1,
                          faces=CHANNEL, streaming=streaming)
        lbm.lbm_set_closure_f32(lat.h, W, 300.0, 30.0)
        lat.set_force(1e-5)
        lat.init_equilibrium(rho, u)
        lat.step(4)
        lat.sync()
        lat.close()
        n += 1
    for prec in ("f32", "f16"):
        sl = slabs.ZSlabs(nx, ny, nz, 2, stencil=19, tau=0.6, precision=prec, closure="smag", faces=CHANNEL)
        sl.set_force(1e-5)
        sl.init_equilibrium(rho, u)
        sl.step(4)
        sl.sync()
        digest.update(sl.get_populations().tobytes())
        sl.close()
        n += 1
    # a boundary list too long to ride in the x-pair grid (D3Q27 FP16 pull tunnel with the
    # landing gear: 325k cells on the free-slip faces alone), so the listed cells get their own launch
    bx, by, bz = 512, 160, 160
    lat = lbm.Lattice(bx, by, bz, stencil=27, tau=0.52, precision="f16", closure="smag", cs_smag=0.1,
                      faces=TUNNEL, u_inflow=(0.05, 0, 0), streaming="pull")
    lat.set_flags(inputs.landing_gear_flags(bx, by, bz, scale=bx / 768))
    lat.init_equilibrium()
    lat.step(3)
    lat.sync()
    digest.update(np.asarray(lat.reduce()).tobytes())
    lat.close()
    n += 1
    # the allocation-free sums read the caller's exported populations and flags
    import torch

    lat = lbm.Lattice(nx, ny, nz, stencil=27, tau=0.6, closure="smag", faces=TUNNEL, u_inflow=(0.04, 0, 0))
    lat.set_flags(flags)
    lat.init_equilibrium(rho, u)
    lat.step(3)
    df = torch.from_numpy(lat.get_populations()).cuda()
    sums = lbm.lbm_reduce_noalloc(df, torch.from_numpy(flags).cuda(), nx, ny, nz, 27)
    digest.update(np.asarray(sums).tobytes())
    lat.close()
    n += 1
    print(f"cases: {n} lattices stepped, populations sha256 {digest.hexdigest()}", flush=True)


if __name__ == "__main__":
    run()
