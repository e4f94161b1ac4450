"""GPU parity of 2:1 grid refinement (lbm_refine_explode / lbm_refine_coalesce through the C ABI)
against the FP64 oracle of the volumetric scheme (oracle/refine.py): the post-collision
populations of both levels after several coarse steps, element by element."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _states(r, seed, noise):
    """Float32 shifted pre-collision populations of both levels: equilibria of smooth seeded
    fields plus a seeded non-equilibrium part, computed by the oracle."""
    import oracle
    from paper_2305_09910_gb300 import inputs

    out = []
    for k, (nz, ny, nx) in enumerate(((r.nz, r.ny, r.nx), (r.nzf, 2 * r.ny, 2 * r.nx))):
        o = oracle.Oracle(nx, ny, nz, q=r.q, faces=("periodic",) * 6)
        rho = 1.0 + inputs.uniform_field(seed, 10 * k + 1, (nz, ny, nx), -0.02, 0.02)
        u = inputs.uniform_field(seed, 10 * k + 2, (3, nz, ny, nx), -0.04, 0.04)
        o.init_equilibrium(rho, u)
        eps = inputs.uniform_field(seed, 10 * k + 3, o.f.shape, -noise, noise)
        o.f += eps * o.w[:, None, None, None]
        out.append(o.shifted().astype(np.float32))
    return out


CASES = [
    # nx, ny, nz, z0, z1, q, walls, closure, force, tau
    (40, 12, 10, 3, 7, 19, False, "none", (0.0, 0.0, 0.0), 0.8),
    (33, 8, 9, 2, 6, 19, True, "smag", (2e-5, -1e-5, 0.0), 0.62),
    (20, 6, 8, 2, 5, 27, False, "smag", (1e-5, 0.0, 1e-5), 0.7),
    (17, 10, 8, 1, 4, 27, True, "none", (0.0, 1e-5, 0.0), 1.1),
]


@pytest.mark.parametrize("case", CASES)
def test_refined_slab_matches_oracle(case):
    from oracle.refine import RefinedOracle
    from paper_2305_09910_gb300.refine import RefinedSlab

    nx, ny, nz, z0, z1, q, walls, closure, force, tau = case
    ora = RefinedOracle(nx, ny, nz, z0, z1, q=q, tau=tau, closure=closure, cs=0.12, force=force, walls=walls)
    dfc, dff = _states(ora, seed=11 + q, noise=0.05)
    ora.set_shifted(dfc, dff)
    gpu = RefinedSlab(nx, ny, nz, z0, z1, stencil=q, tau=tau, walls=walls, force=force, closure=closure,
                      cs_smag=0.12)
    try:
        gpu.set_populations(dfc, dff)
        for steps in (1, 5):
            gpu.step(steps)
            ora.step(steps)
            gpu.sync()
            gc, gf = gpu.get_post_collision()
            oc, of = ora.post_collision()
            w = ora.w[:, None, None, None]
            m = ~ora.covered
            ec = np.abs(gc[:, m].astype(np.float64) - (oc[:, m] - w)).max()
            ef = np.abs(gf.astype(np.float64) - (of - w)).max()
            # FP32 arithmetic and storage against FP64: a few ulps of |f| ~ 0.3 per step
            assert ec <= 1e-6 and ef <= 1e-6, (steps, ec, ef)
    finally:
        gpu.close()


def test_refined_mass_is_conserved_on_the_gpu():
    from paper_2305_09910_gb300.refine import RefinedSlab

    nx, ny, nz, z0, z1 = 64, 32, 24, 8, 16
    gpu = RefinedSlab(nx, ny, nz, z0, z1, tau=0.7)

    class _R:  # the shapes _states needs
        pass

    r = _R()
    r.nx, r.ny, r.nz, r.nzf, r.q = nx, ny, nz, 2 * (z1 - z0), 19
    dfc, dff = _states(r, seed=5, noise=0.02)
    try:
        gpu.set_populations(dfc, dff)
        gpu.step(1)
        m0 = gpu.mass()
        gpu.step(100)
        gpu.sync()
        m1 = gpu.mass()
        # float32 roundings of O(1) populations, 200 fine and 100 coarse updates
        assert abs(m1 - m0) / m0 <= 2e-6, (m0, m1)
    finally:
        gpu.close()


@pytest.mark.parametrize("precision", ["f16", "bf16"])
def test_refined_slab_half_storage(precision):
    from oracle.refine import RefinedOracle
    from paper_2305_09910_gb300.refine import RefinedSlab

    nx, ny, nz, z0, z1 = 32, 8, 10, 3, 7
    ora = RefinedOracle(nx, ny, nz, z0, z1, tau=0.8)
    dfc, dff = _states(ora, seed=3, noise=0.02)
    ora.set_shifted(dfc, dff)
    gpu = RefinedSlab(nx, ny, nz, z0, z1, tau=0.8, precision=precision)
    try:
        gpu.set_populations(dfc, dff)
        gpu.step(4)
        ora.step(4)
        gpu.sync()
        gc, gf = gpu.get_post_collision()
        oc, of = ora.post_collision()
        w = ora.w[:, None, None, None]
        m = ~ora.covered
        err = max(np.abs(gc[:, m] - (oc[:, m] - w)).max(), np.abs(gf - (of - w)).max())
        # one rounding of a shifted population is at most 2^-11 (f16) / 2^-8 (bf16) of |df|, and
        # a value passes through fewer than 10 roundings in 4 coarse steps (8 fine steps and
        # the transfers)
        dmax = max(np.abs(dfc[:, m]).max(), np.abs(dff).max())
        bound = 10 * dmax * (2.0 ** -11 if precision == "f16" else 2.0 ** -8)
        assert err <= bound, err
    finally:
        gpu.close()


def test_refine_argument_checks():
    from paper_2305_09910_gb300 import lbm

    per = ("periodic",) * 4
    c = lbm.Lattice(16, 8, 4, tau=0.8, streaming="pull", faces=per + ("halo", "halo"))
    f = lbm.Lattice(32, 16, 4, tau=0.6, streaming="pull", faces=per + ("halo", "halo"))
    bad = lbm.Lattice(30, 16, 4, tau=0.6, streaming="pull", faces=per + ("halo", "halo"))
    walls = lbm.Lattice(32, 16, 4, tau=0.6, streaming="pull",
                        faces=("periodic", "periodic", "wall", "wall", "halo", "halo"))
    try:
        with pytest.raises(lbm.LbmError, match="ESTATE"):
            lbm.lbm_refine_explode(c.h, 5, f.h, 4, 0)
        c.step(1)
        f.step(1)
        bad.step(1)
        walls.step(1)
        with pytest.raises(lbm.LbmError, match="EINVAL"):
            lbm.lbm_refine_explode(c.h, 5, f.h, 5, 0)  # faces do not meet
        with pytest.raises(lbm.LbmError, match="EINVAL"):
            lbm.lbm_refine_explode(c.h, 5, bad.h, 4, 0)  # not twice as wide
        with pytest.raises(lbm.LbmError, match="EUNSUPPORTED"):
            lbm.lbm_refine_explode(c.h, 5, walls.h, 4, 0)
        with pytest.raises(lbm.LbmError, match="EINVAL"):
            lbm.lbm_refine_explode(c.h, 5, f.h, 4, 2)
        with pytest.raises(lbm.LbmError, match="ESTATE"):
            lbm.lbm_refine_coalesce(f.h, 4, c.h, 5)  # one fine step since the import
        lbm.lbm_refine_explode(c.h, 5, f.h, 4, 0)
        f.step(1)
        lbm.lbm_refine_coalesce(f.h, 4, c.h, 5)
        c.sync()
        f.sync()
        with pytest.raises(lbm.LbmError, match="ESTATE"):
            aa = lbm.Lattice(8, 8, 8, tau=0.8)
            try:
                aa.get_post_collision()
            finally:
                aa.close()
    finally:
        for lat in (c, f, bad, walls):
            lat.close()


MULTI_CASES = [
    # nx, ny, nz, slabs, q, walls, closure, force, tau, precision
    (24, 8, 12, [(0, 3), (9, 12)], 19, True, "smag", (2e-5, 0.0, 0.0), 0.7, "f32"),  # channel: both walls refined
    (20, 6, 12, [(1, 3), (6, 9)], 27, False, "none", (0.0, 1e-5, 0.0), 0.9, "f32"),
    (17, 6, 9, [(0, 3)], 19, True, "smag", (1e-5, 0.0, 1e-5), 0.62, "f32"),  # one wall refined, ragged nx
    (32, 8, 10, [(0, 2), (5, 10)], 19, True, "none", (1e-5, 0.0, 0.0), 0.8, "f16"),
]


def _multi_states(r, seed, noise):
    class _Shape:
        pass

    outs = []
    for k, s in enumerate(r.slabs):
        sh = _Shape()
        sh.nx, sh.ny, sh.nz, sh.nzf, sh.q = r.nx, r.ny, r.nz, s.nzf, r.q
        dfc, dff = _states(sh, seed + 7 * k, noise)
        outs.append(dff)
    return dfc, outs


@pytest.mark.parametrize("case", MULTI_CASES)
def test_several_refined_slabs_match_oracle(case):
    from oracle.refine import RefinedOracle
    from paper_2305_09910_gb300.refine import RefinedSlab

    nx, ny, nz, slabs, q, walls, closure, force, tau, precision = case
    ora = RefinedOracle(nx, ny, nz, q=q, tau=tau, closure=closure, cs=0.12, force=force, walls=walls, slabs=slabs)
    dfc, dffs = _multi_states(ora, seed=31, noise=0.03)
    ora.set_shifted(dfc, dffs if len(dffs) > 1 else dffs[0])
    gpu = RefinedSlab(nx, ny, nz, stencil=q, tau=tau, walls=walls, force=force, closure=closure, cs_smag=0.12,
                      slabs=slabs, precision=precision)
    try:
        gpu.set_populations(dfc, dffs)
        gpu.step(5)
        ora.step(5)
        gpu.sync()
        gc, gf = gpu.get_post_collision()
        oc, of = ora.post_collision()
        gf = gf if isinstance(gf, list) else [gf]
        of = of if isinstance(of, list) else [of]
        w = ora.w[:, None, None, None]
        m = ~ora.covered
        err = np.abs(gc[:, m].astype(np.float64) - (oc[:, m] - w)).max()
        for g, o in zip(gf, of):
            err = max(err, np.abs(g.astype(np.float64) - (o - w)).max())
        if precision == "f32":
            assert err <= 1e-6, err
        else:  # one FP16 rounding of |df| per storage pass, fewer than 20 passes in 5 coarse steps
            dmax = max([np.abs(dfc[:, m]).max()] + [np.abs(d).max() for d in dffs])
            assert err <= 20 * dmax * 2.0 ** -11, err
    finally:
        gpu.close()
