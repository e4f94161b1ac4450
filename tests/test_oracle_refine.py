"""Pins of the FP64 grid-refinement oracle (oracle/refine.py) against what the mathematics and
the scheme's published properties fix, not against itself:

* transport consistency: with collisions left out, one coarse step moves a coarse population
  through the interface by exactly one coarse cell along c_i (spread evenly over that
  cell's 8 fine cells), and moves 8 equal fine populations of a coarse cell's volume out by
  one coarse cell into one coarse population -- what streaming on the coarse lattice does;
* exact conservation of mass and momentum (the volumetric transfer of Rohde et al. 2006);
* a uniform equilibrium is a fixed point on both levels;
* the decay rate nu k^2 of a shear wave that crosses both interfaces (acoustic scaling of
  the viscosity, tau_f - 1/2 = 2 (tau_c - 1/2));
* the analytic Poiseuille profile across a refined slab between no-slip walls (viscosity and
  body-force scaling F_f = F_c / 2);
* with several refined slabs, and slabs on the no-slip walls (halfway bounce-back on the
  fine level): exact mass conservation, the Poiseuille parabola with both walls refined (the
  channel case), the shear-wave rate across four interfaces;
* planted mistakes in the oracle (wrong viscosity scaling, an unshifted coalescence) fail
  these pins.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import oracle.refine as refine
from oracle.refine import RefinedOracle
from paper_2305_09910_gb300 import inputs


def _tracer_in(r, i, X, Y):
    """Post-collision coarse array: 1 in direction i of interface cell (X, Y) below the slab."""
    cstar = np.zeros((r.q, r.nz, r.ny, r.nx))
    cstar[i, r.lo, Y, X] = 1.0
    return cstar


@pytest.mark.parametrize("q", [19, 27])
def test_coarse_to_fine_transport_moves_one_coarse_cell(q):
    r = RefinedOracle(4, 4, 6, 2, 4, q=q)
    X, Y = 1, 2
    for i in range(q):
        cx, cy, cz = (int(v) for v in r.c[i])
        if cz != 1:
            continue
        ext = r.explode(_tracer_in(r, i, X, Y))
        ext[:, 2:-2] = 0.0
        ext = r.fine_stream(r.fine_stream(ext))
        got = ext[i, 2:-2]
        want = np.zeros_like(got)
        xs = [(2 * (X + cx) + a) % (2 * r.nx) for a in (0, 1)]
        ys = [(2 * (Y + cy) + b) % (2 * r.ny) for b in (0, 1)]
        for y in ys:
            for x in xs:
                want[0:2, y, x] = 1.0  # the fine cells of coarse cell (X + cx, Y + cy, z0)
        assert np.array_equal(got, want), i
        # no other direction was touched
        others = np.delete(ext[:, 2:-2], i, axis=0)
        assert np.nansum(np.abs(others)) == 0.0


@pytest.mark.parametrize("q", [19, 27])
def test_fine_to_coarse_transport_moves_one_coarse_cell(q):
    r = RefinedOracle(4, 4, 6, 2, 4, q=q)
    X, Y = 2, 1
    for i in range(q):
        cx, cy, cz = (int(v) for v in r.c[i])
        if cz != -1:
            continue
        ext = np.zeros((q, r.nzf + 4, 2 * r.ny, 2 * r.nx))
        # the 8 fine cells of covered coarse cell (X, Y, z0): fine planes 0, 1 of the slab
        ext[i, 2:4, 2 * Y:2 * Y + 2, 2 * X:2 * X + 2] = 1.0
        ext = r.fine_stream(r.fine_stream(ext))
        coal = r.coalesce(ext)[r.lo]
        want = np.zeros((r.ny, r.nx))
        want[(Y + cy) % r.ny, (X + cx) % r.nx] = 1.0
        assert np.array_equal(coal[i], want), i


def test_coalescence_is_the_volume_mean():
    r = RefinedOracle(4, 4, 6, 2, 4)
    i = int(np.flatnonzero((r.c[:, 2] == 1) & (r.c[:, 0] == 0) & (r.c[:, 1] == 0))[0])
    ext = np.zeros((r.q, r.nzf + 4, 8, 8))
    ext[i, r.nzf + 3, 5, 2] = 0.8  # one fine ghost cell above the slab, coarse cell (1, 2)
    coal = r.coalesce(ext)[r.hi][i]
    want = np.zeros((4, 4))
    want[2, 1] = 0.1
    assert np.array_equal(coal, want)


def _smooth_state(r, seed=7):
    nz, ny, nx = r.nz, r.ny, r.nx
    rc = 1.0 + inputs.uniform_field(seed, 1, (nz, ny, nx), -0.01, 0.01)
    uc = inputs.uniform_field(seed, 2, (3, nz, ny, nx), -0.02, 0.02)
    shp = (r.nzf, 2 * ny, 2 * nx)
    rf = 1.0 + inputs.uniform_field(seed, 3, shp, -0.01, 0.01)
    uf = inputs.uniform_field(seed, 4, (3,) + shp, -0.02, 0.02)
    r.init_equilibrium(rc, uc, rf, uf)


@pytest.mark.parametrize("q", [19, 27])
def test_mass_and_momentum_are_conserved(q):
    r = RefinedOracle(4, 4, 8, 2, 5, q=q, tau=0.7)
    _smooth_state(r)
    m0, j0 = r.mass(), r.momentum()
    r.step(20)
    assert abs(r.mass() - m0) <= 1e-13 * m0
    assert np.abs(r.momentum() - j0).max() <= 1e-13 * m0
    assert not np.isnan(r.ff).any() and not np.isnan(r.fc[:, ~r.covered]).any()


def test_uniform_equilibrium_is_a_fixed_point():
    r = RefinedOracle(4, 2, 6, 1, 3, tau=0.9, closure="smag", cs=0.1)
    u = np.array([0.03, -0.02, 0.01])
    r.init_equilibrium(1.02, u, 1.02, u)
    feq = oracle.equilibrium(19, 1.02, u)
    r.step(5)
    assert np.abs(r.fc[:, ~r.covered] - feq[:, None, None, None]).max() <= 1e-15
    assert np.abs(r.ff - feq[:, None, None, None]).max() <= 1e-15


def _shear_wave_rate(fine_tau=None, T=400):
    nz, z0, z1, tau, U = 32, 8, 24, 0.8, 1e-3
    k = 2 * np.pi / nz
    r = RefinedOracle(2, 2, nz, z0, z1, tau=tau)
    if fine_tau is not None:
        r.fine = oracle.Oracle(4, 4, r.nzf, tau=fine_tau, faces=("periodic",) * 6)
    zc = np.arange(nz, dtype=float)
    zf = z0 + (np.arange(r.nzf) + 0.5) / 2 - 0.5  # fine cell centres in coarse units
    uc = np.zeros((3, nz, 2, 2))
    uc[0] = U * np.sin(k * zc)[:, None, None]
    uf = np.zeros((3, r.nzf, 4, 4))
    uf[0] = U * np.sin(k * zf)[:, None, None]
    r.init_equilibrium(1.0, uc, 1.0, uf)
    cxd = r.c[:, 0].astype(float)
    m = ~r.covered

    def amp():
        f = np.where(np.isnan(r.fc), 0.0, r.fc)
        with np.errstate(invalid="ignore"):
            uxc = (np.tensordot(cxd, f, axes=(0, 0)) / f.sum(0)).mean(axis=(1, 2))
        uxf = (np.tensordot(cxd, r.ff, axes=(0, 0)) / r.ff.sum(0)).mean(axis=(1, 2))
        # least squares over the volume: a fine plane weighs half a coarse plane
        num = (uxc[m] * np.sin(k * zc[m])).sum() + 0.5 * (uxf * np.sin(k * zf)).sum()
        den = (np.sin(k * zc[m]) ** 2).sum() + 0.5 * (np.sin(k * zf) ** 2).sum()
        return num / den

    a0 = amp()
    r.step(T)
    return -np.log(amp() / a0) / T, (tau - 0.5) / 3 * k * k


def test_shear_wave_decays_at_the_viscous_rate():
    rate, ana = _shear_wave_rate()
    # a uniform coarse lattice of this resolution is off by 0.09 %; the refined one by 0.07 %
    assert abs(rate / ana - 1.0) <= 5e-3


def _poiseuille(T=3000, force_fine=None, fine_tau=None):
    nz, z0, z1, tau, F = 16, 4, 12, 1.0, 1e-6
    nu = (tau - 0.5) / 3
    r = RefinedOracle(2, 2, nz, z0, z1, tau=tau, force=(F, 0, 0), walls=True)
    if force_fine is not None or fine_tau is not None:
        r.fine = oracle.Oracle(4, 4, r.nzf, tau=refine.fine_tau(tau) if fine_tau is None else fine_tau,
                               faces=("periodic",) * 6, force=(F / 2 if force_fine is None else force_fine, 0, 0))
    r.init_equilibrium(1.0, np.zeros(3), 1.0, np.zeros(3))
    r.step(T)
    cxd = r.c[:, 0].astype(float)

    def ux(f, fx):  # velocity with the half-force correction of the forcing scheme
        return ((np.tensordot(cxd, f, axes=(0, 0)) + fx / 2) / f.sum(0)).mean(axis=(1, 2))

    ana = lambda z: F / (2 * nu) * (z + 0.5) * (nz - z - 0.5)  # walls at z = -1/2, nz - 1/2
    m = ~r.covered
    zc = np.arange(nz, dtype=float)[m]
    zf = z0 + (np.arange(r.nzf) + 0.5) / 2 - 0.5
    umax = ana(nz / 2 - 0.5)
    ec = np.abs(ux(r.fc[:, m], F) - ana(zc)).max() / umax
    ef = np.abs(ux(r.ff, r.fine.cfg.force[0]) - ana(zf)).max() / umax
    return ec, ef


def test_poiseuille_profile_across_the_refined_slab():
    ec, ef = _poiseuille()
    # observed 3e-9 / 4e-9 of u_max after 3000 steps (the remainder is the start-up transient)
    assert ec <= 1e-6 and ef <= 1e-6


def test_planted_mistakes_fail_the_pins():
    # viscosity not rescaled on the fine level (tau_f = tau_c)
    ec, ef = _poiseuille(T=1500, fine_tau=1.0)
    assert ef > 0.05
    # body force not halved on the fine level
    ec, ef = _poiseuille(T=1500, force_fine=1e-6)
    assert max(ec, ef) > 0.05
    # tau_f = 2 tau_c: the shear wave decays at the wrong rate
    rate, ana = _shear_wave_rate(fine_tau=1.6, T=200)
    assert abs(rate / ana - 1.0) > 0.05


def test_planted_unshifted_coalescence_fails_transport_pin():
    r = RefinedOracle(4, 4, 6, 2, 4)
    i = int(np.flatnonzero((r.c[:, 0] == 1) & (r.c[:, 1] == 0) & (r.c[:, 2] == -1))[0])
    ext = np.zeros((r.q, r.nzf + 4, 8, 8))
    ext[i, 2:4, 2:4, 2:4] = 1.0
    # mistake: the fine populations are averaged where they started, without streaming
    coal_wrong = r.coalesce(np.concatenate([ext[:, 2:4], ext[:, 2:]], axis=1))[r.lo][i]
    coal_right = r.coalesce(r.fine_stream(r.fine_stream(ext)))[r.lo][i]
    assert coal_right[1, 2] == 1.0 and coal_wrong[1, 2] != 1.0


# ---- several slabs, slabs on the walls -------------------------------------------------------
def _smooth_multi(r, seed=9):
    nz, ny, nx = r.nz, r.ny, r.nx
    rc = 1.0 + inputs.uniform_field(seed, 1, (nz, ny, nx), -0.01, 0.01)
    uc = inputs.uniform_field(seed, 2, (3, nz, ny, nx), -0.02, 0.02)
    rf, uf = [], []
    for k, s in enumerate(r.slabs):
        shp = (s.nzf, 2 * ny, 2 * nx)
        rf.append(1.0 + inputs.uniform_field(seed, 10 + k, shp, -0.01, 0.01))
        uf.append(inputs.uniform_field(seed, 20 + k, (3,) + shp, -0.02, 0.02))
    r.init_equilibrium(rc, uc, rf, uf)


@pytest.mark.parametrize("walls,slabs", [(False, [(1, 3), (5, 8)]), (True, [(0, 2), (6, 9)]),
                                         (True, [(0, 3)]), (True, [(3, 5), (7, 9)])])
def test_several_slabs_conserve_mass(walls, slabs):
    r = RefinedOracle(4, 2, 9, q=19, tau=0.7, walls=walls, slabs=slabs)
    _smooth_multi(r)
    m0, j0 = r.mass(), r.momentum()
    r.step(15)
    assert abs(r.mass() - m0) <= 1e-13 * m0
    if not walls:
        assert np.abs(r.momentum() - j0).max() <= 1e-13 * m0
    assert not any(np.isnan(f).any() for f in r.ffs) and not np.isnan(r.fc[:, ~r.covered]).any()


def test_poiseuille_with_refined_wall_slabs():
    """The channel case: both walls inside fine slabs, a coarse core; the analytic parabola
    on both levels (walls half a fine cell beyond the first fine cell centres)."""
    nz, tau, F = 16, 1.0, 1e-6
    nu = (tau - 0.5) / 3
    r = RefinedOracle(2, 2, nz, q=19, tau=tau, force=(F, 0, 0), walls=True, slabs=[(0, 4), (12, 16)])
    r.init_equilibrium(1.0, np.zeros(3), [1.0, 1.0], [np.zeros(3), np.zeros(3)])
    r.step(3000)
    cxd = r.c[:, 0].astype(float)

    def ux(f, fx):
        return ((np.tensordot(cxd, f, axes=(0, 0)) + fx / 2) / f.sum(0)).mean(axis=(1, 2))

    ana = lambda z: F / (2 * nu) * (z + 0.5) * (nz - z - 0.5)
    umax = ana(nz / 2 - 0.5)
    m = ~r.covered
    err = np.abs(ux(r.fc[:, m], F) - ana(np.arange(nz, dtype=float)[m])).max() / umax
    for s, f in zip(r.slabs, r.ffs):
        zf = s.z0 + (np.arange(s.nzf) + 0.5) / 2 - 0.5
        err = max(err, np.abs(ux(f, F / 2) - ana(zf)).max() / umax)
    assert err <= 1e-6, err


def test_shear_wave_with_two_slabs_decays_at_the_viscous_rate():
    nz, tau, U = 32, 0.8, 1e-3
    k = 2 * np.pi / nz
    r = RefinedOracle(2, 2, nz, q=19, tau=tau, slabs=[(4, 10), (18, 26)])
    zc = np.arange(nz, dtype=float)
    uc = np.zeros((3, nz, 2, 2))
    uc[0] = U * np.sin(k * zc)[:, None, None]
    zfs = [s.z0 + (np.arange(s.nzf) + 0.5) / 2 - 0.5 for s in r.slabs]
    ufs = []
    for s, zf in zip(r.slabs, zfs):
        u = np.zeros((3, s.nzf, 4, 4))
        u[0] = U * np.sin(k * zf)[:, None, None]
        ufs.append(u)
    r.init_equilibrium(1.0, uc, [1.0, 1.0], ufs)
    cxd = r.c[:, 0].astype(float)
    m = ~r.covered

    def amp():
        f = np.where(np.isnan(r.fc), 0.0, r.fc)
        with np.errstate(invalid="ignore"):
            uxc = (np.tensordot(cxd, f, axes=(0, 0)) / f.sum(0)).mean(axis=(1, 2))
        num = (uxc[m] * np.sin(k * zc[m])).sum()
        den = (np.sin(k * zc[m]) ** 2).sum()
        for ff, zf in zip(r.ffs, zfs):
            uxf = (np.tensordot(cxd, ff, axes=(0, 0)) / ff.sum(0)).mean(axis=(1, 2))
            num += 0.5 * (uxf * np.sin(k * zf)).sum()
            den += 0.5 * (np.sin(k * zf) ** 2).sum()
        return num / den

    a0 = amp()
    r.step(400)
    rate = -np.log(amp() / a0) / 400
    assert abs(rate / ((tau - 0.5) / 3 * k * k) - 1.0) <= 5e-3
