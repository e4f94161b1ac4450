"""Pins of the oracle functions that the full-size parity tests and the closure rest on.

* ``ora_step_sampled`` (one step from f = f^eq(rho, u), evaluated at chosen cells, used for
  full-size sampled parity) equals the pinned whole-lattice step ``ora_step`` from the same
  state at every cell of channel, wind-tunnel and mixed-face lattices, both stencils, to
  1e-15 (Eq. LBCollision then Eq. LBStreaming, Sec. 2).
* ``ora_step_sampled_pop`` (the same from arbitrary shifted float32 populations, used to
  check a step of the bench's gather kernel at full size) equals ``ora_step`` likewise.
* ``ora_filter2`` (width-2 box filter with Favre velocity, the closure's training data)
  returns, for linear density and momentum fields, the closed form: the box mean is the
  value at the box centre, the Favre velocity the centre momentum over the centre density;
  boxes with solid cells drop exactly those cells' contributions.
* ``ora_stats_sample`` (the channel statistics of Sec. 5.1: plane sums of u and u_a u_b)
  returns the closed-form plane sums of a prescribed field U(y) + Fourier modes in x and z.

Each pin is shown to fail on a planted mistake in a compiled copy of the oracle
(``tests/mutants.py``).
"""
import numpy as np
import pytest

from tests.mutants import mutant

FACES_CHANNEL = ("periodic", "periodic", "wall", "wall", "periodic", "periodic")
FACES_TUNNEL = ("inflow", "outflow", "freeslip", "freeslip", "freeslip", "freeslip")
FACES_MIXED = ("inflow", "outflow", "periodic", "periodic", "wall", "freeslip")


def _fields(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    rho = (1.0 + rng.uniform(-0.02, 0.02, (nz, ny, nx))).astype(np.float32)
    u = rng.uniform(-0.06, 0.06, (3, nz, ny, nx)).astype(np.float32)
    u[0] += 0.04
    return rho, u


def _flags(nx, ny, nz, seed, inflow_cells):
    rng = np.random.default_rng(seed)
    fl = np.zeros((nz, ny, nx), np.uint8)
    for _ in range(3):
        x, y, z = rng.integers(2, nx - 3), rng.integers(1, ny - 2), rng.integers(1, nz - 2)
        fl[z:z + 2, y:y + 2, x:x + 2] = 1
    if inflow_cells:
        fl[nz // 2, ny // 2, 1] = 2
    return fl


CASES = [
    ("channel", FACES_CHANNEL, dict(closure="smag", cs=0.12, force=(2e-5, -1e-5, 3e-6))),
    ("tunnel", FACES_TUNNEL, dict(closure="smag", cs=0.1, u_w=(0.05, 0.01, -0.02))),
    ("mixed", FACES_MIXED, dict(closure="none", u_w=(0.04, 0.0, 0.01), force=(0, 1e-5, 0))),
]


def _sampled_vs_step(O, q, faces, kw, seed=3):
    nx, ny, nz = 13, 9, 7
    flags = _flags(nx, ny, nz, seed, inflow_cells=faces[0] != "inflow" or q == 27)
    o = O.Oracle(nx, ny, nz, q=q, tau=0.57, faces=faces, flags=flags, **kw)
    rho, u = _fields(nx, ny, nz, seed)
    o.init_equilibrium(rho.astype(np.float64), u.astype(np.float64))
    o.step(1, threads=1)
    cells = np.arange(nx * ny * nz)
    got = o.step_sampled(rho, u, cells)  # (N, q)
    ref = o.f.reshape(q, -1).T
    fluid = flags.reshape(-1) == 0
    assert fluid.sum() > 0.8 * fluid.size
    return float(np.abs(got[fluid] - ref[fluid]).max()), float(np.abs(got[~fluid]).max(initial=0.0))


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("name,faces,kw", CASES, ids=[c[0] for c in CASES])
def test_step_sampled_equals_whole_lattice_step(oracle_mod, q, name, faces, kw):
    err, solid = _sampled_vs_step(oracle_mod, q, faces, kw)
    assert err <= 1e-15, err
    assert solid == 0.0


@pytest.mark.parametrize("edit", [
    # the cached post-collision values are the equilibrium itself (the collision is skipped)
    ("uc, f);\n    ora_collide(e->cfg, f, e->cached, NULL);\n", "uc, f);\n    memcpy(e->cached, f, sizeof f);\n"),
    # the one-cell cache is never refreshed: every source reads the first cell looked up
    ("  if (e->cached_cell != cell) {\n    double f[27], uc[3]", "  if (e->cached_cell < 0) {\n    double f[27], uc[3]"),
], ids=["no_collision", "stale_cache"])
def test_planted_mistakes_in_step_sampled_fail_the_pin(oracle_mod, edit):
    with mutant([edit]):
        err, _ = _sampled_vs_step(oracle_mod, 19, FACES_CHANNEL, CASES[0][2])
    assert err > 1e-6, err


def _sampled_pop_vs_step(O, q, faces, kw, seed=4):
    """The sampled step from arbitrary populations (a developed, non-equilibrium state)."""
    nx, ny, nz = 13, 9, 7
    flags = _flags(nx, ny, nz, seed, inflow_cells=faces[0] != "inflow" or q == 27)
    o = O.Oracle(nx, ny, nz, q=q, tau=0.57, faces=faces, flags=flags, **kw)
    rho, u = _fields(nx, ny, nz, seed)
    o.init_equilibrium(rho.astype(np.float64), u.astype(np.float64))
    o.step(2, threads=1)
    df = o.shifted().astype(np.float32)
    o.set_shifted(df)  # both sides start from the same float32 values
    o.step(1, threads=1)
    cells = np.arange(nx * ny * nz)
    got = o.step_sampled_pop(df, cells)
    ref = o.f.reshape(q, -1).T
    fluid = flags.reshape(-1) == 0
    return float(np.abs(got[fluid] - ref[fluid]).max()), float(np.abs(got[~fluid]).max(initial=0.0))


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("name,faces,kw", CASES, ids=[c[0] for c in CASES])
def test_step_sampled_from_populations_equals_whole_lattice_step(oracle_mod, q, name, faces, kw):
    err, solid = _sampled_pop_vs_step(oracle_mod, q, faces, kw)
    assert err <= 1e-15, err
    assert solid == 0.0


def test_planted_mistake_in_step_sampled_from_populations_fails_the_pin(oracle_mod):
    # the populations are unshifted with the D3Q19 weights whatever the stencil
    with mutant([("for (int i = 0; i < e->cfg->q; i++) f[i] = W_(e->cfg->q, i) + (double)e->df",
                  "for (int i = 0; i < e->cfg->q; i++) f[i] = W_(19, i) + (double)e->df")]):
        err, _ = _sampled_pop_vs_step(oracle_mod, 27, FACES_TUNNEL, CASES[1][2])
    assert err > 1e-3, err


# ---- box filter --------------------------------------------------------------------------

def _lin(coef, x, y, z):
    return coef[0] + coef[1] * x + coef[2] * y + coef[3] * z


RHO_C = (1.0, 0.01, -0.02, 0.015)
MOM_C = ((0.02, 0.001, 0.002, -0.003), (-0.01, 0.002, -0.001, 0.0005), (0.005, -0.0015, 0.001, 0.002))
FORCE = (1e-4, -2e-4, 5e-5)


def _filter_case(O, q):
    nx, ny, nz = 8, 6, 4
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rho = _lin(RHO_C, x, y, z)
    mom = np.stack([_lin(c, x, y, z) for c in MOM_C])
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[1, 2, 5] = 1           # one solid cell in box (2, 1, 0)
    flags[2:4, 4:6, 0:2] = 1     # box (0, 2, 1) entirely solid
    o = O.Oracle(nx, ny, nz, q=q, faces=FACES_CHANNEL, force=FORCE, flags=flags)
    # reported velocity = (sum c f + F/2) / rho, so the cell momentum rho u is mom exactly
    u_in = (mom - 0.5 * np.asarray(FORCE)[:, None, None, None]) / rho
    o.init_equilibrium(rho, u_in)
    rb, ub = o.filter2()
    # closed form: the mean of a linear field over a 2x2x2 box is its value at the box centre
    Z, Y, X = np.meshgrid(np.arange(nz // 2), np.arange(ny // 2), np.arange(nx // 2), indexing="ij")
    cxc, cyc, czc = 2 * X + 0.5, 2 * Y + 0.5, 2 * Z + 0.5
    rs = 8.0 * _lin(RHO_C, cxc, cyc, czc)
    ms = np.stack([8.0 * _lin(c, cxc, cyc, czc) for c in MOM_C])
    for fz, fy, fx in zip(*np.nonzero(flags)):  # solid cells drop out of the sums
        rs[fz // 2, fy // 2, fx // 2] -= _lin(RHO_C, fx, fy, fz)
        for d in range(3):
            ms[d, fz // 2, fy // 2, fx // 2] -= _lin(MOM_C[d], fx, fy, fz)
    rs[np.abs(rs) < 1e-12] = 0.0
    ref_rb = rs / 8.0
    ref_ub = np.where(rs > 0, ms / np.where(rs > 0, rs, 1.0), 0.0)
    return rb, ub, ref_rb, ref_ub


@pytest.mark.parametrize("q", [19, 27])
def test_filter2_closed_form_for_linear_fields(oracle_mod, q):
    rb, ub, ref_rb, ref_ub = _filter_case(oracle_mod, q)
    assert ref_rb[1, 2, 0] == 0.0 and rb[1, 2, 0] == 0.0 and np.all(ub[:, 1, 2, 0] == 0.0)
    assert np.abs(rb - ref_rb).max() <= 1e-14
    assert np.abs(ub - ref_ub).max() <= 1e-14
    # the partially solid box differs from the full-box formula, so the drop is exercised
    assert abs(ref_rb[0, 1, 2] - _lin(RHO_C, 4.5, 2.5, 0.5)) > 1e-2


def test_planted_favre_weighting_mistake_fails_the_filter_pin(oracle_mod):
    with mutant([("          for (int d = 0; d < 3; d++) ms[d] += rho * u[d];\n",
                  "          for (int d = 0; d < 3; d++) ms[d] += u[d];\n")]):
        _, ub, _, ref_ub = _filter_case(oracle_mod, 19)
    assert np.abs(ub - ref_ub).max() > 1e-4


def test_planted_box_origin_mistake_fails_the_filter_pin(oracle_mod):
    # the box of coarse cell X starts at fine x = X instead of 2X (still inside the lattice)
    with mutant([("* fine->nx +\n                               2 * X + (c & 1);",
                  "* fine->nx +\n                               X + (c & 1);")]):
        rb, _, ref_rb, _ = _filter_case(oracle_mod, 19)
    assert np.abs(rb - ref_rb).max() > 1e-5


# ---- plane statistics -----------------------------------------------------------------------

A_X, B_Y, C_Z = 0.013, 0.021, 0.017
STATS_FORCE = (3e-5, -2e-5, 1e-5)


def _U(y, ny):
    return 0.08 * y * (ny - 1 - y) / ((ny - 1) ** 2 / 4.0)


def _stats_case(O):
    nx, ny, nz = 8, 6, 6
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kx, kz = 2 * np.pi / nx, 2 * np.pi / nz
    ut = np.stack([_U(y, ny) + A_X * np.cos(kx * x), B_Y * np.sin(kz * z), C_Z * np.cos(kx * x)])
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[:, 0, :] = 1
    flags[:, ny - 1, :] = 1
    solid = (1, 2, 3)  # (z, y, x) of one interior solid cell
    flags[solid] = 1
    o = O.Oracle(nx, ny, nz, q=19, faces=FACES_CHANNEL, force=STATS_FORCE, flags=flags)
    # rho = 1, so the reported velocity is u_in + F/2: prescribe ut by u_in = ut - F/2
    o.init_equilibrium(1.0, ut - 0.5 * np.asarray(STATS_FORCE)[:, None, None, None])
    acc = o.stats_sample()
    # closed form per plane: full periods of cos(kx x) and sin(kz z) sum to zero, their
    # squares to half the count; the solid rows give nothing, the solid cell is taken out
    n = nx * nz
    ref = np.zeros((ny, 10))
    for yy in range(1, ny - 1):
        U = _U(yy, ny)
        ref[yy] = [n, n * U, 0.0, 0.0, n * (U * U + A_X ** 2 / 2), n * B_Y ** 2 / 2, n * C_Z ** 2 / 2,
                   0.0, n * A_X * C_Z / 2, 0.0]
    v = ut[:, solid[0], solid[1], solid[2]]
    ref[solid[1]] -= [1.0, v[0], v[1], v[2], v[0] ** 2, v[1] ** 2, v[2] ** 2, v[0] * v[1], v[0] * v[2], v[1] * v[2]]
    return acc, ref


def test_stats_sample_closed_form_plane_sums(oracle_mod):
    acc, ref = _stats_case(oracle_mod)
    assert np.abs(acc - ref).max() <= 1e-14


def test_planted_index_mistake_fails_the_stats_pin(oracle_mod):
    with mutant([("        a[7] += u[0] * u[1];\n", "        a[7] += u[0] * u[2];\n")]):
        acc, ref = _stats_case(oracle_mod)
    assert np.abs(acc - ref).max() > 1e-4
