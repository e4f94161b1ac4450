"""Pins of the FP64 oracle against what the method and the mathematics fix.

Nothing here compares the oracle with itself: each test checks an identity of the
velocity set or the equilibrium, a closed-form solution, a conservation law, a special
case that reduces to a textbook operator, a hand-traced particle path, or an exact
rational restatement of the step (tests/exact_lbm.py).

Paper anchors: Eq. LBCollision and Eq. LBStreaming (Sec. 2); D3Q19 (Sec. 4, Sec. 5.2);
the wind-tunnel boundary set of Sec. 5.2 (inflow left, outflow right).
"""
import math

import numpy as np
import pytest

from tests import exact_lbm

FACES_CHANNEL = ("periodic", "periodic", "wall", "wall", "periodic", "periodic")


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


# ---------------------------------------------------------------------------------------
# velocity set and equilibrium
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("q", [19, 27])
def test_stencil_isotropy_and_order(O, q):
    c, w, opp = O.stencil(q)
    assert c.shape == (q, 3)
    assert len({tuple(v) for v in c}) == q
    assert abs(w.sum() - 1.0) < 1e-15
    eye = np.eye(3)
    for a in range(3):
        assert abs((w * c[:, a]).sum()) < 1e-16
        for b in range(3):
            assert abs((w * c[:, a] * c[:, b]).sum() - eye[a, b] / 3.0) < 1e-15
            for g in range(3):
                assert abs((w * c[:, a] * c[:, b] * c[:, g]).sum()) < 1e-16
    # fourth-order isotropy needed by the second-order equilibrium
    for a in range(3):
        assert abs((w * c[:, a] ** 4).sum() - 1.0 / 3.0) < 1e-15
        for b in range(3):
            if a != b:
                assert abs((w * c[:, a] ** 2 * c[:, b] ** 2).sum() - 1.0 / 9.0) < 1e-15
    # published order: rest first, then each direction followed by its opposite
    assert tuple(c[0]) == (0, 0, 0) and opp[0] == 0
    for i in range(1, q, 2):
        assert opp[i] == i + 1 and opp[i + 1] == i
        assert tuple(c[i]) == tuple(-c[i + 1])
    if q == 27:
        c19, _, _ = O.stencil(19)
        assert (c[:19] == c19).all()


@pytest.mark.parametrize("q", [19, 27])
def test_equilibrium_moments(O, q):
    c, w, opp = O.stencil(q)
    rng = np.random.default_rng(5)
    for _ in range(50):
        rho = 1.0 + rng.uniform(-0.1, 0.1)
        u = rng.uniform(-0.1, 0.1, 3)
        feq = O.equilibrium(q, rho, u)
        assert abs(feq.sum() - rho) < 1e-14
        assert np.abs(c.T @ feq - rho * u).max() < 1e-15
        second = np.einsum("i,ia,ib->ab", feq, c, c)
        assert np.abs(second - (rho / 3.0 * np.eye(3) + rho * np.outer(u, u))).max() < 1e-14
        # moving-wall identity: f_i^eq - f_opp^eq = 6 w_i rho (c_i . u)
        assert np.abs(feq - feq[opp] - 6.0 * w * rho * (c @ u)).max() < 1e-15


@pytest.mark.parametrize("q", [19, 27])
def test_equilibrium_moments_exact_rational(q):
    from fractions import Fraction as Fr
    lat = exact_lbm.ExactLattice((1, 1, 1), q, 1, Fr(3, 16))
    rho, u = Fr(101, 100), (Fr(3, 100), Fr(-1, 50), Fr(1, 70))
    eq = lat.feq(rho, u)
    assert sum(eq.values()) == rho
    for a in range(3):
        assert sum(cv[a] * v for cv, v in eq.items()) == rho * u[a]
        for b in range(3):
            s = sum(cv[a] * cv[b] * v for cv, v in eq.items())
            assert s == rho * Fr(int(a == b), 3) + rho * u[a] * u[b]


# ---------------------------------------------------------------------------------------
# streaming and boundary rules, traced by hand
# ---------------------------------------------------------------------------------------

def test_streaming_is_a_shift(O):
    """Eq. LBStreaming on a periodic lattice moves each population one cell along c_i."""
    for q in (19, 27):
        o = O.Oracle(5, 6, 7, q=q)
        c, _, _ = O.stencil(q)
        rng = np.random.default_rng(1)
        fstar = rng.random(o.f.shape)
        o.stream(fstar)
        for i in range(q):
            # array axes are (z, y, x)
            expect = np.roll(fstar[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2))
            assert np.array_equal(o.f[i], expect)


def test_streaming_periodic_identity(O):
    o = O.Oracle(5, 5, 5, q=27)
    rng = np.random.default_rng(2)
    f0 = rng.random(o.f.shape)
    cur = f0.copy()
    for _ in range(5):
        o.stream(cur)
        cur = o.f.copy()
    assert np.array_equal(cur, f0)


def _single(O, o, i, cell):
    fstar = np.zeros(o.f.shape)
    x, y, z = cell
    fstar[i, z, y, x] = 1.0
    o.stream(fstar)
    hits = np.argwhere(np.abs(o.f - o.w[:, None, None, None] * 0) > 0)
    return fstar, hits


def _dir(O, q, v):
    c, _, _ = O.stencil(q)
    return int(np.where((c == np.array(v)).all(axis=1))[0][0])


def test_bounce_back_wall_face(O):
    o = O.Oracle(3, 3, 3, q=19, faces=("wall",) * 6)
    i = _dir(O, 19, (-1, 0, 0))
    fstar = np.zeros(o.f.shape)
    fstar[i, 1, 1, 0] = 1.0
    o.stream(fstar)
    j = _dir(O, 19, (1, 0, 0))
    assert o.f[j, 1, 1, 0] == 1.0
    assert np.count_nonzero(o.f) == 1


def test_bounce_back_solid_cell(O):
    flags = np.zeros((3, 3, 3), np.uint8)
    flags[1, 1, 2] = 1  # (x=2, y=1, z=1)
    o = O.Oracle(3, 3, 3, q=19, flags=flags)
    i = _dir(O, 19, (1, 0, 0))
    fstar = np.zeros(o.f.shape)
    fstar[i, 1, 1, 1] = 1.0
    o.stream(fstar)
    j = _dir(O, 19, (-1, 0, 0))
    got = o.f.copy()
    got[:, flags == 1] = 0.0  # solid cells carry w, not populations
    assert got[j, 1, 1, 1] == 1.0 and np.count_nonzero(got) == 1


def test_free_slip_specular(O):
    faces = ("periodic", "periodic", "freeslip", "freeslip", "periodic", "periodic")
    o = O.Oracle(4, 3, 3, q=19, faces=faces)
    i = _dir(O, 19, (1, 1, 0))
    fstar = np.zeros(o.f.shape)
    fstar[i, 1, 2, 1] = 1.0  # x=1, y=ny-1
    o.stream(fstar)
    j = _dir(O, 19, (1, -1, 0))
    assert o.f[j, 1, 2, 2] == 1.0 and np.count_nonzero(o.f) == 1


def test_free_slip_edge_double_reflection(O):
    faces = ("periodic", "periodic", "freeslip", "freeslip", "freeslip", "freeslip")
    o = O.Oracle(4, 3, 3, q=27, faces=faces)
    i = _dir(O, 27, (1, 1, 1))
    fstar = np.zeros(o.f.shape)
    fstar[i, 2, 2, 1] = 1.0  # x=1, y=2, z=2: corner edge
    o.stream(fstar)
    j = _dir(O, 27, (1, -1, -1))
    assert o.f[j, 2, 2, 2] == 1.0 and np.count_nonzero(o.f) == 1


def test_inflow_face_moving_wall(O):
    uw = (0.05, 0.01, 0.0)
    faces = ("inflow", "outflow", "periodic", "periodic", "periodic", "periodic")
    o = O.Oracle(4, 3, 3, q=19, faces=faces, u_w=uw, rho_w=1.0)
    c, w, _ = O.stencil(19)
    fstar = np.zeros(o.f.shape)
    o.stream(fstar)
    # at x=0 every population coming from x=-1 is the moving-wall term alone
    for i in range(19):
        if c[i, 0] == 1:
            assert o.f[i, 1, 1, 0] == pytest.approx(6.0 * w[i] * (c[i] @ np.array(uw)), abs=1e-17)


def test_outflow_copies_upstream(O):
    faces = ("periodic", "outflow", "periodic", "periodic", "periodic", "periodic")
    with pytest.raises(ValueError):
        O.Oracle(4, 3, 3, q=19, faces=faces)  # periodic pairs must match
    faces = ("inflow", "outflow", "periodic", "periodic", "periodic", "periodic")
    o = O.Oracle(5, 3, 4, q=19, faces=faces)
    c, _, _ = O.stencil(19)
    rng = np.random.default_rng(3)
    fstar = rng.random(o.f.shape)
    o.stream(fstar)
    for i in range(19):
        if c[i, 0] == -1:
            assert np.array_equal(o.f[i, :, :, 4], o.f[i, :, :, 3])
            # and what the upstream cell received is the plain shift of fstar
            expect = np.roll(fstar[i], shift=(c[i, 2], c[i, 1]), axis=(0, 1))[:, :, 4]
            assert np.array_equal(o.f[i, :, :, 3], expect)


# ---------------------------------------------------------------------------------------
# collision special cases
# ---------------------------------------------------------------------------------------

def _random_state(O, q, rng, amp=1e-2):
    u = rng.uniform(-0.08, 0.08, 3)
    rho = 1.0 + rng.uniform(-0.02, 0.02)
    feq = O.equilibrium(q, rho, u)
    _, w, _ = O.stencil(q)
    return feq + amp * rng.uniform(-1, 1, q) * w


@pytest.mark.parametrize("q", [19, 27])
def test_trt_reduces_to_bgk(O, q):
    """With Lambda = (tau - 1/2)^2 both rates equal 1/tau: the BGK operator with Guo forcing."""
    tau = 0.73
    F = np.array([1e-4, -2e-4, 5e-5])
    o = O.Oracle(2, 2, 2, q=q, tau=tau, lam=(tau - 0.5) ** 2, force=F)
    c, w, _ = O.stencil(q)
    rng = np.random.default_rng(7)
    for _ in range(20):
        f = _random_state(O, q, rng)
        rho = f.sum()
        u = (c.T @ f + 0.5 * F) / rho
        feq = O.equilibrium(q, rho, u)
        cu = c @ u
        Fi = w * (3.0 * (c @ F - u @ F) + 9.0 * cu * (c @ F))
        bgk = f - (f - feq) / tau + (1.0 - 0.5 / tau) * Fi
        got, tau_eff = o.collide_cell(f)
        assert tau_eff == tau
        assert np.abs(got - bgk).max() < 2e-16


@pytest.mark.parametrize("q", [19, 27])
def test_collision_conserves_mass_and_adds_force(O, q):
    F = np.array([3e-4, 1e-4, -2e-4])
    o = O.Oracle(2, 2, 2, q=q, tau=0.55, closure="smag", cs=0.17, force=F)
    c, _, _ = O.stencil(q)
    rng = np.random.default_rng(8)
    for _ in range(20):
        f = _random_state(O, q, rng)
        fs, _ = o.collide_cell(f)
        assert abs(fs.sum() - f.sum()) < 1e-15
        assert np.abs(c.T @ fs - (c.T @ f + F)).max() < 1e-15


@pytest.mark.parametrize("q", [19, 27])
def test_smagorinsky_solves_implicit_equation(O, q):
    """tau = tau0 + 3 C_s^2 |S|(tau) with |S| = 3 sqrt(2 Pi:Pi) / (2 rho tau)."""
    tau0, cs = 0.5069, 0.1
    o = O.Oracle(2, 2, 2, q=q, tau=tau0, closure="smag", cs=cs)
    c, _, _ = O.stencil(q)
    rng = np.random.default_rng(9)
    for amp in (1e-4, 1e-3, 1e-2, 5e-2):
        f = _random_state(O, q, rng, amp)
        rho = f.sum()
        u = (c.T @ f) / rho
        neq = f - O.equilibrium(q, rho, u)
        pi = np.einsum("i,ia,ib->ab", neq, c, c)
        qn = (pi * pi).sum()
        _, tau = o.collide_cell(f)
        S = 3.0 * math.sqrt(2.0 * qn) / (2.0 * rho * tau)
        assert abs(tau - (tau0 + 3.0 * cs * cs * S)) < 1e-14
        assert tau > tau0


def test_smagorinsky_cs_zero_is_plain_trt(O):
    rng = np.random.default_rng(10)
    for q in (19, 27):
        a = O.Oracle(2, 2, 2, q=q, tau=0.6, closure="smag", cs=0.0, force=(1e-5, 0, 0))
        b = O.Oracle(2, 2, 2, q=q, tau=0.6, closure="none", force=(1e-5, 0, 0))
        for _ in range(10):
            f = _random_state(O, q, rng)
            assert np.array_equal(a.collide_cell(f)[0], b.collide_cell(f)[0])


# ---------------------------------------------------------------------------------------
# conservation laws and closed-form flows
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("q", [19, 27])
def test_mass_conservation_walls_and_solids(O, q):
    """Periodic + halfway bounce-back conserve mass: the drift is FP64 round-off only.

    The bound is 1e-15 relative per step: the FP64 weights sum to 1 - O(1e-17), which the
    equilibrium turns into a systematic loss of that order per collision."""
    nx, ny, nz = 12, 10, 8
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[2:4, 3:5, 4:7] = 1
    o = O.Oracle(nx, ny, nz, q=q, tau=0.6, closure="smag", cs=0.1, force=(1e-5, 2e-6, 0),
                 flags=flags, faces=FACES_CHANNEL)
    rng = np.random.default_rng(11)
    o.init_equilibrium(1 + rng.uniform(-0.01, 0.01, (nz, ny, nx)),
                       rng.uniform(-0.05, 0.05, (3, nz, ny, nx)))
    m0 = o.mass_momentum()[0]
    o.step(1000)
    m1 = o.mass_momentum()[0]
    assert abs(m1 - m0) / m0 < 1000 * 1e-15


@pytest.mark.parametrize("q", [19, 27])
def test_momentum_grows_by_force_when_periodic(O, q):
    """Fully periodic: total momentum changes by exactly F per cell and step."""
    n = (6, 5, 4)
    F = np.array([2e-5, -1e-5, 3e-6])
    o = O.Oracle(*n, q=q, tau=0.7, closure="smag", cs=0.12, force=F)
    rng = np.random.default_rng(12)
    o.init_equilibrium(1 + rng.uniform(-0.01, 0.01, n[::-1]),
                       rng.uniform(-0.05, 0.05, (3,) + n[::-1]))
    p0 = o.mass_momentum()[1:]
    o.step(200)
    p1 = o.mass_momentum()[1:]
    ncell = np.prod(n)
    assert np.abs(p1 - p0 - 200 * ncell * F).max() < 1e-12


@pytest.mark.parametrize("q,lam,tau,walls", [
    (19, 3 / 16, 0.8, "rows"), (19, 1 / 4, 0.8, "rows"), (19, 0.09, 0.8, "rows"),
    (19, 3 / 16, 0.56, "faces"), (27, 3 / 16, 0.8, "rows"), (27, 1 / 12, 1.0, "faces")])
def test_poiseuille_closed_form(O, q, lam, tau, walls):
    """Steady force-driven channel with halfway bounce-back and TRT.

    The steady solution is the parabola between walls halfway between the wall-adjacent
    fluid nodes and the solid nodes, plus a uniform slip (16 Lambda - 3)/12 * g/(2 nu)
    that vanishes for Lambda = 3/16 (Ginzburg and d'Humieres' TRT bounce-back analysis)."""
    ny = 18
    g = 1e-6
    nu = (tau - 0.5) / 3
    if walls == "rows":
        flags = np.zeros((1, ny, 1), np.uint8)
        flags[0, 0, 0] = flags[0, ny - 1, 0] = 1
        o = O.Oracle(1, ny, 1, q=q, tau=tau, lam=lam, force=(g, 0, 0), flags=flags)
        y0, y1 = 0.5, ny - 1.5
        fluid = slice(1, ny - 1)
    else:
        o = O.Oracle(1, ny, 1, q=q, tau=tau, lam=lam, force=(g, 0, 0), faces=FACES_CHANNEL)
        y0, y1 = -0.5, ny - 0.5
        fluid = slice(0, ny)
    o.init_equilibrium(1.0, np.zeros(3))
    H = y1 - y0
    o.step(int(30 * H * H / (math.pi ** 2 * nu)) + 100, threads=1)
    _, u = o.moments()
    y = np.arange(ny, dtype=np.float64)
    ua = g / (2 * nu) * ((y - y0) * (y1 - y) + (16 * lam - 3) / 12)
    umax = g / (2 * nu) * H * H / 4
    err = np.abs(u[0, 0, fluid, 0] - ua[fluid]).max() / umax
    assert err < 1e-9
    assert np.abs(u[1:]).max() < 1e-13  # round-off of sum c_y f with f ~ w


@pytest.mark.parametrize("q", [19, 27])
def test_free_slip_plug_flow(O, q):
    """Free-slip walls exert no friction: a uniform state starting at rest accelerates as
    u(t) = t F / rho (the populations start at the equilibrium of u = -F/2 so that the
    reported velocity, which includes +F/2, is zero at t = 0)."""
    F = 1e-5
    faces = ("periodic", "periodic", "freeslip", "freeslip", "freeslip", "freeslip")
    o = O.Oracle(4, 5, 3, q=q, tau=0.7, force=(F, 0, 0), faces=faces)
    o.init_equilibrium(1.0, np.array([-0.5 * F, 0, 0]))
    o.step(50)
    rho, u = o.moments()
    assert np.abs(rho - 1).max() < 1e-14
    assert np.abs(u[0] - 50 * F).max() < 1e-15
    # the same with bounce-back walls is slowed down at the walls
    o2 = O.Oracle(4, 5, 3, q=q, tau=0.7, force=(F, 0, 0), faces=FACES_CHANNEL)
    o2.init_equilibrium(1.0, np.array([-0.5 * F, 0, 0]))
    o2.step(50)
    assert o2.moments()[1][0, :, 0, :].max() < 50 * F * 0.99


@pytest.mark.parametrize("q", [19, 27])
def test_uniform_tunnel_is_a_fixed_point(O, q):
    """Inflow at u_w, zero-gradient outflow, free-slip sides: uniform (1, u_w) is steady."""
    uw = np.array([0.05, 0.0, 0.0])
    faces = ("inflow", "outflow", "freeslip", "freeslip", "freeslip", "freeslip")
    o = O.Oracle(8, 5, 4, q=q, tau=0.52, closure="smag", cs=0.1, faces=faces, u_w=uw)
    o.init_equilibrium(1.0, uw)
    f0 = o.f.copy()
    o.step(30)
    assert np.abs(o.f - f0).max() < 1e-15


def _tg_decay_rate(O, N, nu, U0):
    """Measured decay rate of the Taylor-Green mode, relative to 2 nu k^2."""
    tau = 3 * nu + 0.5
    o = O.Oracle(N, N, 1, q=19, tau=tau)
    k = 2 * math.pi / N
    x = np.arange(N)[None, :]
    y = np.arange(N)[:, None]
    mode = np.sin(k * x) * np.cos(k * y)
    u = np.zeros((3, 1, N, N))
    u[0, 0] = U0 * mode
    u[1, 0] = -U0 * np.cos(k * x) * np.sin(k * y)
    p = -U0 ** 2 / 4 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    o.init_equilibrium((1 + 3 * p)[None], u)
    t_decay = 1.0 / (2 * nu * k * k)
    t1 = int(round(0.1 * t_decay))
    t2 = int(round(0.6 * t_decay))

    def amplitude():  # projection of u_x on the vortex mode (filters acoustic modes)
        return (o.moments()[1][0, 0] * mode).sum() / (mode * mode).sum()

    o.step(t1)
    a1 = amplitude()
    o.step(t2 - t1)
    a2 = amplitude()
    return math.log(a1 / a2) / (t2 - t1) / (2 * nu * k * k)


def test_taylor_green_decay(O):
    """Taylor-Green vortex: velocity decays as exp(-2 nu k^2 t); the error is second order
    under diffusive scaling (nu fixed, U0 ~ 1/N, times ~ N^2)."""
    nu = 0.04
    errs = {}
    for N in (16, 32, 64):
        errs[N] = abs(_tg_decay_rate(O, N, nu, U0=0.08 / N) - 1.0)
    assert errs[64] < 1e-3
    order1 = math.log2(errs[16] / errs[32])
    order2 = math.log2(errs[32] / errs[64])
    assert 1.6 < order1 < 2.4 and 1.8 < order2 < 2.2, errs


# ---------------------------------------------------------------------------------------
# exact rational restatement of whole steps
# ---------------------------------------------------------------------------------------

def _exact_vs_oracle(O, q, n, tau, lam, force, cs, faces, solid, inflow_cells, u_w, steps,
                     seed):
    from fractions import Fraction as Fr
    nx, ny, nz = n
    flags = np.zeros((nz, ny, nx), np.uint8)
    for (x, y, z) in solid:
        flags[z, y, x] = 1
    for (x, y, z) in inflow_cells:
        flags[z, y, x] = 2
    o = O.Oracle(nx, ny, nz, q=q, tau=tau, lam=lam, closure="smag" if cs else "none",
                 cs=cs or 0.0, faces=faces, u_w=u_w, force=force, flags=flags)
    rng = np.random.default_rng(seed)
    o.init_equilibrium(1 + rng.uniform(-0.02, 0.02, (nz, ny, nx)),
                       rng.uniform(-0.06, 0.06, (3, nz, ny, nx)))
    o.f += rng.uniform(-1e-3, 1e-3, o.f.shape) * o.w[:, None, None, None]
    o.f[:, flags != 0] = o.w[:, None]
    c, _, _ = O.stencil(q)
    ex = exact_lbm.ExactLattice(n, q, Fr(tau), Fr(lam), force=[Fr(a) for a in force],
                                cs=None if not cs else Fr(cs), faces=faces, solid=solid,
                                inflow_cells=inflow_cells, u_w=[Fr(a) for a in u_w])
    for (x, y, z) in ex.cells():
        if ex.fluid((x, y, z)):
            ex.f[(x, y, z)] = {tuple(c[i]): Fr(float(o.f[i, z, y, x])) for i in range(q)}
    for _ in range(steps):
        o.step(1, threads=1)
        ex.step()
    err = 0.0
    for (x, y, z), fc in ex.f.items():
        for i in range(q):
            err = max(err, abs(float(fc[tuple(c[i])]) - o.f[i, z, y, x]))
    return err


def test_exact_channel_4cubed(O):
    """Two steps of a 4^3 channel (walls, one solid cell, force, Smagorinsky), Q19."""
    err = _exact_vs_oracle(O, 19, (4, 4, 4), 0.6, 3 / 16, (1e-4, -3e-5, 2e-5), 0.1,
                           FACES_CHANNEL, [(1, 2, 1)], [], (0, 0, 0), 2, 21)
    assert err < 1e-15


def test_exact_tunnel_4cubed(O):
    """Two steps with inflow, outflow, free-slip, one solid and one inflow cell, Q19."""
    faces = ("inflow", "outflow", "freeslip", "freeslip", "periodic", "periodic")
    err = _exact_vs_oracle(O, 19, (4, 4, 3), 0.55, 3 / 16, (0, 0, 0), 0.1, faces,
                           [(2, 1, 1)], [(1, 3, 0)], (0.05, 0.01, 0.0), 2, 22)
    assert err < 1e-15


def test_exact_tunnel_q27(O):
    """One step of a Q27 tunnel whose corners mix wall, inflow, outflow and free-slip."""
    faces = ("inflow", "outflow", "wall", "freeslip", "freeslip", "freeslip")
    err = _exact_vs_oracle(O, 27, (3, 3, 3), 0.7, 3 / 16, (1e-4, 0, 0), 0.15, faces,
                           [(1, 1, 1)], [], (0.04, 0.0, 0.01), 1, 23)
    assert err < 1e-15


# ---------------------------------------------------------------------------------------
# closure network
# ---------------------------------------------------------------------------------------

def test_mlp_forward_matches_erf_gelu(O):
    from scipy.special import erf
    p = np.zeros(O.MLP_NPARAM)
    W1 = p[:224].reshape(32, 7)
    W1[0, 2] = 1.0
    b2_off = 224 + 32 + 1024
    W2 = p[256:b2_off].reshape(32, 32)
    W2[0, 0] = 1.3
    p[b2_off + 32] = 0.7  # W3[0]
    p[-1] = -0.2
    gelu = lambda a: 0.5 * a * (1 + erf(a / math.sqrt(2)))
    for x2 in (-2.0, -0.3, 0.0, 0.4, 1.7):
        x = np.zeros(7)
        x[2] = x2
        y = O.mlp_forward(p, x)
        assert abs(y - (0.7 * gelu(1.3 * gelu(x2)) - 0.2 + 31 * 0 * 0.7)) < 1e-15


def test_mlp_gradient_central_differences(O):
    rng = np.random.default_rng(13)
    p = rng.normal(0, 0.4, O.MLP_NPARAM)
    for _ in range(3):
        x = rng.normal(0, 1, 7)
        g = O.mlp_backward(p, x, 1.0)
        h = 1e-6
        idx = rng.choice(O.MLP_NPARAM, 60, replace=False)
        for k in idx:
            pp, pm = p.copy(), p.copy()
            pp[k] += h
            pm[k] -= h
            fd = (O.mlp_forward(pp, x) - O.mlp_forward(pm, x)) / (2 * h)
            assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_mlp_zero_output_layer_is_smagorinsky(O):
    """softplus(0) C_s0^2 / ln 2 = C_s0^2: a zero last layer reproduces Smagorinsky."""
    rng = np.random.default_rng(14)
    p = rng.normal(0, 0.3, O.MLP_NPARAM)
    p[224 + 32 + 1024 + 32:] = 0.0
    for q in (19, 27):
        a = O.Oracle(2, 2, 2, q=q, tau=0.52, closure="mlp", cs=0.1, mlp=p, mlp_scale=(100, 10))
        b = O.Oracle(2, 2, 2, q=q, tau=0.52, closure="smag", cs=0.1)
        for _ in range(10):
            f = _random_state(O, q, rng, 1e-2)
            fa, ta = a.collide_cell(f)
            fb, tb = b.collide_cell(f)
            assert abs(ta - tb) < 1e-15
            assert np.abs(fa - fb).max() < 1e-16


def test_stats_sample_matches_moments(O):
    rng = np.random.default_rng(15)
    o = O.Oracle(6, 5, 4, q=19, faces=FACES_CHANNEL)
    o.init_equilibrium(1 + rng.uniform(-0.01, 0.01, (4, 5, 6)), rng.uniform(-0.05, 0.05, (3, 4, 5, 6)))
    acc = o.stats_sample()
    _, u = o.moments()
    assert np.allclose(acc[:, 0], 24)
    assert np.allclose(acc[:, 1], u[0].sum(axis=(0, 2)), rtol=0, atol=1e-15)
    assert np.allclose(acc[:, 7], (u[0] * u[1]).sum(axis=(0, 2)), rtol=0, atol=1e-15)


def test_velocity_set_weights_match_the_published_tables(O):
    """tests/golden/velocity_set_weights.txt: the D3Q19 and D3Q27 weights by squared speed
    (Qian, d'Humieres & Lallemand 1992) and c_s^2 = 1/3."""
    import os
    from fractions import Fraction

    path = os.path.join(os.path.dirname(__file__), "golden", "velocity_set_weights.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    for q in (19, 27):
        c, w, _ = O.stencil(q)
        c2 = (c * c).sum(axis=1)
        for st, speed, count, frac in rows:
            if int(st) != q:
                continue
            sel = c2 == int(speed)
            assert sel.sum() == int(count)
            assert np.all(np.abs(w[sel] - float(Fraction(frac))) <= 1e-17)
        # c_s^2 = sum_i w_i c_ix^2
        assert abs((w * c[:, 0] ** 2).sum() - 1.0 / 3.0) <= 1e-16
