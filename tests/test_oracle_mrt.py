"""Pins of the oracle's D3Q19 MRT collision (d'Humieres, Ginzburg, Krafczyk, Lallemand & Luo,
Phil. Trans. R. Soc. A 360 (2002) 437), the operator of the paper's LAGOON runs (Sec. 5.2):
  * the moment basis is orthogonal with the published row norms;
  * the moments of the polynomial equilibrium are the published closed forms
    (e = -11 rho + 19 rho u^2, eps = 3 rho - 11/2 rho u^2, q = -2/3 j, 3pi = -3p/2, ...);
  * with one rate for all moments it is BGK, with even/odd rates it is TRT;
  * mass is conserved and the momentum grows by F;
  * changing one group's rate moves f* only inside that group's moment subspace;
  * the steady Poiseuille channel with halfway bounce-back is the closed-form parabola when
    (1/s_nu - 1/2)(1/s_q - 1/2) = 3/16, whatever the even ghost rates."""
import numpy as np
import pytest


def _cfg(oracle_mod, **kw):
    return oracle_mod.Oracle(4, 4, 4, q=19, **kw)


def _golden_norms():
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "d3q19_mrt_row_norms.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return [int(v) for v in rows[0]]


def test_basis_orthogonal_with_published_norms(oracle_mod):
    M = oracle_mod.mrt_matrix()
    G = M @ M.T
    assert np.array_equal(G, np.diag(np.diag(G)))
    norms = _golden_norms()
    assert list(np.diag(G)) == norms


def test_equilibrium_moments_closed_forms(oracle_mod):
    M = oracle_mod.mrt_matrix()
    rng = np.random.default_rng(3)
    for _ in range(5):
        rho = 1 + 0.1 * rng.standard_normal()
        u = 0.05 * rng.standard_normal(3)
        m = M @ oracle_mod.equilibrium(19, rho, u)
        j = rho * u
        u2 = u @ u
        p3xx, pww = rho * (3 * u[0] ** 2 - u2), rho * (u[1] ** 2 - u[2] ** 2)
        want = [rho, -11 * rho + 19 * rho * u2, 3 * rho - 5.5 * rho * u2,
                j[0], -2 / 3 * j[0], j[1], -2 / 3 * j[1], j[2], -2 / 3 * j[2],
                p3xx, -0.5 * p3xx, pww, -0.5 * pww,
                rho * u[0] * u[1], rho * u[1] * u[2], rho * u[0] * u[2], 0, 0, 0]
        assert np.allclose(m, want, rtol=0, atol=1e-14)


def _random_f(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.05 * rng.standard_normal()
    u = 0.04 * rng.standard_normal(3)
    _, w, _ = oracle_mod.stencil(19)
    return oracle_mod.equilibrium(19, rho, u) + 1e-3 * w * rng.standard_normal(19)


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.3])
def test_equal_rates_is_bgk_and_even_odd_rates_is_trt(oracle_mod, tau):
    F = (2e-5, -1e-5, 3e-6)
    wp = 1 / tau
    bgk = _cfg(oracle_mod, tau=tau, lam=(tau - 0.5) ** 2, force=F)
    mrt1 = _cfg(oracle_mod, tau=tau, force=F, collision="mrt", mrt_s=(wp,) * 5)
    lam = 3 / 16
    wm = 1 / (lam / (tau - 0.5) + 0.5)
    trt = _cfg(oracle_mod, tau=tau, lam=lam, force=F)
    mrt2 = _cfg(oracle_mod, tau=tau, force=F, collision="mrt", mrt_s=(wp, wp, wm, wp, wm))
    for seed in range(4):
        f = _random_f(oracle_mod, seed)
        assert np.abs(mrt1.collide_cell(f)[0] - bgk.collide_cell(f)[0]).max() <= 1e-15
        assert np.abs(mrt2.collide_cell(f)[0] - trt.collide_cell(f)[0]).max() <= 1e-15


def test_conservation(oracle_mod):
    c, _, _ = oracle_mod.stencil(19)
    F = np.array([3e-5, 1e-5, -2e-5])
    o = _cfg(oracle_mod, tau=0.6, force=F, collision="mrt", mrt_s=(1.19, 1.4, 1.2, 1.4, 1.98))
    for seed in range(4):
        f = _random_f(oracle_mod, 10 + seed)
        fs, _ = o.collide_cell(f)
        assert abs(fs.sum() - f.sum()) <= 1e-15
        assert np.abs(c.T @ fs - c.T @ f - F).max() <= 1e-15


def test_one_rate_moves_only_its_moments(oracle_mod):
    M = oracle_mod.mrt_matrix()
    groups = {2: [4, 6, 8], 3: [10, 12], 4: [16, 17, 18], 0: [1], 1: [2]}
    base = (1.19, 1.4, 1.2, 1.4, 1.98)
    f = _random_f(oracle_mod, 21)
    a = _cfg(oracle_mod, tau=0.7, force=(1e-5, 0, 0), collision="mrt", mrt_s=base).collide_cell(f)[0]
    for g, rows in groups.items():
        s = list(base)
        s[g] = 0.9
        b = _cfg(oracle_mod, tau=0.7, force=(1e-5, 0, 0), collision="mrt", mrt_s=s).collide_cell(f)[0]
        dm = M @ (b - a)
        others = [k for k in range(19) if k not in rows]
        assert np.abs(dm[rows]).max() > 1e-9
        assert np.abs(dm[others]).max() <= 1e-15


def test_poiseuille_exact_with_magic_rates(oracle_mod):
    from paper_2305_09910_gb300 import inputs

    ny, tau, g = 12, 0.9, 1e-5
    nu = (tau - 0.5) / 3
    wnu = 1 / tau
    sq = 1 / (3 / 16 / (tau - 0.5) + 0.5)  # (1/s_nu - 1/2)(1/s_q - 1/2) = 3/16
    flags = inputs.poiseuille_flags(1, ny, 1)
    y = np.arange(ny, dtype=float)
    y0, y1 = 0.5, ny - 1.5
    exact = g / (2 * nu) * (y - y0) * (y1 - y)
    fluid = slice(1, ny - 1)
    err = {}
    for name, s_q in (("magic", sq), ("other", 1.6)):
        o = oracle_mod.Oracle(1, ny, 1, q=19, tau=tau, force=(g, 0, 0), flags=flags, collision="mrt",
                              mrt_s=(1.1, 1.3, s_q, 1.7, s_q))
        o.init_equilibrium(1.0, np.zeros(3))
        o.step(int(30 * (ny - 2) ** 2 / nu))
        _, u = o.moments()
        err[name] = np.abs(u[0, 0, fluid, 0] - exact[fluid]).max() / exact.max()
    assert err["magic"] <= 1e-9        # round-off of ~20k steps
    assert err["other"] >= 1e-4        # the bounce-back slip of a non-magic pair
