"""Pins of the oracle's learned-closure pieces: box-filter samples, loss gradient, Adam.

Fine states are built from the first-order Chapman-Enskog solution
f = f^eq(u) - (rho w tau / c_s^2) Q_i : grad u with Q_i = c_i c_i - c_s^2 I, whose
non-equilibrium stress is exactly -2 rho c_s^2 tau S, so the strain-rate estimate of the
sample builder is known in closed form, as are the filtered subgrid stresses of linear
velocity fields.
"""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def _ce_state(O, o, tau, grad_u, u_of):
    """Chapman-Enskog populations of a velocity field with constant gradient grad_u[a][b] =
    d u_b / d x_a, u_of(x, y, z) -> u (rho = 1)."""
    c, w, _ = O.stencil(o.q)
    cs2 = 1.0 / 3.0
    for z in range(o.nz):
        for y in range(o.ny):
            for x in range(o.nx):
                u = np.array(u_of(x, y, z), dtype=np.float64)
                feq = O.equilibrium(o.q, 1.0, u)
                Qg = np.einsum("ia,ib,ab->i", c, c, grad_u) - cs2 * np.trace(grad_u)
                o.f[:, z, y, x] = feq - w * tau / cs2 * Qg


def test_uniform_state_gives_zero_samples(O):
    o = O.Oracle(4, 6, 4, q=19, tau=0.55, closure="smag", cs=0.1)
    o.init_equilibrium(1.0, np.array([0.03, -0.01, 0.02]))
    x, t, sm, w = o.closure_samples(0.6, 0.1, (100.0, 10.0))
    assert x.shape == (2 * 3 * 2, 7)
    assert np.abs(x).max() < 1e-12 and np.abs(t).max() == 0.0
    assert np.abs(sm).max() < 1e-12 and np.abs(w).max() < 1e-20


def test_linear_shear_strain_and_features(O):
    """u_x = a y: S_c,xy = a (two fine steps per coarse step), |S_c| = 2|a|, the subgrid
    stress is the in-box variance a^2/4 of u_x, orthogonal to S: nu* = 0."""
    a, tau, tau_c, cs0 = 2e-4, 0.6, 0.55, 0.1
    o = O.Oracle(4, 4, 2, q=19, tau=tau)
    g = np.zeros((3, 3))
    g[1, 0] = a  # d u_x / d y
    _ce_state(O, o, tau, g, lambda x, y, z: (a * y, 0.0, 0.0))
    x, t, sm, w = o.closure_samples(tau_c, cs0, (1.0, 1.0))
    assert np.allclose(sm, 2 * a, rtol=1e-9)
    assert np.allclose(w, 4 * a * a, rtol=1e-9)
    assert np.abs(t).max() == 0.0
    tc = tau_c + 3 * cs0 * cs0 * 2 * a
    expect_xy = -(2.0 / 3.0) * tc * a  # rho_bar = 1 to O(a^2)
    assert np.allclose(x[:, 3], expect_xy, rtol=1e-6)
    assert np.abs(x[:, [0, 1, 2, 4, 5]]).max() < 1e-12


def test_aligned_stress_gives_closed_form_eddy_viscosity(O):
    """u_x = u_y = a y: tau_sgs = a^2/4 in xx, yy, xy (zero in zz), trace a^2/2;
    S_c = (xy: a, yy: 2a), S_c:S_c = 6 a^2; tau^d : S_c = (a^2/12)(2a) + 2 (a^2/4) a = 2a^3/3;
    nu* = -(tau^d : S_c) / (2 S_c : S_c) = -a/18, clipped at zero."""
    for a, expect in ((-3e-4, 3e-4 / 18), (3e-4, 0.0)):
        o = O.Oracle(2, 4, 2, q=27, tau=0.7)
        g = np.zeros((3, 3))
        g[1, 0] = g[1, 1] = a
        _ce_state(O, o, 0.7, g, lambda x, y, z: (a * y, a * y, 0.0))
        _, t, sm, _ = o.closure_samples(0.6, 0.1)
        assert np.allclose(sm, math.sqrt(2 * 6) * abs(a), rtol=1e-6)
        assert np.allclose(t, expect, rtol=1e-5, atol=1e-12)


def test_closure_loss_gradient_central_differences(O):
    rng = np.random.default_rng(31)
    p = rng.normal(0, 0.3, O.MLP_NPARAM)
    n = 16
    x = rng.normal(0, 1, (n, 7))
    t = np.abs(rng.normal(0, 1e-4, n))
    sm = np.abs(rng.normal(0, 3e-3, n)) + 1e-4
    w = sm * sm
    L, g = O.closure_loss(p, x, t, sm, w, 0.1)
    assert L > 0
    h = 1e-6
    for k in rng.choice(O.MLP_NPARAM, 40, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (O.closure_loss(pp, x, t, sm, w, 0.1)[0] - O.closure_loss(pm, x, t, sm, w, 0.1)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (k, fd, g[k])


def test_adam_first_step_is_signed_learning_rate(O):
    """With zero moments the bias-corrected first step is lr * g / (|g| + eps)."""
    rng = np.random.default_rng(32)
    p = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    m, v = np.zeros(50), np.zeros(50)
    p0 = p.copy()
    O.adam(p, g, m, v, 1e-3, 1)
    assert np.allclose(p, p0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    # a constant gradient keeps the step at lr * g / (|g| + eps) (bias corrections cancel)
    for t in range(2, 6):
        O.adam(p, g, m, v, 1e-3, t)
    assert np.allclose(p, p0 - 5e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)
