"""Pins of the oracle's regularised collision (projected regularisation, Latt & Chopard 2006)
against facts that do not come from its own formula:

* it conserves mass and adds exactly F to the momentum;
* it has the second moment of BGK with Guo forcing (the oracle's TRT with
  Lambda = (tau - 1/2)^2, itself pinned to BGK) for any pre-collision state, and the same
  effective relaxation time under Smagorinsky;
* its non-equilibrium part f* - f^eq - F/2 lies in the span of w_i H_i (least-squares fit over
  the 6 symmetric components leaves nothing), i.e. it carries no independent
  non-equilibrium above second order: on D3Q19 the third-order (heat-flux and m) moments of
  the published MRT basis of d'Humieres et al. (2002) vanish, where BGK keeps them;
* for a state whose non-equilibrium is already of that form it equals BGK exactly;
* a shear wave decays at nu k^2 with nu = (tau - 1/2)/3;
* planted mistakes (projection without the trace term, half force left out) fail them.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2305_09910_gb300 import inputs


def _cell_oracle(q, tau, collision, force=(0.0, 0.0, 0.0), closure="none", cs=0.0):
    return oracle.Oracle(1, 1, 1, q=q, tau=tau, lam=(tau - 0.5) ** 2, collision=collision, force=force,
                         closure=closure, cs=cs)


def _random_cell(q, seed):
    c, w, _ = oracle.stencil(q)
    rho = 1.0 + float(inputs.uniform_field(seed, 1, (1,), -0.05, 0.05)[0])
    u = inputs.uniform_field(seed, 2, (3,), -0.08, 0.08)
    noise = inputs.uniform_field(seed, 3, (q,), -0.3, 0.3)
    return oracle.equilibrium(q, rho, u) * (1.0 + noise * 0.2), c.astype(np.float64), w


FORCE = (2e-4, -1e-4, 3e-4)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_conserves_mass_and_adds_the_force(q, seed):
    f, c, _ = _random_cell(q, seed)
    fs, _ = _cell_oracle(q, 0.73, "reg", force=FORCE).collide_cell(f)
    assert abs(fs.sum() - f.sum()) <= 1e-15
    assert np.abs(c.T @ fs - c.T @ f - np.array(FORCE)).max() <= 1e-15


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("closure", ["none", "smag"])
def test_second_moment_equals_bgk(q, closure):
    for seed in range(4):
        f, c, _ = _random_cell(q, 10 + seed)
        reg, tau_r = _cell_oracle(q, 0.61, "reg", FORCE, closure, 0.17).collide_cell(f)
        bgk, tau_b = _cell_oracle(q, 0.61, "trt", FORCE, closure, 0.17).collide_cell(f)
        assert tau_r == tau_b
        mom = lambda g: np.einsum("ia,ib,i->ab", c, c, g)
        assert np.abs(mom(reg) - mom(bgk)).max() <= 1e-15
        assert abs(reg.sum() - bgk.sum()) <= 1e-15
        assert np.abs(c.T @ reg - c.T @ bgk).max() <= 1e-15
        # and they differ above second order: the regularised state is not BGK's
        assert np.abs(reg - bgk).max() > 1e-4


def _guo(q, u, F):
    c, w, _ = oracle.stencil(q)
    c = c.astype(np.float64)
    F = np.asarray(F)
    return w * (3.0 * (c - u) @ F + 9.0 * (c @ u) * (c @ F))


def _moments(f, c):
    rho = f.sum()
    return rho, (c.T @ f + 0.5 * np.array(FORCE)) / rho


@pytest.mark.parametrize("q", [19, 27])
def test_non_equilibrium_is_second_order_hermite(q):
    for seed in range(4):
        f, c, w = _random_cell(q, 20 + seed)
        fs, _ = _cell_oracle(q, 0.9, "reg", FORCE).collide_cell(f)
        rho, u = _moments(f, c)
        r = fs - oracle.equilibrium(q, rho, u) - 0.5 * _guo(q, u, FORCE)
        # least squares r_i = w_i sum_ab c_ia c_ib X_ab - w_i tr(X)/3 over symmetric X
        pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
        A = np.zeros((q, 6))
        for k, (a, b) in enumerate(pairs):
            A[:, k] = w * (c[:, a] * c[:, b] * (1 if a == b else 2) - (1.0 / 3.0 if a == b else 0.0))
        x, *_ = np.linalg.lstsq(A, r, rcond=None)
        assert np.abs(A @ x - r).max() <= 1e-16 + 1e-12 * np.abs(r).max()
        assert np.abs(r).max() > 1e-4  # the non-equilibrium part is not trivially zero


def test_third_order_moments_of_the_mrt_basis_vanish():
    M = oracle.mrt_matrix()
    odd_ghost = [4, 6, 8, 16, 17, 18]  # heat flux q_a and the third-order m_a rows
    for seed in range(4):
        f, c, _ = _random_cell(19, 30 + seed)
        rho, u = _moments(f, c)
        base = oracle.equilibrium(19, rho, u) + 0.5 * _guo(19, u, FORCE)
        fs, _ = _cell_oracle(19, 0.8, "reg", FORCE).collide_cell(f)
        assert np.abs(M[odd_ghost] @ (fs - base)).max() <= 1e-15
        assert np.abs(M[[9, 11, 13]] @ (fs - base)).max() > 1e-6  # the stress does relax
        # BGK keeps a third-order non-equilibrium part
        bgk, _ = _cell_oracle(19, 0.8, "trt", FORCE).collide_cell(f)
        assert np.abs(M[odd_ghost] @ (bgk - base)).max() > 1e-6


@pytest.mark.parametrize("q", [19, 27])
def test_equals_bgk_on_hermite_states(q):
    c, w, _ = oracle.stencil(q)
    c = c.astype(np.float64)
    rho, u = 1.03, np.array([0.02, -0.05, 0.04])
    A = inputs.uniform_field(4, 1, (3, 3), -1e-3, 1e-3)
    A = A + A.T
    H = np.einsum("ia,ib->iab", c, c) - np.eye(3) / 3.0
    f = oracle.equilibrium(q, rho, u) + 4.5 * w * np.einsum("iab,ab->i", H, A) - 0.5 * _guo(q, u, FORCE)
    reg, _ = _cell_oracle(q, 0.7, "reg", FORCE).collide_cell(f)
    bgk, _ = _cell_oracle(q, 0.7, "trt", FORCE).collide_cell(f)
    assert np.abs(reg - bgk).max() <= 2e-16


@pytest.mark.parametrize("q", [19, 27])
def test_shear_wave_decays_at_the_viscous_rate(q):
    nz, tau, U = 32, 0.8, 1e-3
    k = 2 * np.pi / nz
    o = oracle.Oracle(2, 2, nz, q=q, tau=tau, collision="reg")
    z = np.arange(nz, dtype=float)
    u = np.zeros((3, nz, 2, 2))
    u[0] = U * np.sin(k * z)[:, None, None]
    o.init_equilibrium(1.0, u)
    cx = oracle.stencil(q)[0][:, 0].astype(float)

    def amp():
        ux = (np.tensordot(cx, o.f, axes=(0, 0)) / o.f.sum(0)).mean(axis=(1, 2))
        return (ux * np.sin(k * z)).sum() / (np.sin(k * z) ** 2).sum()

    a0 = amp()
    T = 400
    o.step(T)
    rate = -np.log(amp() / a0) / T
    assert abs(rate / ((tau - 0.5) / 3 * k * k) - 1.0) <= 5e-3


def test_planted_mistakes_fail_the_pins():
    """The projection written without the trace term, or without the half force in g, as a
    plain restatement here: each breaks one of the pins above."""
    q = 19
    f, c, w = _random_cell(q, 40)
    tau = 0.9
    rho, u = _moments(f, c)
    feq = oracle.equilibrium(q, rho, u)
    fi = _guo(q, u, FORCE)

    def reg(trace=True, half_force=True):
        g = f - feq + (0.5 * fi if half_force else 0.0)
        P = np.einsum("ia,ib,i->ab", c, c, g)
        h = np.einsum("ia,ib,ab->i", c, c, P) - (np.trace(P) / 3.0 if trace else 0.0)
        return feq + 0.5 * fi + (1 - 1 / tau) * 4.5 * w * h

    good, _ = _cell_oracle(q, tau, "reg", FORCE).collide_cell(f)
    assert np.abs(reg() - good).max() <= 1e-15
    assert abs(reg(trace=False).sum() - f.sum()) > 1e-6  # mass no longer conserved
    bgk, _ = _cell_oracle(q, tau, "trt", FORCE).collide_cell(f)
    mom = lambda g: np.einsum("ia,ib,i->ab", c, c, g)
    assert np.abs(mom(reg(half_force=False)) - mom(bgk)).max() > 1e-7  # stress no longer BGK's
