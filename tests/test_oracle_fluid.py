"""Pins of the fluid-step oracle (Sec. 3.1 Steps 1 and 3) against closed forms
and exact properties, so that a wrong sign, index or stencil weight in any
of its operators fails here.  CPU only."""
import numpy as np
import pytest

from oracle import fluid

RNG = np.random.default_rng(2408)


def grid(n):
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h   # cell centres
    nd = np.arange(n) * h          # nodes
    return h, c, nd


def test_gradient_of_a_nodal_mode_is_the_closed_form():
    n = 16
    h, c, nd = grid(n)
    for m in (1, 3):
        Z, Y, X = np.meshgrid(nd, nd, nd, indexing="ij")
        p = np.sin(2 * np.pi * m * X) + 0.5 * np.cos(2 * np.pi * (m + 1) * Z)
        G = fluid.grad_node_to_cell(p, h)
        Zc, Yc, Xc = np.meshgrid(c, c, c, indexing="ij")
        gx = (2 / h) * np.sin(np.pi * m * h) * np.cos(2 * np.pi * m * Xc)
        gz = -0.5 * (2 / h) * np.sin(np.pi * (m + 1) * h) * np.sin(2 * np.pi * (m + 1) * Zc)
        assert np.max(np.abs(G[0] - gx)) < 1e-12
        assert np.max(np.abs(G[1])) < 1e-12
        assert np.max(np.abs(G[2] - gz)) < 1e-12


def test_divergence_is_the_negative_adjoint_of_the_gradient():
    n = (12, 10, 8)
    h = 0.07
    p = RNG.normal(size=(n[2], n[1], n[0]))
    V = RNG.normal(size=(3, n[2], n[1], n[0]))
    lhs = np.sum(fluid.grad_node_to_cell(p, h) * V)
    rhs = -np.sum(p * fluid.div_cell_to_node(V, h))
    assert abs(lhs - rhs) < 1e-12 * np.sum(np.abs(V)) / h


def test_div_grad_of_a_mode_is_its_symbol_times_the_mode():
    n = 16
    h, _, nd = grid(n)
    Z, Y, X = np.meshgrid(nd, nd, nd, indexing="ij")
    for m in ((1, 0, 0), (2, 3, 1), (5, 5, 2)):
        p = np.cos(2 * np.pi * (m[0] * X + m[1] * Y + m[2] * Z))
        Lp = fluid.div_cell_to_node(fluid.grad_node_to_cell(p, h), h)
        th = [2 * np.pi * mm / n for mm in m]
        s = [np.sin(t / 2) ** 2 for t in th]
        cc = [np.cos(t / 2) ** 2 for t in th]
        lam = -(4 / h ** 2) * (s[0] * cc[1] * cc[2] + s[1] * cc[0] * cc[2] + s[2] * cc[0] * cc[1])
        assert np.max(np.abs(Lp - lam * p)) < 1e-9 * abs(lam)


def test_poisson_solve_inverts_div_grad():
    n = (16, 8, 12)
    h = 1.0 / 16
    p = RNG.normal(size=(n[2], n[1], n[0]))
    rhs = fluid.div_cell_to_node(fluid.grad_node_to_cell(p, h), h)
    q = fluid.solve_div_grad(rhs, h)
    assert np.max(np.abs(fluid.div_cell_to_node(fluid.grad_node_to_cell(q, h), h) - rhs)) < 1e-10 * np.max(np.abs(rhs))


def test_projection_is_divergence_free_and_idempotent():
    n = (16, 12, 8)
    h, dt, rho = 1.0 / 16, 1e-3, 1.3
    u = RNG.normal(size=(3, n[2], n[1], n[0]))
    p_old = RNG.normal(size=(n[2], n[1], n[0]))
    u1, p1 = fluid.projection(u, p_old, rho, dt, h)
    assert np.max(np.abs(fluid.div_cell_to_node(u1, h))) < 1e-11 * np.max(np.abs(u)) / h
    # a divergence-free field passes unchanged (with the pressure it came with)
    u2, p2 = fluid.projection(u1, p1, rho, dt, h)
    assert np.max(np.abs(u2 - u1)) < 1e-12 * np.max(np.abs(u1))
    assert np.max(np.abs(p2 - p1)) < 1e-10 * np.max(np.abs(p1))
    # a pure gradient is removed entirely
    g = fluid.grad_node_to_cell(RNG.normal(size=(n[2], n[1], n[0])), h)
    u3, _ = fluid.projection(g, np.zeros(p_old.shape), rho, dt, h)
    assert np.max(np.abs(u3)) < 1e-12 * np.max(np.abs(g))


def test_helmholtz_solve_of_a_mode_is_the_closed_form():
    n = 32
    h, c, _ = grid(n)
    Zc, Yc, Xc = np.meshgrid(c, c, c, indexing="ij")
    m, coef = 3, 0.01
    u = np.stack([np.sin(2 * np.pi * m * Xc), np.zeros_like(Xc), np.cos(2 * np.pi * m * Yc)])
    x = fluid.solve_helmholtz(u, coef, h)
    f = 1.0 / (1.0 + coef * (4 / h ** 2) * np.sin(np.pi * m * h) ** 2)
    assert np.max(np.abs(x - f * u)) < 1e-13


def test_convection_vanishes_for_uniform_and_shear_flows():
    n = 16
    h, c, _ = grid(n)
    Zc, Yc, Xc = np.meshgrid(c, c, c, indexing="ij")
    uni = np.stack([np.full_like(Xc, 0.7), np.full_like(Xc, -0.2), np.full_like(Xc, 0.1)])
    assert np.max(np.abs(fluid.convection(uni, h, 1e-3))) < 1e-13
    shear = np.stack([np.sin(2 * np.pi * Yc) + np.cos(2 * np.pi * Zc), np.zeros_like(Xc), np.zeros_like(Xc)])
    assert np.max(np.abs(fluid.convection(shear, h, 1e-3))) < 1e-13


def test_convection_converges():
    """A smooth divergence-free field: div(u u) = (u . grad) u, analytic.  The
    limited slopes clip to first order at extrema, so the mean error
    converges at nearly second order and the largest at first."""
    errs, means = [], []
    for n in (32, 64):
        h, c, _ = grid(n)
        Zc, Yc, Xc = np.meshgrid(c, c, c, indexing="ij")
        k = 2 * np.pi
        u = np.stack([np.sin(k * Xc) * np.cos(k * Yc), -np.cos(k * Xc) * np.sin(k * Yc), 0.3 * np.ones_like(Xc)])
        exact = np.stack([0.5 * k * np.sin(2 * k * Xc) + 0.3 * 0,
                          0.5 * k * np.sin(2 * k * Yc),
                          np.zeros_like(Xc)])
        A = fluid.convection(u, h, 0.1 * h)
        errs.append(np.max(np.abs(A - exact)))
        means.append(np.mean(np.abs(A - exact)))
    assert means[1] < means[0] / 2.8   # mean error: order > 1.48
    assert errs[1] < errs[0] / 1.8     # largest error: order > 0.85


def test_predictor_of_fluid_at_rest_is_the_body_force_step():
    n = 8
    h = 1.0 / n
    u = np.zeros((3, n, n, n))
    p = np.zeros((n, n, n))
    g = (0.0, 0.0, -9.81)
    out = fluid.predictor(u, p, 1.0, 1e-2, g, 1e-3, h)
    assert np.max(np.abs(out[2] + 9.81e-3)) < 1e-15 and np.max(np.abs(out[:2])) < 1e-15


@pytest.mark.parametrize("nu", [0.0, 0.05])
def test_taylor_green_step_converges_to_the_exact_solution(nu):
    """2D Taylor-Green vortex (uniform in z): u = sin x cos y, v = -cos x sin y
    (k = 2 pi) decays as exp(-2 nu k^2 t) with p = rho/4 (cos 2kx + cos 2ky)
    times exp(-4 nu k^2 t).  One predictor + projection step from the exact
    state at t = 0 (pressure at t = -dt/2) approaches the exact state at dt
    as h shrinks with dt proportional to h (the limiter keeps the largest
    error first order at the vortex extrema); a sign or stencil error in any
    term leaves an error that does not shrink."""
    errs, means, perr = [], [], []
    k, rho = 2 * np.pi, 1.0
    for n in (16, 32):
        h, c, nd = grid(n)
        dt = 0.2 * h
        Zc, Yc, Xc = np.meshgrid(c, c, c, indexing="ij")
        Z, Y, X = np.meshgrid(nd, nd, nd, indexing="ij")

        def vel(t):
            d = np.exp(-2 * nu * k * k * t)
            return np.stack([np.sin(k * Xc) * np.cos(k * Yc) * d, -np.cos(k * Xc) * np.sin(k * Yc) * d,
                             np.zeros_like(Xc)])

        p_half = rho / 4 * (np.cos(2 * k * X) + np.cos(2 * k * Y)) * np.exp(-4 * nu * k * k * (-0.5 * dt))
        us = fluid.predictor(vel(0.0), p_half, rho, nu * rho, (0.0, 0.0, 0.0), dt, h)
        u1, p1 = fluid.projection(us, p_half, rho, dt, h)
        e = np.abs(u1 - vel(dt)) / dt  # error per unit time
        errs.append(np.max(e))
        means.append(np.mean(e))
        # the new pressure approximates p at t + dt/2 (the old pressure's
        # gradient leaves u^{n+1} unchanged, so only p^{n+1/2} checks its sign)
        p_exact = rho / 4 * (np.cos(2 * k * X) + np.cos(2 * k * Y)) * np.exp(-4 * nu * k * k * (0.5 * dt))
        perr.append(np.max(np.abs((p1 - p1.mean()) - (p_exact - p_exact.mean()))))
    assert errs[1] < errs[0] / 1.8 and means[1] < means[0] / 2.0
    assert perr[1] < perr[0] / 1.8 and perr[1] < 0.05 * rho / 2
