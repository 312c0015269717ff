"""Pins of the oracle's viscous terms (Sec. 2: eqs. Terms1, Stresses,
HeatConduct, sutherlandlaw, EulerEquationsDetails and the averaged gradient
with its penalty, eq. viscous_jump).

* uniform flow: no viscous flux (free stream);
* periodic mesh: sum |V| R = 0 (the face flux is the same from both sides);
* Couette flow u = y: interior cells get exactly (0, 0, 0, mu) -- the divergence
  of the constant shear stress vanishes, and the work of the stress,
  d(u tau_xy)/dy = mu (du/dy)^2, heats the gas;
* the penalty term in closed form: cell-mean (first-order) states of u = x on
  uniform squares give the energy residual 4/3 (1 + alpha) mu;
* a manufactured smooth flow: the viscous residual converges to the cell
  averages of the divergence of the viscous flux, derived symbolically here
  (sympy) from the paper's stress tensor, heat flux and Sutherland's law.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_25906_gb300 import inputs as I

MU0 = 0.01


def _visc(m, U, forced=None, **kw):
    """the viscous part of the residual: R(mu0) - R(0), same classes"""
    om = O.Mesh(m)
    Rv = O.Scheme(om, mu0=MU0, **kw).residual(U, forced=forced)[0]
    R0 = O.Scheme(om, **kw).residual(U, forced=forced)[0]
    return Rv, Rv - R0


def test_uniform_flow_has_no_viscous_flux():
    m = I.mixed_tri_quad_mesh(12, seed=5, periodic=True)
    n = m.n_cells
    U = np.stack([np.full(n, 1.3), np.full(n, 0.4), np.full(n, -0.2), np.full(n, 3.1)])
    Rv, dv = _visc(m, U, order=3, flux="hllc")
    assert np.abs(Rv).max() < 1e-12 and np.abs(dv).max() < 1e-12


@pytest.mark.parametrize("order", [2, 3, 4])
def test_viscous_residual_is_conservative(order):
    m = I.mixed_tri_quad_mesh(12, seed=5, periodic=True)
    vm = m.vertex_means()
    rho = 1 + 0.2 * np.sin(2 * np.pi * vm[:, 0]) * np.cos(2 * np.pi * vm[:, 1])
    u = 0.3 * np.sin(2 * np.pi * vm[:, 1])
    v = 0.2 * np.cos(2 * np.pi * vm[:, 0])
    p = 1 + 0.1 * np.cos(2 * np.pi * (vm[:, 0] - vm[:, 1]))
    U = I.conserved_2d(rho, u, v, p)
    _, dv = _visc(m, U, order=order, flux="hllc")
    vol, _ = O.Mesh(m).geometry()
    assert np.abs(dv).max() > 1e-4
    tot = (dv * vol).sum(axis=1)
    assert np.abs(tot).max() < 1e-13 * np.abs(dv).max(), tot


def test_couette_flow_heats_interior_cells_at_mu():
    """u = y, v = 0, rho = 1, p = 1 (T = 1, mu = mu0), on quadrilaterals
    periodic in x; the degree-2 reconstruction is exact for these fields, so
    away from the open walls every cell's residual is (0, 0, 0, mu0)."""
    m = I.structured_quad_mesh(10, 16, periodic=(True, False), jitter=0.1, seed=3)
    rho = np.ones(m.n_cells)
    my = I.cell_average_2d(m, lambda x, y: y)
    E = I.cell_average_2d(m, lambda x, y: 2.5 + 0.5 * y * y)
    U = np.stack([rho, my, 0 * rho, E])
    Rv, _ = _visc(m, U, order=3, scheme="linear", flux="hllc")
    yc = m.vertex_means()[:, 1]
    inner = (yc > 4 / 16) & (yc < 12 / 16)
    assert inner.sum() >= 60
    want = np.array([0, 0, 0, MU0])[:, None]
    assert np.abs(Rv[:, inner] - want).max() < 1e-11, np.abs(Rv[:, inner] - want).max()


@pytest.mark.parametrize("alpha", [4.0 / 3.0, 0.0, 2.0])
def test_penalty_term_closed_form(alpha):
    """Uniform squares (h = 1/16), u = x, rho = 1, cell means of E chosen so
    that every cell-mean pressure is 1; all cells forced first-order, so the
    face states are the cell means while the conserved gradients come from
    the exact degree-2 polynomials (grad rho = 0, grad m_x = e_x).  Across an
    x-face the averaged velocity gradient is e_x, the penalty adds
    alpha (u_j - u_i) / h = alpha: du/dx = 1 + alpha, tau_xx = 4/3 mu (1 +
    alpha), and the work of the stress through the two x-faces,
    (u_i + h/2) tau_xx h - (u_i - h/2) tau_xx h, over the area h^2 gives the
    energy residual 4/3 (1 + alpha) mu0; the other components vanish.  The
    Prandtl number is made huge: at a cell-mean state the temperature
    gradient of the polynomial is not zero, and conduction is not what this
    checks."""
    n = 16
    m = I.structured_quad_mesh(n, n, periodic=(False, True))
    xc = m.vertex_means()[:, 0]
    U = np.stack([np.ones(n * n), xc, 0 * xc, 2.5 + 0.5 * xc * xc])
    forced = np.full(n * n, O.FIRST, np.uint8)
    _, dv = _visc(m, U, forced=forced, order=3, flux="hllc", visc_alpha=alpha, prandtl=1e30)
    inner = (xc > 4 / n) & (xc < 12 / n)
    want = np.array([0, 0, 0, 4.0 / 3.0 * (1 + alpha) * MU0])[:, None]
    assert np.abs(dv[:, inner] - want).max() < 1e-12, np.abs(dv[:, inner] - want).max()


def test_viscous_time_step_keeps_the_quadrant_problem_physical():
    """The CFL step with the diffusion limit (4 max(4/3, gamma/Pr) mu/rho
    sum|S|^2/|V| added to the convective bound) is smaller than the inviscid
    one, and viscous steps across the jumps of the 2D Riemann problem keep
    density and pressure positive."""
    m = I.mixed_tri_quad_mesh(20, seed=2)
    U0 = I.quadrant_state(m)
    om = O.Mesh(m)
    sv = O.Scheme(om, order=3, flux="hllc", mu0=0.02)
    s0 = O.Scheme(om, order=3, flux="hllc")
    assert sv.dt(U0, 0.5) < s0.dt(U0, 0.5)
    U = U0.copy()
    for _ in range(3):
        U = sv.rk3_step(U, sv.dt(U, 0.5))
    p = 0.4 * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])
    assert np.isfinite(U).all() and (U[0] > 0).all() and (p > 0).all()


@pytest.mark.parametrize("prandtl", [0.72, 2.0])
def test_viscous_time_step_closed_form(prandtl):
    """R29 on a uniform hx x hy quadrilateral mesh, where the face sums are
    written by hand: sum_f (|u.n_f| + a)|S_f| = 2(|u| + a) hy + 2(|v| + a) hx
    and sum_f |S_f|^2 / |V| = 2 (hx^2 + hy^2) / (hx hy); the diffusion limit
    adds 4 nu times the latter, nu = max(4/3, gamma/Pr) mu / rho with
    Sutherland's mu(T = p / rho).  Pr = 2 makes 4/3 the larger factor."""
    g, T0, S, mu0 = 1.4, 1.0, 110.4 / 288.15, 0.05
    nx, ny = 6, 4
    hx, hy = 1.0 / nx, 1.0 / ny
    m = I.structured_quad_mesh(nx, ny)
    rng = np.random.default_rng(11)
    n = m.n_cells
    rho, p = 0.5 + rng.random(n), 0.5 + rng.random(n)
    u, v = rng.uniform(-1.0, 1.0, (2, n))
    U = np.stack([rho, rho * u, rho * v, p / (g - 1) + 0.5 * rho * (u * u + v * v)])
    a = np.sqrt(g * p / rho)
    T = p / rho
    mu = mu0 * (T / T0) ** 1.5 * (T0 + S) / (T + S)
    nu = max(4.0 / 3.0, g / prandtl) * mu / rho
    lam = 2 * (np.abs(u) + a) * hy + 2 * (np.abs(v) + a) * hx + 4 * nu * 2 * (hx * hx + hy * hy) / (hx * hy)
    want = 0.5 * np.min(hx * hy / lam)
    got = O.Scheme(O.Mesh(m), order=2, mu0=mu0, t0=T0, suth_s=S, prandtl=prandtl).dt(U, 0.5)
    assert abs(got - want) <= 1e-14 * want


def _manufactured():
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    g, mu0, T0, S, Pr = sp.Rational(7, 5), MU0, 1.0, 110.4 / 288.15, 0.72
    rho = 1 + sp.Rational(1, 10) * sp.sin(2 * sp.pi * x) * sp.cos(2 * sp.pi * y)
    vel = [sp.Rational(1, 5) * sp.sin(2 * sp.pi * y), sp.Rational(1, 10) * sp.cos(2 * sp.pi * x)]
    p = 1 + sp.Rational(1, 10) * sp.cos(2 * sp.pi * (x - y))
    T = p / rho
    mu = mu0 * (T / T0) ** sp.Rational(3, 2) * (T0 + S) / (T + S)
    X = [x, y]
    div = sum(sp.diff(vel[k], X[k]) for k in range(2))
    tau = [[mu * (sp.diff(vel[i], X[j]) + sp.diff(vel[j], X[i]) - (sp.Rational(2, 3) * div if i == j else 0))
            for j in range(2)] for i in range(2)]
    theta = [sum(vel[i] * tau[i][j] for i in range(2)) + mu / Pr * g / (g - 1) * sp.diff(T, X[j]) for j in range(2)]
    src = [sum(sp.diff(tau[i][j], X[j]) for j in range(2)) for i in range(2)]
    src.append(sum(sp.diff(theta[j], X[j]) for j in range(2)))
    f = lambda e: sp.lambdify((x, y), e, "numpy")
    fr, fu, fv, fp = f(rho), f(vel[0]), f(vel[1]), f(p)
    state = [lambda a, b: fr(a, b) + 0 * a, lambda a, b: fr(a, b) * fu(a, b) + 0 * a,
             lambda a, b: fr(a, b) * fv(a, b) + 0 * a,
             lambda a, b: fp(a, b) / 0.4 + 0.5 * fr(a, b) * (fu(a, b) ** 2 + fv(a, b) ** 2)]
    return state, [f(e) for e in src]


@pytest.mark.parametrize("order", [3, 4])
def test_viscous_residual_converges_to_the_analytic_divergence(order):
    """Smooth periodic flow with Sutherland viscosity and heat conduction:
    the viscous residual tends to the cell averages of div F_v (momentum and
    energy), at about r - 1 in the maximum norm on jittered triangles (the
    face gradients are exact to O(h^r), divided by the cell size); measured
    0.78 (order 3) and 1.85 (order 4) from 16 to 32 cells per side."""
    state, src = _manufactured()
    errs = []
    for n in (8, 16, 32):
        m = I.structured_tri_mesh(n, periodic=True, jitter=0.2, seed=1)
        U = np.stack([I.cell_average_2d(m, f, npts=10) for f in state])
        _, dv = _visc(m, U, order=order, scheme="linear", flux="rusanov")
        ex = [I.cell_average_2d(m, lambda a, b, f=f: f(a, b) + 0 * a, npts=10) for f in src]
        errs.append(max(np.abs(dv[1 + k] - ex[k]).max() / np.abs(ex[k]).max() for k in range(3)))
    rate = math.log2(errs[1] / errs[2])
    assert errs[2] < errs[1] < errs[0] and rate > (order - 2) - 0.3, (errs, rate)
