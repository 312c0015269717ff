"""Pins of the oracle's CWENOZ nonlinear weights (Sec. 2.3) with tau > 0.

Three checks that a plausible slip in the weights would fail:

* brute force on small meshes: every polynomial of Sec. 2.3 rebuilt from the
  paper's definitions by an independent route -- the least-squares fits of
  eq. dofMatrix solved by numpy's LAPACK lstsq on cell averages of plain
  monomials, the smoothness indicators of eq. SI1 integrated directly over
  the mapped cell by a Gauss rule (not through the OI matrix), p_1 from the
  p_opt definition, tau and the weights from their printed definitions --
  and compared with the oracle's weights, indicators and CWENOZ face values
  on a front where tau is far from zero;
* smooth data: the weights tend to the linear weights lambda_s as h -> 0,
  at a rate far above the scheme's order (tau is a b-th power of indicator
  differences that vanish with h);
* pure CWENOZ's error on a smooth wave approaches the linear scheme's as h
  shrinks, the behaviour Table tab:2D_Vortex (Sec. 3.1) prints for P3..P7.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_25906_gb300 import inputs as I


# ---------------------------------------------------------------------------
# independent building blocks
# ---------------------------------------------------------------------------

def _exps(r):
    """multi-indices (a, b) with 1 <= a + b <= r"""
    return [(a, t - a) for t in range(1, r + 1) for a in range(t, -1, -1)]


def _tri_rule(n):
    """Gauss rule on the unit triangle (0,0) (1,0) (0,1) by the collapsed
    (Duffy) map of the unit square: exact for degree <= 2n - 2."""
    x, w = np.polynomial.legendre.leggauss(n)
    s, ws = 0.5 * (x + 1), 0.5 * w
    S, T = np.meshgrid(s, s, indexing="ij")
    W = np.outer(ws, ws) * S
    return np.stack([(S * (1 - T)).ravel(), (S * T).ravel()], 1), W.ravel()


def _poly_integral_sq_derivs(coef, r, verts):
    """sum over multi-indices 1 <= |g| <= r (each counted once) of the
    integral over the polygon `verts` (reference coordinates) of
    (D^g p)^2, p = sum_b coef[b] xi^b0 eta^b1 -- eq. SI1 with h_c = 1."""
    pts, wts = _tri_rule(r + 2)
    total = 0.0
    for k in range(1, len(verts) - 1):           # fan of triangles from vertex 0
        a, b, c = verts[0], verts[k], verts[k + 1]
        J = np.stack([b - a, c - a], 1)
        X = a[None, :] + pts @ J.T
        w = wts * abs(np.linalg.det(J))
        for g in _exps(r):
            d = np.zeros(len(X))
            for (e0, e1), cf in coef.items():
                if e0 < g[0] or e1 < g[1]:
                    continue
                f0 = math.perm(e0, g[0]) * math.perm(e1, g[1])
                d += cf * f0 * X[:, 0] ** (e0 - g[0]) * X[:, 1] ** (e1 - g[1])
            total += float((w * d * d).sum())
    return total


def _brute_cweno(m, osch, U, c, v, r, lam1p, eps, b):
    """Sec. 2.3 for cell c, variable v, from the definitions."""
    x0, Ji = osch.refmap(c)
    Ji = Ji[:2, :2]
    xi = lambda x, y: Ji[0, 0] * (x - x0[0]) + Ji[0, 1] * (y - x0[1])
    eta = lambda x, y: Ji[1, 0] * (x - x0[0]) + Ji[1, 1] * (y - x0[1])
    ex = _exps(r)
    # cell averages of every plain monomial psi_b = xi^b0 eta^b1 over every cell
    avg = {e: I.cell_average_2d(m, lambda x, y, e=e: xi(x, y) ** e[0] * eta(x, y) ** e[1], npts=10) for e in ex}
    vol, _ = O.Mesh(m).geometry()
    st, dr = osch.stencil(c)
    nd = osch.operator(c, "nd").astype(int)
    u = U[v]

    def fit(cells, exps):
        # eq. dofMatrix: A_mk = int_{V_m'} phi_k, b_m = |V_m'| (U_m - U_0), phi_k
        # = psi_k minus its mean over the considered cell (the reference map's
        # constant Jacobian is a common factor of every row and drops out)
        A = np.array([[vol[j] * (avg[e][j] - avg[e][c]) for e in exps] for j in cells])
        rhs = np.array([vol[j] * (u[j] - u[c]) for j in cells])
        a, *_ = np.linalg.lstsq(A, rhs, rcond=None)
        return dict(zip(exps, a))

    p_opt = fit(st, ex)
    lin = [e for e in ex if sum(e) == 1]
    p_dir = [fit(st[dr[f, :nd[f]]], lin) for f in range(len(nd))]
    st_tot = len(p_dir) + 1
    lam1 = 1.0 - 1.0 / lam1p
    lams = (1.0 - lam1) / (st_tot - 1)
    p1 = {e: (p_opt[e] - sum(lams * p.get(e, 0.0) for p in p_dir)) / lam1 for e in ex}
    # the cell in reference coordinates
    vx = m.cell_vertices(c)[:, :2]
    vr = np.stack([xi(vx[:, 0], vx[:, 1]), eta(vx[:, 0], vx[:, 1])], 1)
    SI = [_poly_integral_sq_derivs(p1, r, vr)] + [_poly_integral_sq_derivs(p, r, vr) for p in p_dir]
    tau = (sum(abs(SI[s] - SI[0]) for s in range(1, st_tot)) / (st_tot - 1)) ** b
    lam = [lam1] + [lams] * (st_tot - 1)
    wt = [lam[s] * (1.0 + tau / (eps + SI[s])) for s in range(st_tot)]
    om = np.array(wt) / sum(wt)
    pcw = {e: om[0] * p1[e] + sum(om[1 + f] * p_dir[f].get(e, 0.0) for f in range(len(p_dir))) for e in ex}
    # CWENOZ face values: U_0 + sum_k a_k phi_k(x_q)
    P = osch.face_points(c)
    Xq, Yq = xi(P[:, 0], P[:, 1]), eta(P[:, 0], P[:, 1])
    val = u[c] + sum(cf * (Xq ** e[0] * Yq ** e[1] - avg[e][c]) for e, cf in pcw.items())
    return om, np.array(SI), tau, val


def _front(m):
    return lambda x, y: 2.0 + 1.5 * np.tanh((x - 0.47 + 0.3 * (y - 0.5)) / 0.02) + 0.1 * np.sin(2 * np.pi * y)


@pytest.mark.parametrize("order", [3, 4])
def test_cweno_weights_brute_force(order):
    """Weights, indicators and CWENOZ face values equal an independent
    rebuild from the definitions of Sec. 2.3, on triangles and
    quadrilaterals near a front where tau is far from zero."""
    r = order - 1
    m = I.mixed_tri_quad_mesh(14, seed=5)
    lam1p, eps, b = 1e3, 1e-3, 4.0
    osch = O.Scheme(O.Mesh(m), order=order, lambda1p=lam1p)
    rho = I.cell_average_2d(m, _front(m), npts=10)
    U = np.stack([rho, 0.3 * rho, -0.2 * rho, rho + 3.0])
    vm = m.vertex_means()
    near = np.nonzero((np.abs(vm[:, 0] - 0.47 - 0.3 * (0.5 - vm[:, 1])) < 0.12)
                      & (np.abs(vm[:, 1] - 0.5) < 0.3))[0]
    checked, types, nontrivial = 0, set(), 0
    for c in near[:: max(1, len(near) // 10)]:
        om_b, si_b, tau, val_b = _brute_cweno(m, osch, U, c, 0, r, lam1p, eps, b)
        om_o, si_o, _ = osch.cweno_info(U, c, 0)
        assert np.abs(si_o - si_b).max() <= 1e-9 * max(1.0, np.abs(si_b).max()), (c, si_o, si_b)
        assert np.abs(om_o - om_b).max() <= 1e-10, (c, om_o, om_b)
        V = osch.reconstruct(U, c, O.CW)
        assert np.abs(V[:, 0] - val_b).max() <= 1e-10 * (1 + np.abs(val_b).max()), c
        checked += 1
        types.add(int(m.cell_type[c]))
        # a weight far from its linear value: tau matters in this cell
        lam1 = 1 - 1 / lam1p
        lam = np.r_[lam1, np.full(len(om_b) - 1, (1 - lam1) / (len(om_b) - 1))]
        if (np.abs(om_b / lam - 1)).max() > 0.5:
            nontrivial += 1
    assert checked >= 6 and types == {I.TRI, I.QUAD} and nontrivial >= 3, (checked, types, nontrivial)


def _max_weight_gap(n, order, lam1p=1e3):
    """max over sampled cells and the density variable of max_s |omega_s -
    lambda_s| / lambda_s on the smooth density wave, n x n periodic jittered
    triangle mesh"""
    m = I.structured_tri_mesh(n, periodic=True, jitter=0.2, seed=1)
    osch = O.Scheme(O.Mesh(m), order=order, lambda1p=lam1p)
    U = I.density_wave_state(m)
    rng = np.random.default_rng(n)
    cells = rng.choice(m.n_cells, size=min(m.n_cells, 48), replace=False)
    gap = 0.0
    lam1 = 1 - 1 / lam1p
    for c in cells:
        om_, _, _ = osch.cweno_info(U, int(c), 0)
        st = len(om_)
        lam = np.r_[lam1, np.full(st - 1, (1 - lam1) / (st - 1))]
        gap = max(gap, float((np.abs(om_ - lam) / lam).max()))
    return gap


@pytest.mark.parametrize("order,ns,min_rate", [(3, (12, 24, 48), 12.0), (5, (12, 24, 48), 12.0)])
def test_weights_tend_to_linear_weights_on_smooth_data(order, ns, min_rate):
    """Smooth data: omega_s -> lambda_s as h -> 0 (Sec. 2.3: on smooth data the
    optimal polynomial is restored).  The indicators agree to O(h^3) in
    reference coordinates, tau is their mean difference to the power b = 4,
    so the weights approach the linear weights much faster than the scheme's
    order: the gap falls by about 2^16 per halving of h (measured 15.9 and
    16.8 from 24 to 48 cells per side); bar: rate > 12 between refinements."""
    gaps = [_max_weight_gap(n, order) for n in ns]
    rates = [math.log2(gaps[i] / gaps[i + 1]) for i in range(len(gaps) - 1)]
    assert all(x > min_rate for x in rates), (gaps, rates)


@pytest.mark.slow
@pytest.mark.parametrize("order", [3, 5])
def test_pure_cweno_error_approaches_linear_error(order):
    """Table tab:2D_Vortex (Sec. 3.1): on smooth data CWENOZ's error falls onto
    the linear scheme's as the mesh is refined.  Density wave advected to
    t = 0.05 on n x n periodic jittered triangles: |e_cweno / e_linear - 1|
    shrinks with h and is below 1e-3 on the finest mesh."""
    T = 0.05
    gaps, errs = [], []
    for n in (8, 16, 32):
        m = I.structured_tri_mesh(n, periodic=True, jitter=0.2, seed=1)
        om = O.Mesh(m)
        vol, _ = om.geometry()
        ex = I.density_wave_state(m, t=T)
        e = {}
        for scheme in ("linear", "cweno"):
            s = O.Scheme(om, order=order, flux="rusanov", scheme=scheme)
            U = I.density_wave_state(m)
            h = (1.0 / n)
            nsteps = int(math.ceil(T / (0.4 * h ** ((order) / 3.0) / 2.0)))
            dt = T / nsteps
            for _ in range(nsteps):
                U = s.rk3_step(U, dt)
            e[scheme] = math.sqrt(((U[0] - ex[0]) ** 2 * vol).sum() / vol.sum())
        errs.append(e)
        gaps.append(abs(e["cweno"] / e["linear"] - 1.0))
    assert gaps[-1] < gaps[0] and gaps[-1] < 1e-3, (gaps, errs)
