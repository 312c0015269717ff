"""Pins of the oracle's paper variants (CPU): the SSP-RK(5,4) time step of
Spiteri and Ruuth (the paper's integrator, Sec. 2) and Venkatakrishnan's
limiter for the MUSCL reconstruction (the paper's parameter K = 5).

  * SSP-RK(5,4): its Shu-Osher table satisfies the eight order conditions of
    a fourth-order Runge-Kutta method (Butcher form), every coefficient is
    non-negative and every stage is a convex combination; on u' = lambda u
    the error of one step against exp(z) falls as z^5; a step of the Euler
    residual is that same method applied to the residual.
  * Venkatakrishnan: with eps = 0 its limiter value never exceeds
    Barth-Jespersen's at any face point (phi(y) <= min(1, y)), so the face
    values stay inside the neighbour bounds and the cell's limiter is at most
    Barth-Jespersen's; with a large K it does not limit (a plane is
    reproduced exactly); at a jump with the paper's K = 5 it limits (one
    theta in (0, 1) scales every point's increment).
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_25906_gb300 import inputs as I


def _butcher(al, be):
    A = np.zeros((6, 5))
    for i in range(1, 6):
        for j in range(i):
            A[i] += al[i, j] * A[j]
            A[i, j] += be[i, j]
    return A[:5, :5], A[5]


def test_rk54_order_conditions_and_ssp_form():
    al, be = O.rk54_table()
    assert np.allclose(al[1:].sum(axis=1), 1.0, atol=1e-14)
    assert (al >= 0).all() and (be >= 0).all()
    A, b = _butcher(al, be)
    c = A.sum(axis=1)
    conds = [b.sum() - 1, b @ c - 1 / 2, b @ c ** 2 - 1 / 3, b @ A @ c - 1 / 6, b @ c ** 3 - 1 / 4,
             b @ (c * (A @ c)) - 1 / 8, b @ A @ c ** 2 - 1 / 12, b @ A @ A @ c - 1 / 24]
    assert np.abs(conds).max() < 1e-14, conds
    # not fifth order: some fifth-order condition fails
    assert abs(b @ c ** 4 - 1 / 5) > 1e-6 or abs(b @ A @ A @ A @ c - 1 / 120) > 1e-6


def test_rk54_linear_error_is_fifth_power():
    lam = -1.0
    errs = []
    for dt in (0.2, 0.1, 0.05):
        u = O.rk54_generic(np.array([1.0]), dt, lambda x: lam * x)
        errs.append(abs(u[0] - np.exp(lam * dt)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 28 < r1 < 36 and 29 < r2 < 35, (errs, r1, r2)


def test_rk54_step_is_the_method_on_the_residual():
    m = I.mixed_tri_quad_mesh(10, seed=2, periodic=True)
    s = O.Scheme(O.Mesh(m), order=3, flux="hllc")
    U = I.quadrant_state(m)
    dt = 0.5 * s.dt(U, 0.5)
    got = s.rk54_step(U, dt)
    shape = U.shape
    ref = O.rk54_generic(U.ravel(), dt, lambda x: s.residual(x.reshape(shape))[0].ravel()).reshape(shape)
    assert np.array_equal(got, ref)


def _random_state(m, seed):
    rng = np.random.default_rng(seed)
    n = m.n_cells
    return np.stack([1 + rng.random(n), rng.standard_normal(n), rng.standard_normal(n), 5 + rng.random(n)])


def test_venkatakrishnan_without_threshold_is_inside_barth_jespersen():
    m = I.mixed_tri_quad_mesh(14, seed=6)
    sv = O.Scheme(O.Mesh(m), order=3, limiter="venkatakrishnan", venkat_k=0.0)
    sb = O.Scheme(O.Mesh(m), order=3)
    nbr, _ = sv.mesh.connectivity()
    U = _random_state(m, 1)
    strict = 0
    for c in range(0, m.n_cells, 7):
        Vv = sv.reconstruct(U, c, O.MU)
        Vb = sb.reconstruct(U, c, O.MU)
        nb = [j for j in nbr[c] if j >= 0] + [c]
        lo, hi = U[:, nb].min(axis=1), U[:, nb].max(axis=1)
        assert (Vv >= lo - 1e-14).all() and (Vv <= hi + 1e-14).all()
        # same gradient, smaller or equal limiter: |V - u0| shrinks point by point
        dv, db = np.abs(Vv - U[:, c]), np.abs(Vb - U[:, c])
        assert (dv <= db + 1e-14).all()
        strict += int((dv < db - 1e-12).any())
    assert strict > 0


def test_venkatakrishnan_large_threshold_reproduces_a_plane():
    m = I.mixed_tri_quad_mesh(14, seed=6)
    s = O.Scheme(O.Mesh(m), order=3, limiter="venkatakrishnan", venkat_k=1e6)
    rho = I.cell_average_2d(m, lambda x, y: 2.0 + 0.3 * (x - 2 * y))
    U = np.stack([rho, rho, rho, rho + 3])
    for c in (40, 150, 260):
        V = s.reconstruct(U, c, O.MU)
        P = s.face_points(c)
        ex = 2.0 + 0.3 * (P[:, 0] - 2 * P[:, 1])
        assert np.abs(V[:, 0] - ex).max() < 1e-12


def test_venkatakrishnan_limits_at_a_jump():
    m = I.structured_quad_mesh(16, 16, jitter=0.1, seed=3)
    s = O.Scheme(O.Mesh(m), order=3, limiter="venkatakrishnan", venkat_k=5.0)
    vm = m.vertex_means()
    rho = np.where(vm[:, 0] < 0.5, 1.0, 0.2)
    U = np.stack([rho, 0 * rho, 0 * rho, 2.5 + 0 * rho])
    free = O.Scheme(O.Mesh(m), order=3, limiter="venkatakrishnan", venkat_k=1e6)
    for c in (7 * 16 + 7, 7 * 16 + 8):   # the two cells on either side of the jump
        V = s.reconstruct(U, c, O.MU)
        Vf = free.reconstruct(U, c, O.MU)
        d, df = V[:, 0] - rho[c], Vf[:, 0] - rho[c]
        assert np.abs(d).max() > 0                          # not first order
        assert np.abs(d).max() < 0.9 * np.abs(df).max()     # limited: 0 < theta < 1
        assert np.allclose(d[np.abs(df) > 0] / df[np.abs(df) > 0], (d / np.where(df == 0, 1, df))[np.abs(df) > 0][0])


def _venkat_theta(s, sfree, U, c, v):
    """the limiter value of variable v at cell c, read off the reconstruction:
    (V - u0) = theta (V_free - u0) at every face point, V_free the unlimited
    (huge threshold) reconstruction of the same gradient; also the unlimited
    increments"""
    u0 = U[v, c]
    d = s.reconstruct(U, c, O.MU)[:, v] - u0
    df = sfree.reconstruct(U, c, O.MU)[:, v] - u0
    k = int(np.argmax(np.abs(df)))
    th = d[k] / df[k]
    assert np.allclose(d, th * df, rtol=0, atol=1e-13 * (1.0 + abs(u0)))
    return float(th), df


def test_venkatakrishnan_limiter_values():
    """R21, by two properties of the published limiter and its value.
    (a) With K = 0 (eps = 0), phi(y) = (y^2 + 2y) / (y^2 + y + 2) of
    y = Delta_1 / Delta_2 reaches 1 exactly at y = 2: a cell is limited
    (theta < 1) exactly when some face point's increment exceeds half the
    distance to the bound on its side (bounds over the cell and its face
    neighbours); theta then equals the published value.  (b) eps^2 = (K dx)^3:
    phi depends on Delta / eps only, so scaling every difference of the data
    by sigma is the same as scaling K by sigma^(-2/3)."""
    m = I.mixed_tri_quad_mesh(14, seed=6)
    om = O.Mesh(m)
    nbr, _ = om.connectivity()
    vol, _ = om.geometry()
    s0 = O.Scheme(om, order=3, limiter="venkatakrishnan", venkat_k=0.0)
    sf = O.Scheme(om, order=3, limiter="venkatakrishnan", venkat_k=1e6)
    U = _random_state(m, 4)
    v = 1
    limited = free = 0
    for c in range(0, m.n_cells, 3):
        th, df = _venkat_theta(s0, sf, U, c, v)
        nb = [j for j in nbr[c] if j >= 0] + [c]
        hi, lo = U[v, nb].max() - U[v, c], U[v, nb].min() - U[v, c]
        d1 = np.where(df > 0, hi, lo)
        y = d1[df != 0] / df[df != 0]
        phi = np.minimum(1.0, (y * y + 2 * y) / (y * y + y + 2))
        assert (th < 1.0 - 1e-12) == bool((y < 2.0 - 1e-9).any()), (c, th, y.min())
        assert abs(th - phi.min()) < 1e-12
        limited += th < 1.0
        free += th == 1.0
    assert limited >= 20 and free >= 5
    sigma, K = 8.0, 0.3
    Us = U.copy()
    Us[v] = sigma * U[v]
    sk = O.Scheme(om, order=3, limiter="venkatakrishnan", venkat_k=K)
    sk2 = O.Scheme(om, order=3, limiter="venkatakrishnan", venkat_k=K * sigma ** (-2.0 / 3.0))
    moved = 0
    for c in range(0, m.n_cells, 3):
        a, _ = _venkat_theta(sk, sf, Us, c, v)
        b, _ = _venkat_theta(sk2, sf, U, c, v)
        assert abs(a - b) < 1e-10, (c, a, b)
        moved += abs(a - _venkat_theta(sk, sf, U, c, v)[0]) > 1e-6
    assert moved >= 10


# ---------------------------------------------------------------------------
# CWENOZ in characteristic variables
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("u,n", [([1.2, 0.3, -0.4, 2.9], [0.6, 0.8]),
                                 ([0.9, 0.2, -0.1, 0.35, 2.7], [0.36, 0.48, 0.8]),
                                 ([1.1, 0.0, 0.0, 0.5, 3.1], [0.0, 0.0, 1.0])])
def test_euler_eigenvectors_diagonalise_the_flux_jacobian(u, n):
    """L R = I, and L (dF.n/dU) R = diag(u.n - c, u.n, ..., u.n + c) with
    the Jacobian taken by central differences of the physical flux F(U, U)."""
    u, n = np.array(u), np.array(n)
    nv, d = u.size, u.size - 2
    L, R = O.euler_eigen(u, n)
    assert np.abs(L @ R - np.eye(nv)).max() < 1e-14
    A = np.zeros((nv, nv))
    h = 1e-6
    n3 = np.zeros(3)
    n3[:d] = n
    for j in range(nv):
        e = np.zeros(nv)
        e[j] = h
        A[:, j] = (O.flux("rusanov", u + e, u + e, n3) - O.flux("rusanov", u - e, u - e, n3)) / (2 * h)
    D = L @ A @ R
    vel = u[1:1 + d] / u[0]
    p = 0.4 * (u[-1] - 0.5 * u[0] * vel @ vel)
    c, qn = np.sqrt(1.4 * p / u[0]), vel @ n
    ex = np.array([qn - c] + [qn] * (nv - 2) + [qn + c])
    assert np.abs(D - np.diag(ex)).max() < 1e-8
    assert np.abs(np.diag(D) - ex).max() < 1e-8


@pytest.mark.parametrize("maker", [lambda: I.mixed_tri_quad_mesh(12, seed=5),
                                   lambda: I.structured_hex_mesh(6, 1.0, periodic=False, jitter=0.1, seed=3)])
def test_characteristic_cweno_equals_conserved_on_linear_data(maker):
    """On linear data every indicator is equal, the weights are the linear
    weights, and the characteristic projection (linear) commutes with the
    reconstruction: both forms reproduce the plane."""
    m = maker()
    om = O.Mesh(m)
    sc = O.Scheme(om, order=3)
    sw = O.Scheme(om, order=3, cweno_vars="characteristic")
    vm = m.vertex_means()
    vol, cen = om.geometry()
    g = np.array([0.3, -0.2, 0.1])[:m.dim]
    rho = 1.5 + cen[:, :m.dim] @ g
    mom = 0.2 + 0.1 * (cen[:, :m.dim] @ g)
    if m.dim == 2:
        U = np.stack([rho, mom, -mom, 3.0 + mom])
    else:
        U = np.stack([rho, mom, -mom, 0.5 * mom, 3.0 + mom])
    for c in (7, 40, 101):
        Vc = sc.reconstruct(U, c, O.CW)
        Vw = sw.reconstruct(U, c, O.CW)
        assert np.abs(Vc - Vw).max() < 1e-12
        P = sc.face_points(c)
        ex = 1.5 + P[:, :m.dim] @ g
        assert np.abs(Vw[:, 0] - ex).max() < 1e-12


def test_characteristic_cweno_conserves_and_preserves_free_stream():
    m = I.mixed_tri_quad_mesh(10, seed=7, periodic=True)
    om = O.Mesh(m)
    vol, _ = om.geometry()
    s = O.Scheme(om, order=3, flux="hllc", cweno_vars="characteristic", scheme="cweno")
    n = m.n_cells
    Uu = I.conserved_2d(np.full(n, 1.2), np.full(n, 0.4), np.full(n, -0.3), np.full(n, 0.8))
    R, *_ = s.residual(Uu)
    assert np.abs(R).max() < 1e-12
    U = I.quadrant_state(m)
    R, raw, tag, fin = s.residual(U)
    assert (fin == 1).sum() > n // 3
    tot = (R * vol).sum(axis=1)
    assert np.abs(tot).max() < 1e-12 * (np.abs(R) * vol).sum()
    # and it differs from conserved-variable CWENOZ at the discontinuities
    Rc, *_ = O.Scheme(om, order=3, flux="hllc", scheme="cweno").residual(U)
    assert np.abs(R - Rc).max() > 1e-6 * np.abs(Rc).max()


@pytest.mark.parametrize("seed", [3, 5])
def test_characteristic_cweno_respects_the_mirror_symmetry(seed):
    """R24 projects each face's points with the eigenvectors of that face's
    normal.  On unit squares with data symmetric under the reflection x <-> y
    (density and energy symmetric, the two momenta swapped), a cell on the
    diagonal has mirror-image stencils and faces, so the value at each face
    point must be the mirror of the value at the reflected point (momenta
    swapped); projecting every face with one normal breaks that.  Random
    symmetric data: every cell is non-smooth.  Order 3: its stencil is two
    whole face layers, and so are its directional stencils (higher orders
    break distance ties by cell id, which the reflection does not keep)."""
    n = 8
    m = I.structured_quad_mesh(n, n, periodic=(True, True))
    rng = np.random.default_rng(seed)
    r = 1.0 + rng.random((n, n))
    E = 6.0 + rng.random((n, n))
    pu = rng.standard_normal((n, n))
    U = np.stack([(r + r.T).ravel(), pu.ravel(), pu.T.ravel(), (E + E.T).ravel()])   # cell (i, j) at [j, i]
    s = O.Scheme(O.Mesh(m), order=3, cweno_vars="characteristic")
    for c in (2 * n + 2, 5 * n + 5):
        V = s.reconstruct(U, c, O.CW)
        P = s.face_points(c)
        for q in range(P.shape[0]):
            k = int(np.argmin(np.hypot(P[:, 0] - P[q, 1], P[:, 1] - P[q, 0])))
            assert np.hypot(P[k, 0] - P[q, 1], P[k, 1] - P[q, 0]) < 1e-12
            assert np.allclose(V[q], V[k][[0, 2, 1, 3]], rtol=0, atol=1e-12), (c, q)
        assert np.abs(V - U[:, c]).max() > 1e-3        # a real reconstruction, not the mean


def test_characteristic_cweno_on_a_contact_is_density_cweno():
    """Across a contact (u, v and p constant, rho jumps) every difference of
    conserved states is a multiple of the entropy eigenvector (1, u, v, q^2/2),
    which does not depend on rho or on the face normal.  Its characteristic
    projection is then rho's own data in the entropy field and zero in the
    others, so the characteristic reconstruction gives rho exactly as the
    component-wise one does, and rho u, rho v, E follow rho along that
    eigenvector at every face point."""
    m = I.mixed_tri_quad_mesh(16, seed=9)
    om = O.Mesh(m)
    vol, cen = om.geometry()
    rho = 1.0 + 0.1 * np.sin(3 * cen[:, 1]) + np.where(cen[:, 0] < 0.47, 0.8, 0.0)
    u, v, p = 0.3, -0.2, 1.0
    U = I.conserved_2d(rho, np.full_like(rho, u), np.full_like(rho, v), np.full_like(rho, p))
    sc = O.Scheme(om, order=3)
    sw = O.Scheme(om, order=3, cweno_vars="characteristic")
    near = np.argsort(np.abs(cen[:, 0] - 0.47))[:6]
    moved = 0.0
    for c in near:
        Vc = sc.reconstruct(U, c, O.CW)
        Vw = sw.reconstruct(U, c, O.CW)
        assert np.abs(Vw[:, 0] - Vc[:, 0]).max() < 1e-12
        assert np.abs(Vw[:, 1] - u * Vw[:, 0]).max() < 1e-12
        assert np.abs(Vw[:, 2] - v * Vw[:, 0]).max() < 1e-12
        assert np.abs(Vw[:, 3] - (p / 0.4 + 0.5 * (u * u + v * v) * Vw[:, 0])).max() < 1e-12
        moved = max(moved, np.abs(Vw[:, 0] - sc.reconstruct(U, c, O.LIN)[:, 0]).max())
    assert moved > 1e-3            # the nonlinear weights are really at work here
