"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

No test here compares the oracle with itself or retypes one of its formulas:
each check is a closed form, an invariant, a special case reducing to a
library routine, a statement the paper makes, or brute force on a tiny mesh.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2510_25906_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# quadrature and geometry
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_gauss_legendre_exactness(n):
    x, w = O.gauss_legendre(n)
    for k in range(2 * n):
        assert abs((w * x ** k).sum() - 1.0 / (k + 1)) < 1e-14
    # degree 2n is not integrated exactly
    assert abs((w * x ** (2 * n)).sum() - 1.0 / (2 * n + 1)) > 1e-12


def test_cell_monomial_integrals_closed_form():
    # unit right triangle: int x^a y^b = a! b! / (a+b+2)!
    tri = I.Mesh(2, np.array([[0., 0.], [1., 0.], [0., 1.], [1., 1.]]), np.array([1, 1], np.uint8),
                 np.array([0, 3, 6]), np.array([0, 1, 2, 1, 3, 2], np.int32), np.zeros(2))
    om = O.Mesh(tri)
    for a in range(5):
        for b in range(5 - a):
            ex = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(om.monomial_integral(0, a, b) - ex) < 1e-15
    # unit square split as quads / unit cube: int x^a y^b z^c = 1/((a+1)(b+1)(c+1))
    q = I.structured_quad_mesh(1, 1)
    oq = O.Mesh(q)
    for a in range(5):
        for b in range(5):
            assert abs(oq.monomial_integral(0, a, b) - 1.0 / ((a + 1) * (b + 1))) < 1e-15
    h = I.structured_hex_mesh(1, 1.0, periodic=False)
    oh = O.Mesh(h)
    for a, b, c in [(0, 0, 0), (1, 2, 3), (4, 0, 2), (3, 3, 3)]:
        assert abs(oh.monomial_integral(0, a, b, c) - 1.0 / ((a + 1) * (b + 1) * (c + 1))) < 1e-14


def test_bilinear_quad_integral_matches_two_triangles():
    m = I.structured_quad_mesh(3, 3, jitter=0.3, seed=4)
    om = O.Mesh(m)
    c = 4  # the interior, jittered quad
    v = m.cell_vertices(c)
    tri = I.Mesh(2, v, np.array([1, 1], np.uint8), np.array([0, 3, 6]), np.array([0, 1, 2, 0, 2, 3], np.int32), np.zeros(2))
    ot = O.Mesh(tri)
    for a, b in [(0, 0), (1, 0), (0, 1), (2, 3), (4, 1)]:
        assert abs(om.monomial_integral(c, a, b) - ot.monomial_integral(0, a, b) - ot.monomial_integral(1, a, b)) < 1e-14


@pytest.mark.parametrize("maker,measure", [
    (lambda: I.structured_tri_mesh(12, periodic=True, jitter=0.2, seed=1), 1.0),
    (lambda: I.mixed_tri_quad_mesh(14, seed=2), 1.0),
    (lambda: I.mixed_tri_quad_mesh(10, seed=7, periodic=True), 1.0),
    (lambda: I.structured_hex_mesh(6, 2 * math.pi, periodic=True), (2 * math.pi) ** 3),
    (lambda: I.structured_hex_mesh(5, 1.0, periodic=False, jitter=0.2, seed=9), 1.0),
])
def test_geometry_invariants(maker, measure):
    m = maker()
    om = O.Mesh(m)
    vol, cen = om.geometry()
    assert (vol > 0).all()
    assert abs(vol.sum() - measure) < 1e-13 * measure
    nbr, nbrf = om.connectivity()
    fo, fn, nrm, area, sh = om.faces()
    # every interior face has exactly two cells, and the pairing is symmetric
    for c in range(m.n_cells):
        nf = {1: 3, 2: 4, 4: 6}[int(m.cell_type[c])]
        for f in range(nf):
            j = nbr[c, f]
            if j >= 0:
                assert nbr[j, nbrf[c, f]] == c and nbrf[j, nbrf[c, f]] == f
    # closed cells: sum of outward area vectors vanishes
    closure = np.zeros((m.n_cells, 3))
    np.add.at(closure, fo, nrm * area[:, None])
    inner = fn >= 0
    np.add.at(closure, fn[inner], -(nrm * area[:, None])[inner])
    scale = area.max()
    assert np.abs(closure).max() < 1e-13 * scale
    # periodic shifts are whole periods
    per = m.period
    for d in range(m.dim):
        if per[d] > 0:
            k = sh[:, d] / per[d]
            assert np.allclose(k, np.round(k), atol=0)
    if all(p > 0 for p in per[:m.dim]):
        assert (fn >= 0).all()


# ---------------------------------------------------------------------------
# stencils
# ---------------------------------------------------------------------------

def _face_adjacency(m, om):
    nbr, _ = om.connectivity()
    return nbr


def _brute_stencil(m, om, c, M):
    """Independent restatement of the stencil rule: face-adjacency layers,
    whole layers while they fit, then the first layer that does not fit by
    ascending (quantised squared distance / h^2, id)."""
    nbr = _face_adjacency(m, om)
    vol, _ = om.geometry()
    vm = m.vertex_means()
    per = m.period
    h2 = vol[c] if m.dim == 2 else np.cbrt(vol[c]) ** 2
    seen = {c}
    layer = [c]
    taken = []
    for L in range(1, 17):
        nxt = []
        for a in layer:
            for j in nbr[a]:
                if j >= 0 and j not in seen:
                    seen.add(j)
                    nxt.append(j)
        if not nxt:
            break

        def key(j):
            dx = vm[j] - vm[c]
            for d in range(m.dim):
                if per[d] > 0:
                    dx[d] -= per[d] * np.round(dx[d] / per[d])
            return (int(np.rint(np.dot(dx, dx) / h2 * 2 ** 20)), j)

        nxt.sort(key=key)
        room = M - len(taken)
        taken += [(L,) + key(j) for j in nxt[:room]]
        layer = nxt
        if len(taken) == M:
            break
    taken.sort()
    return [t[2] for t in taken]


@pytest.mark.parametrize("maker,order", [
    (lambda: I.structured_tri_mesh(10, periodic=True, jitter=0.2, seed=3), 3),
    (lambda: I.mixed_tri_quad_mesh(10, seed=2), 5),
    (lambda: I.structured_hex_mesh(6, 1.0, periodic=True), 4),
    (lambda: I.structured_tet_mesh(4, periodic=True, jitter=0.1, seed=6), 3),
    (lambda: I.mixed_element_mesh(4, seed=7), 3),
])
def test_stencil_rule_brute_force(maker, order):
    m = maker()
    om = O.Mesh(m)
    s = O.Scheme(om, order=order)
    nbr, _ = om.connectivity()
    for c in range(0, m.n_cells, max(1, m.n_cells // 25)):
        st, _ = s.stencil(c)
        assert len(set(st.tolist())) == s.M and c not in st
        for j in nbr[c]:
            if j >= 0:
                assert j in st  # every face neighbour belongs to the stencil
        assert st.tolist() == _brute_stencil(m, om, c, s.M)


@pytest.mark.parametrize("maker,order", [
    (lambda: I.structured_tri_mesh(10, periodic=True, jitter=0.2, seed=3), 3),
    (lambda: I.mixed_tri_quad_mesh(10, seed=2), 5),
    (lambda: I.structured_quad_mesh(9, 8), 3),
    (lambda: I.structured_hex_mesh(6, 1.0, periodic=True, jitter=0.1, seed=5), 3),
    (lambda: I.structured_tet_mesh(4, periodic=True, jitter=0.1, seed=6), 3),
    (lambda: I.mixed_element_mesh(4, seed=7), 3),
])
def test_directional_stencils_brute_force(maker, order):
    """The directional stencils (reading R7) rebuilt from the reading's own
    words: for each face, the central-stencil cells (in stencil order) whose
    vertex mean, periodic shift included, lies beyond the cell's vertex mean
    along the face's outward unit normal by at least h / 2^21 (the signed
    distance rounded to h / 2^20 is positive; h = |V|^(1/d)), at most Md of
    them; with fewer than d + 1 the first Md central cells.  Compared per cell
    as a multiset over the faces, so independent of the local face order."""
    m = maker()
    om = O.Mesh(m)
    s = O.Scheme(om, order=order)
    d = m.dim
    vm = np.zeros((m.n_cells, 3))
    vm[:, :d] = m.vertex_means()[:, :d]
    vol, _ = om.geometry()
    fo, fn, nrm, _, _ = om.faces()
    normals = [[] for _ in range(m.n_cells)]
    for g in range(len(fo)):
        normals[fo[g]].append(nrm[g])
        if fn[g] >= 0:
            normals[fn[g]].append(-nrm[g])
    checked = 0
    for c in range(0, m.n_cells, max(1, m.n_cells // 40)):
        st, dirs = s.stencil(c)
        nd = s.operator(c, "nd").astype(int)
        shift = s.operator(c, "shift")
        h = vol[c] ** (1.0 / d)
        pos = vm[st] + shift
        got = sorted(tuple(sorted(dirs[f][:nd[f]].tolist())) for f in range(len(nd)))
        assert len(normals[c]) == len(nd)
        want, ambiguous = [], False
        for n in normals[c]:
            x = (pos - vm[c]) @ n / h * 2.0 ** 20
            ambiguous |= bool(np.any(np.abs(x - 0.5) < 1e-3))
            cand = [a for a in range(s.M) if x[a] >= 0.5][:s.Md]
            if len(cand) < d + 1:
                cand = list(range(s.Md))
            want.append(tuple(sorted(cand)))
        if ambiguous:
            continue
        assert got == sorted(want), (c, got, sorted(want))
        checked += 1
    assert checked >= 20


def _hand_mesh(spec):
    if spec["mesh"] == "quad":
        n = spec["n"]
        return I.structured_quad_mesh(n, n, periodic=(spec["periodic"],) * 2)
    return I.structured_hex_mesh(spec["n"], 1.0, periodic=spec["periodic"])


@pytest.mark.parametrize("case", _golden("stencils_hand.json")["cases"],
                         ids=lambda c: f'{c["mesh"]}{c["n"]}_o{c["order"]}_c{c["cell"]}')
def test_stencils_against_hand_enumeration(case):
    """Central and directional stencils of a few cells of uniform 5x5, 4x4
    periodic and 3x3x3 meshes, enumerated by hand (Sec. 2.1, 2.3; readings R3
    and R7); the fixture gives each derivation."""
    m = _hand_mesh(case)
    s = O.Scheme(O.Mesh(m), order=case["order"])
    st, dirs = s.stencil(case["cell"])
    assert st.tolist() == case["stencil"]
    if "directional" in case:
        nd = s.operator(case["cell"], "nd").astype(int)
        got = sorted(sorted(dirs[f][:nd[f]].tolist()) for f in range(len(nd)))
        assert got == sorted(case["directional"])


def test_stencil_construction_fails_on_a_mesh_too_small():
    spec = _golden("stencils_hand.json")["too_small"]
    m = _hand_mesh(spec)
    with pytest.raises(RuntimeError, match="fewer than M cells"):
        s = O.Scheme(O.Mesh(m), order=spec["order"])
        s.stencil(0)


def test_stencil_size_rule():
    # M = 2 K(r, d), K(r, d) = prod_{l=1..d}(r+l)/d!  (Sec. 2.1)
    expect2d = {2: 6, 3: 12, 4: 20, 5: 30, 6: 42}
    m = I.structured_tri_mesh(12, periodic=True, jitter=0.1, seed=1)
    om = O.Mesh(m)
    for order, M in expect2d.items():
        s = O.Scheme(om, order=order)
        assert s.M == M and s.N == M // 2 - 1
    h = I.structured_hex_mesh(8, 1.0, periodic=True)
    oh = O.Mesh(h)
    s = O.Scheme(oh, order=4)
    assert (s.M, s.N) == (40, 19)


def test_uniform_hex_stencil_distance_pattern_translation_invariant():
    m = I.structured_hex_mesh(8, 1.0, periodic=True)
    om = O.Mesh(m)
    s = O.Scheme(om, order=4)
    vm = m.vertex_means()

    def pattern(c):
        st, _ = s.stencil(c)
        dx = vm[st] - vm[c]
        dx -= np.round(dx)
        return sorted(np.round((dx * 8) ** 2 @ np.ones(3)).astype(int).tolist())

    p0 = pattern(0)
    assert p0 == [1] * 6 + [2] * 12 + [3] * 8 + [4] * 6 + [5] * 8
    for c in (17, 100, 511, 300):
        assert pattern(c) == p0


# ---------------------------------------------------------------------------
# least squares and the reconstructions
# ---------------------------------------------------------------------------

def test_pseudo_inverse_against_lapack():
    m = I.mixed_tri_quad_mesh(12, seed=5)
    s = O.Scheme(O.Mesh(m), order=5)
    for c in (3, 50, 111):
        A = s.operator(c, "A")
        Vr = s.operator(c, "Vr")
        P = s.operator(c, "P")
        Ap = P / Vr[1:][None, :]
        assert np.abs(Ap @ A - np.eye(s.N)).max() < 1e-15 * np.linalg.cond(A)
        assert np.abs(Ap - np.linalg.pinv(A)).max() < 1e-10 * np.abs(Ap).max()


def _poly2d(rng, r):
    coef = {(a, b): rng.standard_normal() for a in range(r + 1) for b in range(r + 1 - a)}
    return lambda x, y: sum(c * x ** a * y ** b for (a, b), c in coef.items())


@pytest.mark.parametrize("order", [2, 3, 4, 5])
def test_linear_reconstruction_reproduces_polynomials(order):
    """Cell means of a degree-r polynomial give back its face-point values."""
    r = order - 1
    m = I.mixed_tri_quad_mesh(12, seed=5)
    s = O.Scheme(O.Mesh(m), order=order)
    rng = np.random.default_rng(order)
    f = _poly2d(rng, r)
    rho = I.cell_average_2d(m, f, npts=8)
    U = np.stack([rho, 0.5 * rho, -rho, rho + 4.0])
    for c in range(0, m.n_cells, 5):
        V = s.reconstruct(U, c, O.LIN)
        P = s.face_points(c)
        ex = f(P[:, 0], P[:, 1])
        assert np.abs(V[:, 0] - ex).max() < 1e-11 * (1 + np.abs(ex).max())
        assert np.abs(V[:, 2] + ex).max() < 1e-11 * (1 + np.abs(ex).max())


def test_hex_reconstruction_reproduces_cubics():
    m = I.structured_hex_mesh(7, 1.0, periodic=False, jitter=0.15, seed=4)
    s = O.Scheme(O.Mesh(m), order=4)
    rng = np.random.default_rng(11)
    terms = [(a, b, c) for a in range(4) for b in range(4 - a) for c in range(4 - a - b)]
    coef = rng.standard_normal(len(terms))
    om = s.mesh
    vol, _ = om.geometry()
    rho = np.array([sum(k * om.monomial_integral(c, *t, npts=6) for k, t in zip(coef, terms)) for c in range(m.n_cells)]) / vol
    U = np.stack([rho, 0 * rho, 0 * rho, 0 * rho, rho + 5.0])
    for c in (0, 57, 171, 200, 342):
        V = s.reconstruct(U, c, O.LIN)
        P = s.face_points(c)
        ex = sum(k * P[:, 0] ** t[0] * P[:, 1] ** t[1] * P[:, 2] ** t[2] for k, t in zip(coef, terms))
        assert np.abs(V[:, 0] - ex).max() < 1e-10 * (1 + np.abs(ex).max())


def test_cweno_exact_on_linear_data_and_weights_reduce_to_linear():
    """Degree-1 data: every stencil gives the same polynomial, so all
    indicators agree, tau = 0, omega = lambda (Sec. 2.3) and CWENOZ is exact."""
    m = I.mixed_tri_quad_mesh(12, seed=5)
    lam1p = 1e3
    s = O.Scheme(O.Mesh(m), order=4, lambda1p=lam1p)
    rho = I.cell_average_2d(m, lambda x, y: 1.0 + 0.3 * x - 0.7 * y)
    U = np.stack([rho, rho, rho, rho + 3])
    for c in (10, 77, 150):
        om_, si, _ = s.cweno_info(U, c, 0)
        st = len(om_)
        lam1 = 1 - 1 / lam1p
        lam = np.r_[lam1, np.full(st - 1, (1 - lam1) / (st - 1))]
        assert np.abs(si - si[0]).max() < 1e-12 * max(1.0, si[0])
        assert np.abs(om_ - lam).max() < 1e-12
        V = s.reconstruct(U, c, O.CW)
        P = s.face_points(c)
        assert np.abs(V[:, 0] - (1.0 + 0.3 * P[:, 0] - 0.7 * P[:, 1])).max() < 1e-12


def test_smoothness_indicator_closed_form():
    """SI of p = xi^2 on the reference triangle (h_c = 1): int (2 xi)^2 +
    int 2^2 over the unit right triangle = 1/3 + 2 = 7/3; of p = xi: 1/2."""
    m = I.structured_tri_mesh(10, periodic=False, jitter=0.2, seed=2)
    s = O.Scheme(O.Mesh(m), order=3)
    for c in (42, 97, 121):
        x0, Ji = s.refmap(c)
        xi = lambda x, y: Ji[0, 0] * (x - x0[0]) + Ji[0, 1] * (y - x0[1])
        for f, ex in ((lambda x, y: xi(x, y) ** 2, 7.0 / 3.0), (lambda x, y: xi(x, y), 0.5)):
            rho = I.cell_average_2d(m, f, npts=8)
            st, _ = s.stencil(c)
            a = s.operator(c, "P") @ (rho[st] - rho[c])
            si = a @ s.operator(c, "OI") @ a
            assert abs(si - ex) < 1e-11


def _tri_quadratic_integral(f, a, b, c):
    """Exact integral of a quadratic over the triangle abc: the area times the
    mean of f at the edge midpoints."""
    area = 0.5 * abs((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))
    return area / 3.0 * (f((a + b) / 2) + f((b + c) / 2) + f((c + a) / 2))


def test_reference_map_and_indicator_on_quadrilaterals():
    """R4 and R5 on jittered quadrilaterals, independently of the oracle's own
    map: the reference map is the affine map of the corner simplex v0 v1 v3
    (v0 -> 0, v1 -> e1, v3 -> e2), so the cell's image has corners 0, e1,
    w = J^-1 (v2 - v0), e2; the indicator of p = xi^2 is int (2 xi)^2 + 2^2
    over that image (h_c = 1, Sec. 2.3), and of p = xi its area, both
    integrated exactly over the image's two triangles."""
    m = I.structured_quad_mesh(8, 8, jitter=0.2, seed=4)
    s = O.Scheme(O.Mesh(m), order=3)
    for c in (9, 27, 36, 50):
        v = m.cell_vertices(c)
        J = np.stack([v[1] - v[0], v[3] - v[0]], axis=1)
        Ji = np.linalg.inv(J)
        x0, Jo = s.refmap(c)
        assert np.allclose(x0[:2], v[0], rtol=0, atol=1e-15)
        assert np.allclose(Jo[:2, :2], Ji, rtol=1e-13, atol=0)
        w = Ji @ (v[2] - v[0])
        e0, e1, e2 = np.zeros(2), np.array([1.0, 0.0]), np.array([0.0, 1.0])
        tris = ((e0, e1, w), (e0, w, e2))
        area = sum(_tri_quadratic_integral(lambda q: 1.0, *t) for t in tris)
        ixx = sum(_tri_quadratic_integral(lambda q: q[0] ** 2, *t) for t in tris)
        xi = lambda x, y: Ji[0, 0] * (x - v[0][0]) + Ji[0, 1] * (y - v[0][1])
        for f, ex in ((lambda x, y: xi(x, y) ** 2, 4.0 * ixx + 4.0 * area), (lambda x, y: xi(x, y), area)):
            rho = I.cell_average_2d(m, f, npts=8)
            st, _ = s.stencil(c)
            a = s.operator(c, "P") @ (rho[st] - rho[c])
            assert abs(a @ s.operator(c, "OI") @ a - ex) < 1e-10 * ex


@pytest.mark.parametrize("h", [1.0, 1e-2])
def test_indicator_is_scale_free_on_hexahedra(h):
    """Uniform hexahedra of edge h: the corner simplex v0 v1 v3 v4 maps the
    cell onto the unit cube whatever h is, so the indicator of p = xi^2
    (xi = x / h about the cell's corner) is int (2 xi)^2 + 2^2 over the cube =
    4/3 + 4 = 16/3 at every h (R4, R5); cell averages of the quadratic are
    taken in closed form."""
    n = 6
    m = I.structured_hex_mesh(n, n * h, periodic=False)
    s = O.Scheme(O.Mesh(m), order=3)
    c = (2 * n + 2) * n + 3          # cell (3, 2, 2)
    x0, Jo = s.refmap(c)
    lo = m.cell_vertices(c)[0]
    assert np.allclose(x0, lo, rtol=0, atol=1e-15 * n * h)
    assert np.allclose(Jo, np.eye(3) / h, rtol=1e-13, atol=0)
    # mean of ((x - lo_x) / h)^2 over the cell whose lower corner is at x = k h
    # relative to lo_x: ((k + 1)^3 - k^3) / 3
    vm = m.vertex_means()
    k = np.rint((vm[:, 0] - h / 2 - lo[0]) / h)
    rho = ((k + 1) ** 3 - k ** 3) / 3.0
    st, _ = s.stencil(c)
    a = s.operator(c, "P") @ (rho[st] - rho[c])
    assert abs(a @ s.operator(c, "OI") @ a - 16.0 / 3.0) < 1e-10


def test_cweno_weights_are_convex_and_favour_smooth_stencils():
    m = I.structured_quad_mesh(16, 16, jitter=0.1, seed=3)
    s = O.Scheme(O.Mesh(m), order=3)
    vm = m.vertex_means()
    rho = np.where(vm[:, 0] < 0.5, 1.0, 0.2)
    U = np.stack([rho, 0 * rho, 0 * rho, 2.5 + 0 * rho])
    c = 7 * 16 + 8  # cell just right of the jump
    om_, si, _ = s.cweno_info(U, c, 0)
    assert abs(om_.sum() - 1) < 1e-14 and (om_ >= 0).all()
    # the directional stencil pointing away from the jump (+x face, local face 1)
    # is smooth: SI = 0 and its weight is the largest relative to lambda
    assert si[1 + 1] < 1e-14
    assert np.argmax(om_[1:]) == 1


def test_muscl_barth_jespersen_bounds():
    m = I.mixed_tri_quad_mesh(14, seed=6)
    s = O.Scheme(O.Mesh(m), order=3)
    om = s.mesh
    nbr, _ = om.connectivity()
    rng = np.random.default_rng(1)
    U = np.stack([1 + rng.random(m.n_cells), rng.standard_normal(m.n_cells), rng.standard_normal(m.n_cells),
                  5 + rng.random(m.n_cells)])
    for c in range(0, m.n_cells, 11):
        V = s.reconstruct(U, c, O.MU)
        nb = [j for j in nbr[c] if j >= 0] + [c]
        lo, hi = U[:, nb].min(axis=1), U[:, nb].max(axis=1)
        assert (V >= lo - 1e-14).all() and (V <= hi + 1e-14).all()
    # linear data well inside the bounds: theta = 1 reproduces the plane
    rho = I.cell_average_2d(m, lambda x, y: 2.0 + 1e-3 * (x + 2 * y))
    U = np.stack([rho, rho, rho, rho + 3])
    inside = 0
    for c in range(m.n_cells):
        P = s.face_points(c)
        ex = 2.0 + 1e-3 * (P[:, 0] + 2 * P[:, 1])
        nb = [j for j in nbr[c] if j >= 0] + [c]
        if ex.min() >= rho[nb].min() and ex.max() <= rho[nb].max():
            V = s.reconstruct(U, c, O.MU)
            assert np.abs(V[:, 0] - ex).max() < 1e-13, c
            inside += 1
    assert inside >= m.n_cells // 2


def test_harten_bound_closed_form():
    """|q - qbar| <= 0.9 max(|qbar|, 1e-14) on density and pressure (Sec. 2.4)."""
    m = I.structured_tri_mesh(8, periodic=True, jitter=0.1, seed=1)
    s = O.Scheme(O.Mesh(m), order=3)
    U = np.tile(np.array([[2.0], [0.0], [0.0], [2.5]]), (1, m.n_cells))  # p = 1
    Q = s.Q(0)
    base = np.tile(U[:, 0], (Q, 1))
    for frac, ok in ((0.85, True), (0.95, False), (-0.85, True), (-0.95, False)):
        V = base.copy()
        V[2, 0] = 2.0 * (1 + frac)
        V[2, 3] = 2.5 + 0.5 * (V[2, 0] - 2.0) * 0  # keep pressure: E unchanged, zero velocity
        V[2, 3] = 2.5
        assert s.harten_ok(U, 0, V) == ok
    for frac, ok in ((0.89, True), (0.91, False)):
        V = base.copy()
        V[1, 3] = 2.5 * (1 + frac)  # p scales with E at rest
        assert s.harten_ok(U, 0, V) == ok


# ---------------------------------------------------------------------------
# detector (Sec. 2.5) and the paper's presets
# ---------------------------------------------------------------------------

def _evolved_quadrant(n=16, steps=3):
    m = I.mixed_tri_quad_mesh(n, seed=2)
    U = I.quadrant_state(m)
    s = O.Scheme(O.Mesh(m), order=3, flux="hllc")
    for _ in range(steps):
        U = s.rk3_step(U, s.dt(U, 0.5))
    return m, s, U


def test_quadrant_states_golden():
    g = _golden("quadrant_states.json")
    for k, v in I.QUADRANT_STATES.items():
        assert list(v) == g[k]


def test_nad_presets_are_invariants():
    presets = _golden("nad_presets.json")
    m, s0, U = _evolved_quadrant()
    om = s0.mesh
    counts = {}
    for name in ("default", "linear_cweno", "linear_muscl", "muscl_cweno"):
        s = O.Scheme(om, order=3, flux="hllc", **presets[name])
        _, raw, tag, fin = s.residual(U)
        counts[name] = np.bincount(raw, minlength=3)
        if name == "linear_cweno":
            assert counts[name][O.MU] == 0
        if name == "linear_muscl":
            assert counts[name][O.CW] == 0
        if name == "muscl_cweno":
            # only deactivated cells stay linear: compare with a detector that is never deactivated
            s_on = O.Scheme(om, order=3, flux="hllc", kappa=0.0, **presets[name])
            _, raw_on, _, _ = s_on.residual(U)
            assert (raw_on != O.LIN).all()
    assert counts["default"][O.MU] > 0 and counts["default"][O.CW] > 0


def test_uniform_state_is_all_linear():
    m = I.mixed_tri_quad_mesh(10, seed=2)
    s = O.Scheme(O.Mesh(m), order=3, flux="hllc")
    U = I.conserved_2d(np.full(m.n_cells, 1.3), np.full(m.n_cells, 0.2), np.full(m.n_cells, -0.1), np.full(m.n_cells, 0.9))
    _, raw, tag, fin = s.residual(U)
    assert (raw == O.LIN).all() and (fin == O.LIN).all()


def test_step_on_quad_strip_flags_jump_and_its_neighbourhood():
    """A density/pressure jump across x = 0.5 on a uniform quad strip.  The
    linear candidate over- and under-shoots next to the jump, but by less
    than beta_m = 0.5 of the local range, so the default detector puts the two
    cells at the jump in the CWENOZ band (eqs. NADMUSCL, NADCWENOZ); the
    all-zero margins of panel (d) put them in MUSCL.  Tagging spreads the class
    to the face neighbours; cells whose neighbours all agree are deactivated
    (eq. NADDeactivatedCriteria) and stay linear."""
    presets = _golden("nad_presets.json")
    nx, ny = 24, 12
    m = I.structured_quad_mesh(nx, ny, 1.0, 0.5, periodic=(False, True))
    vm = m.vertex_means()
    left = vm[:, 0] < 0.5
    U = I.conserved_2d(np.where(left, 1.0, 0.125), 0 * vm[:, 0], 0 * vm[:, 0], np.where(left, 1.0, 0.1))
    col = np.arange(m.n_cells) % nx
    at_jump = (col == 11) | (col == 12)
    near = (col >= 10) & (col <= 13)
    for order in (3, 5):
        for name, cls in (("default", O.CW), ("linear_muscl", O.MU)):
            s = O.Scheme(O.Mesh(m), order=order, flux="hllc", **presets[name])
            _, raw, tag, fin = s.residual(U)
            assert (raw[at_jump] == cls).all() and (raw[~at_jump] == O.LIN).all()
            assert (tag[near] == cls).all() and (tag[~near] == O.LIN).all()


def test_detector_watches_density_and_pressure_only():
    """R10: the detector checks rho and p (the Harten variables of Sec. 2.4).
    A shear layer -- tangential velocity jumping from +0.5 to -0.5 across
    x = 0.5 with rho and p uniform -- leaves both flat, so every cell stays
    linear, although momentum and energy jump; checking every conserved
    variable instead flags the two cells at the jump.  A contact (rho jumps, p
    uniform) is flagged under the default."""
    nx, ny = 24, 12
    m = I.structured_quad_mesh(nx, ny, 1.0, 0.5, periodic=(False, True))
    vm = m.vertex_means()
    left = vm[:, 0] < 0.5
    one = np.ones(m.n_cells)
    col = np.arange(m.n_cells) % nx
    at_jump = (col == 11) | (col == 12)
    shear = I.conserved_2d(one, 0 * one, np.where(left, 0.5, -0.5), one)
    contact = I.conserved_2d(np.where(left, 1.0, 0.5), 0 * one, 0 * one, one)
    for order in (3, 5):
        s = O.Scheme(O.Mesh(m), order=order, flux="hllc")
        assert (s.residual(shear)[1] == O.LIN).all()
        raw = s.residual(contact)[1]
        assert (raw[at_jump] != O.LIN).all() and (raw[~at_jump] == O.LIN).all()
        s_all = O.Scheme(O.Mesh(m), order=order, flux="hllc", nad_vars=7)
        raw = s_all.residual(shear)[1]
        assert (raw[at_jump] != O.LIN).all() and (raw[~at_jump] == O.LIN).all()


def test_detector_margins_act_in_the_direction_the_paper_describes():
    """R11 and R12 on the quadrant problem: a larger beta_w > 0 widens the
    linear band (Sec. 2.5 -- under the printed sign it would narrow it), so
    the linear cells only ever grow with it, and a larger kappa deactivates
    more cells.  With kappa = 0 nothing is deactivated and no raw class is
    linear, not even in the uniform quadrants (the candidate there equals the
    neighbours' extremes, outside the open band); with a huge kappa every cell
    is deactivated."""
    m = I.mixed_tri_quad_mesh(24, seed=2)
    U = I.quadrant_state(m)

    def linear(**kw):
        return O.Scheme(O.Mesh(m), order=3, flux="hllc", **kw).residual(U)[1] == O.LIN

    prev = None
    for bw in (-0.5, 0.0, 1e-2, 0.1, 0.5):
        lin = linear(beta_w=bw)
        if prev is not None:
            assert (lin >= prev).all(), bw
        prev = lin
    assert linear(beta_w=0.5).sum() > linear(beta_w=0.0).sum()
    prev = None
    for k in (0.0, 0.5, 1.0, 4.0, 1e3):
        lin = linear(kappa=k)
        if prev is not None:
            assert (lin >= prev).all(), k
        prev = lin
    assert not linear(kappa=0.0).any() and linear(kappa=1e3).all()


@pytest.mark.parametrize("n_exp", [1.0, 2.0])
def test_deactivation_threshold_flips_where_the_closed_form_says(n_exp):
    """R12 (eq. NADDeactivatedCriteria): a cell is deactivated when the spread
    of |U_j - U_i| over its face neighbours is below (kappa dx)^n, dx =
    |V|^(1/d).  At a density contact (pressure and velocity uniform) on unit
    squares of edge h, the two cells at the jump J see |dU| = {0, J, 0, 0}, a
    spread of J, so they turn linear exactly when kappa passes J^(1/n) / h;
    pressure, uniform, is deactivated for any kappa > 0."""
    nx, ny = 24, 12
    m = I.structured_quad_mesh(nx, ny, 1.0, 0.5, periodic=(False, True))
    h = 1.0 / nx
    vm = m.vertex_means()
    J = 0.875
    one = np.ones(m.n_cells)
    U = I.conserved_2d(np.where(vm[:, 0] < 0.5, 1.0, 1.0 - J), 0 * one, 0 * one, one)
    col = np.arange(m.n_cells) % nx
    at_jump = (col == 11) | (col == 12)
    k_flip = J ** (1.0 / n_exp) / h
    below = O.Scheme(O.Mesh(m), order=3, flux="hllc", kappa=0.98 * k_flip, n_exp=n_exp).residual(U)[1]
    above = O.Scheme(O.Mesh(m), order=3, flux="hllc", kappa=1.02 * k_flip, n_exp=n_exp).residual(U)[1]
    assert (below[at_jump] != O.LIN).all() and (below[~at_jump] == O.LIN).all()
    assert (above == O.LIN).all()


def test_hybrid_equals_linear_when_detector_is_deactivated():
    """Sec. 3.1: with no troubled cell the hybrid operates as the linear scheme."""
    m = I.structured_tri_mesh(16, periodic=True, jitter=0.2, seed=1)
    U = I.density_wave_state(m)
    om = O.Mesh(m)
    hy = O.Scheme(om, order=3, kappa=1.0, n_exp=2.0 / 3.0)
    li = O.Scheme(om, order=3, scheme="linear")
    Rh, raw, _, fin = hy.residual(U)
    Rl, _, _, _ = li.residual(U)
    assert (raw == O.LIN).all()
    assert np.array_equal(Rh, Rl)


# ---------------------------------------------------------------------------
# fluxes
# ---------------------------------------------------------------------------

def _cons(rho, u, p, g=1.4):
    u = np.asarray(u, float)
    return np.r_[rho, rho * u, p / (g - 1) + 0.5 * rho * u @ u]


def _phys(U, n, g=1.4):
    rho, m, E = U[0], U[1:-1], U[-1]
    u = m / rho
    p = (g - 1) * (E - 0.5 * rho * u @ u)
    un = u @ n
    return np.r_[rho * un, m * un + p * n, (E + p) * un]


@pytest.mark.parametrize("kind", ["rusanov", "hllc", "hll"])
def test_flux_consistency_and_antisymmetry(kind):
    rng = np.random.default_rng(3)
    for d in (2, 3):
        for _ in range(20):
            n = rng.standard_normal(d); n /= np.linalg.norm(n)
            UL = _cons(0.5 + rng.random(), rng.standard_normal(d), 0.5 + rng.random())
            UR = _cons(0.5 + rng.random(), rng.standard_normal(d), 0.5 + rng.random())
            assert np.allclose(O.flux(kind, UL, UL, n), _phys(UL, n), rtol=1e-14, atol=1e-14)
            assert np.allclose(O.flux(kind, UL, UR, n), -O.flux(kind, UR, UL, -n), rtol=1e-12, atol=1e-13)


def test_supersonic_upwinding():
    n = np.array([1.0, 0.0])
    UL = _cons(1.0, [3.0, 0.2], 1.0)
    UR = _cons(0.5, [2.8, -0.1], 0.7)
    for kind in ("hllc", "hll"):
        assert np.allclose(O.flux(kind, UL, UR, n), _phys(UL, n), rtol=1e-14)
        assert np.allclose(O.flux(kind, UR, UL, -n), _phys(UL, -n), rtol=1e-14)


def test_hllc_preserves_stationary_contact():
    """Toro: HLLC resolves an isolated stationary contact exactly; HLL and
    Rusanov smear it (mass flux != 0)."""
    n = np.array([0.0, 1.0, 0.0])
    UL, UR = _cons(1.0, [0.3, 0.0, -0.2], 1.0), _cons(0.2, [0.3, 0.0, -0.2], 1.0)
    F = O.flux("hllc", UL, UR, n)
    assert abs(F[0]) < 1e-15 and abs(F[2] - 1.0) < 1e-15 and abs(F[4]) < 1e-15
    assert abs(O.flux("hll", UL, UR, n)[0]) > 1e-3
    assert abs(O.flux("rusanov", UL, UR, n)[0]) > 1e-3


def test_rusanov_textbook():
    n = np.array([0.6, 0.8])
    UL, UR = _cons(1.0, [0.1, 0.2], 1.0), _cons(0.8, [-0.3, 0.1], 0.6)
    cl, cr = math.sqrt(1.4 * 1.0 / 1.0), math.sqrt(1.4 * 0.6 / 0.8)
    s = max(abs(0.1 * 0.6 + 0.2 * 0.8) + cl, abs(-0.3 * 0.6 + 0.1 * 0.8) + cr)
    ex = 0.5 * (_phys(UL, n) + _phys(UR, n)) - 0.5 * s * (UR - UL)
    assert np.allclose(O.flux("rusanov", UL, UR, n), ex, rtol=1e-14)


def test_hllc_star_flux_from_the_rankine_hugoniot_conditions():
    """HLLC (R18) in the form derived from the Rankine-Hugoniot conditions
    across the wave S_K and the contact (Toro, Riemann Solvers, Sec. 10.4):
    F*_K = [S* (S_K U_K - F_K) + S_K p* D*] / (S_K - S*), D* = (0, n, S*),
    p* = p_K + rho_K (S_K - u_K)(S* - u_K), which equals the flux of the
    explicit star state F_K + S_K (U*_K - U_K) the oracle evaluates.  Random
    subsonic pairs in 2D and 3D, on both sides of the contact."""
    rng = np.random.default_rng(7)
    g = 1.4
    checked = [0, 0]
    for trial in range(400):
        d = 2 + trial % 2
        n = rng.standard_normal(d)
        n /= np.linalg.norm(n)
        rl, rr = 0.5 + rng.random(2)
        pl, pr = 0.5 + rng.random(2)
        ul, ur = 0.6 * rng.standard_normal((2, d))
        UL, UR = _cons(rl, ul, pl), _cons(rr, ur, pr)
        unl, unr = ul @ n, ur @ n
        cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
        SL, SR = min(unl - cl, unr - cr), max(unl + cl, unr + cr)
        if SL >= 0 or SR <= 0:
            continue
        Ss = (pr - pl + rl * unl * (SL - unl) - rr * unr * (SR - unr)) / (rl * (SL - unl) - rr * (SR - unr))
        K = (UL, SL, rl, unl, pl) if Ss >= 0 else (UR, SR, rr, unr, pr)
        UK, SK, rk, uk, pk = K
        ps = pk + rk * (SK - uk) * (Ss - uk)
        D = np.r_[0.0, n, Ss]
        want = (Ss * (SK * UK - _phys(UK, n)) + SK * ps * D) / (SK - Ss)
        got = O.flux("hllc", UL, UR, n)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12), (trial, got, want)
        checked[int(Ss >= 0)] += 1
    assert min(checked) >= 50


def _tiled_twice(small, shape):
    """the periodic mesh `small` (structured, nodes numbered x fastest) and
    its two periodic images side by side along x as one periodic mesh of
    twice the length; returns (big, tile, first): big cell -> small cell, and
    the big cells of the first image in small-cell order"""
    dims = list(shape)                      # cells per direction, x first
    nx = dims[0]
    L = small.period[0]
    if small.dim == 2:
        big = I.structured_quad_mesh(2 * nx, dims[1], 2 * L, small.period[1], periodic=(True, True))
    else:
        big = I.structured_hex_mesh(2 * nx, 2 * L, periodic=True, ny=dims[1], nz=dims[2])
        big = I.Mesh(3, big.nodes, big.cell_type, big.cell_ptr, big.cell_idx,
                     np.array([2 * L, small.period[1], small.period[2]]))
    npd = [d + 1 for d in dims]
    nodes = big.nodes.copy()
    for b in range(nodes.shape[0]):
        i, rest = b % (2 * nx + 1), b // (2 * nx + 1)
        k, r = divmod(i, nx)
        if i == 2 * nx:
            k, r = 1, nx
        nodes[b] = small.nodes[rest * npd[0] + r] + np.r_[k * L, np.zeros(small.dim - 1)]
    big = I.Mesh(small.dim, nodes, big.cell_type, big.cell_ptr, big.cell_idx, big.period)
    rows = int(np.prod(dims[1:]))
    tile = np.array([q * nx + (i % nx) for q in range(rows) for i in range(2 * nx)])
    first = np.array([q * 2 * nx + i for q in range(rows) for i in range(nx)])
    return big, tile, first


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_images_give_the_same_residual(dim):
    """A jittered periodic mesh and two of its periodic images joined into
    one periodic mesh describe the same flow: each cell of the first image
    must get the small mesh's residual (hybrid, HLLC, with and without the
    viscous terms) and class.  The small mesh's periodic seam is an interior
    face of the big one, so every use of a periodic shift -- stencil cells,
    directional stencils, face pairing, the viscous centre distance L_int --
    is checked against the same computation without one."""
    rng = np.random.default_rng(3 + dim)
    if dim == 2:
        shape = (8, 6)
        small = I.structured_quad_mesh(*shape, 1.0, 1.0, periodic=(True, True), jitter=0.2, seed=5)
        order = 3
    else:
        shape = (6, 6, 6)
        small = I.structured_hex_mesh(6, 1.0, periodic=True, jitter=0.15, seed=5)
        order = 2
    big, tile, first = _tiled_twice(small, shape)
    n = small.n_cells
    rho, p = 0.8 + 0.4 * rng.random(n), 0.8 + 0.4 * rng.random(n)
    vel = rng.uniform(-0.5, 0.5, (dim, n))
    Us = np.concatenate([rho[None], rho * vel, (p / 0.4 + 0.5 * rho * (vel ** 2).sum(0))[None]])
    vm = small.vertex_means()

    def band(jump):     # a smooth wave and a density band: linear, CWENOZ, MUSCL and first-order cells
        r = 1.0 + 0.2 * np.sin(2 * math.pi * vm[:, 0]) + np.where(np.abs(vm[:, 1] - 0.5) < 0.2, jump, 0.0)
        return np.concatenate([r[None], 0.3 * r[None], np.zeros((dim - 1, n)), (1.0 / 0.4 + 0.045 * r)[None]])

    for U in (Us, band(0.5), band(4.0)):
        for kw in ({}, {"mu0": 0.05}):
            Rs, _, _, fs = O.Scheme(O.Mesh(small), order=order, flux="hllc", **kw).residual(U)
            Rb, _, _, fb = O.Scheme(O.Mesh(big), order=order, flux="hllc", **kw).residual(U[:, tile])
            assert np.array_equal(fb[first], fs)
            assert np.abs(Rb[:, first] - Rs).max() <= 1e-12 * np.abs(Rs).max(), kw


# ---------------------------------------------------------------------------
# residual, time stepping and order of accuracy
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("maker,order,flux", [
    (lambda: I.structured_tri_mesh(12, periodic=True, jitter=0.2, seed=1), 3, "rusanov"),
    (lambda: I.mixed_tri_quad_mesh(12, seed=8, periodic=True), 5, "hllc"),
    (lambda: I.structured_hex_mesh(6, 2 * math.pi, periodic=True), 4, "hllc"),
])
def test_free_stream_and_conservation(maker, order, flux):
    m = maker()
    om = O.Mesh(m)
    vol, _ = om.geometry()
    s = O.Scheme(om, order=order, flux=flux)
    n = m.n_cells
    if m.dim == 2:
        Uu = I.conserved_2d(np.full(n, 1.2), np.full(n, 0.4), np.full(n, -0.3), np.full(n, 0.8))
    else:
        Uu = np.tile(np.array([[1.2], [0.3], [-0.2], [0.1], [3.0]]), (1, n))
    R, *_ = s.residual(Uu)
    scale = np.abs(Uu).max() * 4 / vol.min() ** (1.0 / m.dim)
    assert np.abs(R).max() < 64 * 2.2e-16 * scale
    # periodic: volume-weighted residuals sum to zero (no boundary flux)
    rng = np.random.default_rng(0)
    if m.dim == 2:
        U = I.conserved_2d(1 + 0.3 * rng.random(n), rng.standard_normal(n) * 0.3, rng.standard_normal(n) * 0.3, 1 + 0.3 * rng.random(n))
    else:
        U = I.turbulence_state(m, seed=1)
        U[0] *= 1 + 0.2 * rng.random(n)
    R, raw, tag, fin = s.residual(U)
    tot = (R * vol).sum(axis=1)
    assert np.abs(tot).max() < 1e-12 * (np.abs(R) * vol).sum()


def test_transmissive_boundary_conserves_up_to_boundary_flux():
    """Non-periodic domain, uniform state: the boundary flux F(U).n sums to
    zero over the closed boundary, so the residual vanishes."""
    m = I.mixed_tri_quad_mesh(10, seed=2)
    s = O.Scheme(O.Mesh(m), order=3, flux="hllc")
    n = m.n_cells
    U = I.conserved_2d(np.full(n, 0.7), np.full(n, 1.1), np.full(n, 0.4), np.full(n, 1.3))
    R, *_ = s.residual(U)
    assert np.abs(R).max() < 1e-11


@pytest.mark.parametrize("dim,periodic", [(2, False), (2, True), (3, False)])
def test_time_step_closed_form(dim, periodic):
    """R16 on uniform meshes, where the face sum is written by hand: the
    faces of an hx x hy rectangle are two of length hy with normals +-x and
    two of length hx with normals +-y, so sum_f (|u.n_f| + a)|S_f| =
    2(|u| + a) hy + 2(|v| + a) hx (in 3D, 2 h^2 per axis); dt = CFL min |V| / that."""
    g = 1.4
    rng = np.random.default_rng(3 + dim)
    if dim == 2:
        nx, ny = 6, 4
        m = I.structured_quad_mesh(nx, ny, periodic=(periodic, periodic))
        hs = np.array([1.0 / nx, 1.0 / ny])
    else:
        m = I.structured_hex_mesh(4, 1.0, periodic=periodic)
        hs = np.full(3, 0.25)
    n = m.n_cells
    rho, p = 0.5 + rng.random(n), 0.5 + rng.random(n)
    vel = rng.uniform(-1.0, 1.0, (dim, n))
    U = np.concatenate([rho[None], rho * vel, (p / (g - 1) + 0.5 * rho * (vel ** 2).sum(0))[None]])
    a = np.sqrt(g * p / rho)
    vol = np.prod(hs)
    lam = sum(2.0 * (np.abs(vel[k]) + a) * vol / hs[k] for k in range(dim))
    want = 0.5 * np.min(vol / lam)
    got = O.Scheme(O.Mesh(m), order=2).dt(U, 0.5)
    assert abs(got - want) <= 1e-14 * want


def test_ssp_rk3_amplification_factor():
    lam = np.array([-1.0, -0.3, 0.5, -2.0])
    dt = 0.4
    U = O.rk3_generic(np.ones(4), dt, lambda u: lam * u)
    z = lam * dt
    assert np.allclose(U, 1 + z + z ** 2 / 2 + z ** 3 / 6, rtol=1e-15, atol=1e-15)


def test_sampled_residual_matches_full():
    m = I.mixed_tri_quad_mesh(14, seed=2)
    U = I.quadrant_state(m)
    s = O.Scheme(O.Mesh(m), order=3, flux="hllc")
    U = s.rk3_step(U, s.dt(U, 0.5))
    R, raw, tag, fin = s.residual(U)
    smp = np.array([0, 5, 101, 200, m.n_cells - 1])
    Rs, raws, tags, fins = s.residual(U, sample=smp)
    assert np.array_equal(Rs[:, smp], R[:, smp])
    assert np.array_equal(fins[smp], fin[smp])


@pytest.mark.slow
def test_order_of_accuracy_density_wave():
    """The smooth density wave rho(x - t, y - t) converges at the design
    order r + 1 = 3 in the volume-weighted L2 norm (eq. NormsofErrors)."""
    errs = []
    T = 0.1
    for n in (12, 24, 48):
        m = I.structured_tri_mesh(n, periodic=True, jitter=0.2, seed=1)
        om = O.Mesh(m)
        vol, _ = om.geometry()
        s = O.Scheme(om, order=3, flux="rusanov", scheme="linear")
        U = I.density_wave_state(m)
        dt0 = s.dt(U, 0.5)
        nsteps = int(math.ceil(T / dt0))
        dt = T / nsteps
        for _ in range(nsteps):
            U = s.rk3_step(U, dt)
        ex = I.density_wave_state(m, t=T)
        errs.append(math.sqrt(((U[0] - ex[0]) ** 2 * vol).sum() / vol.sum()))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert 2.6 < rates[-1] < 3.6, (errs, rates)
