"""Pins of the oracle on tetrahedra (CPU): the element the adjoint workload's
mesh is made of (unit cube, hexahedra cut into six tetrahedra).

  * int x^a y^b z^c over the unit tetrahedron = a! b! c! / (a+b+c+3)!
  * the six-tetrahedra cut: measures sum to the domain, every cell closed
    (sum of outward area vectors = 0), interior faces paired symmetrically,
    periodic pairing complete
  * triangle-face rule: weights sum to the face area and integrate degree-r
    polynomials exactly (checked on the faces of the unit tetrahedron)
  * linear reconstruction reproduces degree-r polynomials (orders 2, 3) on a
    jittered tetrahedral mesh
  * free stream preserved, volume-weighted residuals sum to zero on a
    periodic mesh
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_25906_gb300 import inputs as I


def _unit_tet():
    nodes = np.array([[0., 0., 0.], [1., 0., 0.], [0., 1., 0.], [0., 0., 1.]])
    return I.Mesh(3, nodes, np.array([I.TET], np.uint8), np.array([0, 4]), np.array([0, 1, 2, 3], np.int32),
                  np.zeros(3), "unit_tet", {})


def test_tet_monomial_integrals_closed_form():
    om = O.Mesh(_unit_tet())
    for a, b, c in [(0, 0, 0), (1, 0, 0), (1, 1, 1), (2, 0, 3), (4, 1, 0), (2, 2, 2)]:
        ex = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
        assert abs(om.monomial_integral(0, a, b, c, npts=6) - ex) < 1e-15


@pytest.mark.parametrize("periodic,jitter", [(False, 0.1), (True, 0.0)])
def test_tet_mesh_geometry(periodic, jitter):
    m = I.structured_tet_mesh(4, 1.0, periodic=periodic, jitter=jitter, seed=3)
    om = O.Mesh(m)
    vol, cen = om.geometry()
    assert (vol > 0).all() and abs(vol.sum() - 1.0) < 1e-13
    nbr, nbrf = om.connectivity()
    for c in range(m.n_cells):
        for f in range(4):
            j = nbr[c, f]
            if j >= 0:
                assert nbr[j, nbrf[c, f]] == c and nbrf[j, nbrf[c, f]] == f
    if periodic:
        assert (nbr[:, :4] >= 0).all()
    fo, fn, nrm, area, sh = om.faces()
    closure = np.zeros((m.n_cells, 3))
    np.add.at(closure, fo, nrm * area[:, None])
    inner = fn >= 0
    np.add.at(closure, fn[inner], -(nrm * area[:, None])[inner])
    assert np.abs(closure).max() < 1e-13 * area.max()


@pytest.mark.parametrize("order", [2, 3])
def test_tet_face_rule(order):
    """On each face of the unit tetrahedron the rule integrates every
    monomial of degree <= r exactly: sum_p w_p x^a y^b z^c against the
    closed form of the face triangle (its barycentric integral)."""
    om = O.Mesh(_unit_tet())
    s = O.Scheme(om, order=order)
    r = order - 1
    P = s.face_points(0)             # [4 * nfp, 3]
    W = s.face_weights(0)            # [4 * nfp]
    nfp = P.shape[0] // 4
    verts = np.array([[0., 0., 0.], [1., 0., 0.], [0., 1., 0.], [0., 0., 1.]])
    faces = [(1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1)]
    rng = np.random.default_rng(order)
    for f, (i, j, k) in enumerate(faces):
        A, B, Cc = verts[i], verts[j], verts[k]
        area = 0.5 * np.linalg.norm(np.cross(B - A, Cc - A))
        pts, w = P[f * nfp:(f + 1) * nfp], W[f * nfp:(f + 1) * nfp]
        assert abs(w.sum() - area) < 1e-15
        for _ in range(4):
            e = rng.integers(0, r + 1, 3)
            while e.sum() > r:
                e = rng.integers(0, r + 1, 3)
            q = sum(wp * np.prod(x ** e) for wp, x in zip(w, pts))
            # exact: a dense product rule of high order on the same triangle
            g, gw = np.polynomial.legendre.leggauss(12)
            g, gw = 0.5 * (g + 1), 0.5 * gw
            ex = 0.0
            for a, wa in zip(g, gw):
                for b, wb in zip(g, gw):
                    x = A + a * (B - A) + a * b * (Cc - B)
                    ex += wa * wb * 2 * area * a * np.prod(x ** e)
            assert abs(q - ex) < 1e-14, (f, e, q, ex)


@pytest.mark.parametrize("order", [2, 3])
def test_tet_reconstruction_reproduces_polynomials(order):
    r = order - 1
    m = I.structured_tet_mesh(5, 1.0, periodic=False, jitter=0.1, seed=6)
    s = O.Scheme(O.Mesh(m), order=order)
    rng = np.random.default_rng(order + 20)
    terms = [(a, b, c) for a in range(r + 1) for b in range(r + 1 - a) for c in range(r + 1 - a - b)]
    coef = rng.standard_normal(len(terms))
    om = s.mesh
    vol, _ = om.geometry()
    rho = np.array([sum(k * om.monomial_integral(c, *t, npts=5) for k, t in zip(coef, terms))
                    for c in range(m.n_cells)]) / vol
    U = np.stack([rho, 0 * rho, 0 * rho, 0 * rho, rho + 5.0])
    for c in (0, 101, 377, 512, 749):
        V = s.reconstruct(U, c, O.LIN)
        P = s.face_points(c)
        ex = sum(k * P[:, 0] ** t[0] * P[:, 1] ** t[1] * P[:, 2] ** t[2] for k, t in zip(coef, terms))
        assert np.abs(V[:, 0] - ex).max() < 1e-10 * (1 + np.abs(ex).max())


def test_tet_free_stream_and_conservation():
    m = I.structured_tet_mesh(4, 1.0, periodic=True, jitter=0.0)
    om = O.Mesh(m)
    vol, _ = om.geometry()
    s = O.Scheme(om, order=3, flux="hllc")
    n = m.n_cells
    Uu = np.tile(np.array([[1.2], [0.3], [-0.2], [0.1], [3.0]]), (1, n))
    R, *_ = s.residual(Uu)
    scale = np.abs(Uu).max() * 4 / vol.min() ** (1.0 / 3)
    assert np.abs(R).max() < 64 * 2.2e-16 * scale
    rng = np.random.default_rng(0)
    U = Uu * (1 + 0.2 * rng.random((1, n)))
    U[1:4] += 0.1 * rng.standard_normal((3, n))
    R, raw, tag, fin = s.residual(U)
    tot = (R * vol).sum(axis=1)
    assert np.abs(tot).max() < 1e-12 * (np.abs(R) * vol).sum()
