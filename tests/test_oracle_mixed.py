"""Pins of the oracle on 3D meshes that mix tetrahedra, prisms, pyramids
and hexahedra (CPU).

  * int x^a y^b z^c over the unit prism (triangle (0,0) (1,0) (0,1) times
    [0,1]) = a! b! / (a+b+2)! / (c+1), and over the pyramid on the unit
    square with its apex over the origin at height 1
    = c! (a+b+2)! / ((a+1) (b+1) (a+b+c+3)!)
  * a prism cut into three tetrahedra, and a pyramid into two, give the
    same moments as the pieces (flat faces)
  * the mixed mesh (every type present): measures sum to the cube, each
    cell closed (sum of outward area vectors = 0), interior faces paired
    symmetrically, a triangle only ever meets a triangle
  * the face rule on triangles and quadrilaterals integrates degree-r
    polynomials exactly on the unit prism's and pyramid's faces
  * the linear reconstruction reproduces degree-r polynomials (orders 2, 3)
    in every cell type of a jittered mixed mesh
  * free stream and conservation of the residual
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_25906_gb300 import inputs as I


def _single(nodes, t, conn):
    nodes = np.asarray(nodes, float)
    return I.Mesh(3, nodes, np.array([t], np.uint8), np.array([0, len(conn)]), np.asarray(conn, np.int32),
                  np.zeros(3), "single", {})


PRISM = [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [0, 1, 1]]
PYRAMID = [[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1]]


@pytest.mark.parametrize("a,b,c", [(0, 0, 0), (1, 0, 0), (0, 1, 2), (2, 1, 1), (3, 0, 2), (1, 2, 3)])
def test_prism_and_pyramid_monomials_closed_form(a, b, c):
    f = math.factorial
    om = O.Mesh(_single(PRISM, I.PRISM, range(6)))
    ex = f(a) * f(b) / f(a + b + 2) / (c + 1)
    assert abs(om.monomial_integral(0, a, b, c, npts=6) - ex) < 1e-15
    om = O.Mesh(_single(PYRAMID, I.PYRAMID, range(5)))
    ex = f(c) * f(a + b + 2) / ((a + 1) * (b + 1) * f(a + b + c + 3))
    assert abs(om.monomial_integral(0, a, b, c, npts=6) - ex) < 1e-15


def test_prism_and_pyramid_equal_their_tetrahedra():
    rng = np.random.default_rng(3)
    pr = np.array(PRISM, float) + 0.15 * rng.standard_normal((6, 3)) * [1, 1, 0]
    pr[3:, :2] = pr[:3, :2] + 0.1 * rng.standard_normal(2)       # flat quadrilateral sides: parallel top
    pr[3:, 2] = 1.0 + 0.0 * pr[3:, 2]
    py = np.array(PYRAMID, float)
    py[4] = [0.3, 0.2, 0.9]
    cases = [(pr, I.PRISM, [[0, 1, 2, 3], [1, 2, 3, 4], [2, 3, 4, 5]]), (py, I.PYRAMID, [[0, 1, 2, 4], [0, 2, 3, 4]])]
    for nodes, t, tets in cases:
        om = O.Mesh(_single(nodes, t, range(len(nodes))))
        for e in [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 2, 1), (2, 0, 2)]:
            whole = om.monomial_integral(0, *e, npts=6)
            parts = 0.0
            for tt in tets:
                x = nodes[tt]
                det = np.dot(x[1] - x[0], np.cross(x[2] - x[0], x[3] - x[0]))
                if det < 0:
                    tt = [tt[0], tt[2], tt[1], tt[3]]
                parts += O.Mesh(_single(nodes[tt], I.TET, range(4))).monomial_integral(0, *e, npts=6)
            assert abs(whole - parts) < 1e-14 * max(1.0, abs(whole)), (t, e, whole, parts)


def test_mixed_mesh_geometry():
    m = I.mixed_element_mesh(4, seed=7)
    assert set(np.unique(m.cell_type)) == {I.TET, I.PRISM, I.PYRAMID, I.HEX}
    om = O.Mesh(m)
    vol, cen = om.geometry()
    assert (vol > 0).all() and abs(vol.sum() - 1.0) < 1e-13
    nbr, nbrf = om.connectivity()
    nf = {I.TET: 4, I.PRISM: 5, I.PYRAMID: 5, I.HEX: 6}
    tri = {I.TET: {0, 1, 2, 3}, I.PRISM: {0, 1}, I.PYRAMID: {0, 1, 2, 3}, I.HEX: set()}
    for c in range(m.n_cells):
        t = int(m.cell_type[c])
        for f in range(nf[t]):
            j = nbr[c, f]
            if j >= 0:
                assert nbr[j, nbrf[c, f]] == c and nbrf[j, nbrf[c, f]] == f
                assert (f in tri[t]) == (int(nbrf[c, f]) in tri[int(m.cell_type[j])])
    fo, fn, nrm, area, sh = om.faces()
    closure = np.zeros((m.n_cells, 3))
    np.add.at(closure, fo, nrm * area[:, None])
    inner = fn >= 0
    np.add.at(closure, fn[inner], -(nrm * area[:, None])[inner])
    assert np.abs(closure).max() < 1e-13 * area.max()


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("shape", ["prism", "pyramid"])
def test_face_rule_on_mixed_faces(order, shape):
    """Each face of the unit prism / pyramid (triangles by the collapsed
    rule, quadrilaterals by the tensor rule) integrates every monomial of
    degree <= r exactly against a dense product rule on the same face."""
    nodes, t, nfaces = (PRISM, I.PRISM, 5) if shape == "prism" else (PYRAMID, I.PYRAMID, 5)
    om = O.Mesh(_single(nodes, t, range(len(nodes))))
    s = O.Scheme(om, order=order)
    r = order - 1
    P = s.face_points(0)
    W = s.face_weights(0)
    nfp = P.shape[0] // nfaces
    g, gw = np.polynomial.legendre.leggauss(12)
    g, gw = 0.5 * (g + 1), 0.5 * gw
    rng = np.random.default_rng(order)
    faces = {"prism": [(0, 2, 1), (3, 4, 5), (0, 1, 4, 3), (1, 2, 5, 4), (2, 0, 3, 5)],
             "pyramid": [(0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4), (0, 3, 2, 1)]}[shape]
    X = np.asarray(nodes, float)
    for f, fv in enumerate(faces):
        pts, w = P[f * nfp:(f + 1) * nfp], W[f * nfp:(f + 1) * nfp]
        for _ in range(4):
            e = rng.integers(0, r + 1, 3)
            while e.sum() > r:
                e = rng.integers(0, r + 1, 3)
            q = sum(wp * np.prod(x ** e) for wp, x in zip(w, pts))
            ex = 0.0
            if len(fv) == 3:
                A, B, C = X[list(fv)]
                area = 0.5 * np.linalg.norm(np.cross(B - A, C - A))
                for a, wa in zip(g, gw):
                    for b, wb in zip(g, gw):
                        ex += wa * wb * 2 * area * a * np.prod((A + a * (B - A) + a * b * (C - B)) ** e)
            else:
                A, B, C, D = X[list(fv)]           # planar here: |S| w is the exact weight
                area = 0.5 * np.linalg.norm(np.cross(C - A, D - B))
                for a, wa in zip(g, gw):
                    for b, wb in zip(g, gw):
                        x = (1 - a) * (1 - b) * A + a * (1 - b) * B + a * b * C + (1 - a) * b * D
                        ex += wa * wb * area * np.prod(x ** e)
            assert abs(q - ex) < 1e-14, (shape, f, e, q, ex)


@pytest.mark.parametrize("order", [2, 3])
def test_mixed_reconstruction_reproduces_polynomials(order):
    r = order - 1
    m = I.mixed_element_mesh(4, seed=11)
    s = O.Scheme(O.Mesh(m), order=order)
    rng = np.random.default_rng(order + 40)
    terms = [(a, b, c) for a in range(r + 1) for b in range(r + 1 - a) for c in range(r + 1 - a - b)]
    coef = rng.standard_normal(len(terms))
    om = s.mesh
    vol, _ = om.geometry()
    rho = np.array([sum(k * om.monomial_integral(c, *t, npts=5) for k, t in zip(coef, terms))
                    for c in range(m.n_cells)]) / vol
    U = np.stack([rho, 0 * rho, 0 * rho, 0 * rho, rho + 5.0])
    picks = [int(np.nonzero(m.cell_type == t)[0][k]) for t in (I.TET, I.PRISM, I.PYRAMID, I.HEX) for k in (0, -1)]
    for c in picks:
        V = s.reconstruct(U, c, O.LIN)
        P = s.face_points(c)
        ex = sum(k * P[:, 0] ** t[0] * P[:, 1] ** t[1] * P[:, 2] ** t[2] for k, t in zip(coef, terms))
        assert np.abs(V[:, 0] - ex).max() < 1e-10 * (1 + np.abs(ex).max()), (c, int(m.cell_type[c]))


def test_mixed_free_stream_and_conservation():
    m = I.mixed_element_mesh(4, seed=5)
    om = O.Mesh(m)
    vol, _ = om.geometry()
    s = O.Scheme(om, order=3, flux="hllc")
    n = m.n_cells
    Uu = np.tile(np.array([[1.2], [0.3], [-0.2], [0.1], [3.0]]), (1, n))
    R, *_ = s.residual(Uu)
    scale = np.abs(Uu).max() * 6 / vol.min() ** (1.0 / 3)
    assert np.abs(R).max() < 64 * 2.2e-16 * scale
    rng = np.random.default_rng(0)
    U = Uu * (1 + 0.2 * rng.random((1, n)))
    U[1:4] += 0.1 * rng.standard_normal((3, n))
    R, raw, tag, fin = s.residual(U)
    assert len(np.unique(fin)) >= 2
    # open boundary: interior fluxes cancel pairwise, so the volume-weighted
    # residuals sum to minus the boundary fluxes (transmissive: the physical
    # flux of the cell's own face-point state)
    faces = {I.TET: [(1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1)],
             I.PRISM: [(0, 2, 1), (3, 4, 5), (0, 1, 4, 3), (1, 2, 5, 4), (2, 0, 3, 5)],
             I.PYRAMID: [(0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4), (0, 3, 2, 1)],
             I.HEX: [(0, 3, 2, 1), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7)]}
    nbr, _ = om.connectivity()
    bsum = np.zeros(5)
    for c in range(n):
        t = int(m.cell_type[c])
        X = m.cell_vertices(c)
        V = s.reconstruct(U, c, int(fin[c]))
        w = s.face_weights(c)
        nfp = s.nfp
        for f, fv in enumerate(faces[t]):
            if nbr[c, f] >= 0:
                continue
            P = X[list(fv)]
            A = 0.5 * np.cross(P[1] - P[0], P[2] - P[0]) if len(fv) == 3 else 0.5 * np.cross(P[2] - P[0], P[3] - P[1])
            nrm = A / np.linalg.norm(A)
            for q in range(f * nfp, (f + 1) * nfp):
                bsum += w[q] * O.flux("rusanov", V[q], V[q], nrm)
    tot = (R * vol).sum(axis=1)
    assert np.abs(tot + bsum).max() < 1e-12 * (np.abs(R) * vol).sum()
