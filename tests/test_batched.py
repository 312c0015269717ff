"""Batched problems: many independent open 2D meshes of uneven size and order.

A batch of problems is one mesh (hfv_mesh_create_batch) per order; problem k
is a run of consecutive cells.  Bars:
  * host: batched connectivity = each problem's connectivity, cell ids
    offset (bit-exact); the recipe's sizes, orders and states
  * oracle (host): the residual of a union of problems = each problem's own
    residual (no coupling), to the last bit
  * GPU: the residual, classes and one SSP-RK3 step of a batch equal those of
    the problems run one at a time (bit-exact, FP64 and FP32, each problem
    with its own CFL step); hfv_step_many (one stream per order) equals
    stepping the batches one after the other; the batch against the oracle
    with forced classes (1e-12 FP64) and free-running classes (>= 99.9 %)
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_25906_gb300 import build as B
from paper_2510_25906_gb300 import inputs as I


@pytest.fixture(scope="module")
def Hc():
    B.build()
    import paper_2510_25906_gb300.hfv as H
    H.load()
    return H


def _small_batch(count=7, seed=9):
    return I.batched_problems(count, seed=seed, min_cells=120, max_cells=1500, orders=(3,))


def test_batched_recipe_is_seeded_and_in_range():
    a = I.batched_problems(24, seed=5)
    b = I.batched_problems(24, seed=5)
    for p, q in zip(a, b):
        assert p["order"] == q["order"] and p["kind"] == q["kind"]
        assert np.array_equal(p["U"], q["U"]) and np.array_equal(p["mesh"].nodes, q["mesh"].nodes)
    cells = np.array([p["mesh"].n_cells for p in a])
    assert cells.min() >= 2 * 22 * 22 * 0.9 and cells.max() <= 200000 * 1.01
    assert set(p["order"] for p in a) <= {2, 3, 4, 5}
    assert set(p["kind"] for p in a) == {"sine", "sod"}
    for p in a:
        assert (p["mesh"].period == 0).all()
        rho, e = p["U"][0], p["U"][3]
        assert (rho > 0).all() and (e > 0).all()


def test_batched_connectivity_is_offset_concatenation(Hc):
    P = _small_batch()
    gm = Hc.Mesh.batch([p["mesh"] for p in P])
    nbr, nbrf = gm.connectivity()
    off = np.cumsum([0] + [p["mesh"].n_cells for p in P])
    assert np.array_equal(gm.segments, off)
    assert gm.n_segments == len(P)
    for k, p in enumerate(P):
        n1, f1 = Hc.Mesh(p["mesh"]).connectivity()
        exp = np.where(n1 >= 0, n1 + off[k], -1)
        assert np.array_equal(nbr[off[k]:off[k + 1]], exp), k
        assert np.array_equal(nbrf[off[k]:off[k + 1]], f1), k


def test_batched_mesh_rejects_periodic_and_mixed_dims(Hc):
    m_open = I.structured_tri_mesh(6, periodic=False)
    m_per = I.structured_tri_mesh(6, periodic=True)
    with pytest.raises(Hc.HfvError) as e:
        Hc.Mesh.batch([m_open, m_per])
    assert e.value.code == Hc.HFV_ERR_ARG
    m3 = I.structured_hex_mesh(3, 1.0, periodic=False)
    with pytest.raises(Hc.HfvError):
        Hc.Mesh.batch([m_open, m3])


def test_oracle_union_residual_equals_each_problem():
    """The oracle on a disjoint union of open meshes computes each problem's
    residual exactly: stencils, detector bounds and fluxes never cross."""
    P = _small_batch(4, seed=3)
    union = I.concat_meshes([p["mesh"] for p in P])
    U = np.concatenate([p["U"] for p in P], axis=1)
    Ru, _, _, fu = O.Scheme(O.Mesh(union), order=3, flux="hllc").residual(U)
    off = np.cumsum([0] + [p["mesh"].n_cells for p in P])
    for k, p in enumerate(P):
        Rk, _, _, fk = O.Scheme(O.Mesh(p["mesh"]), order=3, flux="hllc").residual(p["U"])
        assert np.array_equal(Ru[:, off[k]:off[k + 1]], Rk), k
        assert np.array_equal(fu[off[k]:off[k + 1]], fk), k


# --------------------------------------------------------------------------- GPU

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    import paper_2510_25906_gb300.hfv as H
    H.load()
    return H


def _groups(P):
    g = {}
    for k, p in enumerate(P):
        g.setdefault(p["order"], []).append(k)
    return g


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_residual_and_step_bit_exact(H, precision):
    P = I.batched_problems(12, seed=21, min_cells=200, max_cells=6000)
    dtp = torch.float64 if precision == "fp64" else torch.float32
    for order, ks in _groups(P).items():
        gm = H.Mesh.batch([P[k]["mesh"] for k in ks])
        gb = H.Scheme(gm, order=order, flux="hllc", precision=precision)
        Ub = np.concatenate([P[k]["U"] for k in ks], axis=1)
        cb = torch.empty(gm.n_cells, dtype=torch.uint8, device="cuda")
        Rb = gb.residual(torch.tensor(Ub, dtype=dtp, device="cuda"), class_out=cb).cpu().numpy()
        Us = torch.tensor(Ub, device="cuda")
        dtb = np.atleast_1d(gb.step(Us, cfl=0.5, want_dt=True))
        Us = Us.cpu().numpy()
        for j, k in enumerate(ks):
            a, b = gm.segments[j], gm.segments[j + 1]
            g1 = H.Scheme(H.Mesh(P[k]["mesh"]), order=order, flux="hllc", precision=precision)
            c1 = torch.empty(b - a, dtype=torch.uint8, device="cuda")
            R1 = g1.residual(torch.tensor(P[k]["U"], dtype=dtp, device="cuda"), class_out=c1).cpu().numpy()
            assert np.array_equal(Rb[:, a:b], R1), (order, k)
            assert np.array_equal(cb[a:b].cpu().numpy(), c1.cpu().numpy()), (order, k)
            U1 = torch.tensor(P[k]["U"], device="cuda")
            dt1 = g1.step(U1, cfl=0.5, want_dt=True)
            assert dtb[j] == dt1, (order, k, dtb[j], dt1)
            assert np.array_equal(Us[:, a:b], U1.cpu().numpy()), (order, k)


@pytest.mark.gpu
def test_step_many_equals_sequential_and_captures(H):
    P = I.batched_problems(10, seed=33, min_cells=200, max_cells=4000)
    groups = _groups(P)
    schemes, states, ref = [], [], []
    for order, ks in groups.items():
        gm = H.Mesh.batch([P[k]["mesh"] for k in ks])
        g = H.Scheme(gm, order=order, flux="hllc", precision="fp32")
        U0 = np.concatenate([P[k]["U"] for k in ks], axis=1)
        schemes.append(g)
        states.append(torch.tensor(U0, device="cuda"))
        Ur = torch.tensor(U0, device="cuda")
        for _ in range(2):
            g.step(Ur, cfl=0.5)
        ref.append(Ur.cpu().numpy())
    assert len(schemes) >= 2
    H.step_many(schemes, states, cfl=0.5)
    torch.cuda.synchronize()
    # the second step inside a CUDA graph (one branch per order)
    st = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        work = [s.clone() for s in states]
        with torch.cuda.graph(graph, stream=st):
            H.step_many(schemes, work, cfl=0.5, stream=st)
        for w, s in zip(work, states):
            w.copy_(s)
        graph.replay()
    torch.cuda.synchronize()
    for w, r in zip(work, ref):
        assert np.array_equal(w.cpu().numpy(), r)
    # a scheme listed twice would share its scratch between two branches
    with pytest.raises(H.HfvError) as e:
        H.step_many([schemes[0], schemes[0]], [states[0], states[0].clone()], cfl=0.5)
    assert e.value.code == H.HFV_ERR_ARG


@pytest.mark.gpu
def test_batched_against_oracle(H):
    """A batch of small order-3 problems against the oracle on their union."""
    P = _small_batch(6, seed=41)
    union = I.concat_meshes([p["mesh"] for p in P])
    U = np.concatenate([p["U"] for p in P], axis=1)
    Ro, raw, tag, fin = O.Scheme(O.Mesh(union), order=3, flux="hllc").residual(U)
    gm = H.Mesh.batch([p["mesh"] for p in P])
    g = H.Scheme(gm, order=3, flux="hllc", precision="fp64")
    forced = torch.tensor(fin, dtype=torch.uint8, device="cuda")
    R = g.residual(torch.tensor(U, device="cuda"), forced=forced).cpu().numpy()
    scale = np.abs(Ro).max(axis=1)
    assert (np.abs(R - Ro).max(axis=1) / scale).max() <= 1e-12
    cls = torch.empty(gm.n_cells, dtype=torch.uint8, device="cuda")
    g.residual(torch.tensor(U, device="cuda"), class_out=cls)
    agree = (cls.cpu().numpy() == fin).mean()
    assert agree >= 0.999, agree
    assert len(np.unique(fin)) >= 2


@pytest.mark.gpu
def test_autotune_keeps_results(H):
    """hfv_autotune changes launch shapes only: the residual is bit-identical
    before and after, and the chosen shape is within the candidate ranges."""
    P = I.batched_problems(8, seed=51, min_cells=2000, max_cells=20000, orders=(3,))
    gm = H.Mesh.batch([p["mesh"] for p in P])
    g = H.Scheme(gm, order=3, flux="hllc", precision="fp32")
    U = torch.tensor(np.concatenate([p["U"] for p in P], axis=1), dtype=torch.float32, device="cuda")
    R0 = g.residual(U).cpu().numpy()
    shape = g.autotune(U, reps=2)
    assert 1 <= shape[0] <= 8 and shape[1] in (2, 4, 8, 16, 32) and shape[2] in (50, 67, 75, 85, 95), shape
    assert shape[3] in (0, 1), shape
    R1 = g.residual(U).cpu().numpy()
    assert np.array_equal(R0, R1)


@pytest.mark.gpu
@pytest.mark.parametrize("order", [2, 3, 4])
def test_candidate_tile_shapes_give_the_same_bits(H, order):
    """The candidate kernel's two tile shapes (48-cell tiles at three CTAs
    per SM, 64-cell tiles at two; 2D FP32 orders 2-3) and any CTA count give
    the same residual bits; at order 4, which has one shape, the second
    falls back to it."""
    P = I.batched_problems(6, seed=53, min_cells=2000, max_cells=30000, orders=(order,))
    gm = H.Mesh.batch([p["mesh"] for p in P])
    g = H.Scheme(gm, order=order, flux="hllc", precision="fp32")
    U = torch.tensor(np.concatenate([p["U"] for p in P], axis=1), dtype=torch.float32, device="cuda")
    out = []
    for shape in ((0, 16, 75, 0), (0, 16, 75, 1), (1, 4, 50, 0), (1, 4, 50, 1)):
        g.set_shape(shape)
        cls = torch.empty(U.shape[1], dtype=torch.uint8, device="cuda")
        out.append((g.residual(U, class_out=cls).cpu().numpy(), cls.cpu().numpy()))
    for R, c in out[1:]:
        assert np.array_equal(R, out[0][0]) and np.array_equal(c, out[0][1])
    with pytest.raises(H.HfvError):
        g.set_shape((0, 16, 75, 2))
