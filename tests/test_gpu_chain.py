"""Chained steps (step_chain = 1): the last stage of a step writes the next
step's stage copy and time step, and the next hfv_step on the same state skips
its stage-in pass.  The results must be the same bits as unchained steps:
states and time steps, in CFL and fixed-step modes, on a batched mesh with one
time step per problem, and when the chain is broken by a residual call or by
stepping another state in between."""
import numpy as np
import pytest

from paper_2510_25906_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25906_gb300 import build as B
    B.build()
    import paper_2510_25906_gb300.hfv as H
    H.load()
    return H


def _run(g, U0, steps, cfl=0.5, dt=None, interleave=None):
    U = torch.tensor(U0, device="cuda")
    dts = []
    for k in range(steps):
        if dt is None:
            dts.append(g.step(U, cfl=cfl, want_dt=True))
        else:
            g.step(U, dt=dt)
        if interleave is not None:
            interleave(k, U)
    torch.cuda.synchronize()
    return U.cpu().numpy(), np.array(dts)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_chained_steps_are_bit_identical(H, precision):
    m = I.mixed_tri_quad_mesh(40, seed=2)
    U0 = I.quadrant_state(m)
    gm = H.Mesh(m)
    kw = dict(order=3, flux="hllc", precision=precision)
    g0 = H.Scheme(gm, **kw)
    g1 = H.Scheme(gm, step_chain=1, **kw)
    Ua, da = _run(g0, U0, 6)
    Ub, db = _run(g1, U0, 6)
    assert np.array_equal(da, db), (da, db)
    assert np.array_equal(Ua, Ub)
    # fixed step
    Ua, _ = _run(g0, U0, 4, dt=1e-4)
    Ub, _ = _run(g1, U0, 4, dt=1e-4)
    assert np.array_equal(Ua, Ub)


@pytest.mark.parametrize("case", ["hex_o4_fp32", "mixed3d_o3_fp32", "hex_o3_fp64"])
def test_chained_steps_are_bit_identical_in_3d(H, case):
    """the chained epilogue on eight-lane groups (hexahedra, mixed elements:
    up to six faces per cell), with a shock in the mixed case"""
    if case.startswith("hex"):
        m = I.structured_hex_mesh(12, jitter=0.1, seed=3)
        U0 = I.turbulence_state(m, seed=3)
        order = 4 if "o4" in case else 3
    else:
        m = I.mixed_element_mesh(6, seed=7)
        U0 = I.shock_pulse_state(m)
        order = 3
    kw = dict(order=order, flux="hllc", precision=case.rsplit("_", 1)[1])
    gm = H.Mesh(m)
    g0 = H.Scheme(gm, **kw)
    g1 = H.Scheme(gm, step_chain=1, **kw)
    Ua, da = _run(g0, U0, 4, cfl=0.4)
    Ub, db = _run(g1, U0, 4, cfl=0.4)
    assert np.array_equal(da, db), (da, db)
    assert np.array_equal(Ua, Ub)


def test_chain_broken_by_residual_and_by_another_state(H):
    m = I.mixed_tri_quad_mesh(32, seed=4)
    U0 = I.quadrant_state(m)
    gm = H.Mesh(m)
    g0 = H.Scheme(gm, order=3, flux="hllc", precision="fp32")
    g1 = H.Scheme(gm, order=3, flux="hllc", precision="fp32", step_chain=1)
    other = torch.tensor(I.quadrant_state(m)[:, ::-1].copy(), device="cuda")

    def meddle(g):
        def f(k, U):
            if k == 1:
                g.residual(U.float().contiguous())       # overwrites the stage copy
            if k == 3:
                g.step(other, cfl=0.5)                    # another state in between
        return f
    Ua, da = _run(g0, U0, 6, interleave=meddle(g0))
    Ub, db = _run(g1, U0, 6, interleave=meddle(g1))
    assert np.array_equal(da, db) and np.array_equal(Ua, Ub)


def test_chained_steps_on_a_batched_mesh(H):
    """one time step per problem: the chained minimum is per problem too"""
    P = I.batched_problems(6, seed=5, min_cells=800, max_cells=6000)
    orders = {}
    for p in P:
        orders.setdefault(p["order"], []).append(p)
    for order, ps in orders.items():
        gm = H.Mesh.batch([p["mesh"] for p in ps])
        U0 = np.concatenate([p["U"] for p in ps], axis=1)
        g0 = H.Scheme(gm, order=order, flux="hllc", precision="fp32")
        g1 = H.Scheme(gm, order=order, flux="hllc", precision="fp32", step_chain=1)
        Ua, da = _run(g0, U0, 4)
        Ub, db = _run(g1, U0, 4)
        assert np.array_equal(da, db), (order, da, db)
        assert np.array_equal(Ua, Ub), order
