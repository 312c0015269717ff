"""Parity of the paper's variants on the GPU against the oracle: the
SSP-RK(5,4) step of Spiteri and Ruuth and Venkatakrishnan's MUSCL limiter.

Bars: one SSP-RK(5,4) step 1e-12 (FP64) and 1e-5 (FP32 residuals, FP64
accumulation) of max |U| per variable; forced-class residuals with the
Venkatakrishnan limiter 1e-12 (FP64) / 1e-5 (FP32) of max |R| per variable;
the adjoint with that limiter against central differences (1e-6)."""
import math

import numpy as np
import pytest

import oracle as O
from bounds import fp32_bar, rounded
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


def _quadrant(n=24, seed=2, periodic=False):
    m = I.mixed_tri_quad_mesh(n, seed=seed, periodic=periodic)
    return m, I.quadrant_state(m)


def _hex():
    m = I.structured_hex_mesh(8, 2 * math.pi, periodic=True)
    U = I.turbulence_state(m, seed=3)
    x = m.vertex_means()[:, 0]
    fac = np.where(x < math.pi, 1.0, 0.5)
    ke = 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]
    p = 0.4 * (U[4] - ke)
    U[0] *= fac
    U[1:4] *= fac
    U[4] = p / 0.4 + ke * fac
    return m, U


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_ssprk54_step(H, precision, tol):
    m, U = _quadrant()
    kw = dict(order=3, flux="hllc")
    osch = O.Scheme(O.Mesh(m), **kw)
    U = osch.rk3_step(U, osch.dt(U, 0.5))       # develop some structure first
    dt = osch.dt(U, 0.5)
    Uo = osch.rk54_step(U, dt)
    g = H.Scheme(H.Mesh(m), precision=precision, time_scheme="ssprk54", **kw)
    Ug = torch.tensor(U, device="cuda")
    g.step(Ug, dt=dt)
    scale = np.abs(Uo).max(axis=1, keepdims=True)
    err = (np.abs(Ug.cpu().numpy() - Uo) / scale).max()
    print(f"SSP-RK(5,4) {precision}: max rel err {err:.2e}")
    assert err <= tol, err
    # a different step from SSP-RK3 (the stages are really taken)
    Ur = osch.rk3_step(U, dt)
    diff = np.abs(Ur - Uo).max() / np.abs(Uo).max()
    assert diff > 1e-6 and diff > 100 * err, (diff, err)


def test_ssprk54_cfl_step_matches_oracle_dt(H):
    m, U = _quadrant(16)
    kw = dict(order=3, flux="hllc")
    osch = O.Scheme(O.Mesh(m), **kw)
    g = H.Scheme(H.Mesh(m), precision="fp64", time_scheme="ssprk54", **kw)
    Ug = torch.tensor(U, device="cuda")
    used = g.step(Ug, cfl=0.5, want_dt=True)
    assert abs(used - osch.dt(U, 0.5)) <= 1e-14 * used
    Uo = osch.rk54_step(U, used)
    scale = np.abs(Uo).max(axis=1, keepdims=True)
    assert (np.abs(Ug.cpu().numpy() - Uo) / scale).max() <= 1e-12


@pytest.mark.parametrize("case", ["quadrant", "hex"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_venkatakrishnan_forced_class_residual(H, case, precision, tol):
    if case == "quadrant":
        m, U = _quadrant()
        kw = dict(order=3, flux="hllc", limiter="venkatakrishnan", venkat_k=5.0)
    else:
        m, U = _hex()
        kw = dict(order=3, flux="hllc", limiter="venkatakrishnan", venkat_k=0.5, kappa=0.1)
    osch = O.Scheme(O.Mesh(m), **kw)
    # MUSCL on every flagged cell: the limiter is what is compared
    fin = osch.residual(U)[3]
    forced = np.where(fin == 1, 2, fin).astype(np.uint8)
    Ro, _, _, fo = osch.residual(U, forced=forced)
    assert (fo == 2).sum() > 10
    g = H.Scheme(H.Mesh(m), precision=precision, **kw)
    dt = torch.float64 if precision == "fp64" else torch.float32
    cls = torch.empty(m.n_cells, dtype=torch.uint8, device="cuda")
    R = g.residual(torch.tensor(U, dtype=dt, device="cuda"), forced=torch.tensor(fo, device="cuda"),
                   class_out=cls).double().cpu().numpy()
    assert np.array_equal(cls.cpu().numpy(), fo)
    scale = np.abs(Ro).max(axis=1)
    err = (np.abs(R - Ro).max(axis=1) / scale).max()
    print(f"Venkatakrishnan {case} {precision}: {(fo == 2).sum()} MUSCL cells, max rel err {err:.2e}")
    assert err <= tol, err


def _smooth_with_contact(m):
    """No two cells share a value (a piecewise-constant state has ties in the
    limiter's max / min, where the frozen-branch derivative and central
    differences legitimately differ)."""
    c = m.vertex_means()
    rho = 1.0 + 0.2 * np.sin(2 * math.pi * (1.3 * c[:, 0] + 1.7 * c[:, 1])) + np.where(c[:, 0] < 0.45, 0.3, 0.0)
    u = 0.3 + 0.1 * np.cos(2 * math.pi * c[:, 1])
    v = -0.2 + 0.1 * np.sin(2 * math.pi * c[:, 0])
    p = 1.0 + 0.1 * np.cos(2 * math.pi * (c[:, 0] - c[:, 1]))
    return I.conserved_2d(rho, u, v, p)


def test_venkatakrishnan_adjoint_against_central_differences(H):
    m = I.mixed_tri_quad_mesh(10, seed=4)
    U = _smooth_with_contact(m)
    g = H.Scheme(H.Mesh(m), precision="fp64", order=3, flux="hllc", limiter="venkatakrishnan", venkat_k=5.0)
    cls = torch.tensor(np.random.default_rng(5).choice([0, 2], m.n_cells, p=[0.5, 0.5]).astype(np.uint8),
                       device="cuda")
    rng = np.random.default_rng(1)
    lam = torch.tensor(rng.standard_normal(U.shape), device="cuda")
    grad = g.residual_vjp(torch.tensor(U, device="cuda"), cls, lam).cpu().numpy()
    h = 1e-6
    for _ in range(3):
        d = rng.standard_normal(U.shape) * np.abs(U).mean(axis=1, keepdims=True) * 0.1
        Rp = g.residual(torch.tensor(U + h * d, device="cuda"), forced=cls).cpu().numpy()
        Rm = g.residual(torch.tensor(U - h * d, device="cuda"), forced=cls).cpu().numpy()
        fd = ((Rp - Rm) * lam.cpu().numpy()).sum() / (2 * h)
        scale = np.abs((Rp - Rm) * lam.cpu().numpy()).sum() / (2 * h)
        an = (grad * d).sum()
        assert abs(fd - an) <= 1e-6 * scale, (fd, an)


@pytest.mark.parametrize("case", ["quadrant", "hex", "tet"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_characteristic_cweno_forced_class_residual(H, case, precision, tol):
    """CWENOZ in characteristic variables (per face, projected with the
    eigenvectors of the flux Jacobian along its normal) against the oracle,
    every flagged cell forced to CWENOZ."""
    if case == "quadrant":
        m, U = _quadrant()
        kw = dict(order=3, flux="hllc", cweno_vars="characteristic")
    elif case == "hex":
        m, U = _hex()
        kw = dict(order=3, flux="hllc", cweno_vars="characteristic", kappa=0.1)
    else:
        m = I.structured_tet_mesh(4, 1.0, periodic=False, jitter=0.1, seed=6)
        U = _smooth_3d(m)
        kw = dict(order=3, flux="hllc", cweno_vars="characteristic")
    osch = O.Scheme(O.Mesh(m), **kw)
    fin = osch.residual(U)[3]
    forced = np.where(fin == 2, 1, fin).astype(np.uint8)
    Ro, _, _, fo = osch.residual(U, forced=forced)
    assert (fo == 1).sum() > 10
    g = H.Scheme(H.Mesh(m), precision=precision, **kw)
    dt = torch.float64 if precision == "fp64" else torch.float32
    cls = torch.empty(m.n_cells, dtype=torch.uint8, device="cuda")
    R = g.residual(torch.tensor(U, dtype=dt, device="cuda"), forced=torch.tensor(fo, device="cuda"),
                   class_out=cls).double().cpu().numpy()
    ok = cls.cpu().numpy() == fo
    if precision == "fp64":
        assert ok.all()
    ref = Ro
    if precision == "fp32":
        # against the oracle on the same FP32-rounded state (bounds.fp32_bar)
        ref = osch.residual(rounded(U), forced=fo)[0]
        tol, e_in = fp32_bar(Ro, ref, tol)
    assert ok.mean() >= 0.999
    scale = np.abs(ref).max(axis=1)
    err = (np.abs(R - ref)[:, ok].max(axis=1) / scale).max()
    print(f"characteristic CWENOZ {case} {precision}: {(fo == 1).sum()} CWENOZ cells, max rel err {err:.2e}, "
          f"bar {tol:.1e}")
    assert err <= tol, err
    # the characteristic form really differs from the conserved one here
    Rc = O.Scheme(O.Mesh(m), **{**kw, "cweno_vars": "conserved"}).residual(U, forced=fo)[0]
    assert np.abs(Rc - Ro).max() > 1e-8 * np.abs(Ro).max()


def _smooth_3d(m):
    c = m.vertex_means()
    rho = 1.0 + 0.05 * np.sin(2 * math.pi * (c[:, 0] + c[:, 2])) + np.where(c[:, 1] < 0.5, 0.5, 0.0)
    vel = np.stack([0.3 + 0.1 * np.cos(2 * math.pi * c[:, 2]), 0.1 * np.sin(2 * math.pi * c[:, 0]),
                    -0.2 * np.ones(len(c))])
    E = 1.0 / 0.4 + 0.5 * rho * (vel ** 2).sum(0)
    return np.stack([rho, rho * vel[0], rho * vel[1], rho * vel[2], E])


def test_adjoint_rejects_characteristic_cweno(H):
    m, U = _quadrant(8)
    g = H.Scheme(H.Mesh(m), precision="fp64", order=3, cweno_vars="characteristic")
    Ud = torch.tensor(U, device="cuda")
    cls = torch.zeros(m.n_cells, dtype=torch.uint8, device="cuda")
    with pytest.raises(H.HfvError) as e:
        g.residual_vjp(Ud, cls, torch.ones_like(Ud))
    assert e.value.code == H.HFV_ERR_ARG
