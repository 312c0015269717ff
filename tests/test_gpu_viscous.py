"""GPU parity of the viscous (Navier-Stokes) residual against the oracle.

Bars as for the Euler residual: forced classes 1e-12 (FP64) of max |R| per
variable; FP32 against the oracle on the same FP32-rounded state,
max(1e-5, 8 E_in) (bounds.fp32_bar).  On a smooth periodic flow the viscous
part alone, R(mu0) - R(0), is compared as well (1e-11 in FP64), so that a
mistake in it cannot hide under the convective fluxes.  A viscous SSP-RK3
step matches the oracle's step."""
import math

import numpy as np
import pytest

import oracle as O
from bounds import fp32_bar, rounded
from paper_2510_25906_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VISC = dict(mu0=0.02, t0=1.0, prandtl=0.72, visc_alpha=4.0 / 3.0)
S_SUTH = 110.4 / 288.15


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25906_gb300 import build as B
    B.build()
    import paper_2510_25906_gb300.hfv as H
    H.load()
    return H


def _smooth_2d(m):
    c = m.vertex_means()
    rho = 1 + 0.2 * np.sin(2 * np.pi * c[:, 0]) * np.cos(2 * np.pi * c[:, 1])
    u = 0.3 * np.sin(2 * np.pi * c[:, 1])
    v = 0.2 * np.cos(2 * np.pi * c[:, 0])
    p = 1 + 0.1 * np.cos(2 * np.pi * (c[:, 0] - c[:, 1]))
    return I.conserved_2d(rho, u, v, p)


def _smooth_3d(m, contact=True):
    c = m.vertex_means()
    rho = 1.0 + 0.05 * np.sin(2 * math.pi * (c[:, 0] + c[:, 2])) + (np.where(c[:, 1] < 0.5, 0.5, 0.0) if contact else 0)
    vel = np.stack([0.3 + 0.1 * np.cos(2 * math.pi * c[:, 2]), 0.1 * np.sin(2 * math.pi * c[:, 0]),
                    -0.2 + 0.1 * np.sin(2 * math.pi * c[:, 1])])
    p = 1.0 + 0.05 * np.cos(2 * math.pi * c[:, 1])
    E = p / 0.4 + 0.5 * rho * (vel ** 2).sum(0)
    return np.stack([rho, rho * vel[0], rho * vel[1], rho * vel[2], E])


def _case(name):
    if name == "quadrant_r2":
        m = I.mixed_tri_quad_mesh(20, seed=2)
        return m, I.quadrant_state(m), dict(order=3, flux="hllc")
    if name == "smooth_periodic_r3":
        m = I.mixed_tri_quad_mesh(16, seed=5, periodic=True)
        return m, _smooth_2d(m), dict(order=4, flux="rusanov")
    if name == "hex_r3":
        m = I.structured_hex_mesh(8, 1.0, periodic=True, jitter=0.0)
        return m, _smooth_3d(m), dict(order=4, flux="hllc", kappa=0.1)
    if name == "tet_r2":
        m = I.structured_tet_mesh(4, 1.0, periodic=False, jitter=0.1, seed=6)
        return m, _smooth_3d(m), dict(order=3, flux="hllc")
    if name == "mixed3d_r2":
        m = I.mixed_element_mesh(5, seed=7)
        return m, _smooth_3d(m), dict(order=3, flux="hll")
    raise KeyError(name)


CASES = ["quadrant_r2", "smooth_periodic_r3", "hex_r3", "tet_r2", "mixed3d_r2"]
_cache = {}


def _oracle(name):
    if name not in _cache:
        m, U, kw = _case(name)
        om = O.Mesh(m)
        osch = O.Scheme(om, suth_s=S_SUTH, **VISC, **kw)
        R, raw, tag, fin = osch.residual(U)
        R0 = O.Scheme(om, **kw).residual(U, forced=fin)[0]
        _cache[name] = (m, U, kw, osch, R, fin, R0)
    return _cache[name]


def _scheme(H, m, kw, precision, viscous=True):
    extra = dict(sutherland_s=S_SUTH, **VISC) if viscous else {}
    return H.Scheme(H.Mesh(m), precision=precision, **extra, **kw)


def _rel(a, b, mask=None):
    sc = np.abs(b).max(axis=1)
    sc[sc == 0] = 1
    d = np.abs(a - b)
    if mask is not None:
        d = d[:, mask]
    return (d.max(axis=1) / sc).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("name", CASES)
def test_viscous_forced_class_residual(H, name, precision, tol):
    m, U, kw, osch, R, fin, R0 = _oracle(name)
    assert np.abs(R - R0).max() > 1e-6 * np.abs(R).max()      # the viscous part is there
    g = _scheme(H, m, kw, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    cls = torch.empty(m.n_cells, dtype=torch.uint8, device="cuda")
    Rg = g.residual(torch.tensor(U, dtype=dt, device="cuda"), forced=torch.tensor(fin, device="cuda"),
                    class_out=cls).double().cpu().numpy()
    ok = cls.cpu().numpy() == fin
    assert ok.mean() >= 0.999 and (precision == "fp32" or ok.all())
    ref = R
    if precision == "fp32":
        ref = osch.residual(rounded(U), forced=fin)[0]
        tol, _ = fp32_bar(R, ref, tol)
    err = _rel(Rg, ref, ok)
    print(f"viscous {name} {precision}: classes {np.bincount(fin, minlength=4)}, max rel err {err:.2e} (bar {tol:.1e})")
    assert err <= tol, err


@pytest.mark.parametrize("name", ["smooth_periodic_r3", "hex_r3"])
def test_viscous_part_alone(H, name):
    """R(mu0) - R(0) with the same classes, GPU against oracle (FP64)."""
    m, U, kw, osch, R, fin, R0 = _oracle(name)
    Ug = torch.tensor(U, device="cuda")
    f = torch.tensor(fin, device="cuda")
    Rv = _scheme(H, m, kw, "fp64").residual(Ug, forced=f).cpu().numpy()
    Re = _scheme(H, m, kw, "fp64", viscous=False).residual(Ug, forced=f).cpu().numpy()
    dv_g, dv_o = Rv - Re, R - R0
    err = _rel(dv_g[1:], dv_o[1:])
    print(f"viscous part {name}: max |dv| {np.abs(dv_o).max():.3e}, rel err {err:.2e}")
    assert np.abs(dv_o[1:]).max() > 1e-3 and err <= 1e-11, err


def test_viscous_free_running_classes_and_step(H):
    m, U, kw, osch, R, fin, R0 = _oracle("quadrant_r2")
    g = _scheme(H, m, kw, "fp64")
    Ug = torch.tensor(U, device="cuda")
    cls = torch.empty(m.n_cells, dtype=torch.uint8, device="cuda")
    g.residual(Ug, class_out=cls)
    assert (cls.cpu().numpy() == fin).mean() >= 0.999
    # the CFL step with the viscous diffusion limit, as the oracle takes it
    dt = osch.dt(U, 0.5)
    used = g.step(Ug, cfl=0.5, want_dt=True)
    assert abs(used - dt) <= 1e-13 * dt, (used, dt)
    Uo = osch.rk3_step(U, used)
    assert np.isfinite(Uo).all()
    scale = np.abs(Uo).max(axis=1, keepdims=True)
    err = (np.abs(Ug.cpu().numpy() - Uo) / scale).max()
    print(f"viscous SSP-RK3 step: dt {used:.6e}, max rel err {err:.2e}")
    assert err <= 1e-12, err


def test_viscous_scheme_rejects_adjoint(H):
    m, U, kw, *_ = _oracle("smooth_periodic_r3")
    g = _scheme(H, m, kw, "fp64")
    Ug = torch.tensor(U, device="cuda")
    cls = torch.zeros(m.n_cells, dtype=torch.uint8, device="cuda")
    with pytest.raises(H.HfvError) as e:
        g.residual_vjp(Ug, cls, torch.ones_like(Ug))
    assert e.value.code == H.HFV_ERR_ARG
