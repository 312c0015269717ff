"""Adjoint of the residual (hfv_residual_vjp) and of SSP-RK3 trajectories.

Bars (FP64, classes frozen at the base state, central differences h = 1e-6):
  * lam^T dR/dU against central differences of the GPU residual along random
    directions: <= 1e-6 of the directional derivative's scale
  * against the gradient the oracle gives by central differences of its own
    residual, component by component: <= 1e-6 of max |g|
  * dJ/dU0 of J = sum |V| rho^2 after SSP-RK3 steps against central
    differences of the same trajectory: <= 1e-6
Every class (linear, CWENOZ, MUSCL, first order) is present in each case.
"""
import math

import numpy as np
import pytest

import oracle as O
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


def _mixed_state(m, seed):
    """A smooth wave on the quadrant states' density scale plus a moderate
    contact: smooth, weakly non-smooth and discontinuous cells."""
    c = m.vertex_means()
    rng = np.random.default_rng(seed)
    k = rng.uniform(1.0, 2.0, 2)
    rho = 1.0 + 0.2 * np.sin(2 * math.pi * (k[0] * c[:, 0] + k[1] * c[:, 1])) + np.where(c[:, 0] < 0.45, 0.3, 0.0)
    u = 0.3 + 0.1 * np.cos(2 * math.pi * c[:, 1])
    v = -0.2 + 0.1 * np.sin(2 * math.pi * c[:, 0])
    p = 1.0 + 0.1 * np.cos(2 * math.pi * (c[:, 0] - c[:, 1]))
    return I.conserved_2d(rho, u, v, p)


def _hex_state(m, seed):
    c = m.vertex_means()
    rng = np.random.default_rng(seed)
    k = rng.uniform(1.0, 2.0, 3)
    rho = 1.0 + 0.2 * np.sin(2 * math.pi * (c @ k)) + np.where(c[:, 1] < 0.5, 0.25, 0.0)
    vel = np.stack([0.3 + 0.1 * np.cos(2 * math.pi * c[:, 2]), -0.1 + 0.1 * np.sin(2 * math.pi * c[:, 0]),
                    0.2 * np.ones(len(c))])
    p = 1.0 + 0.1 * np.cos(2 * math.pi * (c[:, 0] - c[:, 2]))
    E = p / 0.4 + 0.5 * rho * (vel ** 2).sum(0)
    return np.stack([rho, rho * vel[0], rho * vel[1], rho * vel[2], E])


def _classes(n, seed):
    """Every class present: a seeded assignment (a forced linear or CWENOZ
    cell that breaks the Harten bound falls back to first order)."""
    return np.random.default_rng(seed).choice(4, n, p=[0.4, 0.25, 0.25, 0.1]).astype(np.uint8)


CASES = {
    "mixed_r2_hllc": (lambda: I.mixed_tri_quad_mesh(10, seed=4), _mixed_state, dict(order=3, flux="hllc")),
    "mixed_r3_rusanov": (lambda: I.mixed_tri_quad_mesh(10, seed=6), _mixed_state, dict(order=4, flux="rusanov")),
    "mixed_r4_hll": (lambda: I.mixed_tri_quad_mesh(12, seed=8), _mixed_state, dict(order=5, flux="hll")),
    "hex_r2_hllc": (lambda: I.structured_hex_mesh(5, 1.0, periodic=False, jitter=0.15, seed=5), _hex_state,
                    dict(order=3, flux="hllc")),
    "hex_r3_hllc": (lambda: I.structured_hex_mesh(6, 1.0, periodic=False, jitter=0.1, seed=7), _hex_state,
                    dict(order=4, flux="hllc")),
    "tet_r2_hllc": (lambda: I.structured_tet_mesh(4, 1.0, periodic=False, jitter=0.1, seed=8), _hex_state,
                    dict(order=3, flux="hllc")),
    "mixed3d_r2_hllc": (lambda: I.mixed_element_mesh(4, seed=7), _hex_state, dict(order=3, flux="hllc")),
}


def _setup(H, name):
    mk, st, kw = CASES[name]
    m = mk()
    U = st(m, 3)
    g = H.Scheme(H.Mesh(m), precision="fp64", **kw)
    cls = torch.tensor(_classes(m.n_cells, 5), device="cuda")
    return m, U, kw, g, cls


@pytest.mark.parametrize("name", list(CASES))
def test_vjp_against_central_differences(H, name):
    m, U, kw, g, cls = _setup(H, name)
    rng = np.random.default_rng(1)
    Ud = torch.tensor(U, device="cuda")
    lam = torch.tensor(rng.standard_normal(U.shape), device="cuda")
    grad = g.residual_vjp(Ud, cls, lam).cpu().numpy()
    h = 1e-6
    for k in range(3):
        d = rng.standard_normal(U.shape) * np.abs(U).mean(axis=1, keepdims=True) * 0.1
        Rp = g.residual(torch.tensor(U + h * d, device="cuda"), forced=cls).cpu().numpy()
        Rm = g.residual(torch.tensor(U - h * d, device="cuda"), forced=cls).cpu().numpy()
        fd = ((Rp - Rm) * lam.cpu().numpy()).sum() / (2 * h)
        an = (grad * d).sum()
        scale = (np.abs((Rp - Rm) * lam.cpu().numpy()).sum() / (2 * h))
        print(f"{name} dir {k}: fd {fd:.10e} adjoint {an:.10e} rel {abs(fd - an) / scale:.2e}")
        assert abs(fd - an) <= 1e-6 * scale, (fd, an, scale)


@pytest.mark.parametrize("name", ["mixed_r2_hllc", "hex_r2_hllc", "tet_r2_hllc", "mixed3d_r2_hllc"])
def test_vjp_against_oracle_gradient(H, name):
    """The oracle's gradient: central differences of the oracle's FP64
    residual (classes forced), one input at a time."""
    mk, st, kw = CASES[name]
    if name.startswith("mixed3d"):
        m = I.mixed_element_mesh(3, nz=2, seed=1, p_pyramid=0.6)   # every element type
    elif name.startswith("mixed"):
        m = I.mixed_tri_quad_mesh(5, seed=4)
    elif name.startswith("hex"):
        m = I.structured_hex_mesh(3, 1.0, periodic=False, jitter=0.15, seed=5)
    else:
        m = I.structured_tet_mesh(2, 1.0, periodic=False, jitter=0.1, seed=5)
    U = st(m, 3)
    cls_np = _classes(m.n_cells, 7)
    g = H.Scheme(H.Mesh(m), precision="fp64", **kw)
    # the classes the GPU ends with (Harten fallbacks) are the ones to force on the oracle
    fin = torch.empty(m.n_cells, dtype=torch.uint8, device="cuda")
    g.residual(torch.tensor(U, device="cuda"), forced=torch.tensor(cls_np, device="cuda"), class_out=fin)
    fin_np = fin.cpu().numpy()
    lam = np.random.default_rng(2).standard_normal(U.shape)
    grad = g.residual_vjp(torch.tensor(U, device="cuda"), fin, torch.tensor(lam, device="cuda")).cpu().numpy()
    osch = O.Scheme(O.Mesh(m), **kw)
    h = 1e-6
    ref = np.zeros_like(U)
    for v in range(U.shape[0]):
        for c in range(U.shape[1]):
            Up = U.copy(); Up[v, c] += h
            Um = U.copy(); Um[v, c] -= h
            Rp = osch.residual(Up, forced=fin_np)[0]
            Rm = osch.residual(Um, forced=fin_np)[0]
            ref[v, c] = ((Rp - Rm) * lam).sum() / (2 * h)
    err = np.abs(grad - ref).max() / np.abs(ref).max()
    print(f"{name}: {m.n_cells} cells, classes {np.bincount(fin_np, minlength=4)}, max rel err {err:.2e}")
    assert err <= 1e-6, err


@pytest.mark.parametrize("name", ["mixed_r2_hllc", "hex_r2_hllc"])
def test_rk3_trajectory_gradient(H, name):
    from paper_2510_25906_gb300 import adjoint as A
    mk, st, kw = CASES[name]
    m = mk()
    U = torch.tensor(st(m, 3), device="cuda")
    gm = H.Mesh(m)
    g = H.Scheme(gm, precision="fp64", **kw)
    J = A.density_square_integral(gm.volumes())
    dt = 0.4 * float(g.compute_dt(U, 0.5)[0].item())
    steps = 3
    Jv, dJ, UN, dts = A.rk3_gradient(g, U, steps, J, dt=dt)
    # the base trajectory's classes, frozen for the differences
    cls, W = [], U.clone()
    for _ in range(steps):
        _, _, W3, c = A._stages(g, W, dt)
        cls.append(c)
        W = W3.contiguous()

    def traj(U0):
        W = U0.clone()
        for c in cls:
            W = A._stages(g, W, dt, classes=c)[2].contiguous()
        return J(W)[0]

    rng = np.random.default_rng(4)
    h = 1e-6
    for k in range(2):
        d = torch.tensor(rng.standard_normal(U.shape), device="cuda") * U.abs().mean(dim=1, keepdim=True) * 0.1
        fd = (traj(U + h * d) - traj(U - h * d)) / (2 * h)
        an = float((dJ * d).sum().item())
        print(f"{name}: dJ fd {fd:.10e} adjoint {an:.10e} rel {abs(fd - an) / abs(fd):.2e}")
        assert abs(fd - an) <= 1e-6 * abs(fd)


def test_autograd_function_matches_vjp(H):
    from paper_2510_25906_gb300 import adjoint as A
    m, U, kw, g, _ = _setup(H, "mixed_r2_hllc")
    Ud = torch.tensor(U, device="cuda", requires_grad=True)
    R = A.ResidualFunction.apply(Ud, g)
    lam = torch.randn_like(R)
    (gr,) = torch.autograd.grad((R * lam).sum(), Ud)
    c = torch.empty(m.n_cells, dtype=torch.uint8, device="cuda")
    g.residual(Ud.detach(), class_out=c)
    ref = g.residual_vjp(Ud.detach(), c, lam)
    assert torch.equal(gr, ref)


def test_adjoint_workload_trajectory_gradient(H):
    """The adjoint workload's shape at 6 * 12^3 tetrahedra: a Gaussian pulse
    ahead of a planar Mach 2 shock, Venkatakrishnan's limiter (K = 5), ten
    CFL steps.  Along the density pulse (no cell at a tie of the limiter's
    bounds moves) the gradient matches central differences to 1e-6.  Along
    a random direction the piecewise-constant states on both sides of the
    shock put cells at ties of max / min (U_0 equal to a neighbour), where
    the frozen-branch derivative is one of the one-sided ones and central
    differences average them: the bar there is 1e-3."""
    from paper_2510_25906_gb300 import adjoint as A
    m, U0 = I.adjoint_problem(12)
    gm = H.Mesh(m)
    g = H.Scheme(gm, order=3, flux="hllc", precision="fp64", limiter="venkatakrishnan", venkat_k=5.0)
    J = A.density_square_integral(gm.volumes())
    U = torch.tensor(U0, device="cuda")
    steps = 10
    Jv, dJ, UN, dts = A.rk3_gradient(g, U, steps, J, cfl=0.5)
    assert torch.isfinite(dJ).all()
    cls, W = [], U.clone()
    for h_ in dts:
        _, _, W3, c = A._stages(g, W, h_)
        cls.append(c)
        W = W3.contiguous()
    hist = np.bincount(torch.cat([c for stage in cls for c in stage]).cpu().numpy(), minlength=4)
    assert (hist[1:] > 0).all(), hist

    def traj(U0_):
        W = U0_.clone()
        for c, h_ in zip(cls, dts):
            W = A._stages(g, W, h_, classes=c)[2].contiguous()
        return J(W)[0]

    cen = torch.tensor(m.vertex_means(), device="cuda")
    pulse = torch.zeros_like(U)
    pulse[0] = torch.exp(-((cen - torch.tensor([0.75, 0.5, 0.5], device="cuda")) ** 2).sum(1) / (2 * 0.08 ** 2))
    rng = np.random.default_rng(1)
    rand = torch.tensor(rng.standard_normal(U.shape), device="cuda") * U.abs().mean(dim=1, keepdim=True)
    for d, bar in ((pulse, 1e-6), (rand, 1e-3)):
        fd = (traj(U + 1e-6 * d) - traj(U - 1e-6 * d)) / 2e-6
        an = float((dJ * d).sum().item())
        print(f"adjoint workload: fd {fd:.10e} adjoint {an:.10e} rel {abs(fd - an) / abs(fd):.2e}")
        assert abs(fd - an) <= bar * abs(fd)
