"""The seeded synthetic inputs are what their recipe says: cell counts and
element mixes, the states' defining properties (periodic mean, uniform
sound speed, a divergence-free velocity at the stated turbulent Mach number
with its spectral peak at k0, shock states that satisfy the Rankine-Hugoniot
conditions), and open or periodic boundaries as stated."""
import math

import numpy as np

from paper_2510_25906_gb300 import inputs as I

G = 1.4


def _prim(U, d):
    rho = U[0]
    vel = U[1:d + 1] / rho
    p = (G - 1.0) * (U[d + 1] - 0.5 * rho * (vel ** 2).sum(0))
    return rho, vel, p


def _areas(m):
    out = np.zeros(m.n_cells)
    for c in range(m.n_cells):
        v = m.cell_vertices(c)
        x, y = v[:, 0], v[:, 1]
        out[c] = 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))
    return out


def test_density_wave_workload():
    m, U, d = I.workload("density_wave")
    assert m.n_cells == 2048 and (m.cell_type == I.TRI).all() and (m.period[:2] == 1.0).all()
    rho, vel, p = _prim(U, 2)
    assert np.allclose(vel, 1.0, atol=1e-12) and np.allclose(p, 1.0, atol=1e-12)
    # the cell averages of 1 + 0.2 sin(2 pi (x + y)) over a periodic domain average to 1
    a = _areas(m)
    assert abs(a.sum() - 1.0) < 1e-13 and abs((a * rho).sum() - 1.0) < 1e-12
    assert 1.19 < rho.max() < 1.2 and 0.8 < rho.min() < 0.81
    assert d == {"order": 3, "flux": "rusanov", "cfl": 0.5, "steps": 10}


def test_quadrant_workload():
    m, U, d = I.workload("quadrant")
    ntri = int((m.cell_type == I.TRI).sum())
    assert m.n_cells == 249_601 and (ntri, m.n_cells - ntri) == (166_274, 83_327)
    assert (m.period == 0).all()
    rho, vel, p = _prim(U, 2)
    states = np.unique(np.round(np.stack([rho, vel[0], vel[1], p], axis=1), 12), axis=0)
    assert states.shape[0] == 4                                    # four constant quadrants
    assert d["order"] == 3 and d["flux"] == "hllc"


def test_solenoidal_velocity():
    """rms |u| = M_t c; the sampled field's spectral divergence vanishes; the
    shell spectrum peaks at k0 (E(k) ~ k^4 exp(-2 k^2 / k0^2) peaks there)."""
    n, k0 = 32, 4.0
    u = I.solenoidal_velocity(n, seed=3, k0=k0, mach_t=0.6)
    assert u.shape == (3, n, n, n)
    assert abs(math.sqrt((u * u).sum(0).mean()) - 0.6) < 1e-12
    uh = np.fft.fftn(u, axes=(1, 2, 3))
    kk = np.fft.fftfreq(n, d=1.0 / n)
    KZ, KY, KX = np.meshgrid(kk, kk, kk, indexing="ij")
    div = KX * uh[0] + KY * uh[1] + KZ * uh[2]
    # the Nyquist planes (a component at n/2, where +k and -k are one sample
    # frequency) are left out: the real part of the field folds them
    inner = (np.abs(KX) < n // 2) & (np.abs(KY) < n // 2) & (np.abs(KZ) < n // 2)
    assert np.abs(div[inner]).max() <= 1e-12 * np.abs(uh).max() * n
    kmag = np.rint(np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)).astype(int)
    e = np.bincount(kmag.ravel(), weights=(np.abs(uh) ** 2).sum(0).ravel())
    assert 3 <= int(np.argmax(e[1:n // 2])) + 1 <= 5


def test_turbulence_state_has_unit_sound_speed():
    m, U, d = I.workload("turbulence", scale=16)
    assert m.n_cells == 16 ** 3 and (m.cell_type == I.HEX).all()
    assert np.allclose(m.period, 2 * math.pi)
    rho, vel, p = _prim(U, 3)
    assert np.allclose(rho, 1.0) and np.allclose(p, 1.0 / G)      # c = sqrt(gamma p / rho) = 1
    assert abs(math.sqrt((vel ** 2).sum(0).mean()) - 0.6) < 1e-12
    assert d["order"] == 4 and d["flux"] == "hllc"


def test_mach2_shock_satisfies_rankine_hugoniot():
    """Mass, momentum and energy fluxes through the shock, in its frame
    (speed s = M c0 into gas at rest, rho0 = p0 = 1), balance."""
    post, pre = I.mach2_shock_states(G, 2.0)
    s = 2.0 * math.sqrt(G)
    r1, u1, p1 = post[0], post[1], post[4]
    r0, u0, p0 = pre[0], pre[1], pre[4]
    w1, w0 = u1 - s, u0 - s
    h = lambda r, p, w: G / (G - 1.0) * p / r + 0.5 * w * w
    assert abs(r1 * w1 - r0 * w0) < 1e-12
    assert abs(r1 * w1 * w1 + p1 - (r0 * w0 * w0 + p0)) < 1e-12
    assert abs(h(r1, p1, w1) - h(r0, p0, w0)) < 1e-12
    assert abs(r1 - 8.0 / 3.0) < 1e-12 and abs(p1 - 4.5) < 1e-12    # the textbook Mach 2 ratios at gamma 1.4


def test_adjoint_and_mixed_workloads():
    m, U = I.adjoint_problem(n=4)
    assert m.n_cells == 6 * 4 ** 3 and (m.cell_type == I.TET).all() and (m.period == 0).all()
    rho, vel, p = _prim(U, 3)
    post, pre = I.mach2_shock_states(G, 2.0)
    behind = m.vertex_means()[:, 0] < 0.4
    assert np.allclose(rho[behind], post[0]) and np.allclose(p[behind], post[4])
    assert np.allclose(p[~behind], 1.0) and np.allclose(vel[:, ~behind], 0.0)
    assert rho[~behind].max() > 1.05                               # the pulse
    mm = I.mixed_element_mesh(6)
    assert set(np.unique(mm.cell_type).tolist()) == {I.TET, I.PRISM, I.PYRAMID, I.HEX}


def test_batched_problems():
    P = I.batched_problems(count=24, seed=5)
    assert len(P) == 24
    kinds = {p["kind"] for p in P}
    assert kinds == {"sine", "sod"}
    for p in P:
        m = p["mesh"]
        assert 2 <= p["order"] <= 5 and (m.period == 0).all() and (m.cell_type == I.TRI).all()
        assert 900 <= m.n_cells <= 201_000
        rho, vel, pr = _prim(p["U"], 2)
        assert (rho > 0).all() and (pr > 0).all()
    again = I.batched_problems(count=24, seed=5)
    assert all(np.array_equal(a["U"], b["U"]) for a, b in zip(P, again))      # seeded
