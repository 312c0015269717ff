"""Parity at the benchmark sizes, in the benchmark's launch configuration.

The GPU computes the whole mesh (hfv_residual, free-running detector); the
FP64 oracle computes a sample of cells (plus the two face layers they depend
on).  Sampled cells are taken near the discontinuities and at random.
Bars: class agreement >= 99.9 % on the sample, residuals where the class of a
cell and of its face neighbours agree: 1e-12 (FP64) of the largest |R| over
the sample per variable; FP32 against the oracle on the same FP32-rounded
state (classes as the oracle's), max(1e-5, 8 E_in) with E_in the change of
the exact residual under that rounding (bounds.fp32_bar)."""
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


_oracle = {}


def _sample(rng, near, n, k_near, k_rand):
    cand = np.nonzero(near)[0]
    pick = rng.choice(cand, min(k_near, cand.size), replace=False)
    rand = rng.choice(n, k_rand, replace=False)
    return np.unique(np.concatenate([pick, rand])).astype(np.int64)


def _oracle_run(key, mesh, U, kw, smp):
    """The oracle's sampled residual, computed once per workload and order,
    and the same on the FP32-rounded state with the oracle's classes forced."""
    if key not in _oracle:
        om = O.Mesh(mesh)
        sch = O.Scheme(om, **kw)
        Ro, raw, tag, fin = sch.residual(U, sample=smp)
        forced = np.where(fin == 255, 0, fin).astype(np.uint8)
        Ro32 = sch.residual(rounded(U), forced=forced, sample=smp)[0]
        nbr, _ = om.connectivity()
        _oracle[key] = (Ro, Ro32, fin, nbr)
    return _oracle[key]


def _check(H, mesh, U, kw, precision, near, n_near, n_rand, tol, seed, key):
    rng = np.random.default_rng(seed)
    smp = _sample(rng, near, mesh.n_cells, n_near, n_rand)
    gm = H.Mesh(mesh)
    g = H.Scheme(gm, precision=precision, **kw)
    dt = torch.float32 if precision == "fp32" else torch.float64
    cls = torch.empty(mesh.n_cells, dtype=torch.uint8, device="cuda")
    Rg = g.residual(torch.tensor(U, dtype=dt, device="cuda"), class_out=cls).double().cpu().numpy()
    cg = cls.cpu().numpy()
    del g, gm
    torch.cuda.empty_cache()
    Ro, Ro32, fin, nbr = _oracle_run(key, mesh, U, kw, smp)
    e_in = 0.0
    if precision == "fp32":
        tol, e_in = fp32_bar(Ro, Ro32, tol, cells=smp)
        Ro = Ro32
    agree = (cg[smp] == fin[smp]).mean()
    assert agree >= 0.999, (agree, [(int(c), int(cg[c]), int(fin[c])) for c in smp[cg[smp] != fin[smp]][:10]])
    good = np.array([cg[c] == fin[c] and all(cg[j] == fin[j] for j in nbr[c] if j >= 0 and fin[j] != 255)
                     for c in smp])
    scale = np.abs(Ro[:, smp]).max(axis=1)
    per_var = np.abs(Rg[:, smp] - Ro[:, smp])[:, good].max(axis=1) / scale
    err = per_var.max()
    print(f"{mesh.name} {kw} {precision}: {smp.size} sampled cells, classes {np.bincount(fin[smp], minlength=4)}, "
          f"agreement {agree:.4f}, max rel err {err:.2e} per variable {np.array2string(per_var, precision=2)} "
          f"max|R| {np.array2string(scale, precision=3)} bar {tol:.1e} (input rounding {e_in:.1e})")
    assert err <= tol, err
    assert len(np.unique(fin[smp])) >= 2


@pytest.mark.parametrize("order,precision,tol", [(3, "fp64", 1e-12), (3, "fp32", 1e-5), (5, "fp64", 1e-12),
                                                 (5, "fp32", 1e-5)])
def test_quadrant_full_size(H, order, precision, tol):
    mesh, U, d = I.workload("quadrant")
    vm = mesh.vertex_means()
    near = (np.abs(vm[:, 0] - 0.5) < 3.0 / 408) | (np.abs(vm[:, 1] - 0.5) < 3.0 / 408)
    _check(H, mesh, U, dict(order=order, flux="hllc"), precision, near, 300, 300, tol, seed=order,
           key=("quadrant", order))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_turbulence_full_size(H, precision, tol):
    """128^3 hexahedra, order 4; the seeded solenoidal field plus a density
    jump across x = pi in pressure equilibrium (the detector flags the contact
    at t = 0)."""
    mesh, U, d = I.workload("turbulence")
    x = mesh.vertex_means()[:, 0]
    fac = np.where(x < math.pi, 1.0, 0.5)
    ke = 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]
    p = 0.4 * (U[4] - ke)
    U[0] *= fac
    U[1:4] *= fac
    U[4] = p / 0.4 + ke * fac
    h = 2 * math.pi / 128
    near = (np.abs(x - math.pi) < 3 * h) | (x < 3 * h) | (x > 2 * math.pi - 3 * h)
    _check(H, mesh, U, dict(order=4, flux="hllc"), precision, near, 40, 24, tol, seed=11, key=("turbulence", 4))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_mixed_elements_full_size(H, precision, tol):
    """The 3D mixed-element workload (250,828 tetrahedra, prisms, pyramids and
    hexahedra), order 3, the Mach 2 shock ahead of the density pulse; sampled
    near the shock and at random."""
    mesh = I.mixed_element_mesh(48)
    U = I.shock_pulse_state(mesh)
    near = np.abs(mesh.vertex_means()[:, 0] - 0.4) < 3.0 / 48
    _check(H, mesh, U, dict(order=3, flux="hllc"), precision, near, 300, 300, tol, seed=11, key=("mixed", 3))
