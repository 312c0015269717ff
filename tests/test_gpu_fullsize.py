"""Parity at the benchmark sizes, in the benchmark's launch configuration.

The GPU computes the whole mesh (hfv_residual, free-running detector); the
FP64 oracle computes a sample of cells (plus the two face layers they depend
on).  Sampled cells are taken near the discontinuities and at random.
Bars: class agreement >= 99.9 % on the sample, residuals where the class of a
cell and of its face neighbours agree: 1e-12 (FP64) and 1e-5 (FP32) of the
largest |R| over the sample per variable; on the smooth-dominated 3D field
the FP32 bar is the bound of the FP32 arithmetic (fp32_bound), since its
residuals are small next to the face fluxes they are the difference of."""
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


_oracle = {}


def _sample(rng, near, n, k_near, k_rand):
    cand = np.nonzero(near)[0]
    pick = rng.choice(cand, min(k_near, cand.size), replace=False)
    rand = rng.choice(n, k_rand, replace=False)
    return np.unique(np.concatenate([pick, rand])).astype(np.int64)


def _oracle_run(key, mesh, U, kw, smp):
    """The oracle's sampled residual, computed once per workload and order,
    and max_c sum_f |S_f| / |V_c| for the FP32 arithmetic bound."""
    if key not in _oracle:
        om = O.Mesh(mesh)
        Ro, raw, tag, fin = O.Scheme(om, **kw).residual(U, sample=smp)
        nbr, _ = om.connectivity()
        vol, _ = om.geometry()
        fo, fn, nrm, area, sh = om.faces()
        ssum = np.zeros(mesh.n_cells)
        np.add.at(ssum, fo, area)
        np.add.at(ssum, fn[fn >= 0], area[fn >= 0])
        _oracle[key] = (Ro, fin, nbr, (ssum / vol).max())
    return _oracle[key]


def fp32_bound(U, s_over_v, rmax):
    """FP32 bound relative to max |R| of a variable: rounding the state and
    the face fluxes to FP32 moves each face flux by ~eps32 |F|; the residual
    sums them with weights |S| w / |V|:  4 eps32 (4 max|U|) max(sum |S| / |V|) / max|R|."""
    return 4 * 6e-8 * 4 * np.abs(U).max() * s_over_v / rmax


def _check(H, mesh, U, kw, precision, near, n_near, n_rand, tol, seed, key, smooth=False):
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
    Ro, fin, nbr, s_over_v = _oracle_run(key, mesh, U, kw, smp)
    agree = (cg[smp] == fin[smp]).mean()
    assert agree >= 0.999, (agree, [(int(c), int(cg[c]), int(fin[c])) for c in smp[cg[smp] != fin[smp]][:10]])
    good = np.array([cg[c] == fin[c] and all(cg[j] == fin[j] for j in nbr[c] if j >= 0 and fin[j] != 255)
                     for c in smp])
    scale = np.abs(Ro[:, smp]).max(axis=1)
    per_var = np.abs(Rg[:, smp] - Ro[:, smp])[:, good].max(axis=1) / scale
    err = per_var.max()
    if precision == "fp32" and smooth:
        # residuals of smooth flow are small next to the face fluxes they are
        # the difference of: the bar is the FP32 arithmetic bound
        tol = max(tol, fp32_bound(U, s_over_v, scale).max())
    print(f"{mesh.name} {kw} {precision}: {smp.size} sampled cells, classes {np.bincount(fin[smp], minlength=4)}, "
          f"agreement {agree:.4f}, max rel err {err:.2e} per variable {np.array2string(per_var, precision=2)} "
          f"max|R| {np.array2string(scale, precision=3)} bar {tol:.1e}")
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
    _check(H, mesh, U, dict(order=4, flux="hllc"), precision, near, 40, 24, tol, seed=11, key=("turbulence", 4),
           smooth=True)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_mixed_elements_full_size(H, precision, tol):
    """The 3D mixed-element workload (250,828 tetrahedra, prisms, pyramids and
    hexahedra), order 3, the Mach 2 shock ahead of the density pulse; sampled
    near the shock and at random.  FP32 bar: the larger of 1e-5 and the
    bound of the FP32 arithmetic (tetrahedra and pyramids have the largest
    surface-to-volume ratios)."""
    mesh = I.mixed_element_mesh(48)
    U = I.shock_pulse_state(mesh)
    near = np.abs(mesh.vertex_means()[:, 0] - 0.4) < 3.0 / 48
    _check(H, mesh, U, dict(order=3, flux="hllc"), precision, near, 300, 300, tol, seed=11, key=("mixed", 3),
           smooth=True)
