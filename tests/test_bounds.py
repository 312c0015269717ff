"""The FP32 parity bar's helpers (tests/bounds.py) on the CPU: the relative
error they take, and the bar max(1e-5, 8 E_in) on a well-conditioned case (a
discontinuous quadrant problem: the plain 1e-5) and an ill-conditioned one
(the smooth density wave, whose residual is small next to its fluxes)."""
import numpy as np

import oracle as O
from bounds import FP32_INPUT_FACTOR, fp32_bar, rel_err, rounded
from paper_2510_25906_gb300 import inputs as I


def test_rel_err_is_per_variable_and_masked():
    B = np.array([[1.0, -2.0, 0.5], [0.0, 0.0, 0.0], [10.0, 10.0, 10.0]])
    A = B.copy()
    assert rel_err(A, B) == 0.0
    A[0, 1] += 0.02                      # 0.01 of variable 0's max |B| = 2
    A[2, 0] += 0.05                      # 0.005 of variable 2's 10
    A[1, 2] = 1e-3                       # a variable that is zero everywhere: absolute
    assert abs(rel_err(A, B) - 1e-2) < 1e-15
    # the scale is taken over the selected cells too
    assert abs(rel_err(A, B, cells=[0, 2]) - 5e-3) < 1e-15
    assert abs(rel_err(A, B, cells=[1]) - 1e-2) < 1e-15
    mask = np.array([True, False, False])
    assert abs(rel_err(A, B, cells=mask) - 5e-3) < 1e-15


def test_rounded_is_the_fp32_state():
    U = np.array([[1.0, 1.0 + 2.0 ** -30, np.pi]])
    r = rounded(U)
    assert r.dtype == np.float64 and r[0, 0] == 1.0 and r[0, 1] == 1.0
    assert r[0, 2] == float(np.float32(np.pi))


def _bar(mesh, U, **kw):
    s = O.Scheme(O.Mesh(mesh), **kw)
    R, _, _, fin = s.residual(U)
    Rr = s.residual(rounded(U), forced=fin)[0]
    return fp32_bar(R, Rr)


def test_bar_is_plain_on_a_discontinuous_case_and_rises_on_a_smooth_one():
    m = I.mixed_tri_quad_mesh(24, seed=2)
    bar, e_in = _bar(m, I.quadrant_state(m), order=3, flux="hllc")
    assert bar == 1e-5 and 0.0 < e_in < 1e-5 / FP32_INPUT_FACTOR
    m = I.structured_tri_mesh(32, periodic=True, jitter=0.2, seed=1)
    bar, e_in = _bar(m, I.density_wave_state(m), order=3, flux="rusanov")
    assert 1e-5 < e_in < 1e-4 and bar == FP32_INPUT_FACTOR * e_in
