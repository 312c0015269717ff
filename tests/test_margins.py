"""The margin diagnostic of tests/margins.py on cases whose margins are known:
a density contact at the deactivation flip (kappa = J^(1/n) / h, margin 0 up
to the kappa offset), well away from it, and a uniform state."""
import numpy as np

import oracle as O
from margins import detector_margins
from paper_2510_25906_gb300 import inputs as I


def _contact():
    nx, ny = 24, 12
    m = I.structured_quad_mesh(nx, ny, 1.0, 0.5, periodic=(False, True))
    vm = m.vertex_means()
    one = np.ones(m.n_cells)
    U = I.conserved_2d(np.where(vm[:, 0] < 0.5, 1.0, 0.125), 0 * one, 0 * one, one)
    return m, U, 1.0 / nx, 0.875, 11          # mesh, state, h, jump, a cell at the jump (row 0)


def test_deactivation_margin_vanishes_at_the_flip():
    m, U, h, J, c = _contact()
    om = O.Mesh(m)
    nbr, _ = om.connectivity()
    vol, _ = om.geometry()
    for n_exp in (1.0, 2.0):
        k_flip = J ** (1.0 / n_exp) / h
        s = O.Scheme(om, order=3, flux="hllc", kappa=k_flip * (1 - 1e-9), n_exp=n_exp)
        det, deact, _ = detector_margins(s, U, c, nbr, vol)
        assert deact < 1e-8 and np.isfinite(det)      # density still active, just below the flip
        s = O.Scheme(om, order=3, flux="hllc", kappa=k_flip * (1 + 1e-9), n_exp=n_exp)
        det, deact, _ = detector_margins(s, U, c, nbr, vol)
        assert deact < 1e-8 and det == np.inf         # just above it: deactivated
        s2 = O.Scheme(om, order=3, flux="hllc", kappa=2 * k_flip, n_exp=n_exp)
        _, deact2, _ = detector_margins(s2, U, c, nbr, vol)
        assert abs(deact2 - (1.0 - 2.0 ** -n_exp)) < 1e-9      # |J - 2^n J| / (2^n J)


def test_margins_of_a_uniform_state():
    """Uniform flow: every neighbour difference is zero (deactivation margin
    = thr / thr = 1, so the detector is not consulted: infinite margin) and
    the face values equal the mean (Harten margin 1)."""
    m = I.structured_quad_mesh(8, 8, periodic=(True, True))
    one = np.ones(m.n_cells)
    U = I.conserved_2d(one, 0.3 * one, 0 * one, one)
    om = O.Mesh(m)
    nbr, _ = om.connectivity()
    vol, _ = om.geometry()
    s = O.Scheme(om, order=3)
    det, deact, harten = detector_margins(s, U, 20, nbr, vol, cls=O.LIN)
    assert abs(deact - 1.0) < 1e-12 and abs(harten - 1.0) < 1e-12 and det == np.inf
