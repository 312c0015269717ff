"""Tolerances derived from the arithmetic (shared by the GPU parity tests)."""
import numpy as np


def fp32_bound(m, om, U, R):
    """Arithmetic bound of an FP32 residual relative to max |R|: rounding the
    state to FP32 moves every face flux by ~eps32 |F|, and the residual sums
    them with weights |S| w / |V|:  c * eps32 * max_c sum_f |S_f| |F| / |V_c|."""
    vol, _ = om.geometry()
    fo, fn, nrm, area, sh = om.faces()
    ssum = np.zeros(m.n_cells)
    np.add.at(ssum, fo, area)
    np.add.at(ssum, fn[fn >= 0], area[fn >= 0])
    fscale = np.abs(U).max() * 4.0
    return (4 * 6e-8 * fscale * (ssum / vol).max()) / np.abs(R).max(axis=1).min()
