"""How close a cell sits to a decision of the detector or of the Harten bound
(Sec. 2.4, 2.5), for listing free-running class mismatches with their
margins.  Computed from the oracle's own linear candidate and cell means:

* detector: over the checked variables (density, pressure) that are not
  deactivated and the face points, the smallest distance of U(x) to a class
  boundary -- min - delta_m, min - delta_w, max + delta_w, max + delta_m,
  with min / max over the cell and its face neighbours -- relative to that
  variable's local range (infinite when every variable is deactivated);
* deactivation: |spread - (kappa dx)^n| relative to the threshold, spread =
  max - min of |U_j - U_i| over the face neighbours;
* harten: over density and pressure of the final face values, the smallest
  |theta max(|q_bar|, eps) - |q - q_bar|| relative to theta max(|q_bar|, eps).

A mismatch between two implementations of the same decision is expected only
where one of these is at rounding level.  Diagnostic only: the parity tests
print it and never assert on it.
"""
import numpy as np

import oracle as O


def _pressure(W, d, gamma):
    W = np.atleast_2d(W)
    return (gamma - 1.0) * (W[:, d + 1] - 0.5 * (W[:, 1:d + 1] ** 2).sum(axis=1) / W[:, 0])


def detector_margins(osch, U, c, nbr, vol, cls=None):
    """(detector, deactivation, harten) relative margins of cell c; nbr and
    vol from the oracle mesh (connectivity, geometry); cls the cell's class
    before the Harten bound (linear, CWENOZ or MUSCL: the face values the bound
    is checked on; default the linear candidate)."""
    p = osch.params
    d = osch.dim
    g = p["gamma"]
    u = U[:, c]
    nb = [int(j) for j in nbr[c] if j >= 0]
    V = osch.reconstruct(U, c, O.LIN)
    dx = vol[c] ** (1.0 / d)
    thr = (p["kappa"] * dx) ** p["n_exp"]
    q_of = [lambda X: np.atleast_2d(X)[:, 0], lambda X: _pressure(X, d, g)]
    det, deact = np.inf, np.inf
    for q in q_of:
        qi = q(u[None, :])[0]
        qn = np.array([q(U[:, j][None, :])[0] for j in nb])
        lo, hi = min(qi, qn.min()), max(qi, qn.max())
        dd = np.abs(qn - qi)
        spread = dd.max() - dd.min()
        deact = min(deact, abs(spread - thr) / thr if thr > 0 else np.inf)
        if spread < thr:
            continue                       # deactivated: the detector does not look at this variable
        rng = hi - lo
        dm = max(p["alpha_m"], p["beta_m"] * rng)
        sg = np.sign(p["beta_w"])
        dw = sg * max(p["alpha_w"], abs(p["beta_w"] * rng))
        scale = rng if rng > 0 else max(abs(qi), 1e-300)
        for x in q(V):
            for t in (lo - dm, lo - dw, hi + dw, hi + dm):
                det = min(det, abs(x - t) / scale)
    harten = np.inf
    th, ep = p["harten_theta"], p["harten_eps"]
    Vh = osch.reconstruct(U, c, cls) if cls in (O.LIN, O.CW, O.MU) else V
    for q in q_of:
        qb = q(u[None, :])[0]
        lim = th * max(abs(qb), ep)
        for x in q(Vh):
            harten = min(harten, abs(lim - abs(x - qb)) / lim)
    return det, deact, harten
