"""The FP32 parity bar, derived from where FP32 rounding enters the path.

The FP32 path takes its state in FP32, so its residual is compared with the
oracle's FP64 residual of the same FP32-rounded state: the comparison then
measures the path's own arithmetic.  That arithmetic is bounded below by the
conditioning of the residual.  Every face-point state the path reconstructs
and stores in FP32 carries a relative rounding of ~eps32, and the residual is
a weighted sum of the face fluxes over the cell's faces, divided by |V|.
Where the residual is small next to the fluxes it is the difference of (smooth
flow; cells with a large surface-to-volume ratio), those roundings are
amplified by sum_f |F_f| |S_f| / (|V| max|R|).

E_in, the change of the exact (FP64) residual when its input is rounded to
FP32, measures that amplification on each case from the oracle alone.  On one
GB300 the path's arithmetic error measured 1.1 to 6.2 times E_in over every
forced-class parity case and the characteristic variants.  The same runs
showed where the error comes from: computing the Riemann fluxes and the face
sum in FP64, with IEEE division and square root or compensated sums, left it
unchanged.  Rounding only the oracle's FP64 face states to FP32 (a one-off
experiment) gave about half of E_in.  What remains is the FP32
reconstruction itself: the stored L operators and the candidate contraction
sum_m L_qm (U_m - U_0).

Bar: max(1e-5, FP32_INPUT_FACTOR * E_in).  Where the case is well conditioned
(8 E_in < 1e-5) this is the plain 1e-5."""
import numpy as np

FP32_INPUT_FACTOR = 8.0


def rounded(U):
    """the FP32 state the FP32 path receives, as FP64"""
    return np.asarray(U, np.float64).astype(np.float32).astype(np.float64)


def rel_err(A, B, cells=None):
    """max over variables of max_c |A - B| / max_c |B| (cells: index or mask)"""
    if cells is not None:
        A, B = A[:, cells], B[:, cells]
    scale = np.abs(B).max(axis=1)
    scale[scale == 0] = 1.0
    d = np.abs(A - B)
    return float((d.max(axis=1) / scale).max()) if d.size else 0.0


def fp32_bar(R_exact, R_of_rounded, tol=1e-5, cells=None):
    """(bar, E_in): E_in = rel_err(R(fl32 U), R(U)) over `cells`"""
    e_in = rel_err(R_of_rounded, R_exact, cells)
    return max(tol, FP32_INPUT_FACTOR * e_in), e_in
