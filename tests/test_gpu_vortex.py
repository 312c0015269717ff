"""The isentropic vortex accuracy test of the paper (Sec. 3.1): the hybrid
scheme on periodic jittered triangle meshes of the [0, 10]^2 square reaches
its design order on a smooth flow (the detector leaves every cell linear)
and agrees with pure linear reconstruction there.

Bar: L2 error of the cell-averaged density against the exact translated
vortex at t = 1 falls at least as fast as h^(order - 0.3) between 64 and 128
cells per side (orders 3, 5 and 7), with SSP-RK(5,4) steps small enough that
the spatial error dominates (at 32 -> 64 the vortex core spans too few cells
for the asymptotic rate); at order 7 the step shrinks as h^(7/4) so that the
fourth-order time error falls with the spatial one."""
import math

import numpy as np
import pytest

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


def _l2(H, n, order, scheme, t_end=1.0):
    m = I.structured_tri_mesh(n, periodic=True, jitter=0.2, seed=7, lx=10.0, ly=10.0)
    U0 = I.isentropic_vortex_state(m, 0.0)
    gm = H.Mesh(m)
    g = H.Scheme(gm, order=order, flux="hllc", precision="fp64", scheme=scheme, time_scheme="ssprk54")
    U = torch.tensor(U0, device="cuda")
    h = 10.0 / n
    cfl = 0.2 * (n / 64.0) ** (-max(0, order - 4) / 4.0)
    steps = int(math.ceil(t_end / (cfl * h)))
    dt = t_end / steps
    for _ in range(steps):
        g.step(U, dt=dt)
    cls = torch.empty(m.n_cells, dtype=torch.uint8, device="cuda")
    g.residual(U, class_out=cls)
    ex = I.isentropic_vortex_state(m, t_end)
    vol = gm.volumes()
    err = math.sqrt((vol * (U[0].cpu().numpy() - ex[0]) ** 2).sum() / vol.sum())
    return err, np.bincount(cls.cpu().numpy(), minlength=4)


@pytest.mark.parametrize("order", [3, 5, 7])
def test_vortex_design_order(H, order):
    """Order 7: Table tab:2D_Vortex prints an L2 rate of 6.41 from 64 to 128
    edges per side for P7 and an L2 error of 4.045e-07 at 128; the bar is
    rate >= 6.3 and an error at 128 below the paper's."""
    e1, c1 = _l2(H, 64, order, "hybrid")
    e2, c2 = _l2(H, 128, order, "hybrid")
    rate = math.log2(e1 / e2)
    l1, _ = _l2(H, 64, order, "linear")
    print(f"order {order}: L2 {e1:.3e} -> {e2:.3e}, rate {rate:.2f}; classes {c1} / {c2}; linear {l1:.3e}")
    if order == 7:
        assert rate >= 6.3 and e2 < 4.045e-07, (rate, e2)
    else:
        assert rate >= order - 0.3, rate
    assert abs(e1 - l1) <= 1e-3 * l1   # smooth flow: the hybrid scheme is the linear scheme
