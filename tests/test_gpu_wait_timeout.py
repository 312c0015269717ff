"""The candidate kernel's bounded waits, made to run out on purpose without
faulting or hanging anything: with hfv_debug_wait the producer warp issues no
bulk copy (nothing completes the barrier phase the consumers wait on) and
the consumers' limit is 1 ms.  The launch must record the timeout for
hfv_status (HFV_ERR_TIMEOUT, bit 2) and return; no copy is ever in flight.
After restoring normal operation the same scheme must give the oracle's
residual again, so the context and the scheme are intact."""
import time

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


def test_withheld_copies_time_out_and_the_scheme_recovers(H):
    m = I.mixed_tri_quad_mesh(16, seed=2)
    U = I.quadrant_state(m)
    g = H.Scheme(H.Mesh(m), order=3, flux="hllc", precision="fp64")
    Ug = torch.tensor(U, device="cuda")
    g.residual(Ug)
    torch.cuda.synchronize()
    assert g.status(reset=True) == 0
    g.debug_wait(consumer_wait_ns=1_000_000, withhold_copies=True)
    t0 = time.perf_counter()
    g.residual(Ug)
    torch.cuda.synchronize()
    took = time.perf_counter() - t0
    with pytest.raises(H.HfvError) as e:
        g.status()
    assert e.value.code == H.HFV_ERR_TIMEOUT
    assert took < 1.0, took                     # the 1 ms limit, not the default 2 s
    g.debug_wait(0, False)
    with pytest.raises(H.HfvError):
        g.status(reset=True)                    # read and clear the sticky bit
    assert g.status() == 0
    R = g.residual(Ug).cpu().numpy()
    assert g.status() == 0
    Ro = O.Scheme(O.Mesh(m), order=3, flux="hllc").residual(U)[0]
    scale = np.abs(Ro).max(axis=1, keepdims=True)
    assert (np.abs(R - Ro) / scale).max() < 1e-12
