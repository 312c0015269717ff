"""The compaction entry point that allocates nothing (for callers that cannot
call cudaMalloc when they need the queues, e.g. inside a stream capture).

It must produce the same counts and queues as the compaction inside
hfv_residual: with classes forced, the residual compacts exactly the given
CWENOZ and MUSCL cells, so both are compared bit for bit, on two calls in a
row (the static scratch keeps the previous call's contents; the residual's
queues are read back sorted).  On a mesh of more than 1,024 blocks of 256
cells (where the scan here takes several block counts per thread) both are
also compared with numpy's list of the class-1 and class-2 cells."""
import ctypes

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


def test_static_scratch_compaction_matches_residual_queues(H):
    m = I.mixed_tri_quad_mesh(80, seed=2)       # 9,600-odd cells: 38 blocks and a ragged tail
    U = I.quadrant_state(m)
    g = H.Scheme(H.Mesh(m), order=3, flux="hllc")
    rng = np.random.default_rng(7)
    for trial in range(2):
        forced = torch.tensor(rng.integers(0, 4, m.n_cells).astype(np.uint8), device="cuda")
        g.residual(torch.tensor(U, device="cuda"), forced=forced)
        ref_counts, (ref_c, ref_m) = g.queues()
        for call in range(2):                   # two calls in a row share the scratch
            counts, queues = H.class_queues_static(forced)
            torch.cuda.synchronize()
            cnt = counts.cpu().numpy()
            q = queues.cpu().numpy()
            assert np.array_equal(cnt, ref_counts), (trial, call, cnt, ref_counts)
            assert np.array_equal(q[:cnt[0]], ref_c)
            assert np.array_equal(q[m.n_cells:m.n_cells + cnt[1]], ref_m)


def test_static_scratch_compaction_beyond_1024_blocks_matches_numpy(H):
    """300,000-odd cells (1,178 blocks and a ragged tail), seeded random
    classes: counts and ascending queues equal np.nonzero, for this entry
    point (two calls in a row) and for the residual's own compaction."""
    m = I.structured_quad_mesh(548, 548, jitter=0.1, seed=3)   # 300,304 cells
    nb = (m.n_cells + 255) // 256
    assert nb > 1024 and m.n_cells % 256 != 0
    U = I.quadrant_state(m)
    g = H.Scheme(H.Mesh(m), order=2, flux="hllc", precision="fp32")
    rng = np.random.default_rng(11)
    for trial in range(2):
        cls = rng.integers(0, 4, m.n_cells).astype(np.uint8)
        want_c, want_m = np.nonzero(cls == 1)[0], np.nonzero(cls == 2)[0]
        forced = torch.tensor(cls, device="cuda")
        g.residual(torch.tensor(U, dtype=torch.float32, device="cuda"), forced=forced)
        rc, (qc, qm) = g.queues()
        assert rc.tolist() == [len(want_c), len(want_m)]
        assert np.array_equal(qc, want_c) and np.array_equal(qm, want_m)
        for call in range(2):
            counts, queues = H.class_queues_static(forced)
            torch.cuda.synchronize()
            cnt = counts.cpu().numpy()
            q = queues.cpu().numpy()
            assert cnt.tolist() == [len(want_c), len(want_m)], (trial, call)
            assert np.array_equal(q[:cnt[0]], want_c)
            assert np.array_equal(q[m.n_cells:m.n_cells + cnt[1]], want_m)


def test_static_scratch_rejects_oversized_input(H):
    lib = H.load()
    tiny = torch.zeros(4, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = lib.hfv_class_queues_static(ctypes.c_void_p(tiny.data_ptr()), (1 << 24) + 1, ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), None)
    assert rc == H.HFV_ERR_ARG
    assert b"static scratch limit" in lib.hfv_last_error()
