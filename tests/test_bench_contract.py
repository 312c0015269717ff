"""Host-side pieces of bench.py (CPU): the reference arm's JSON line (the
oracle timed on the host cores) carries the contract's keys, the DRAM
traffic figure is reported only while the candidate kernel's sources hash to
the build it was captured on, per-kernel times are medians over steps, and
the roofline's byte model and ceiling choice match counts made by hand."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["value"] > 0 and line["higher_is_better"] is True and line["warmup"] >= 3
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]
    # the arm times the FP64 oracle: its config must say so
    assert line["dtype"] == "f64" and line["config"]["precision"] == "fp64"


def test_traffic_figure_follows_the_kernel_sources(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    h = bench.kernel_source_hash()
    monkeypatch.setitem(bench.TRAFFIC, ("quadrant", 3, "fp32", "hybrid"), {"bytes_per_cell": 400.0, "sources": h})
    assert bench._traffic("quadrant", 3, "fp32", "hybrid", 1000) == 400000
    assert bench._traffic("quadrant", 3, "fp64", "hybrid", 1000) is None
    monkeypatch.setitem(bench.TRAFFIC, ("quadrant", 3, "fp32", "hybrid"), {"bytes_per_cell": 400.0, "sources": "0"})
    assert bench._traffic("quadrant", 3, "fp32", "hybrid", 1000) is None


def test_kernel_times_are_the_median_over_steps():
    """One step whose first launch waited on the host does not move a
    kernel's reported time; kernels that ran in one step only report zero
    time (their steady-state share) but keep their launch count."""
    sys.path.insert(0, ROOT)
    import bench
    steps = [{"linear": (0.030 * 3, 3), "tag": (0.005 * 3, 3), "cvt": (0.0, 0)} for _ in range(9)]
    steps[4] = {"linear": (0.030 * 3 + 0.110, 3), "tag": (0.005 * 3, 3), "cvt": (0.0, 0)}
    steps[0]["cvt"] = (0.011, 1)
    t = bench.median_kernel_times(steps)
    assert t["linear"][1] == 27 and abs(t["linear"][0] / t["linear"][1] - 0.030) < 1e-12
    assert abs(t["tag"][0] - 0.005 * 27) < 1e-12
    assert t["cvt"] == (0.0, 1)


def test_byte_model_against_hand_counts():
    """The algorithmic bytes behind the roofline, counted by hand at FP32
    (b = 4): order 3 in 2D (M = 12, two points per face, nv = 4) a triangle
    reads U 16 + stencil ids 48 + L 6*12*4 = 288 + face geometry 1.5*3*4 = 18 +
    1/|V| 4 + face neighbours 12 and writes R 16: 402 B; a quadrilateral
    16 + 48 + 384 + 24 + 4 + 16 + 16 = 508 B.  Order 4 on hexahedra (M = 40,
    four points per face, nv = 5): 20 + 160 + 3840 + 48 + 4 + 24 + 20 = 4116 B.
    The candidate kernel's own bytes add the face states written and drop the
    flux kernel's geometry and R: 462 B per triangle, 590 B per quadrilateral,
    125,981,518 B per launch on the 249,601-cell quadrant mesh."""
    from types import SimpleNamespace as NS

    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from paper_2510_25906_gb300 import inputs as I
    s2 = NS(nv=4, M=12, N=5, Md=6, nfp=2)
    tri = NS(dim=2, cell_type=np.full(5, I.TRI, np.uint8), n_cells=5)
    quad = NS(dim=2, cell_type=np.full(5, I.QUAD, np.uint8), n_cells=5)
    assert bench.path_model(tri, s2, 4)["B_lin"] == 402.0
    assert bench.path_model(quad, s2, 4)["B_lin"] == 508.0
    hexes = NS(dim=3, cell_type=np.full(5, I.HEX, np.uint8), n_cells=5)
    assert bench.path_model(hexes, NS(nv=5, M=40, N=19, Md=8, nfp=4), 4)["B_lin"] == 4116.0
    assert bench._k1_bytes(tri, s2, 4) == 5 * 462 and bench._k1_bytes(quad, s2, 4) == 5 * 590
    m, _, _ = I.workload("quadrant")
    ntri = int((m.cell_type == I.TRI).sum())
    assert (ntri, m.n_cells - ntri) == (166_274, 83_327)
    assert bench._k1_bytes(m, s2, 4) == 125_981_518
    assert abs(bench.path_model(m, s2, 4)["B_lin"] * m.n_cells - 109_172_264) < 1.0


def test_path_roofline_takes_the_lower_ceiling():
    """frac = value / min(HBM ceiling, FP64 FMA ceiling) for an FP64 path,
    value x B_alg / HBM peak for an FP32 one; B_alg adds the queued classes'
    bytes at their measured fractions."""
    from types import SimpleNamespace as NS

    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from paper_2510_25906_gb300 import inputs as I
    mesh = NS(dim=2, cell_type=np.full(8, I.QUAD, np.uint8), n_cells=8)
    sz = dict(nv=4, M=12, N=5, Md=6, nfp=2)
    peaks = {"hbm_gbs": 6000.0, "fp64_flops": 1.0e12}
    r32 = bench.path_roofline(mesh, NS(fp32=True, **sz), 1.0e9, (0.1, 0.05), peaks)
    pm = bench.path_model(mesh, NS(**sz), 4)
    B = pm["B_lin"] + 0.1 * pm["B_cweno"] + 0.05 * pm["B_muscl"]
    assert r32["bound"] == "hbm" and abs(r32["frac"] - B * 1e9 / 6e12) < 1e-12
    r64 = bench.path_roofline(mesh, NS(fp32=False, **sz), 1.0e8, (0.1, 0.05), peaks)
    pm = bench.path_model(mesh, NS(**sz), 8)
    B = pm["B_lin"] + 0.1 * pm["B_cweno"] + 0.05 * pm["B_muscl"]
    F = pm["F_lin"] + 0.1 * pm["F_cweno"] + 0.05 * pm["F_muscl"]
    hbm, alu = 6e12 / B, 1e12 / F
    assert r64["bound"] == ("fp64_alu" if alu < hbm else "hbm")
    assert abs(r64["frac"] - 1e8 / min(alu, hbm)) < 1e-12
