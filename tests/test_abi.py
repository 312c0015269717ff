"""Host-side checks of libhfv without a GPU: it builds, loads, exports every
symbol the header declares, and its host mesh ingestion and stencil builder
(pure CPU code) agree bit for bit with the oracle's connectivity and
stencils, and with stencils enumerated by hand."""
import json
import math
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2510_25906_gb300 import build as B
from paper_2510_25906_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    B.build()
    import paper_2510_25906_gb300.hfv as H
    H.load()
    return H


def _declared():
    src = open(os.path.join(ROOT, "include", "hfv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hfv_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(H):
    lib = H.load()
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n


def test_unknown_scheme_parameters_raise(H):
    """A misspelt field or an unknown name raises instead of leaving the
    default silently in place."""
    p = H.default_params(order=5, flux="hll", precision="fp32", limiter="venkatakrishnan", step_chain=1)
    assert (p.order, p.flux, p.precision, p.limiter, p.step_chain) == (5, H.HFV_HLL, H.HFV_FP32,
                                                                       H.LIMITER["venkatakrishnan"], 1)
    with pytest.raises(TypeError):
        H.default_params(presicion="fp32")
    with pytest.raises(ValueError):
        H.default_params(flux="roe")
    with pytest.raises(ValueError):
        H.default_params(precision="fp16")


def test_default_params(H):
    p = H.default_params()
    assert (p.order, p.flux, p.scheme, p.nad_vars, p.precision) == (3, H.HFV_HLLC, H.HFV_HYBRID, 3, H.HFV_FP64)
    assert (p.alpha_m, p.beta_m, p.alpha_w, p.beta_w) == (5e-3, 0.5, 0.0, 0.0)
    assert (p.cweno_eps, p.cweno_b, p.harten_theta, p.harten_eps, p.lambda1_prime) == (1e-3, 4.0, 0.9, 1e-14, 1e3)


@pytest.mark.parametrize("maker", [
    lambda: I.structured_tri_mesh(32, periodic=True, jitter=0.2, seed=1),
    lambda: I.mixed_tri_quad_mesh(40, seed=2),
    lambda: I.mixed_tri_quad_mesh(20, seed=9, periodic=True),
    lambda: I.structured_hex_mesh(10, 2 * math.pi, periodic=True),
    lambda: I.structured_hex_mesh(7, 1.0, periodic=False, jitter=0.2, seed=3),
    lambda: I.structured_tet_mesh(5, 1.0, periodic=False, jitter=0.1, seed=3),
    lambda: I.structured_tet_mesh(4, 1.0, periodic=True),
    lambda: I.mixed_element_mesh(4, seed=7),
    lambda: I.mixed_element_mesh(5, nz=3, seed=13),
])
def test_connectivity_bit_exact_with_oracle(H, maker):
    m = maker()
    g = H.Mesh(m)
    o = O.Mesh(m)
    nbr_g, nbrf_g = g.connectivity()
    nbr_o, nbrf_o = o.connectivity()
    assert np.array_equal(nbr_g, nbr_o)
    assert np.array_equal(nbrf_g, nbrf_o)
    assert g.n_faces == o.n_faces


def test_mesh_errors(H):
    m = I.structured_tri_mesh(4, periodic=False, jitter=0.0)
    bad = I.Mesh(m.dim, m.nodes, m.cell_type.copy(), m.cell_ptr, m.cell_idx, m.period)
    bad.cell_type[3] = 7
    with pytest.raises(H.HfvError) as e:
        H.Mesh(bad)
    assert e.value.code == H.HFV_ERR_MESH
    # clockwise triangle: non-positive measure
    idx = m.cell_idx.copy()
    idx[0:3] = idx[0:3][::-1]
    with pytest.raises(H.HfvError) as e:
        H.Mesh(I.Mesh(m.dim, m.nodes, m.cell_type, m.cell_ptr, idx, m.period))
    assert e.value.code == H.HFV_ERR_MESH
    # a period so small that a cell meets itself
    one = I.structured_quad_mesh(1, 3, periodic=(True, False))
    with pytest.raises(H.HfvError) as e:
        H.Mesh(one)
    assert e.value.code == H.HFV_ERR_MESH


@pytest.mark.parametrize("maker", [
    lambda: I.mixed_element_mesh(5, seed=7),
    lambda: I.mixed_tri_quad_mesh(20, seed=2),
    lambda: I.structured_tri_mesh(12, periodic=True, jitter=0.2, seed=1),
    lambda: I.structured_hex_mesh(6, 1.0, periodic=False, jitter=0.2, seed=3),
    lambda: I.structured_tet_mesh(4, 1.0, periodic=False, jitter=0.1, seed=3),
])
def test_volumes_match_oracle(H, maker):
    """The library's measures (prisms and pyramids by the divergence theorem
    over their faces) against the oracle's volume rules, and their sum
    against the measure of the domain (the unit square or cube)."""
    m = maker()
    vg = H.Mesh(m).volumes()
    vo, _ = O.Mesh(m).geometry()
    assert np.abs(vg - vo).max() <= 1e-14 * vo.max()
    assert (vg > 0).all() and abs(vg.sum() - 1.0) <= 1e-13


def test_mesh_edge_cases(H):
    """Descriptors the library must refuse: no cells, a 3D type in a 2D
    mesh, a vertex count that does not match the type, an inverted prism,
    a face shared by three cells."""
    tri = I.structured_tri_mesh(2, periodic=False, jitter=0.0)
    empty = I.Mesh(2, tri.nodes, tri.cell_type[:0], tri.cell_ptr[:1], tri.cell_idx[:0], tri.period)
    with pytest.raises(H.HfvError) as e:
        H.Mesh(empty)
    assert e.value.code == H.HFV_ERR_ARG
    bad = I.Mesh(2, tri.nodes, tri.cell_type.copy(), tri.cell_ptr, tri.cell_idx, tri.period)
    bad.cell_type[0] = I.PRISM
    with pytest.raises(H.HfvError) as e:
        H.Mesh(bad)
    assert e.value.code == H.HFV_ERR_MESH
    m = I.mixed_element_mesh(2, seed=1, p_pyramid=0.6)
    pyr = int(np.nonzero(m.cell_type == I.PYRAMID)[0][0])
    t = m.cell_type.copy()
    t[pyr] = I.PRISM                                   # five vertices listed for a prism
    with pytest.raises(H.HfvError) as e:
        H.Mesh(I.Mesh(3, m.nodes, t, m.cell_ptr, m.cell_idx, m.period))
    assert e.value.code == H.HFV_ERR_MESH
    pr = int(np.nonzero(m.cell_type == I.PRISM)[0][0])
    idx = m.cell_idx.copy()
    a, b = m.cell_ptr[pr], m.cell_ptr[pr + 1]
    idx[a:b] = np.concatenate([idx[a + 3:b], idx[a:a + 3]])   # top and bottom swapped: inverted
    with pytest.raises(H.HfvError) as e:
        H.Mesh(I.Mesh(3, m.nodes, m.cell_type, m.cell_ptr, idx, m.period))
    assert e.value.code == H.HFV_ERR_MESH
    nodes = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 1.0], [0.5, -1.0], [0.2, 0.8]])
    fan = I.Mesh(2, nodes, np.full(3, I.TRI, np.uint8), np.array([0, 3, 6, 9]),
                 np.array([0, 1, 2, 1, 0, 3, 0, 1, 4], np.int32), np.zeros(2))
    with pytest.raises(H.HfvError) as e:
        H.Mesh(fan)
    assert e.value.code == H.HFV_ERR_MESH


# ---------------------------------------------------------------------------
# the library's host stencil builder (hfv_stencils_host) without a GPU
# ---------------------------------------------------------------------------

def _compare_stencils(H, m, order, step=1):
    """Central and directional stencils of every step-th cell, bit for bit
    against the oracle's; entries past a directional stencil's size and the
    rows of faces a cell does not have are -1."""
    cen, dr = H.Mesh(m).stencils(order)
    osch = O.Scheme(O.Mesh(m), order=order)
    assert cen.shape[1] == osch.M and dr.shape[2] == osch.Md
    for c in range(0, m.n_cells, step):
        st, od = osch.stencil(c)
        assert np.array_equal(cen[c], st), c
        nd = osch.operator(c, "nd").astype(int)
        nf = od.shape[0]
        for f in range(nf):
            assert np.array_equal(dr[c, f, :nd[f]], od[f, :nd[f]]), (c, f)
            assert (dr[c, f, nd[f]:] == -1).all(), (c, f)
        assert (dr[c, nf:] == -1).all(), c


@pytest.mark.parametrize("maker,orders", [
    (lambda: I.structured_tri_mesh(24, periodic=True, jitter=0.2, seed=1), (2, 3, 5, 7)),
    (lambda: I.mixed_tri_quad_mesh(30, seed=2), (3, 4, 6)),
    (lambda: I.mixed_tri_quad_mesh(20, seed=9, periodic=True), (3, 5)),
    (lambda: I.structured_hex_mesh(12, 2 * math.pi, periodic=True), (2, 4, (6, 17))),
    (lambda: I.structured_hex_mesh(7, 1.0, periodic=False, jitter=0.2, seed=3), (3, 4)),
    (lambda: I.structured_tet_mesh(5, 1.0, periodic=False, jitter=0.1, seed=3), (2, 3)),
    (lambda: I.structured_tet_mesh(4, 1.0, periodic=True), (3,)),
    (lambda: I.mixed_element_mesh(5, nz=3, seed=13), (2, 3)),
])
def test_host_stencils_bit_exact_with_oracle(H, maker, orders):
    """orders given as (order, step) compare every step-th cell (the oracle
    builds a cell's operators when its stencil is asked for, slow at order 6
    in 3D)."""
    m = maker()
    for order in orders:
        order, step = order if isinstance(order, tuple) else (order, 1)
        _compare_stencils(H, m, order, step)


def test_host_stencils_bit_exact_on_the_quadrant_mesh(H):
    """The 249,601-cell mixed mesh of the quadrant workload at order 3: every
    seventh cell."""
    m, _, kw = I.workload("quadrant")
    _compare_stencils(H, m, kw["order"], step=7)


def _hand_mesh(spec):
    if spec["mesh"] == "quad":
        return I.structured_quad_mesh(spec["n"], spec["n"], periodic=(spec["periodic"],) * 2)
    return I.structured_hex_mesh(spec["n"], 1.0, periodic=spec["periodic"])


def _hand():
    with open(os.path.join(ROOT, "tests", "golden", "stencils_hand.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("case", _hand()["cases"], ids=lambda c: f'{c["mesh"]}{c["n"]}_o{c["order"]}_c{c["cell"]}')
def test_host_stencils_against_hand_enumeration(H, case):
    cen, dr = H.Mesh(_hand_mesh(case)).stencils(case["order"])
    c = case["cell"]
    assert cen[c].tolist() == case["stencil"]
    if "directional" in case:
        got = sorted(sorted(x for x in row.tolist() if x >= 0) for row in dr[c] if (row >= 0).any())
        assert got == sorted(case["directional"])


def test_host_stencils_errors(H):
    g = H.Mesh(_hand_mesh(_hand()["too_small"]))
    with pytest.raises(H.HfvError) as e:
        g.stencils(_hand()["too_small"]["order"])
    assert e.value.code == H.HFV_ERR_STENCIL
    g = H.Mesh(I.structured_quad_mesh(5, 5))
    for order in (1, 8):
        with pytest.raises(H.HfvError) as e:
            g.stencils(order)
        assert e.value.code == H.HFV_ERR_ARG


def test_descriptor_checked_before_its_offsets_are_followed(H):
    """Offsets, vertex ids, coordinates and periods are checked before the
    library reads through the CSR offsets; a descriptor whose offsets start
    past 0 (with that many unused leading ids) describes the same mesh."""
    m = I.mixed_tri_quad_mesh(6, seed=3)

    def with_(**kw):
        f = dict(dim=m.dim, nodes=m.nodes, cell_type=m.cell_type, cell_ptr=m.cell_ptr, cell_idx=m.cell_idx,
                 period=m.period)
        f.update(kw)
        return I.Mesh(f["dim"], f["nodes"], f["cell_type"], f["cell_ptr"], f["cell_idx"], f["period"])

    def code(mesh, batch=False):
        with pytest.raises(H.HfvError) as e:
            H.Mesh.batch([m, mesh]) if batch else H.Mesh(mesh)
        return e.value.code

    neg = m.cell_ptr - 1                                  # offsets from -1
    assert code(with_(cell_ptr=neg)) == H.HFV_ERR_MESH
    jump = m.cell_ptr.copy()
    jump[5:] += 1                                         # cell 4 claims one vertex too many
    assert code(with_(cell_ptr=jump)) == H.HFV_ERR_MESH
    huge = m.cell_ptr.copy()
    huge[-1] = 1 << 40                                    # the last cell would read far past the ids
    assert code(with_(cell_ptr=huge)) == H.HFV_ERR_MESH
    assert code(with_(cell_ptr=huge), batch=True) == H.HFV_ERR_MESH
    bad_id = m.cell_idx.copy()
    bad_id[7] = m.n_nodes
    assert code(with_(cell_idx=bad_id)) == H.HFV_ERR_MESH
    assert code(with_(cell_idx=bad_id), batch=True) == H.HFV_ERR_MESH
    nan = m.nodes.copy()
    nan[3, 1] = np.nan
    assert code(with_(nodes=nan)) == H.HFV_ERR_MESH
    assert code(with_(period=np.array([-1.0, 0.0]))) == H.HFV_ERR_ARG
    assert code(with_(period=np.array([np.inf, 0.0]))) == H.HFV_ERR_ARG
    shifted = with_(cell_ptr=m.cell_ptr + 3, cell_idx=np.concatenate([np.zeros(3, np.int32), m.cell_idx]))
    a, b = H.Mesh(m).connectivity(), H.Mesh(shifted).connectivity()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(H.Mesh(m).volumes(), H.Mesh(shifted).volumes())
    g = H.Mesh.batch([m, shifted])
    assert g.n_cells == 2 * m.n_cells


def test_elementwise_entry_points_check_sizes_before_any_cuda_call(H):
    """hfv_convert and hfv_rcp64 refuse a negative count, a count whose grid
    would pass 2^31 - 1 blocks and null buffers, and do nothing for n = 0,
    all before any CUDA call (so without a GPU)."""
    lib = H.load()
    big = ((1 << 31) - 1) * 255 + 1
    for n, buf in ((-1, 8), (big, 8), (4, None)):
        assert lib.hfv_convert(1, n, buf, buf, None) == H.HFV_ERR_ARG
        assert lib.hfv_rcp64(n, buf, buf, None) == H.HFV_ERR_ARG
    assert lib.hfv_convert(2, 4, 8, 8, None) == H.HFV_ERR_ARG
    assert lib.hfv_convert(0, 0, None, None, None) == H.HFV_OK
    assert lib.hfv_rcp64(0, None, None, None) == H.HFV_OK


def test_static_queues_check_arguments_before_any_cuda_call(H):
    lib = H.load()
    for n, p in ((0, 8), (-5, 8), (16_777_217, 8), (10, None)):
        assert lib.hfv_class_queues_static(p, n, p, p, None) == H.HFV_ERR_ARG
    lib.hfv_class_queues_static(8, 16_777_217, 8, 8, None)
    assert "static scratch limit of 16777216" in lib.hfv_last_error().decode()


def test_abi_from_plain_c(H, tmp_path):
    """include/hfv.h compiles as C99 and a C program linked against
    libhfv.so builds a mesh, reads its measures and host stencils, and sees
    the error codes and messages (tests/c/abi_from_c.c)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib_dir = os.path.dirname(H.LIB_PATH)
    exe = str(tmp_path / "abi_from_c")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-O1", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_from_c.c"), "-o", exe, "-L", lib_dir, "-lhfv", "-lm",
           f"-Wl,-rpath,{lib_dir}"]
    subprocess.run(cmd, check=True, capture_output=True, text=True, timeout=120)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr


def test_every_entry_point_documents_its_errors():
    """Each declaration in include/hfv.h follows a comment that states its
    error behaviour (the codes it returns, or that it never fails / is a
    no-op)."""
    src = open(os.path.join(ROOT, "include", "hfv.h")).read()
    documented = set()
    for m in re.finditer(r"(/\*(?:(?!\*/).)*\*/)\s*\n\s*((?:HFV_API[^;]*;\s*)+)", src, re.S):
        com = m.group(1)
        if re.search(r"Errors?:|HFV_ERR_|Never fails|no-op", com):
            documented.update(re.findall(r"HFV_API[^;]*?(hfv_\w+)\s*\(", m.group(2)))
    missing = sorted(set(_declared()) - documented)
    assert not missing, missing


def test_library_defaults_are_the_cited_constants(H):
    """hfv_default_params against the cited fixtures: the detector margins of
    Fig. NADMargin (a) and the CWENOZ / Harten / gas constants of Sec. 2,
    2.3 and 2.4 -- the same files the oracle's pins read."""
    gold = os.path.join(ROOT, "tests", "golden")
    nad = json.load(open(os.path.join(gold, "nad_presets.json")))["default"]
    cw = json.load(open(os.path.join(gold, "cweno_constants.json")))
    p = H.default_params()
    assert (p.alpha_m, p.beta_m, p.alpha_w, p.beta_w) == (nad["alpha_m"], nad["beta_m"], nad["alpha_w"], nad["beta_w"])
    assert (p.cweno_eps, p.cweno_b, p.harten_theta, p.harten_eps, p.gamma) == (
        cw["cw_eps"], cw["cw_b"], cw["harten_theta"], cw["harten_eps"], cw["gamma"])
    assert p.lambda1_prime == cw["lambda1p_default"]
    assert p.nad_vars == 3                       # density and pressure


def test_batch_segments(H):
    a = I.mixed_tri_quad_mesh(5, seed=1)
    b = I.structured_tri_mesh(4, periodic=False)
    g = H.Mesh.batch([a, b, a])
    assert g.n_segments == 3
    assert g.segments.tolist() == [0, a.n_cells, a.n_cells + b.n_cells, 2 * a.n_cells + b.n_cells]
    assert g.n_cells == g.segments[-1]
