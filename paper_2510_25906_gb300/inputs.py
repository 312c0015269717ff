"""Seeded synthetic workloads: meshes and initial cell averages.

This module generates inputs only. It holds none of the method's arithmetic:
no faces, stencils, reconstructions, detectors or fluxes. Both the CUDA path
and the CPU oracle consume exactly the arrays built here.

Mesh format (shared by every consumer):
    dim        2 or 3
    nodes      float64 [n_nodes, dim]
    cell_type  uint8   [n_cells]   TRI=1, QUAD=2, TET=3, HEX=4, PRISM=5, PYRAMID=6
    cell_ptr   int64   [n_cells+1] CSR offsets into cell_idx
    cell_idx   int32   [...]       vertex ids in the fixed local order below
    period     float64 [dim]       periodic length per axis, 0 = not periodic

Local vertex order: TRI and QUAD counter-clockwise; TET v0..v3 of positive
volume; HEX v0..v3 the bottom face counter-clockwise seen from +z, v4..v7 the
top face above them; PRISM the triangles v0 v1 v2 and v3 v4 v5 (v3 above
v0); PYRAMID the base v0..v3 counter-clockwise seen from the apex v4.
Periodic meshes carry separate nodes on opposite sides (x=0 and x=L); faces
are paired across the period by their positions.

State format: conserved variables, float64 [nv, n_cells] (structure of
arrays), nv = dim + 2, order (rho, rho*u, rho*v[, rho*w], E).

Workloads (seeded, synthetic, shaped like the paper's):
  * ``density_wave``: periodic unit square, structured n x n quads cut
    along one diagonal, interior nodes jittered by +-0.2h; rho = 1 + 0.2
    sin(2 pi (x + y)), u = v = 1, p = 1 (the smooth advected wave).
  * ``quadrant``: [0,1]^2, n x n quads of which a seeded half are cut
    into two triangles along a seeded diagonal, interior nodes jittered; the
    four constant states of the paper's 2D Riemann problem (Sec. 3.5, the
    2D Riemann problem equation), placed by quadrant about (0.5, 0.5).
  * ``turbulence``: periodic [0, 2 pi]^3, n^3 uniform hexahedra; uniform
    density and pressure (rho = 1, p = 1/gamma, so c = 1) and a seeded
    solenoidal velocity with energy spectrum E(k) ~ k^4 exp(-2 k^2 / k0^2),
    k0 = 4, scaled to turbulent Mach number 0.6 (the decaying-turbulence
    stand-in for the paper's 128^3 Taylor-Green mesh, Sec. 3.6).
  * the adjoint workload (``adjoint_problem``): 6 n^3 jittered tetrahedra of
    the open unit cube with a density pulse ahead of a Mach 2 shock
    (``shock_pulse_state``); the 3D mixed-element mesh
    (``mixed_element_mesh``) carries the same state;
  * the batched workload (``batched_problems``): independent open 2D
    problems of uneven size and order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TRI, QUAD, TET, HEX, PRISM, PYRAMID = 1, 2, 3, 4, 5, 6
GAMMA = 1.4


@dataclass
class Mesh:
    dim: int
    nodes: np.ndarray
    cell_type: np.ndarray
    cell_ptr: np.ndarray
    cell_idx: np.ndarray
    period: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        """Number of cells."""
        return int(self.cell_type.shape[0])

    @property
    def n_nodes(self) -> int:
        """Number of nodes."""
        return int(self.nodes.shape[0])

    def cell_vertices(self, c: int) -> np.ndarray:
        """Coordinates of cell c's vertices in its local order, [nv, dim]."""
        return self.nodes[self.cell_idx[self.cell_ptr[c]:self.cell_ptr[c + 1]]]

    def vertex_means(self) -> np.ndarray:
        """Arithmetic mean of each cell's vertices, [n_cells, dim]."""
        counts = np.diff(self.cell_ptr)
        out = np.zeros((self.n_cells, self.dim))
        for k in np.unique(counts):
            sel = np.nonzero(counts == k)[0]
            idx = self.cell_idx[self.cell_ptr[sel][:, None] + np.arange(k)[None, :]]
            out[sel] = self.nodes[idx].mean(axis=1)
        return out


def _finish(dim, nodes, types, conn_lists, period, name, **meta) -> Mesh:
    counts = np.array([len(c) for c in conn_lists], dtype=np.int64)
    ptr = np.zeros(len(conn_lists) + 1, dtype=np.int64)
    np.cumsum(counts, out=ptr[1:])
    idx = np.concatenate([np.asarray(c, dtype=np.int32) for c in conn_lists]) if conn_lists else np.zeros(0, np.int32)
    return Mesh(dim, np.ascontiguousarray(nodes, dtype=np.float64), np.asarray(types, dtype=np.uint8),
                ptr, idx, np.asarray(period, dtype=np.float64), name, dict(meta))


def _grid_nodes_2d(n: int, lx: float, ly: float, jitter: float, rng) -> np.ndarray:
    """(n+1)^2 nodes, node (i, j) at id j*(n+1)+i; interior nodes jittered."""
    i = np.arange(n + 1)
    xs = (i * lx) / n
    ys = (i * ly) / n
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    nodes = np.stack([X.ravel(), Y.ravel()], axis=1)
    if jitter > 0:
        hx, hy = lx / n, ly / n
        jj, ii = np.meshgrid(i, i, indexing="ij")
        interior = ((ii > 0) & (ii < n) & (jj > 0) & (jj < n)).ravel()
        d = rng.random((nodes.shape[0], 2)) * 2.0 - 1.0
        nodes[interior, 0] += jitter * hx * d[interior, 0]
        nodes[interior, 1] += jitter * hy * d[interior, 1]
    return nodes


def structured_tri_mesh(n: int, periodic: bool = True, jitter: float = 0.2, seed: int = 1,
                        lx: float = 1.0, ly: float = 1.0) -> Mesh:
    """n x n quads, each cut along its (i,j)->(i+1,j+1) diagonal: 2 n^2 triangles."""
    rng = np.random.default_rng(seed)
    nodes = _grid_nodes_2d(n, lx, ly, jitter, rng)
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    a = (j * (n + 1) + i).ravel()
    b, c, d = a + 1, a + n + 2, a + n + 1
    conn = np.stack([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], 1).reshape(-1, 3).astype(np.int32)
    period = [lx, ly] if periodic else [0.0, 0.0]
    ptr = np.arange(0, 3 * conn.shape[0] + 1, 3, dtype=np.int64)
    return Mesh(2, np.ascontiguousarray(nodes, dtype=np.float64), np.full(conn.shape[0], TRI, np.uint8), ptr,
                conn.ravel(), np.asarray(period, dtype=np.float64), f"tri{n}", dict(n=n, seed=seed))


def structured_quad_mesh(nx: int, ny: int, lx: float = 1.0, ly: float = 1.0, periodic=(False, False),
                         jitter: float = 0.0, seed: int = 0) -> Mesh:
    """nx x ny quadrilaterals on [0,lx]x[0,ly] (node (i,j) at id j*(nx+1)+i)."""
    rng = np.random.default_rng(seed)
    xs = (np.arange(nx + 1) * lx) / nx
    ys = (np.arange(ny + 1) * ly) / ny
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    nodes = np.stack([X.ravel(), Y.ravel()], axis=1)
    if jitter > 0:
        jj, ii = np.meshgrid(np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        interior = ((ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)).ravel()
        d = rng.random((nodes.shape[0], 2)) * 2.0 - 1.0
        nodes[interior, 0] += jitter * (lx / nx) * d[interior, 0]
        nodes[interior, 1] += jitter * (ly / ny) * d[interior, 1]
    nid = lambda i, j: j * (nx + 1) + i
    conn = [(nid(i, j), nid(i + 1, j), nid(i + 1, j + 1), nid(i, j + 1)) for j in range(ny) for i in range(nx)]
    period = [lx if periodic[0] else 0.0, ly if periodic[1] else 0.0]
    return _finish(2, nodes, [QUAD] * len(conn), conn, period, f"quad{nx}x{ny}")


def mixed_tri_quad_mesh(n: int, seed: int = 2, p_split: float = 0.5, jitter: float = 0.2,
                        periodic: bool = False) -> Mesh:
    """[0,1]^2 with n x n quads; each is cut into two triangles with probability
    p_split along a seeded diagonal, the rest stay quadrilaterals."""
    rng = np.random.default_rng(seed)
    nodes = _grid_nodes_2d(n, 1.0, 1.0, jitter, rng)
    split = rng.random(n * n) < p_split
    diag = rng.random(n * n) < 0.5
    nid = lambda i, j: j * (n + 1) + i
    conn, types = [], []
    for j in range(n):
        for i in range(n):
            a, b, c, d = nid(i, j), nid(i + 1, j), nid(i + 1, j + 1), nid(i, j + 1)
            q = j * n + i
            if not split[q]:
                conn.append((a, b, c, d)); types.append(QUAD)
            elif diag[q]:
                conn.append((a, b, c)); types.append(TRI)
                conn.append((a, c, d)); types.append(TRI)
            else:
                conn.append((a, b, d)); types.append(TRI)
                conn.append((b, c, d)); types.append(TRI)
    period = [1.0, 1.0] if periodic else [0.0, 0.0]
    return _finish(2, nodes, types, conn, period, f"mixed{n}", n=n, seed=seed)


def structured_hex_mesh(n: int, length: float = 2.0 * math.pi, periodic: bool = True,
                        jitter: float = 0.0, seed: int = 3, ny: int | None = None, nz: int | None = None) -> Mesh:
    """n x ny x nz uniform hexahedra on [0,L]^3, cell (i,j,k) at id (k*ny+j)*n+i."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed)
    hx, hy, hz = length / n, length / ny, length / nz
    xs = (np.arange(n + 1) * length) / n
    ys = (np.arange(ny + 1) * length) / ny
    zs = (np.arange(nz + 1) * length) / nz
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    nodes = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    if jitter > 0:
        K, J, I = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(n + 1), indexing="ij")
        interior = ((I > 0) & (I < n) & (J > 0) & (J < ny) & (K > 0) & (K < nz)).ravel()
        d = rng.random((nodes.shape[0], 3)) * 2.0 - 1.0
        nodes[interior] += jitter * np.array([hx, hy, hz]) * d[interior]
    sx, sy = n + 1, (n + 1) * (ny + 1)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(n), indexing="ij")
    base = (k * sy + j * sx + i).ravel()
    offs = np.array([0, 1, 1 + sx, sx, sy, sy + 1, sy + 1 + sx, sy + sx])
    conn = (base[:, None] + offs[None, :]).astype(np.int32)
    ncell = conn.shape[0]
    ptr = np.arange(ncell + 1, dtype=np.int64) * 8
    period = [length] * 3 if periodic else [0.0] * 3
    return Mesh(3, np.ascontiguousarray(nodes), np.full(ncell, HEX, np.uint8), ptr, conn.ravel().copy(),
                np.asarray(period, np.float64), f"hex{n}", {"n": n, "seed": seed})


def structured_tet_mesh(n: int, length: float = 1.0, periodic: bool = False, jitter: float = 0.0,
                        seed: int = 4) -> Mesh:
    """n^3 hexahedra of [0,L]^3 each cut into six tetrahedra along its
    (0,0,0)-(1,1,1) diagonal (one per ordering of the axes: the path
    000 -> e_a -> e_a + e_b -> 111), conforming across the grid; 6 n^3 cells,
    vertices of each tetrahedron ordered to positive volume.  Interior nodes
    jittered by up to `jitter` h per coordinate."""
    hx = structured_hex_mesh(n, length, periodic=periodic, jitter=jitter, seed=seed)
    corner = {(0, 0, 0): 0, (1, 0, 0): 1, (1, 1, 0): 2, (0, 1, 0): 3, (0, 0, 1): 4, (1, 0, 1): 5, (1, 1, 1): 6,
              (0, 1, 1): 7}
    tets = []
    for perm in ((0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1), (2, 1, 0), (1, 0, 2)):
        b = [0, 0, 0]
        path = [corner[tuple(b)]]
        for ax in perm:
            b[ax] = 1
            path.append(corner[tuple(b)])
        tets.append(path)
    hc = hx.cell_idx.reshape(-1, 8)
    conn = np.concatenate([hc[:, t] for t in tets], axis=0)          # [6 n^3, 4], grouped by pattern
    order = np.arange(conn.shape[0]).reshape(6, -1).T.ravel()       # the six of each hexahedron together
    conn = np.ascontiguousarray(conn[order]).astype(np.int32)
    x = hx.nodes[conn]
    det = np.einsum("ij,ij->i", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]))
    flip = det < 0
    conn[flip, 1], conn[flip, 2] = conn[flip, 2].copy(), conn[flip, 1].copy()
    x = hx.nodes[conn]
    det = np.einsum("ij,ij->i", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]))
    if not (det > 0).all():
        raise ValueError("jitter too large: inverted tetrahedra")
    ncell = conn.shape[0]
    return Mesh(3, hx.nodes, np.full(ncell, TET, np.uint8), np.arange(ncell + 1, dtype=np.int64) * 4, conn.ravel(),
                hx.period, f"tet{n}", {"n": n, "seed": seed})


def mixed_element_mesh(n: int, nz: int | None = None, seed: int = 7, jitter: float = 0.15,
                       p_pyramid: float = 0.3) -> Mesh:
    """Open unit cube of all four 3D element types, conforming: the seeded
    mixed triangle / quadrilateral mesh of [0,1]^2 (n x n, interior nodes
    jittered) extruded through nz layers gives prisms and hexahedra
    (interior layer heights jittered by up to `jitter` h); a seeded share
    p_pyramid of the hexahedra is cut into six pyramids about its vertex
    mean (each pyramid's base is a face of the hexahedron, so every
    neighbour still sees that face whole), and in the bottom layer the
    pyramid standing on the boundary z = 0 is cut into two tetrahedra."""
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed)
    base = mixed_tri_quad_mesh(n, seed=seed, jitter=jitter)
    nb = base.n_nodes
    zs = np.arange(nz + 1) / nz
    z = np.repeat(zs[:, None], nb, axis=1)
    z[1:nz] += jitter / nz * (rng.random((nz - 1, nb)) * 2.0 - 1.0)
    nodes = np.concatenate([np.concatenate([base.nodes, z[k][:, None]], axis=1) for k in range(nz + 1)], axis=0)
    nodes = [tuple(x) for x in nodes]
    hex_faces = ((0, 3, 2, 1), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7))
    conn, types = [], []
    for k in range(nz):
        for c in range(base.n_cells):
            v = base.cell_idx[base.cell_ptr[c]:base.cell_ptr[c + 1]]
            bot, top = [int(x) + k * nb for x in v], [int(x) + (k + 1) * nb for x in v]
            if base.cell_type[c] == TRI:
                conn.append(bot + top); types.append(PRISM)
                continue
            h = bot + top
            if rng.random() >= p_pyramid:
                conn.append(h); types.append(HEX)
                continue
            centre = len(nodes)
            nodes.append(tuple(np.mean([nodes[i] for i in h], axis=0)))
            for f, (a, b, cc, d) in enumerate(hex_faces):
                pyr = [h[a], h[d], h[cc], h[b]]     # base counter-clockwise seen from the centre
                if k == 0 and f == 0:
                    conn.append([pyr[0], pyr[1], pyr[2], centre]); types.append(TET)
                    conn.append([pyr[0], pyr[2], pyr[3], centre]); types.append(TET)
                else:
                    conn.append(pyr + [centre]); types.append(PYRAMID)
    return _finish(3, np.asarray(nodes), types, conn, [0.0, 0.0, 0.0], f"mixed3d{n}", n=n, seed=seed)


# ---------------------------------------------------------------------------
# Initial states
# ---------------------------------------------------------------------------

def _gl(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def cell_average_2d(mesh: Mesh, f, npts: int = 8) -> np.ndarray:
    """Cell averages of f(x, y) over triangles and quadrilaterals by a
    collapsed / tensor Gauss-Legendre rule with npts points per direction."""
    s, ws = _gl(npts)
    S, T = np.meshgrid(s, s, indexing="ij")
    W = np.outer(ws, ws)
    out = np.zeros(mesh.n_cells)
    counts = np.diff(mesh.cell_ptr)
    for nv in (3, 4):
        sel = np.nonzero(counts == nv)[0]
        if sel.size == 0:
            continue
        v = mesh.nodes[mesh.cell_idx[mesh.cell_ptr[sel][:, None] + np.arange(nv)[None, :]]]  # [c, nv, 2]
        if nv == 3:
            p0, p1, p2 = v[:, 0], v[:, 1], v[:, 2]
            X = p0[:, None, None, :] + S[None, :, :, None] * (p1 - p0)[:, None, None, :] \
                + (S * T)[None, :, :, None] * (p2 - p1)[:, None, None, :]
            e1, e2 = p1 - p0, p2 - p1
            det = np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
            J = det[:, None, None] * S[None]
        else:
            p0, p1, p2, p3 = v[:, 0], v[:, 1], v[:, 2], v[:, 3]
            Sx, Tx = S[None, :, :, None], T[None, :, :, None]
            X = (1 - Sx) * (1 - Tx) * p0[:, None, None] + Sx * (1 - Tx) * p1[:, None, None] \
                + Sx * Tx * p2[:, None, None] + (1 - Sx) * Tx * p3[:, None, None]
            dXs = (1 - Tx) * (p1 - p0)[:, None, None] + Tx * (p2 - p3)[:, None, None]
            dXt = (1 - Sx) * (p3 - p0)[:, None, None] + Sx * (p2 - p1)[:, None, None]
            J = np.abs(dXs[..., 0] * dXt[..., 1] - dXs[..., 1] * dXt[..., 0])
        vals = f(X[..., 0], X[..., 1])
        out[sel] = (vals * J * W[None]).sum(axis=(1, 2)) / (J * W[None]).sum(axis=(1, 2))
    return out


def conserved_2d(rho, u, v, p, gamma: float = GAMMA) -> np.ndarray:
    """Conserved 2D state [4, n] (rho, rho u, rho v, E) of primitive arrays."""
    rho, u, v, p = (np.asarray(a, dtype=np.float64) for a in (rho, u, v, p))
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def density_wave_state(mesh: Mesh, t: float = 0.0, amp: float = 0.2, gamma: float = GAMMA) -> np.ndarray:
    """Cell averages of rho = 1 + amp sin(2 pi (x - t + y - t)), u = v = 1, p = 1.
    With constant velocity and pressure the averages of rho*u, rho*v and E
    follow from the average of rho."""
    rb = cell_average_2d(mesh, lambda x, y: 1.0 + amp * np.sin(2.0 * np.pi * ((x - t) + (y - t))))
    return np.stack([rb, rb, rb, 1.0 / (gamma - 1.0) + rb])


QUADRANT_STATES = {  # (rho, u, v, p), paper Sec. 3.5 (2D Riemann problem), domain shifted by +0.5
    "left_top": (0.5323, 1.206, 0.0, 0.3),
    "right_top": (1.5, 0.0, 0.0, 1.5),
    "left_bottom": (0.138, 1.206, 1.206, 0.029),
    "right_bottom": (0.5323, 0.0, 1.206, 0.3),
}


def quadrant_state(mesh: Mesh, gamma: float = GAMMA) -> np.ndarray:
    """Four constant states by quadrant about (0.5, 0.5); the value at each
    cell's vertex mean is taken as its cell average."""
    c = mesh.vertex_means()
    left, top = c[:, 0] < 0.5, c[:, 1] >= 0.5
    prim = np.zeros((mesh.n_cells, 4))
    prim[left & top] = QUADRANT_STATES["left_top"]
    prim[~left & top] = QUADRANT_STATES["right_top"]
    prim[left & ~top] = QUADRANT_STATES["left_bottom"]
    prim[~left & ~top] = QUADRANT_STATES["right_bottom"]
    return conserved_2d(prim[:, 0], prim[:, 1], prim[:, 2], prim[:, 3], gamma)


def solenoidal_velocity(n: int, seed: int = 3, k0: float = 4.0, mach_t: float = 0.6, c: float = 1.0) -> np.ndarray:
    """Seeded divergence-free velocity on an n^3 periodic grid of [0, 2 pi)^3
    sampled at cell centres, [3, n, n, n] indexed (k, j, i) = (z, y, x).
    Spectrum E(k) ~ k^4 exp(-2 k^2 / k0^2); rms |u| = mach_t * c."""
    rng = np.random.default_rng(seed)
    kk = np.fft.fftfreq(n, d=1.0 / n)
    KZ, KY, KX = np.meshgrid(kk, kk, kk, indexing="ij")
    K2 = KX * KX + KY * KY + KZ * KZ
    Kmag = np.sqrt(K2)
    amp = np.zeros_like(Kmag)
    nz = Kmag > 0
    # per-mode amplitude so that the shell-summed energy follows E(k)
    amp[nz] = np.sqrt(Kmag[nz] ** 4 * np.exp(-2.0 * K2[nz] / (k0 * k0)) / (4.0 * np.pi * K2[nz]))
    uh = (rng.standard_normal((3, n, n, n)) + 1j * rng.standard_normal((3, n, n, n))) * amp[None]
    kvec = np.stack([KX, KY, KZ])
    kdotu = (kvec * uh).sum(axis=0)
    with np.errstate(invalid="ignore", divide="ignore"):
        proj = np.where(nz, kdotu / np.where(nz, K2, 1.0), 0.0)
    uh = uh - kvec * proj[None]
    # sample at cell centres x = (i + 1/2) h: phase shift exp(i k h / 2)
    h = 2.0 * np.pi / n
    shift = np.exp(1j * (KX + KY + KZ) * 0.5 * h)
    u = np.real(np.fft.ifftn(uh * shift[None], axes=(1, 2, 3)))
    rms = math.sqrt(float((u * u).sum(axis=0).mean()))
    return u * (mach_t * c / rms)


def turbulence_state(mesh: Mesh, seed: int = 3, k0: float = 4.0, mach_t: float = 0.6,
                     gamma: float = GAMMA) -> np.ndarray:
    """Conserved state on the n^3 periodic hexahedra of structured_hex_mesh:
    rho = 1, p = 1 / gamma (unit sound speed) and solenoidal_velocity."""
    n = int(mesh.meta["n"])
    assert mesh.n_cells == n ** 3
    u = solenoidal_velocity(n, seed, k0, mach_t).reshape(3, -1)  # cell id (k*n+j)*n+i matches (k,j,i)
    rho = np.ones(mesh.n_cells)
    p = np.full(mesh.n_cells, 1.0 / gamma)
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u).sum(axis=0)
    return np.stack([rho, rho * u[0], rho * u[1], rho * u[2], E])


# ---------------------------------------------------------------------------
# Named workloads (sizes as the paper's workloads; small variants for tests)
# ---------------------------------------------------------------------------

def isentropic_vortex_state(mesh: Mesh, t: float = 0.0, eps: float = 5.0, L: float = 10.0,
                            gamma: float = GAMMA, npts: int = 8) -> np.ndarray:
    """Cell averages of the isentropic vortex of the paper's 2D accuracy test
    (Sec. 3.1): strength eps centred at (L/2, L/2) at t = 0, carried by the
    free stream (u, v) = (1, 1) on the periodic square [0, L]^2:
      du = -eps/(2 pi) e^((1-r^2)/2) (y - yc),  dv = eps/(2 pi) e^((1-r^2)/2) (x - xc),
      T = 1 - (gamma-1) eps^2/(8 gamma pi^2) e^(1-r^2),  rho = T^(1/(gamma-1)),  p = rho T,
    the centre at (L/2 + t, L/2 + t) wrapped into the square."""
    xc = (0.5 * L + t) % L
    yc = (0.5 * L + t) % L

    def prim(x, y):
        dx = (x - xc + 0.5 * L) % L - 0.5 * L
        dy = (y - yc + 0.5 * L) % L - 0.5 * L
        r2 = dx * dx + dy * dy
        e = np.exp(0.5 * (1.0 - r2))
        u = 1.0 - eps / (2 * math.pi) * e * dy
        v = 1.0 + eps / (2 * math.pi) * e * dx
        T = 1.0 - (gamma - 1.0) * eps * eps / (8.0 * gamma * math.pi ** 2) * e * e
        rho = T ** (1.0 / (gamma - 1.0))
        return rho, u, v, rho * T

    comps = []
    for k in range(4):
        def f(x, y, k=k):
            rho, u, v, p = prim(x, y)
            return (rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v))[k]
        comps.append(cell_average_2d(mesh, f, npts=npts))
    return np.stack(comps)


SOD_STATES = ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1))   # (rho, u, v, p) left / right of the membrane


def batched_problems(count: int = 256, seed: int = 5, min_cells: int = 1000, max_cells: int = 200000,
                     orders=(2, 3, 4, 5)):
    """Independent open 2D problems of uneven size: jittered triangle meshes of
    the unit square with 2 n^2 cells, n^2 log-uniform between min_cells / 2
    and max_cells / 2; the order drawn uniformly from ``orders``; the state
    either a smooth density wave  rho = 1 + 0.2 sin(2 pi k (x cos a + y sin a)),
    (u, v) = 0.5 (cos a, sin a), p = 1, or a Sod shock tube whose membrane
    passes through the centre with normal (cos a, sin a); the angle a uniform.
    Wave averages by a 4 x 4 collapsed Gauss rule, Sod states at the vertex
    mean.  Returns a list of dicts with keys mesh, U, order, kind, angle."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        cells = math.exp(rng.uniform(math.log(min_cells), math.log(max_cells)))
        n = max(4, int(round(math.sqrt(cells / 2.0))))
        order = int(rng.choice(orders))
        ang = float(rng.uniform(0.0, 2.0 * math.pi))
        sine = bool(rng.random() < 0.5)
        m = structured_tri_mesh(n, periodic=False, jitter=0.2, seed=seed * 100003 + k)
        ca, sa = math.cos(ang), math.sin(ang)
        if sine:
            kw = int(rng.integers(1, 4))
            rb = cell_average_2d(m, lambda x, y: 1.0 + 0.2 * np.sin(2.0 * np.pi * kw * (x * ca + y * sa)), npts=4)
            U = np.stack([rb, 0.5 * ca * rb, 0.5 * sa * rb, 1.0 / (GAMMA - 1.0) + 0.125 * rb])
        else:
            c = m.vertex_means()
            left = (c[:, 0] - 0.5) * ca + (c[:, 1] - 0.5) * sa < 0.0
            prim = np.where(left[:, None], np.array(SOD_STATES[0]), np.array(SOD_STATES[1]))
            U = conserved_2d(prim[:, 0], prim[:, 1], prim[:, 2], prim[:, 3])
        out.append({"mesh": m, "U": np.ascontiguousarray(U), "order": order, "kind": "sine" if sine else "sod",
                    "angle": ang})
    return out


def concat_meshes(meshes) -> Mesh:
    """Disjoint union of open meshes (node and cell ids offset per mesh), in
    order: the layout a batch of problems has as one mesh."""
    nodes = np.concatenate([m.nodes for m in meshes])
    types = np.concatenate([m.cell_type for m in meshes])
    noff = np.cumsum([0] + [m.n_nodes for m in meshes])
    idx = np.concatenate([m.cell_idx.astype(np.int64) + noff[k] for k, m in enumerate(meshes)]).astype(np.int32)
    counts = np.concatenate([np.diff(m.cell_ptr) for m in meshes])
    ptr = np.zeros(types.size + 1, np.int64)
    np.cumsum(counts, out=ptr[1:])
    return Mesh(meshes[0].dim, nodes, types, ptr, idx, np.zeros(meshes[0].dim), "batch", {"count": len(meshes)})


def mach2_shock_states(gamma: float = GAMMA, mach: float = 2.0):
    """Pre- and post-shock primitive states (rho, u, v, w, p) of a normal shock
    of Mach number `mach` running along +x into gas at rest with rho = p = 1
    (Rankine-Hugoniot relations)."""
    m2 = mach * mach
    r = (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    pr = 1.0 + 2.0 * gamma / (gamma + 1.0) * (m2 - 1.0)
    s = mach * math.sqrt(gamma)
    return (r, s * (1.0 - 1.0 / r), 0.0, 0.0, pr), (1.0, 0.0, 0.0, 0.0, 1.0)


def shock_pulse_state(m: Mesh, gamma: float = GAMMA) -> np.ndarray:
    """Conserved state on a 3D mesh of the unit cube: a Gaussian density pulse
    rho = 1 + 0.5 exp(-|x - (0.75, 0.5, 0.5)|^2 / (2 0.08^2)) in gas at rest
    (p = 1) ahead of a planar Mach 2 shock at x = 0.4 moving along +x,
    evaluated at the cells' vertex means."""
    c = m.vertex_means()
    post, pre = mach2_shock_states(gamma)
    behind = c[:, 0] < 0.4
    prim = np.where(behind[:, None], np.array(post), np.array(pre))
    r2 = ((c - np.array([0.75, 0.5, 0.5])) ** 2).sum(1)
    prim[:, 0] = np.where(behind, prim[:, 0], 1.0 + 0.5 * np.exp(-r2 / (2 * 0.08 ** 2)))
    rho, u, v, w, p = prim.T
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, rho * w, E]))


def adjoint_problem(n: int = 55, seed: int = 4, gamma: float = GAMMA):
    """Open unit cube of n^3 hexahedra cut into 6 n^3 jittered tetrahedra
    (55^3 * 6 = 998,250 cells by default) holding shock_pulse_state."""
    m = structured_tet_mesh(n, 1.0, periodic=False, jitter=0.1, seed=seed)
    return m, shock_pulse_state(m, gamma)


def workload(name: str, scale: int | None = None):
    """Return (mesh, U0, defaults) for a named workload.

    density_wave   2,048 periodic jittered triangles (n=32), r=2, Rusanov, FP64
    quadrant       ~249,696 mixed tri/quad cells (n=408), HLLC
    turbulence     128^3 = 2,097,152 periodic hexahedra, r=3, HLLC
    ``scale`` overrides n for a smaller (or larger) instance of the same shape.
    """
    if name == "density_wave":
        n = 32 if scale is None else scale
        m = structured_tri_mesh(n, periodic=True, jitter=0.2, seed=1)
        return m, density_wave_state(m), {"order": 3, "flux": "rusanov", "cfl": 0.5, "steps": 10}
    if name == "quadrant":
        n = 408 if scale is None else scale
        m = mixed_tri_quad_mesh(n, seed=2)
        return m, quadrant_state(m), {"order": 3, "flux": "hllc", "cfl": 0.5, "steps": 200}
    if name == "turbulence":
        n = 128 if scale is None else scale
        m = structured_hex_mesh(n, 2.0 * math.pi, periodic=True, seed=3)
        return m, turbulence_state(m, seed=3), {"order": 4, "flux": "hllc", "cfl": 0.5, "steps": 100}
    raise KeyError(name)
