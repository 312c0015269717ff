"""ctypes front-end of the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA path never
imports this package and this package never imports the CUDA path; the two
share only the seeded input generator.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FLUX = {"rusanov": 0, "hllc": 1, "hll": 2}
SCHEME = {"hybrid": 0, "linear": 1, "cweno": 2, "muscl": 3}
LIMITER = {"barth": 0, "venkatakrishnan": 1}
CWENO_VARS = {"conserved": 0, "characteristic": 1}
LIN, CW, MU, FIRST = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with plain IEEE semantics (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("order", C.c_int), ("flux", C.c_int), ("scheme", C.c_int), ("nad_vars", C.c_int),
                ("gamma", C.c_double), ("alpha_m", C.c_double), ("beta_m", C.c_double),
                ("alpha_w", C.c_double), ("beta_w", C.c_double), ("kappa", C.c_double),
                ("n_exp", C.c_double), ("lambda1p", C.c_double), ("cw_eps", C.c_double),
                ("cw_b", C.c_double), ("harten_theta", C.c_double), ("harten_eps", C.c_double),
                ("stencil_factor", C.c_double), ("limiter", C.c_int), ("cweno_vars", C.c_int), ("venkat_k", C.c_double),
                ("mu0", C.c_double), ("t0", C.c_double), ("suth_s", C.c_double),
                ("prandtl", C.c_double), ("visc_alpha", C.c_double)]


def default_params(**kw) -> dict:
    """Defaults: the paper's default detector margins (Fig. NADMargin (a),
    alpha_m read as 5e-3), CWENOZ eps = 1e-3, b = 4, lambda_1' = 1e3,
    Harten theta = 0.9, eps = 1e-14, deactivation (kappa dx)^n with kappa = 1, n = 1."""
    p = dict(order=3, flux="rusanov", scheme="hybrid", nad_vars=3, gamma=1.4, alpha_m=5e-3, beta_m=0.5,
             alpha_w=0.0, beta_w=0.0, kappa=1.0, n_exp=1.0, lambda1p=1e3, cw_eps=1e-3, cw_b=4.0,
             harten_theta=0.9, harten_eps=1e-14, stencil_factor=2.0, limiter="barth", cweno_vars="conserved", venkat_k=5.0,
             mu0=0.0, t0=1.0, suth_s=110.4 / 288.15, prandtl=0.72, visc_alpha=4.0 / 3.0)
    p.update(kw)
    return p


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P, D, I64, U8, I32, I8 = (C.POINTER(C.c_double), C.c_double, C.c_int64, C.POINTER(C.c_uint8),
                                  C.POINTER(C.c_int32), C.POINTER(C.c_int8))
        lib.or_last_error.restype = C.c_char_p
        lib.or_mesh_create.restype = C.c_void_p
        lib.or_mesh_create.argtypes = [C.c_int, I64, I64, P, U8, C.POINTER(C.c_int64), I32, P]
        lib.or_mesh_free.argtypes = [C.c_void_p]
        lib.or_mesh_nfaces.restype = I64
        lib.or_mesh_nfaces.argtypes = [C.c_void_p]
        lib.or_mesh_connectivity.argtypes = [C.c_void_p, I32, I8]
        lib.or_mesh_geometry.argtypes = [C.c_void_p, P, P]
        lib.or_mesh_faces.argtypes = [C.c_void_p, I32, I32, P, P, P]
        lib.or_cell_monomial_integral.restype = D
        lib.or_cell_monomial_integral.argtypes = [C.c_void_p, I64, C.c_int, C.c_int, C.c_int, C.c_int]
        lib.or_gauss_legendre.argtypes = [C.c_int, P, P]
        lib.or_scheme_create.restype = C.c_void_p
        lib.or_scheme_create.argtypes = [C.c_void_p, C.POINTER(Params)]
        lib.or_scheme_free.argtypes = [C.c_void_p]
        lib.or_scheme_sizes.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
        lib.or_stencil.argtypes = [C.c_void_p, I64, I32, I32]
        lib.or_cell_operator.argtypes = [C.c_void_p, I64, C.c_int, P]
        lib.or_cell_face_points.argtypes = [C.c_void_p, I64, P]
        lib.or_cell_face_weights.argtypes = [C.c_void_p, I64, P]
        lib.or_cell_refmap.argtypes = [C.c_void_p, I64, P, P]
        lib.or_reconstruct.argtypes = [C.c_void_p, P, I64, C.c_int, P]
        lib.or_harten_ok.argtypes = [C.c_void_p, P, I64, P]
        lib.or_nad_raw_cell.argtypes = [C.c_void_p, P, I64]
        lib.or_cweno_info.argtypes = [C.c_void_p, P, I64, C.c_int, P, P, P]
        lib.or_flux.argtypes = [C.c_int, C.c_int, D, P, P, P, P]
        lib.or_residual.argtypes = [C.c_void_p, P, P, U8, U8, U8, U8, C.POINTER(C.c_int64), I64]
        lib.or_dt.restype = D
        lib.or_dt.argtypes = [C.c_void_p, P, D]
        lib.or_rk3_step.argtypes = [C.c_void_p, P, D]
        lib.RHS = C.CFUNCTYPE(None, C.c_void_p, P, P)
        lib.or_rk3_generic.argtypes = [I64, P, D, lib.RHS, C.c_void_p]
        lib.or_rk54_step.argtypes = [C.c_void_p, P, D]
        lib.or_rk54_generic.argtypes = [I64, P, D, lib.RHS, C.c_void_p]
        lib.or_rk54_table.argtypes = [P, P]
        lib.or_euler_eigen.argtypes = [C.c_int, D, P, P, P, P]
        lib.or_ops_built.restype = I64
        lib.or_ops_built.argtypes = [C.c_void_p]
        _lib = lib
        return lib


def _p(a, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct))


def _err(lib):
    return lib.or_last_error().decode()


def euler_eigen(u, n, gamma: float = 1.4):
    """Left (rows) and right (columns) eigenvectors of dF.n/dU at the
    conserved state u along the unit normal n."""
    lib = _load()
    u = np.ascontiguousarray(u, np.float64)
    d = u.size - 2
    n = np.ascontiguousarray(n, np.float64)
    L, R = np.zeros(d * 0 + (d + 2) ** 2), np.zeros((d + 2) ** 2)
    lib.or_euler_eigen(d, gamma, _p(u), _p(n), _p(L), _p(R))
    return L.reshape(d + 2, d + 2), R.reshape(d + 2, d + 2)


def rk54_table():
    """The Shu-Osher coefficients (alpha, beta) [6][5] of the SSP-RK(5,4) step."""
    lib = _load()
    a, b = np.zeros(30), np.zeros(30)
    lib.or_rk54_table(_p(a), _p(b))
    return a.reshape(6, 5), b.reshape(6, 5)


def rk54_generic(U: np.ndarray, dt: float, rhs) -> np.ndarray:
    """One SSP-RK(5,4) step of u' = rhs(u) for a flat FP64 vector (pins)."""
    lib = _load()
    U = np.ascontiguousarray(U, np.float64).copy()
    n = U.size

    def cb(ctx, u, r):
        uu = np.ctypeslib.as_array(u, shape=(n,))
        rr = np.ctypeslib.as_array(r, shape=(n,))
        rr[:] = rhs(uu.copy())
    f = lib.RHS(cb)
    lib.or_rk54_generic(n, _p(U), dt, f, None)
    return U


def gauss_legendre(n: int):
    """The oracle's n-point Gauss-Legendre rule on [0, 1]: (points, weights)."""
    lib = _load()
    x, w = np.zeros(n), np.zeros(n)
    lib.or_gauss_legendre(n, _p(x), _p(w))
    return x, w


def flux(kind: str, UL, UR, n, gamma: float = 1.4) -> np.ndarray:
    """Riemann flux F(UL, UR, n) of kind rusanov / hll / hllc (Sec. 2.4), n a unit normal."""
    lib = _load()
    UL, UR = np.ascontiguousarray(UL, np.float64), np.ascontiguousarray(UR, np.float64)
    nn = np.ascontiguousarray(n, np.float64)
    F = np.zeros_like(UL)
    lib.or_flux(FLUX[kind], len(UL) - 2, gamma, _p(UL), _p(UR), _p(nn), _p(F))
    return F


def rk3_generic(U: np.ndarray, dt: float, rhs) -> np.ndarray:
    """One Shu-Osher SSP-RK3 step of dU/dt = rhs(U) through the oracle's stage code."""
    lib = _load()
    U = np.ascontiguousarray(U, np.float64).copy()
    n = U.size

    def cb(_ctx, u_ptr, r_ptr):
        u = np.ctypeslib.as_array(u_ptr, shape=(n,))
        r = np.ctypeslib.as_array(r_ptr, shape=(n,))
        r[:] = rhs(u.copy())

    cfun = lib.RHS(cb)
    lib.or_rk3_generic(n, _p(U), dt, cfun, None)
    return U


class Mesh:
    def __init__(self, mesh):
        self.lib = _load()
        self.src = mesh
        self.dim = mesh.dim
        self.n_cells = mesh.n_cells
        nodes = np.ascontiguousarray(mesh.nodes, np.float64)
        self._keep = (nodes, np.ascontiguousarray(mesh.cell_type, np.uint8),
                      np.ascontiguousarray(mesh.cell_ptr, np.int64), np.ascontiguousarray(mesh.cell_idx, np.int32),
                      np.ascontiguousarray(mesh.period, np.float64))
        n, t, ptr, idx, per = self._keep
        self.h = self.lib.or_mesh_create(mesh.dim, mesh.n_nodes, mesh.n_cells, _p(n), _p(t, C.c_uint8),
                                         _p(ptr, C.c_int64), _p(idx, C.c_int32), _p(per))
        if not self.h:
            raise RuntimeError("oracle mesh: " + _err(self.lib))
        self.n_faces = int(self.lib.or_mesh_nfaces(self.h))

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.or_mesh_free(self.h)
            self.h = None

    def connectivity(self):
        """(nbr, nbrf): [n_cells, 6] neighbour across each local face (-1 open
        or unused) and that face's local index inside the neighbour."""
        nbr = np.zeros((self.n_cells, 6), np.int32)
        nbrf = np.zeros((self.n_cells, 6), np.int8)
        self.lib.or_mesh_connectivity(self.h, _p(nbr, C.c_int32), _p(nbrf, C.c_int8))
        return nbr, nbrf

    def geometry(self):
        """(|V| [n_cells], centroids [n_cells, 3]) by the oracle's volume rules."""
        vol = np.zeros(self.n_cells)
        cen = np.zeros((self.n_cells, 3))
        self.lib.or_mesh_geometry(self.h, _p(vol), _p(cen))
        return vol, cen

    def faces(self):
        """Per face: owner, neighbour (-1 open), unit normal out of the owner,
        area, and the periodic shift that brings the neighbour next to the owner."""
        nf = self.n_faces
        fo, fn = np.zeros(nf, np.int32), np.zeros(nf, np.int32)
        nrm, area, sh = np.zeros((nf, 3)), np.zeros(nf), np.zeros((nf, 3))
        self.lib.or_mesh_faces(self.h, _p(fo, C.c_int32), _p(fn, C.c_int32), _p(nrm), _p(area), _p(sh))
        return fo, fn, nrm, area, sh

    def monomial_integral(self, c: int, a: int, b: int, cz: int = 0, npts: int = 8) -> float:
        """Integral of x^a y^b z^cz over cell c with npts points per direction."""
        return float(self.lib.or_cell_monomial_integral(self.h, c, a, b, cz, npts))


class Scheme:
    def __init__(self, mesh: Mesh, **kw):
        self.lib = mesh.lib
        self.mesh = mesh
        p = default_params(**kw)
        self.params = p
        cp = Params()
        for k, _ in Params._fields_:
            v = p[k]
            if k == "flux":
                v = FLUX[v] if isinstance(v, str) else v
            if k == "scheme":
                v = SCHEME[v] if isinstance(v, str) else v
            if k == "limiter":
                v = LIMITER[v] if isinstance(v, str) else v
            if k == "cweno_vars":
                v = CWENO_VARS[v] if isinstance(v, str) else v
            setattr(cp, k, v)
        self._cp = cp
        self.h = self.lib.or_scheme_create(mesh.h, C.byref(cp))
        if not self.h:
            raise RuntimeError("oracle scheme: " + _err(self.lib))
        sz = (C.c_int * 6)()
        self.lib.or_scheme_sizes(self.h, sz)
        self.N, self.M, self.Md, self.nq, self.nfp, self.nv = list(sz)
        self.dim = mesh.dim
        nf_of = {1: 3, 2: 4, 3: 4, 4: 6, 5: 5, 6: 5}
        self.nf = np.array([nf_of[int(t)] for t in mesh.src.cell_type], np.int32) if mesh.n_cells < 300000 else None

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.or_scheme_free(self.h)
            self.h = None

    def _nf(self, c):
        return {1: 3, 2: 4, 3: 4, 4: 6, 5: 5, 6: 5}[int(self.mesh.src.cell_type[c])]

    def Q(self, c):
        """Face points of cell c."""
        return self._nf(c) * self.nfp

    def stencil(self, c: int):
        """(central stencil [M] in stencil order, directional stencils [nf, Md]
        as local indices; entries past each size are padding)."""
        s = np.zeros(self.M, np.int32)
        d = np.zeros(self._nf(c) * self.Md, np.int32)
        if self.lib.or_stencil(self.h, c, _p(s, C.c_int32), _p(d, C.c_int32)) != 0:
            raise RuntimeError(_err(self.lib))
        return s, d.reshape(self._nf(c), self.Md)

    def operator(self, c: int, which: str) -> np.ndarray:
        """One of cell c's operators by name (P, Phi, OI, A, Vr, D, G, shift, nd)."""
        N, M, Md, d, nf, Q = self.N, self.M, self.Md, self.dim, self._nf(c), self.Q(c)
        shapes = {"P": (0, (N, M)), "Phi": (1, (Q, N)), "OI": (2, (N, N)), "A": (3, (M, N)),
                  "Vr": (4, (M + 1,)), "D": (5, (nf, d, Md)), "G": (6, (d, Md)), "shift": (7, (M, 3)), "nd": (8, (nf,))}
        w, shp = shapes[which]
        out = np.zeros(int(np.prod(shp)))
        if self.lib.or_cell_operator(self.h, c, w, _p(out)) != 0:
            raise RuntimeError(_err(self.lib))
        return out.reshape(shp)

    def face_points(self, c: int) -> np.ndarray:
        """Physical coordinates of cell c's face quadrature points, [Q, 3]."""
        out = np.zeros((self.Q(c), 3))
        self.lib.or_cell_face_points(self.h, c, _p(out))
        return out

    def face_weights(self, c: int) -> np.ndarray:
        """Quadrature weight times |S| of each face point of cell c."""
        out = np.zeros(self.Q(c))
        self.lib.or_cell_face_weights(self.h, c, _p(out))
        return out

    def refmap(self, c: int):
        """(x0, J^-1) of cell c's reference map xi = J^-1 (x - x0)."""
        x0, Ji = np.zeros(3), np.zeros((3, 3))
        self.lib.or_cell_refmap(self.h, c, _p(x0), _p(Ji))
        return x0, Ji

    def reconstruct(self, U: np.ndarray, c: int, cls: int) -> np.ndarray:
        """Face-point states [Q, nv] of cell c reconstructed as class cls
        (LIN, CW or MU), before the Harten bound."""
        U = np.ascontiguousarray(U, np.float64)
        out = np.zeros((self.Q(c), self.nv))
        if self.lib.or_reconstruct(self.h, _p(U), c, cls, _p(out)) != 0:
            raise RuntimeError(_err(self.lib))
        return out

    def harten_ok(self, U: np.ndarray, c: int, V: np.ndarray) -> bool:
        """Whether face states V [Q, nv] of cell c pass the Harten bound (Sec. 2.4)."""
        U = np.ascontiguousarray(U, np.float64)
        V = np.ascontiguousarray(V, np.float64)
        return bool(self.lib.or_harten_ok(self.h, _p(U), c, _p(V)))

    def nad_raw(self, U: np.ndarray, c: int) -> int:
        """The detector's raw class of cell c (Sec. 2.5), before tagging."""
        U = np.ascontiguousarray(U, np.float64)
        return int(self.lib.or_nad_raw_cell(self.h, _p(U), c))

    def cweno_info(self, U: np.ndarray, c: int, v: int):
        """(weights, indicators, CWENOZ coefficients) of variable v at cell c (Sec. 2.3)."""
        U = np.ascontiguousarray(U, np.float64)
        st = self._nf(c) + 1
        om, si, acw = np.zeros(st), np.zeros(st), np.zeros(self.N)
        self.lib.or_cweno_info(self.h, _p(U), c, v, _p(om), _p(si), _p(acw))
        return om, si, acw

    def residual(self, U: np.ndarray, forced=None, sample=None):
        """Residual R(U) [nv, n] and the raw / tagged / final classes.  With
        ``sample`` only those cells' residuals (and the classes they depend
        on) are computed; other entries are NaN / 255."""
        n = self.mesh.n_cells
        U = np.ascontiguousarray(U, np.float64)
        R = np.full((self.nv, n), np.nan)
        raw = np.full(n, 255, np.uint8)
        tag = np.full(n, 255, np.uint8)
        fin = np.full(n, 255, np.uint8)
        fp = None
        if forced is not None:
            forced = np.ascontiguousarray(forced, np.uint8)
            fp = _p(forced, C.c_uint8)
        sp, ns = None, 0
        if sample is not None:
            sample = np.ascontiguousarray(sample, np.int64)
            sp, ns = _p(sample, C.c_int64), sample.size
        rc = self.lib.or_residual(self.h, _p(U), _p(R), fp, _p(raw, C.c_uint8), _p(tag, C.c_uint8),
                                  _p(fin, C.c_uint8), sp, ns)
        if rc != 0:
            raise RuntimeError("oracle residual: " + _err(self.lib))
        return R, raw, tag, fin

    def dt(self, U: np.ndarray, cfl: float) -> float:
        """The CFL time step of state U (with the diffusion limit when mu0 > 0)."""
        U = np.ascontiguousarray(U, np.float64)
        return float(self.lib.or_dt(self.h, _p(U), cfl))

    def rk54_step(self, U: np.ndarray, dt: float) -> np.ndarray:
        """One step of the five-stage, fourth-order SSP Runge-Kutta method of
        Spiteri and Ruuth (the paper's integrator)."""
        U = np.ascontiguousarray(U, np.float64).copy()
        if self.lib.or_rk54_step(self.h, _p(U), dt) != 0:
            raise RuntimeError("oracle step: " + _err(self.lib))
        return U

    def rk3_step(self, U: np.ndarray, dt: float) -> np.ndarray:
        """One three-stage SSP-RK step of U with step dt (a new array)."""
        U = np.ascontiguousarray(U, np.float64).copy()
        if self.lib.or_rk3_step(self.h, _p(U), dt) != 0:
            raise RuntimeError("oracle step: " + _err(self.lib))
        return U
