"""Thin Python binding of libhfv (include/hfv.h): argument marshalling only.

Every step of the residual path runs in the library's CUDA kernels; PyTorch
supplies device memory and streams.  The binding never falls back to CPU
arithmetic: if the shared library is missing it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhfv.so")

HFV_OK, HFV_ERR_ARG, HFV_ERR_CUDA, HFV_ERR_OOM, HFV_ERR_MESH, HFV_ERR_STENCIL, HFV_ERR_NONPHYSICAL, \
    HFV_ERR_TIMEOUT, HFV_ERR_STATE = 0, -1, -2, -3, -4, -5, -6, -7, -8
HFV_TRI, HFV_QUAD, HFV_TET, HFV_HEX, HFV_PRISM, HFV_PYRAMID = 1, 2, 3, 4, 5, 6
HFV_RUSANOV, HFV_HLLC, HFV_HLL = 0, 1, 2
HFV_HYBRID, HFV_PURE_LINEAR, HFV_PURE_CWENOZ, HFV_PURE_MUSCL = 0, 1, 2, 3
HFV_FP64, HFV_FP32 = 0, 1
HFV_CLASS_LINEAR, HFV_CLASS_CWENOZ, HFV_CLASS_MUSCL, HFV_CLASS_FIRST = 0, 1, 2, 3

KERNELS = ["linear", "tag", "count", "scan", "scatter", "cweno", "muscl", "flux", "rk", "dt", "cvt", "grad",
           "vjp_flux", "vjp_recon", "vjp_gather"]
FLUX = {"rusanov": HFV_RUSANOV, "hllc": HFV_HLLC, "hll": HFV_HLL}
SCHEME = {"hybrid": HFV_HYBRID, "linear": HFV_PURE_LINEAR, "cweno": HFV_PURE_CWENOZ, "muscl": HFV_PURE_MUSCL}
PRECISION = {"fp64": HFV_FP64, "fp32": HFV_FP32}
TIME_SCHEME = {"ssprk3": 0, "ssprk54": 1}
LIMITER = {"barth": 0, "venkatakrishnan": 1}
CWENO_VARS = {"conserved": 0, "characteristic": 1}


class HfvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libhfv error {code}: {msg}")
        self.code = code


class hfv_mesh_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_nodes", C.c_int64), ("n_cells", C.c_int64), ("node_xyz", C.c_void_p),
                ("cell_type", C.c_void_p), ("cell_node_ptr", C.c_void_p), ("cell_node_idx", C.c_void_p),
                ("period", C.c_void_p)]


class hfv_scheme_params(C.Structure):
    _fields_ = [("order", C.c_int), ("flux", C.c_int), ("scheme", C.c_int), ("nad_vars", C.c_int),
                ("precision", C.c_int), ("time_scheme", C.c_int), ("gamma", C.c_double), ("alpha_m", C.c_double),
                ("beta_m", C.c_double), ("alpha_w", C.c_double), ("beta_w", C.c_double), ("kappa", C.c_double),
                ("n_exp", C.c_double), ("lambda1_prime", C.c_double), ("cweno_eps", C.c_double),
                ("cweno_b", C.c_double), ("harten_theta", C.c_double), ("harten_eps", C.c_double),
                ("stencil_factor", C.c_double), ("limiter", C.c_int), ("cweno_vars", C.c_int), ("venkat_k", C.c_double),
                ("mu0", C.c_double), ("t0", C.c_double), ("sutherland_s", C.c_double), ("prandtl", C.c_double),
                ("visc_alpha", C.c_double), ("step_chain", C.c_int)]


_lib = None


def load():
    """Load libhfv.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhfv.so not built at {LIB_PATH}; run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i64, d = C.c_void_p, C.c_int64, C.c_double
    sig = {
        "hfv_default_params": [vp],
        "hfv_mesh_create": [vp, vp],
        "hfv_mesh_create_batch": [vp, C.c_int, vp],
        "hfv_mesh_segments": [vp, vp, vp],
        "hfv_mesh_info": [vp, vp, vp, vp],
        "hfv_mesh_connectivity": [vp, vp, vp],
        "hfv_scheme_create": [vp, vp, vp, vp],
        "hfv_scheme_info": [vp, vp],
        "hfv_get_stencils": [vp, vp, vp],
        "hfv_stencils_host": [vp, C.c_int, vp, vp, vp],
        "hfv_residual": [vp, vp, vp, vp, vp, vp],
        "hfv_compute_dt": [vp, vp, d, vp, vp],
        "hfv_step": [vp, vp, d, d, vp, vp],
        "hfv_step_many": [vp, vp, C.c_int, d, d, vp],
        "hfv_autotune": [vp, vp, C.c_int, vp, vp],
        "hfv_residual_vjp": [vp, vp, vp, vp, vp, vp],
        "hfv_mesh_volumes": [vp, vp],
        "hfv_advance_host": [vp, vp, C.c_int, d, d, vp],
        "hfv_get_queues": [vp, vp, vp],
        "hfv_status": [vp, vp, C.c_int],
        "hfv_scheme_device_bytes": [vp, vp],
        "hfv_kernel_timer": [vp, C.c_int],
        "hfv_kernel_times": [vp, vp, vp, C.c_int],
        "hfv_launch_count": [vp],
        "hfv_class_queues_static": [vp, C.c_int64, vp, vp, vp],
        "hfv_fma_rate": [C.c_int, d, vp, vp],
        "hfv_convert": [C.c_int, C.c_int64, vp, vp, vp],
        "hfv_rcp64": [C.c_int64, vp, vp, vp],
        "hfv_debug_wait": [vp, C.c_int64, C.c_int],
        "hfv_step_classes": [vp, vp, d, vp, C.c_int, vp, vp],
        "hfv_step_vjp": [vp, vp, vp, d, vp, vp],
        "hfv_scheme_setup_ms": [vp, vp],
        "hfv_scheme_set_kind": [vp, C.c_int],
        "hfv_scheme_set_shape": [vp, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.hfv_last_error.restype = C.c_char_p
    lib.hfv_last_error.argtypes = []
    lib.hfv_scheme_destroy.argtypes = [vp]
    lib.hfv_scheme_destroy.restype = None
    lib.hfv_mesh_destroy.argtypes = [vp]
    lib.hfv_mesh_destroy.restype = None
    _lib = lib
    return lib


def _check(rc: int):
    if rc != HFV_OK:
        raise HfvError(rc, load().hfv_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def default_params(**kw) -> hfv_scheme_params:
    """hfv_default_params with the given fields replaced; enumerated fields
    also take their names ("hllc", "fp32", ...).  An unknown field or name
    raises instead of being ignored."""
    p = hfv_scheme_params()
    _check(load().hfv_default_params(C.byref(p)))
    fields = {f[0] for f in hfv_scheme_params._fields_}
    names = {"flux": FLUX, "scheme": SCHEME, "precision": PRECISION, "time_scheme": TIME_SCHEME,
             "limiter": LIMITER, "cweno_vars": CWENO_VARS}
    for k, v in kw.items():
        if k not in fields:
            raise TypeError(f"unknown scheme parameter {k!r}; the fields are {sorted(fields)}")
        if k in names and isinstance(v, str):
            if v not in names[k]:
                raise ValueError(f"{k} = {v!r}: one of {sorted(names[k])}")
            v = names[k][v]
        setattr(p, k, v)
    return p


def _desc(mesh):
    keep = [np.ascontiguousarray(mesh.nodes, np.float64), np.ascontiguousarray(mesh.cell_type, np.uint8),
            np.ascontiguousarray(mesh.cell_ptr, np.int64), np.ascontiguousarray(mesh.cell_idx, np.int32),
            np.ascontiguousarray(mesh.period, np.float64)]
    return hfv_mesh_desc(mesh.dim, mesh.n_nodes, mesh.n_cells, *[k.ctypes.data for k in keep]), keep


class Mesh:
    """hfv_mesh_create / hfv_mesh_connectivity over an ``inputs.Mesh``;
    ``Mesh.batch`` = hfv_mesh_create_batch over a list of them."""

    def __init__(self, mesh, _batch=None):
        lib = load()
        self.src = mesh
        h = C.c_void_p()
        if _batch is None:
            desc, keep = _desc(mesh)
            _check(lib.hfv_mesh_create(C.byref(desc), C.byref(h)))
        else:
            pairs = [_desc(m) for m in _batch]
            arr = (hfv_mesh_desc * len(pairs))(*[d for d, _ in pairs])
            _check(lib.hfv_mesh_create_batch(arr, len(pairs), C.byref(h)))
        self.h = h
        nc, nf, dim = C.c_int64(), C.c_int64(), C.c_int()
        lib.hfv_mesh_info(self.h, C.byref(nc), C.byref(nf), C.byref(dim))
        self.n_cells, self.n_faces, self.dim = nc.value, nf.value, dim.value
        ns = C.c_int()
        _check(lib.hfv_mesh_segments(self.h, C.byref(ns), None))
        self.segments = np.zeros(ns.value + 1, np.int64)
        _check(lib.hfv_mesh_segments(self.h, C.byref(ns), self.segments.ctypes.data))

    def volumes(self) -> np.ndarray:
        """hfv_mesh_volumes: |V_c| per cell."""
        v = np.zeros(self.n_cells)
        _check(load().hfv_mesh_volumes(self.h, v.ctypes.data))
        return v

    @classmethod
    def batch(cls, meshes):
        """Independent open problems as one mesh, problem k = cells
        segments[k] .. segments[k+1] - 1."""
        return cls(None, _batch=list(meshes))

    @property
    def n_segments(self) -> int:
        """Independent problems in the mesh (hfv_mesh_segments)."""
        return self.segments.size - 1

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hfv_mesh_destroy(self.h)
            self.h = None

    def connectivity(self):
        """hfv_mesh_connectivity: (nbr, nbrf), [n_cells, 6] neighbour across
        each local face (-1 open / unused) and that face's index inside it."""
        nbr = np.zeros((self.n_cells, 6), np.int32)
        nbrf = np.zeros((self.n_cells, 6), np.int8)
        _check(load().hfv_mesh_connectivity(self.h, nbr.ctypes.data, nbrf.ctypes.data))
        return nbr, nbrf

    def stencils(self, order: int):
        """hfv_stencils_host: (central [n_cells, M], dir [n_cells, 6, Md]) of
        this mesh at `order`, built on the host (no GPU)."""
        lib = load()
        sz = np.zeros(2, np.int32)
        _check(lib.hfv_stencils_host(self.h, order, sz.ctypes.data, None, None))
        cen = np.zeros((self.n_cells, int(sz[0])), np.int32)
        dr = np.zeros((self.n_cells, 6, int(sz[1])), np.int32)
        _check(lib.hfv_stencils_host(self.h, order, sz.ctypes.data, cen.ctypes.data, dr.ctypes.data))
        return cen, dr


class Scheme:
    """hfv_scheme_create and the calls on a scheme handle."""

    def __init__(self, mesh: Mesh, stream=None, **kw):
        lib = load()
        self.mesh = mesh
        self.params = default_params(**kw)
        h = C.c_void_p()
        _check(lib.hfv_scheme_create(mesh.h, C.byref(self.params), _stream(stream), C.byref(h)))
        self.h = h
        info = (C.c_int64 * 8)()
        _check(lib.hfv_scheme_info(self.h, info))
        self.N, self.M, self.Md, self.nq, self.nfp, self.nv, self.qtot, prec = list(info)
        self.fp32 = prec == HFV_FP32
        self.n_cells = mesh.n_cells

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hfv_scheme_destroy(self.h)
            self.h = None

    @property
    def dtype(self):
        """torch dtype of the residual's state and output (FP32 or FP64)."""
        import torch
        return torch.float32 if self.fp32 else torch.float64

    def device_bytes(self) -> int:
        """hfv_scheme_device_bytes: device memory the scheme holds."""
        b = C.c_int64()
        _check(load().hfv_scheme_device_bytes(self.h, C.byref(b)))
        return b.value

    def stencils(self):
        """hfv_get_stencils: (central [n_cells, M], dir [n_cells, 6, Md])
        of the scheme, the directional entries local indices or -1."""
        cen = np.zeros((self.n_cells, self.M), np.int32)
        dr = np.zeros((self.n_cells, 6, self.Md), np.int32)
        _check(load().hfv_get_stencils(self.h, cen.ctypes.data, dr.ctypes.data))
        return cen, dr

    def _state(self, U, dtype):
        import torch
        if not (isinstance(U, torch.Tensor) and U.is_cuda and U.dtype == dtype and U.is_contiguous()
                and tuple(U.shape) == (self.nv, self.n_cells)):
            raise ValueError(f"expected a contiguous CUDA {dtype} tensor of shape {(self.nv, self.n_cells)}")
        return C.c_void_p(U.data_ptr())

    def residual(self, U, R=None, forced=None, class_out=None, stream=None):
        """hfv_residual: returns R (and fills class_out if given)."""
        import torch
        u = self._state(U, self.dtype)
        if R is None:
            R = torch.empty_like(U)
        r = self._state(R, self.dtype)
        f = C.c_void_p(forced.data_ptr()) if forced is not None else None
        co = C.c_void_p(class_out.data_ptr()) if class_out is not None else None
        for t in (forced, class_out):
            if t is not None and not (t.is_cuda and t.dtype == torch.uint8 and t.numel() == self.n_cells):
                raise ValueError("classes must be CUDA uint8 tensors of n_cells entries")
        _check(load().hfv_residual(self.h, u, r, f, co, _stream(stream)))
        return R

    def compute_dt(self, U, cfl: float, dt_out=None, stream=None):
        """hfv_compute_dt: the CFL step of each problem from the FP64 CUDA
        state U, as a device FP64 tensor (one entry per problem)."""
        import torch
        u = self._state(U, torch.float64)
        if dt_out is None:
            dt_out = torch.empty(self.mesh.n_segments, dtype=torch.float64, device=U.device)
        _check(load().hfv_compute_dt(self.h, u, cfl, C.c_void_p(dt_out.data_ptr()), _stream(stream)))
        return dt_out

    def residual_vjp(self, U, cls, lam, g=None, stream=None):
        """hfv_residual_vjp: g = lam^T dR/dU at U (FP64) with the classes cls frozen."""
        import torch
        u = self._state(U, torch.float64)
        l = self._state(lam, torch.float64)
        if not (isinstance(cls, torch.Tensor) and cls.is_cuda and cls.dtype == torch.uint8 and cls.numel() == self.n_cells):
            raise ValueError("classes must be a CUDA uint8 tensor of n_cells entries")
        if g is None:
            g = torch.empty_like(lam)
        _check(load().hfv_residual_vjp(self.h, u, C.c_void_p(cls.data_ptr()), l, self._state(g, torch.float64),
                                       _stream(stream)))
        return g

    def autotune(self, U, reps: int = 5, stream=None):
        """hfv_autotune on a state in the scheme's precision; returns the shape
        (candidate-kernel CTAs per SM, nonlinear blocks per SM, CWENOZ share %,
        candidate-kernel tile shape)."""
        u = self._state(U, self.dtype)
        shape = (C.c_int * 4)()
        _check(load().hfv_autotune(self.h, u, reps, _stream(stream), shape))
        return tuple(shape)

    def set_shape(self, shape):
        """hfv_scheme_set_shape: a launch shape as autotune returns it."""
        arr = (C.c_int * 4)(*[int(x) for x in shape])
        _check(load().hfv_scheme_set_shape(self.h, arr))

    def step(self, U, cfl: float = 0.5, dt: float = -1.0, want_dt: bool = False, stream=None):
        """hfv_step on an FP64 state in place; returns dt when want_dt (a
        float, or one per problem of a batched mesh)."""
        import torch
        u = self._state(U, torch.float64)
        out = np.zeros(self.mesh.n_segments)
        _check(load().hfv_step(self.h, u, cfl, dt, out.ctypes.data if want_dt else None, _stream(stream)))
        if not want_dt:
            return None
        return float(out[0]) if out.size == 1 else out

    def advance_host(self, U: np.ndarray, n_steps: int, cfl: float = 0.5, dt: float = -1.0, stream=None):
        """hfv_advance_host: U (host FP64 [nv, n]) advanced in place."""
        if not (U.dtype == np.float64 and U.flags.c_contiguous and U.shape == (self.nv, self.n_cells)):
            raise ValueError("expected a C-contiguous float64 array [nv, n_cells]")
        _check(load().hfv_advance_host(self.h, U.ctypes.data, n_steps, cfl, dt, _stream(stream)))
        return U

    def step_classes(self, U, dt: float, cls=None, forced: bool = False, U_out=None, stream=None):
        """hfv_step_classes: one SSP-RK3 step of U into U_out (returned) with
        the stages' classes recorded into (or, forced, taken from) cls [3, n]."""
        import torch
        u = self._state(U, torch.float64)
        if U_out is None:
            U_out = torch.empty_like(U)
        if cls is None:
            cls = torch.empty((3, self.n_cells), dtype=torch.uint8, device=U.device)
        if not (cls.is_cuda and cls.dtype == torch.uint8 and cls.is_contiguous() and cls.numel() == 3 * self.n_cells):
            raise ValueError("cls must be a contiguous CUDA uint8 tensor of 3 x n_cells")
        _check(load().hfv_step_classes(self.h, u, float(dt), C.c_void_p(cls.data_ptr()), 1 if forced else 0,
                                       self._state(U_out, torch.float64), _stream(stream)))
        return U_out, cls

    def step_vjp(self, U, cls, dt: float, lam, stream=None):
        """hfv_step_vjp: lam (dJ/dU after the step) becomes dJ/dU before it, in place."""
        import torch
        if not (cls.is_cuda and cls.dtype == torch.uint8 and cls.is_contiguous() and cls.numel() == 3 * self.n_cells):
            raise ValueError("cls must be a contiguous CUDA uint8 tensor of 3 x n_cells")
        _check(load().hfv_step_vjp(self.h, self._state(U, torch.float64), C.c_void_p(cls.data_ptr()), float(dt),
                                   self._state(lam, torch.float64), _stream(stream)))
        return lam

    def setup_ms(self):
        """hfv_scheme_setup_ms: (stencils, operators) wall time of the setup, ms."""
        ms = np.zeros(2)
        _check(load().hfv_scheme_setup_ms(self.h, ms.ctypes.data))
        return float(ms[0]), float(ms[1])

    def set_kind(self, scheme: str):
        """hfv_scheme_set_kind: hybrid or a pure scheme on the same operators."""
        _check(load().hfv_scheme_set_kind(self.h, SCHEME[scheme]))

    def debug_wait(self, consumer_wait_ns: int = 0, withhold_copies: bool = False):
        """hfv_debug_wait: testing aid of the bounded waits."""
        _check(load().hfv_debug_wait(self.h, int(consumer_wait_ns), 1 if withhold_copies else 0))

    def queues(self):
        """hfv_get_queues: (counts, [CWENOZ cells, MUSCL cells]) of the last
        residual, each queue ascending."""
        counts = np.zeros(2, np.int32)
        q = np.zeros((2, self.n_cells), np.int32)
        _check(load().hfv_get_queues(self.h, counts.ctypes.data, q.ctypes.data))
        return counts, [q[0, :counts[0]].copy(), q[1, :counts[1]].copy()]

    def kernel_timer(self, enable: bool = True):
        """hfv_kernel_timer: bracket every later launch with CUDA events."""
        _check(load().hfv_kernel_timer(self.h, 1 if enable else 0))

    def kernel_times(self, reset: bool = False):
        """hfv_kernel_times: {kernel name: (total ms, launches)}."""
        ms = np.zeros(16)
        n = np.zeros(16, np.int64)
        _check(load().hfv_kernel_times(self.h, ms.ctypes.data, n.ctypes.data, 1 if reset else 0))
        return {KERNELS[k]: (float(ms[k]), int(n[k])) for k in range(len(KERNELS))}

    def status(self, reset: bool = False):
        """hfv_status: the sticky status bits (bit 0 non-physical state);
        raises HfvError on a timed-out device wait or a CUDA error."""
        flags = C.c_int(0)
        rc = load().hfv_status(self.h, C.byref(flags), 1 if reset else 0)
        if rc not in (HFV_OK, HFV_ERR_NONPHYSICAL):
            _check(rc)
        return flags.value


def step_many(schemes, states, cfl: float = 0.5, dt: float = -1.0, stream=None):
    """hfv_step_many: one step of every (scheme, FP64 state) pair, the schemes
    on their own streams forked from and joined into ``stream``."""
    import torch
    if len(schemes) != len(states) or not schemes:
        raise ValueError("one state per scheme")
    hs = (C.c_void_p * len(schemes))(*[s.h.value for s in schemes])
    us = (C.c_void_p * len(states))(*[s._state(U, torch.float64).value for s, U in zip(schemes, states)])
    _check(load().hfv_step_many(hs, us, len(schemes), cfl, dt, _stream(stream)))


def launch_count() -> int:
    """hfv_launch_count: kernels this library launched in the process."""
    n = C.c_int64()
    _check(load().hfv_launch_count(C.byref(n)))
    return n.value


def fma_rate(kind: str = "fp64", target_ms: float = 100.0, stream=None) -> float:
    """hfv_fma_rate: the device's fused multiply-add rate in FLOP/s (2 per
    FMA); kind "fp64" (DFMA), "fp32" (FFMA) or "fp32x2" (packed FFMA2)."""
    k = {"fp64": 0, "fp32": 1, "fp32x2": 2}[kind]
    out = C.c_double()
    _check(load().hfv_fma_rate(k, float(target_ms), C.byref(out), _stream(stream)))
    return out.value


def convert(x, stream=None):
    """hfv_convert: the FP32 kernels' integer conversions applied to a
    contiguous CUDA tensor; float64 -> float32 (round to nearest even) or
    float32 -> float64 (exact)."""
    import torch
    if not x.is_cuda or not x.is_contiguous() or x.dtype not in (torch.float32, torch.float64):
        raise ValueError("convert: a contiguous CUDA float32 or float64 tensor")
    to_f32 = x.dtype == torch.float64
    out = torch.empty(x.shape, dtype=torch.float32 if to_f32 else torch.float64, device=x.device)
    _check(load().hfv_convert(1 if to_f32 else 0, x.numel(), C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                              _stream(stream)))
    return out


def rcp64(x, stream=None):
    """hfv_rcp64: the FP64 kernels' reciprocal of a contiguous CUDA float64 tensor."""
    import torch
    if not x.is_cuda or not x.is_contiguous() or x.dtype != torch.float64:
        raise ValueError("rcp64: a contiguous CUDA float64 tensor")
    out = torch.empty_like(x)
    _check(load().hfv_rcp64(x.numel(), C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def class_queues_static(classes, counts=None, queues=None, stream=None):
    """hfv_class_queues_static: compaction of a CUDA uint8 class tensor into the
    CWENOZ / MUSCL queues with the library's static scratch (no allocation in
    the library; the outputs are allocated here unless given)."""
    import torch
    if not (isinstance(classes, torch.Tensor) and classes.is_cuda and classes.dtype == torch.uint8):
        raise ValueError("classes must be a CUDA uint8 tensor")
    n = classes.numel()
    if counts is None:
        counts = torch.empty(2, dtype=torch.int32, device=classes.device)
    if queues is None:
        queues = torch.empty(2 * n, dtype=torch.int32, device=classes.device)
    _check(load().hfv_class_queues_static(C.c_void_p(classes.data_ptr()), n, C.c_void_p(counts.data_ptr()),
                                          C.c_void_p(queues.data_ptr()), _stream(stream)))
    return counts, queues
