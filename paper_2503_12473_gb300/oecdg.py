"""Thin Python binding of the OECDG C-ABI (include/oecdg.h).

Argument marshalling only: every step of the path runs in the CUDA library
``paper_2503_12473_gb300/_build/liboecdg.so``.  There is no CPU fallback: if the
library is missing or no GPU is present, the calls raise.

Device memory and streams come from PyTorch: state arrays are contiguous
float64 CUDA tensors, passed by ``data_ptr()``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import build as _build

CDG_OK, CDG_EINVAL, CDG_ENOMEM, CDG_ECUDA, CDG_ENONPHYSICAL, CDG_ETIMEOUT, CDG_EUNSUPPORTED = range(7)
ADVECTION, BURGERS, EULER = 0, 1, 2
BASIS_Q, BASIS_P = 0, 1
PERIODIC, TRANSMISSIVE, REFLECTIVE = 0, 1, 2
RK_EULER1, RK_SSP2, RK_SSP3, RK_RK4 = 1, 2, 3, 4
MATH_RCP, MATH_SQRT = 0, 1
BATCH_GRAPH, BATCH_PERSISTENT = 1, 2

STATUS_NAMES = {0: "CDG_OK", 1: "CDG_EINVAL", 2: "CDG_ENOMEM", 3: "CDG_ECUDA", 4: "CDG_ENONPHYSICAL",
                5: "CDG_ETIMEOUT", 6: "CDG_EUNSUPPORTED"}

EXPORTED = [
    "cdg_init_mesh", "cdg_free", "cdg_last_error", "cdg_state_numel", "cdg_quad_points", "cdg_project_ic",
    "cdg_rhs", "cdg_compute_dt", "cdg_set_dt", "cdg_get_dt", "cdg_rk_stage", "cdg_oe_damp",
    "cdg_oe_coefficients", "cdg_step", "cdg_step_async", "cdg_get_time", "cdg_check_status", "cdg_launch_count",
    "cdg_profile_begin", "cdg_profile_end", "cdg_oe_damp_noalloc",
    "cdg_init_batch", "cdg_batch_free", "cdg_batch_last_error", "cdg_batch_step", "cdg_batch_check_status",
    "cdg_batch_get_time", "cdg_batch_launch_count", "cdg_batch_rows", "cdg_batch_autotune",
    "cdg_step_adjoint", "cdg_batch_set_rows", "cdg_record_numel", "cdg_step_record", "cdg_step_adjoint_recorded",
    "cdg_rk_combine", "cdg_step_graph", "cdg_math_eval",
    "cdg_batch_set_wait", "cdg_batch_set_grid", "cdg_batch_grid", "cdg_step_persistent", "cdg_set_wait",
]


class CdgError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class cdg_mesh_desc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("k", ctypes.c_int),
        ("basis", ctypes.c_int), ("system", ctypes.c_int), ("bc", ctypes.c_int * 4), ("oe", ctypes.c_int),
        ("rk", ctypes.c_int),
        ("ax", ctypes.c_double), ("bx", ctypes.c_double), ("ay", ctypes.c_double), ("by", ctypes.c_double),
        ("gamma", ctypes.c_double), ("adv_x", ctypes.c_double), ("adv_y", ctypes.c_double),
        ("cfl", ctypes.c_double),
    ]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it in-tree if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"OECDG CUDA library missing: {path}")
        _build.build()
    L = ctypes.CDLL(path)
    vp, dp, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t
    st = ctypes.c_int
    L.cdg_init_mesh.restype = st
    L.cdg_init_mesh.argtypes = [ctypes.POINTER(cdg_mesh_desc), vp, ctypes.POINTER(vp)]
    L.cdg_free.restype = st
    L.cdg_free.argtypes = [vp]
    L.cdg_last_error.restype = ctypes.c_char_p
    L.cdg_last_error.argtypes = [vp]
    L.cdg_state_numel.restype = st
    L.cdg_state_numel.argtypes = [vp, ctypes.POINTER(sz)]
    L.cdg_quad_points.restype = st
    L.cdg_quad_points.argtypes = [vp, vp, ctypes.POINTER(sz)]
    L.cdg_project_ic.restype = st
    L.cdg_project_ic.argtypes = [vp, vp, vp]
    L.cdg_rhs.restype = st
    L.cdg_rhs.argtypes = [vp, vp, ctypes.c_double, vp]
    L.cdg_compute_dt.restype = st
    L.cdg_compute_dt.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double]
    L.cdg_set_dt.restype = st
    L.cdg_set_dt.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    L.cdg_get_dt.restype = st
    L.cdg_get_dt.argtypes = [vp, dp, dp]
    L.cdg_rk_stage.restype = st
    L.cdg_rk_stage.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    L.cdg_rk_combine.restype = st
    L.cdg_rk_combine.argtypes = [vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                 ctypes.POINTER(ctypes.c_double), ctypes.c_double, vp]
    L.cdg_oe_damp.restype = st
    L.cdg_oe_damp.argtypes = [vp, vp, vp]
    L.cdg_oe_coefficients.restype = st
    L.cdg_oe_coefficients.argtypes = [vp, vp, vp, vp]
    L.cdg_step.restype = st
    L.cdg_step.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    L.cdg_step_async.restype = st
    L.cdg_step_async.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    L.cdg_step_graph.restype = st
    L.cdg_step_graph.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    L.cdg_step_persistent.restype = st
    L.cdg_step_persistent.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    L.cdg_set_wait.restype = st
    L.cdg_set_wait.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    L.cdg_get_time.restype = st
    L.cdg_get_time.argtypes = [vp, dp]
    L.cdg_check_status.restype = st
    L.cdg_check_status.argtypes = [vp]
    L.cdg_profile_begin.restype = st
    L.cdg_profile_begin.argtypes = [vp, ctypes.c_int]
    L.cdg_profile_end.restype = st
    L.cdg_profile_end.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_longlong), dp,
                                  ctypes.POINTER(ctypes.c_longlong)]
    L.cdg_oe_damp_noalloc.restype = st
    L.cdg_oe_damp_noalloc.argtypes = [ctypes.POINTER(cdg_mesh_desc), vp, ctypes.c_double, vp, vp]
    L.cdg_math_eval.restype = st
    L.cdg_math_eval.argtypes = [ctypes.c_int, vp, sz, vp, vp]
    L.cdg_init_batch.restype = st
    L.cdg_init_batch.argtypes = [ctypes.POINTER(cdg_mesh_desc), ctypes.c_int, vp, ctypes.POINTER(vp)]
    L.cdg_batch_free.restype = st
    L.cdg_batch_free.argtypes = [vp]
    L.cdg_batch_last_error.restype = ctypes.c_char_p
    L.cdg_batch_last_error.argtypes = [vp]
    L.cdg_batch_step.restype = st
    L.cdg_batch_step.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int]
    L.cdg_batch_check_status.restype = st
    L.cdg_batch_check_status.argtypes = [vp]
    L.cdg_batch_get_time.restype = st
    L.cdg_batch_get_time.argtypes = [vp, dp]
    L.cdg_batch_launch_count.restype = st
    L.cdg_batch_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.cdg_batch_set_rows.restype = st
    L.cdg_batch_set_rows.argtypes = [vp, ctypes.c_int]
    L.cdg_batch_rows.restype = st
    L.cdg_batch_rows.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.cdg_batch_autotune.restype = st
    L.cdg_batch_autotune.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]
    L.cdg_batch_set_wait.restype = st
    L.cdg_batch_set_wait.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    L.cdg_batch_set_grid.restype = st
    L.cdg_batch_set_grid.argtypes = [vp, ctypes.c_int]
    L.cdg_batch_grid.restype = st
    L.cdg_batch_grid.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.cdg_launch_count.restype = st
    L.cdg_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.cdg_step_adjoint.restype = st
    L.cdg_step_adjoint.argtypes = [vp, vp, vp, vp, vp]
    L.cdg_record_numel.restype = st
    L.cdg_record_numel.argtypes = [vp, ctypes.POINTER(sz)]
    L.cdg_step_record.restype = st
    L.cdg_step_record.argtypes = [vp, vp, vp]
    L.cdg_step_adjoint_recorded.restype = st
    L.cdg_step_adjoint_recorded.argtypes = [vp, vp, vp, vp, vp]
    _lib = L
    return L


def _ptr(t) -> int:
    """Device pointer of a contiguous float64 CUDA tensor (or None)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


@dataclass
class MeshDesc:
    dim: int = 2
    nx: int = 64
    ny: int = 64
    k: int = 2
    basis: int = BASIS_Q
    system: int = EULER
    bc: object = PERIODIC  # one condition for every side, or (x-low, x-high, y-low, y-high)
    oe: int = 1
    rk: int = RK_SSP3
    ax: float = 0.0
    bx: float = 1.0
    ay: float = 0.0
    by: float = 1.0
    gamma: float = 1.4
    adv_x: float = 1.0
    adv_y: float = 0.0
    cfl: float = 0.1

    @property
    def sides(self):
        b = self.bc
        return tuple(b) if isinstance(b, (tuple, list)) else (b, b, b, b)

    def c(self) -> cdg_mesh_desc:
        return cdg_mesh_desc(self.dim, self.nx, self.ny if self.dim == 2 else 1, self.k, self.basis, self.system,
                             (ctypes.c_int * 4)(*self.sides), self.oe, self.rk, self.ax, self.bx, self.ay, self.by,
                             self.gamma, self.adv_x, self.adv_y, self.cfl)

    @property
    def nfields(self) -> int:
        return self.dim + 2 if self.system == EULER else 1

    @property
    def nmodes(self) -> int:
        if self.dim == 1:
            return self.k + 1
        return (self.k + 1) ** 2 if self.basis == BASIS_Q else (self.k + 1) * (self.k + 2) // 2

    @property
    def shape(self):
        """The state's shape: both meshes in the padded layout, one more column
        (row) where the low x (y) side is a reflective wall."""
        nxs = self.nx + (self.sides[0] == REFLECTIVE)
        nys = (self.ny + (self.sides[2] == REFLECTIVE)) if self.dim == 2 else 1
        return (2, self.nfields, self.nmodes, nys, nxs)


def desc_from_workload(w, **over) -> MeshDesc:
    d = MeshDesc(dim=w.dim, nx=w.nx, ny=w.ny, k=w.k, basis=w.basis, system=w.system, bc=w.bc, oe=w.oe,
                 rk=w.rk, ax=w.ax, bx=w.bx, ay=w.ay, by=w.by, gamma=w.gamma, adv_x=w.adv[0], adv_y=w.adv[1],
                 cfl=w.cfl)
    for k_, v in over.items():
        setattr(d, k_, v)
    return d


def cdg_oe_damp_noalloc(desc: MeshDesc, d_uh, tau: float, d_usig, stream=None) -> None:
    """The context-free, allocation-free OE step (see include/oecdg.h).

    The C entry point takes its sizes from `desc` alone and its scratch from
    the current device, so the binding checks, before anything is launched,
    that both tensors hold exactly the state of `desc` and sit on one device,
    and makes the call with that device current on its current stream (or on
    `stream`, which must belong to the same device)."""
    import torch
    numel = 1
    for n in desc.shape:
        numel *= n
    for name, t in (("d_uh", d_uh), ("d_usig", d_usig)):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name}: expected a torch.Tensor")
        if t.numel() != numel:
            raise ValueError(f"{name} has {t.numel()} elements; the mesh description needs {numel}")
    if d_uh.device != d_usig.device:
        raise ValueError(f"d_uh is on {d_uh.device} and d_usig on {d_usig.device}: both must be on one device")
    pu, ps = _ptr(d_uh), _ptr(d_usig)
    L = load()
    with torch.cuda.device(d_uh.device):
        if stream is None:
            stream = torch.cuda.current_stream(d_uh.device)
        elif stream.device != d_uh.device:
            raise ValueError(f"stream is on {stream.device}, the states on {d_uh.device}")
        cd = desc.c()
        s = L.cdg_oe_damp_noalloc(ctypes.byref(cd), pu, tau, ps, ctypes.c_void_p(stream.cuda_stream))
    if s != CDG_OK:
        raise CdgError(s, "cdg_oe_damp_noalloc")


def cdg_math_eval(op: int, d_x, d_y, stream=None) -> None:
    """The kernels' FP64 reciprocal / square root applied elementwise (see include/oecdg.h)."""
    import torch
    L = load()
    if stream is None:
        stream = torch.cuda.current_stream()
    s = L.cdg_math_eval(op, _ptr(d_x), d_x.numel(), _ptr(d_y), ctypes.c_void_p(stream.cuda_stream))
    if s != CDG_OK:
        raise CdgError(s, "cdg_math_eval")


class Context:
    """Owner of a cdg_ctx; methods map one-to-one onto the C-ABI calls."""

    def __init__(self, desc: MeshDesc, stream=None):
        import torch
        L = load()
        self.desc = desc
        self._L = L
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        self._cdesc = desc.c()
        s = L.cdg_init_mesh(ctypes.byref(self._cdesc), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if s != CDG_OK:
            raise CdgError(s, "cdg_init_mesh")
        self.h = h

    def _ck(self, s: int, what: str):
        if s != CDG_OK:
            msg = self._L.cdg_last_error(self.h)
            raise CdgError(s, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._L.cdg_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- the C-ABI -------------------------------------------------------
    def cdg_state_numel(self) -> int:
        n = ctypes.c_size_t()
        self._ck(self._L.cdg_state_numel(self.h, ctypes.byref(n)), "cdg_state_numel")
        return n.value

    def cdg_quad_points(self, d_xy=None) -> int:
        n = ctypes.c_size_t()
        self._ck(self._L.cdg_quad_points(self.h, _ptr(d_xy), ctypes.byref(n)), "cdg_quad_points")
        return n.value

    def cdg_project_ic(self, d_vals, d_u):
        self._ck(self._L.cdg_project_ic(self.h, _ptr(d_vals), _ptr(d_u)), "cdg_project_ic")

    def cdg_rhs(self, d_u, tau_max: float, d_L):
        self._ck(self._L.cdg_rhs(self.h, _ptr(d_u), tau_max, _ptr(d_L)), "cdg_rhs")

    def cdg_compute_dt(self, d_u, t: float = 0.0, T_end: float = 0.0):
        self._ck(self._L.cdg_compute_dt(self.h, _ptr(d_u), t, T_end), "cdg_compute_dt")

    def cdg_set_dt(self, tau: float, tau_max: float):
        self._ck(self._L.cdg_set_dt(self.h, tau, tau_max), "cdg_set_dt")

    def cdg_get_dt(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        self._ck(self._L.cdg_get_dt(self.h, ctypes.byref(a), ctypes.byref(b)), "cdg_get_dt")
        return a.value, b.value

    def cdg_rk_stage(self, l: int, d_un, d_ul, d_out):
        self._ck(self._L.cdg_rk_stage(self.h, l, _ptr(d_un), _ptr(d_ul), _ptr(d_out)), "cdg_rk_stage")

    def cdg_rk_combine(self, d_ul, terms, coefs, ct: float, d_out):
        n = len(terms)
        tp = (ctypes.c_void_p * max(n, 1))(*[_ptr(t) for t in terms])
        cp = (ctypes.c_double * max(n, 1))(*[float(c) for c in coefs])
        self._ck(self._L.cdg_rk_combine(self.h, _ptr(d_ul), n, tp, cp, float(ct), _ptr(d_out)), "cdg_rk_combine")

    def cdg_oe_damp(self, d_uh, d_usig):
        self._ck(self._L.cdg_oe_damp(self.h, _ptr(d_uh), _ptr(d_usig)), "cdg_oe_damp")

    def cdg_oe_coefficients(self, d_uh, d_delta=None, d_sigma=None):
        self._ck(self._L.cdg_oe_coefficients(self.h, _ptr(d_uh), _ptr(d_delta), _ptr(d_sigma)),
                 "cdg_oe_coefficients")

    def cdg_step(self, d_u, t: float = 0.0, T_end: float = 0.0, nsteps: int = 1):
        self._ck(self._L.cdg_step(self.h, _ptr(d_u), t, T_end, nsteps), "cdg_step")

    def cdg_step_async(self, d_u, t: float = 0.0, T_end: float = 0.0, nsteps: int = 1):
        self._ck(self._L.cdg_step_async(self.h, _ptr(d_u), t, T_end, nsteps), "cdg_step_async")

    def cdg_step_graph(self, d_u, t: float = 0.0, T_end: float = 0.0, nsteps: int = 1):
        self._ck(self._L.cdg_step_graph(self.h, _ptr(d_u), t, T_end, nsteps), "cdg_step_graph")

    def cdg_step_persistent(self, d_u, t: float = 0.0, T_end: float = 0.0, nsteps: int = 1):
        self._ck(self._L.cdg_step_persistent(self.h, _ptr(d_u), t, T_end, nsteps), "cdg_step_persistent")

    def cdg_set_wait(self, limit_s: float, withheld: int = 0):
        self._ck(self._L.cdg_set_wait(self.h, ctypes.c_double(limit_s), withheld), "cdg_set_wait")

    def cdg_step_adjoint(self, d_un, d_lam_next, d_lam, d_gtau=None):
        self._ck(self._L.cdg_step_adjoint(self.h, _ptr(d_un), _ptr(d_lam_next), _ptr(d_lam), _ptr(d_gtau)),
                 "cdg_step_adjoint")

    def cdg_record_numel(self) -> int:
        n = ctypes.c_size_t()
        self._ck(self._L.cdg_record_numel(self.h, ctypes.byref(n)), "cdg_record_numel")
        return n.value

    def cdg_step_record(self, d_u, d_rec):
        self._ck(self._L.cdg_step_record(self.h, _ptr(d_u), _ptr(d_rec)), "cdg_step_record")

    def cdg_step_adjoint_recorded(self, d_rec, d_lam_next, d_lam, d_gtau=None):
        self._ck(self._L.cdg_step_adjoint_recorded(self.h, _ptr(d_rec), _ptr(d_lam_next), _ptr(d_lam), _ptr(d_gtau)),
                 "cdg_step_adjoint_recorded")

    def cdg_get_time(self) -> float:
        t = ctypes.c_double()
        self._ck(self._L.cdg_get_time(self.h, ctypes.byref(t)), "cdg_get_time")
        return t.value

    def cdg_check_status(self) -> int:
        return self._L.cdg_check_status(self.h)

    def cdg_launch_count(self) -> int:
        n = ctypes.c_longlong()
        self._ck(self._L.cdg_launch_count(self.h, ctypes.byref(n)), "cdg_launch_count")
        return n.value

    def cdg_profile_begin(self, max_launches: int):
        self._ck(self._L.cdg_profile_begin(self.h, max_launches), "cdg_profile_begin")

    def cdg_profile_end(self):
        """Returns {'stage': (ms_total, launches), 'oe': (ms_total, launches)}."""
        a, c = ctypes.c_double(), ctypes.c_double()
        b, d = ctypes.c_longlong(), ctypes.c_longlong()
        self._ck(self._L.cdg_profile_end(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                         ctypes.byref(d)), "cdg_profile_end")
        return {"stage": (a.value, b.value), "oe": (c.value, d.value)}

    # ---- conveniences (marshalling only) ----------------------------------
    def zeros(self):
        import torch
        return torch.zeros(self.desc.shape, dtype=torch.float64, device="cuda")

    def project(self, fn):
        """Sample u0 = fn(xy[npts, dim]) -> [npts, F] at the context's points and project."""
        import numpy as np
        import torch
        n = self.cdg_quad_points(None)
        xy = torch.empty((n, self.desc.dim), dtype=torch.float64, device="cuda")
        self.cdg_quad_points(xy)
        vals = np.ascontiguousarray(fn(xy.cpu().numpy()), dtype=np.float64).reshape(n, self.desc.nfields)
        dv = torch.from_numpy(vals).cuda()
        u = self.zeros()
        self.cdg_project_ic(dv, u)
        return u


class Batch:
    """Owner of a cdg_batch (many independent 2D Euler Q^2 meshes stepped together).

    Without a stream the library creates its own non-blocking stream: results
    are ready after cdg_batch_check_status() (or torch.cuda.synchronize())."""

    def __init__(self, descs, stream=None):
        L = load()
        self._L = L
        self.descs = list(descs)
        self.n = len(self.descs)
        arr = (cdg_mesh_desc * self.n)(*[d.c() for d in self.descs])
        self._arr = arr
        h = ctypes.c_void_p()
        sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else ctypes.c_void_p()
        s = L.cdg_init_batch(arr, self.n, sp, ctypes.byref(h))
        if s != CDG_OK:
            raise CdgError(s, "cdg_init_batch")
        self.h = h

    def _ck(self, s, what):
        if s != CDG_OK:
            msg = self._L.cdg_batch_last_error(self.h)
            raise CdgError(s, f"{what}: {msg.decode() if msg else ''}")

    def _ptrs(self, states):
        if len(states) != self.n:
            raise ValueError("one state per instance")
        return (ctypes.c_void_p * self.n)(*[_ptr(u) for u in states])

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._L.cdg_batch_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cdg_batch_step(self, states, nsteps: int = 1, use_graph: bool = False, persistent: bool = False):
        self._keep = self._ptrs(states)
        flags = (BATCH_GRAPH if use_graph else 0) | (BATCH_PERSISTENT if persistent else 0)
        self._ck(self._L.cdg_batch_step(self.h, self._keep, nsteps, flags), "cdg_batch_step")

    def cdg_batch_set_wait(self, limit_s: float, withheld: int = 0):
        self._ck(self._L.cdg_batch_set_wait(self.h, ctypes.c_double(limit_s), withheld), "cdg_batch_set_wait")

    def cdg_batch_set_grid(self, blocks_per_sm: int):
        self._ck(self._L.cdg_batch_set_grid(self.h, blocks_per_sm), "cdg_batch_set_grid")

    def cdg_batch_grid(self):
        """(blocks per SM, total blocks) of the persistent grid."""
        b, g = ctypes.c_int(), ctypes.c_int()
        self._ck(self._L.cdg_batch_grid(self.h, ctypes.byref(b), ctypes.byref(g)), "cdg_batch_grid")
        return b.value, g.value

    def cdg_batch_check_status(self) -> int:
        return self._L.cdg_batch_check_status(self.h)

    def cdg_batch_get_time(self):
        import numpy as np
        t = np.zeros(self.n)
        self._ck(self._L.cdg_batch_get_time(self.h, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                 "cdg_batch_get_time")
        return t

    def cdg_batch_launch_count(self) -> int:
        n = ctypes.c_longlong()
        self._ck(self._L.cdg_batch_launch_count(self.h, ctypes.byref(n)), "cdg_batch_launch_count")
        return n.value

    def cdg_batch_set_rows(self, rows: int):
        self._ck(self._L.cdg_batch_set_rows(self.h, rows), "cdg_batch_set_rows")

    def cdg_batch_rows(self) -> int:
        r = ctypes.c_int()
        self._ck(self._L.cdg_batch_rows(self.h, ctypes.byref(r)), "cdg_batch_rows")
        return r.value

    def cdg_batch_autotune(self, states, cache_path=None) -> int:
        self._keep = self._ptrs(states)
        r = ctypes.c_int()
        cp = cache_path.encode() if cache_path else None
        self._ck(self._L.cdg_batch_autotune(self.h, self._keep, cp, ctypes.byref(r)), "cdg_batch_autotune")
        return r.value
