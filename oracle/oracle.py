"""ctypes binding of the plain FP64 CPU oracle (oracle/oecdg_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and
by the CPU-baseline leg of ``bench.py``.  The product path never imports it.

The C library is compiled on first use with gcc (``-ffp-contract=off`` so that
no multiply-add is fused: the oracle rounds every operation separately) into
``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oecdg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboecdg_oracle.so")
_SRC_CS = os.path.join(_HERE, "oecdg_oracle_cs.c")
_LIB_CS = os.path.join(_BUILD, "liboecdg_oracle_cs.so")

ADVECTION, BURGERS, EULER = 0, 1, 2
BASIS_Q, BASIS_P = 0, 1
PERIODIC, TRANSMISSIVE, REFLECTIVE = 0, 1, 2
OK, EINVAL, ENONPHYSICAL = 0, 1, 4


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("k", ctypes.c_int),
        ("basis", ctypes.c_int), ("system", ctypes.c_int), ("bc", ctypes.c_int * 4), ("oe", ctypes.c_int),
        ("rk", ctypes.c_int),
        ("ax", ctypes.c_double), ("bx", ctypes.c_double), ("ay", ctypes.c_double), ("by", ctypes.c_double),
        ("gamma", ctypes.c_double), ("adv_x", ctypes.c_double), ("adv_y", ctypes.c_double),
        ("cfl", ctypes.c_double),
    ]


def _compile(src: str, out: str, deps, force: bool) -> None:
    if force or not os.path.exists(out) or any(os.path.getmtime(out) < os.path.getmtime(d) for d in deps):
        tmp = out + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
               "-D_GNU_SOURCE", "-o", tmp, src, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle library and its complex-step build (idempotent).
    Returns the path of the former."""
    os.makedirs(_BUILD, exist_ok=True)
    _compile(_SRC, _LIB, [_SRC], force)
    _compile(_SRC_CS, _LIB_CS, [_SRC, _SRC_CS], force)
    return _LIB


_lib_handle = None


def lib():
    global _lib_handle
    if _lib_handle is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER(_Problem)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_legendre.restype = ctypes.c_double
        L.orc_legendre.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.orc_gauss.argtypes = [ctypes.c_int, dp, dp]
        L.orc_rhs.argtypes = [P, dp, ctypes.c_double, dp]
        L.orc_bilinear.restype = ctypes.c_double
        L.orc_bilinear.argtypes = [P, dp, dp, ctypes.c_double]
        L.orc_oe_coefficients.restype = ctypes.c_int
        L.orc_oe_coefficients.argtypes = [P, dp, dp, dp, dp]
        L.orc_oe_apply.argtypes = [P, dp, ctypes.c_double, dp]
        L.orc_oe.restype = ctypes.c_int
        L.orc_oe.argtypes = [P, dp, ctypes.c_double]
        L.orc_tau_max.restype = ctypes.c_int
        L.orc_tau_max.argtypes = [P, dp, dp]
        L.orc_step_tau.restype = ctypes.c_int
        L.orc_step_tau.argtypes = [P, dp, ctypes.c_double, ctypes.c_double]
        L.orc_advance.restype = ctypes.c_int
        L.orc_advance.argtypes = [P, dp, dp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.orc_quad_points.restype = ctypes.c_size_t
        L.orc_quad_points.argtypes = [P, dp]
        L.orc_project.argtypes = [P, dp, dp]
        L.orc_eval_cells.argtypes = [P, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.orc_eval_points.argtypes = [P, dp, ctypes.c_int, ctypes.c_size_t, dp, dp]
        ip = ctypes.POINTER(ctypes.c_int)
        L.orc_rhs_cells.argtypes = [P, dp, ctypes.c_double, ctypes.c_int, ip, dp]
        L.orc_oe_cells.restype = ctypes.c_int
        L.orc_oe_cells.argtypes = [P, dp, ctypes.c_double, ctypes.c_int, ip, dp, dp, dp, dp]
        L.orc_check.restype = ctypes.c_int
        L.orc_check.argtypes = [P]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib_handle = L
    return _lib_handle


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Problem:
    """Oracle problem description (Section 2 / Section 4 of the paper)."""
    dim: int = 2
    nx: int = 8
    ny: int = 8
    k: int = 2
    basis: int = BASIS_Q
    system: int = EULER
    bc: int = PERIODIC
    oe: int = 1
    rk: int = 3
    ax: float = 0.0
    bx: float = 1.0
    ay: float = 0.0
    by: float = 1.0
    gamma: float = 1.4
    adv_x: float = 1.0
    adv_y: float = 1.0
    cfl: float = 0.1
    _c: _Problem = field(default=None, repr=False, compare=False)

    @property
    def sides(self):
        """Boundary condition of each side: (x-low, x-high, y-low, y-high)."""
        b = self.bc
        return tuple(b) if isinstance(b, (tuple, list)) else (b, b, b, b)

    def c(self) -> _Problem:
        ny = self.ny if self.dim == 2 else 1
        pc = _Problem(self.dim, self.nx, ny, self.k, self.basis, self.system, (ctypes.c_int * 4)(*self.sides),
                      self.oe, self.rk, self.ax, self.bx, self.ay, self.by, self.gamma, self.adv_x, self.adv_y,
                      self.cfl)
        if lib().orc_check(ctypes.byref(pc)) != OK:
            raise ValueError(f"invalid boundary conditions {self.sides} for system {self.system}")
        return pc

    @property
    def nxs(self) -> int:
        """Stored cells per row: nx, plus the slot of the dual cell centred on a
        reflective x-low wall (both meshes share this padded layout)."""
        return self.nx + (self.sides[0] == REFLECTIVE)

    @property
    def nys(self) -> int:
        return (self.ny + (self.sides[2] == REFLECTIVE)) if self.dim == 2 else 1

    @property
    def nfields(self) -> int:
        return self.dim + 2 if self.system == EULER else 1

    @property
    def nmodes(self) -> int:
        k = self.k
        if self.dim == 1:
            return k + 1
        return (k + 1) ** 2 if self.basis == BASIS_Q else (k + 1) * (k + 2) // 2

    def modes(self):
        """(a, b) degree pairs in storage order."""
        k = self.k
        if self.dim == 1:
            return [(a, 0) for a in range(k + 1)]
        if self.basis == BASIS_Q:
            return [(a, b) for b in range(k + 1) for a in range(k + 1)]
        return [(a, s - a) for s in range(k + 1) for a in range(s, -1, -1)]

    @property
    def shape(self):
        return (2, self.nfields, self.nmodes, self.nys, self.nxs)

    @property
    def hx(self) -> float:
        return (self.bx - self.ax) / self.nx

    @property
    def hy(self) -> float:
        return (self.by - self.ay) / self.ny if self.dim == 2 else 1.0

    def zeros(self) -> np.ndarray:
        return np.zeros(self.shape, dtype=np.float64)


def legendre(n: int, d: int, x: float) -> float:
    return lib().orc_legendre(n, d, x)


def gauss(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss(n, _dp(x), _dp(w))
    return x, w


def rhs(p: Problem, u: np.ndarray, tau_max: float) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    L = np.zeros_like(u)
    pc = p.c()
    lib().orc_rhs(ctypes.byref(pc), _dp(u), tau_max, _dp(L))
    return L


def bilinear(p: Problem, u: np.ndarray, phi: np.ndarray, tau_max: float) -> float:
    """H(u, phi) of Eq. (equcdg) for a test function given by modal coefficients."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    pc = p.c()
    return lib().orc_bilinear(ctypes.byref(pc), _dp(u), _dp(phi), tau_max)


def oe_coefficients(p: Problem, u: np.ndarray):
    """(delta [2,ny,nx,k+1], sigma [2,F], avg [2,F], status)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    delta = np.zeros((2, p.nys, p.nxs, p.k + 1))
    sigma = np.zeros((2, p.nfields))
    avg = np.zeros((2, p.nfields))
    pc = p.c()
    st = lib().orc_oe_coefficients(ctypes.byref(pc), _dp(u), _dp(delta), _dp(sigma), _dp(avg))
    return delta, sigma, avg, st


def _cells(cells) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 3))


def rhs_cells(p: Problem, u: np.ndarray, tau_max: float, cells) -> np.ndarray:
    """L of the listed cells ((mesh, i, j) rows): [n, F, M]."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    c = _cells(cells)
    out = np.zeros((len(c), p.nfields, p.nmodes))
    pc = p.c()
    lib().orc_rhs_cells(ctypes.byref(pc), _dp(u), tau_max, len(c), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                        _dp(out))
    return out


def oe_cells(p: Problem, u: np.ndarray, tau: float, cells):
    """(delta [n, k+1], sigma [2, F], avg [2, F], damped coefficients [n, F, M],
    status) for the listed cells, sigma and avg over the whole meshes."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    c = _cells(cells)
    delta = np.zeros((len(c), p.k + 1))
    sigma = np.zeros((2, p.nfields))
    avg = np.zeros((2, p.nfields))
    usig = np.zeros((len(c), p.nfields, p.nmodes))
    pc = p.c()
    st = lib().orc_oe_cells(ctypes.byref(pc), _dp(u), tau, len(c), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            _dp(delta), _dp(sigma), _dp(avg), _dp(usig))
    return delta, sigma, avg, usig, st


def oe_apply(p: Problem, u: np.ndarray, delta: np.ndarray, tau: float) -> np.ndarray:
    u = np.array(u, dtype=np.float64, copy=True, order="C")
    delta = np.ascontiguousarray(delta, dtype=np.float64)
    pc = p.c()
    lib().orc_oe_apply(ctypes.byref(pc), _dp(delta), tau, _dp(u))
    return u


def oe(p: Problem, u: np.ndarray, tau: float):
    """F_tau u (Eq. (OEstep2D) solved exactly).  Returns (u_sigma, status)."""
    u = np.array(u, dtype=np.float64, copy=True, order="C")
    pc = p.c()
    st = lib().orc_oe(ctypes.byref(pc), _dp(u), tau)
    return u, st


def tau_max(p: Problem, u: np.ndarray):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = ctypes.c_double(0.0)
    pc = p.c()
    st = lib().orc_tau_max(ctypes.byref(pc), _dp(u), ctypes.byref(out))
    return out.value, st


def step_tau(p: Problem, u: np.ndarray, tau: float, tmax: float):
    u = np.array(u, dtype=np.float64, copy=True, order="C")
    pc = p.c()
    st = lib().orc_step_tau(ctypes.byref(pc), _dp(u), tau, tmax)
    return u, st


def advance(p: Problem, u: np.ndarray, t: float = 0.0, T_end: float = 0.0, nsteps: int = 1 << 30):
    """Advance nsteps steps (or to T_end).  Returns (u, t, steps_done, status)."""
    u = np.array(u, dtype=np.float64, copy=True, order="C")
    tt = ctypes.c_double(t)
    done = ctypes.c_int(0)
    pc = p.c()
    st = lib().orc_advance(ctypes.byref(pc), _dp(u), ctypes.byref(tt), T_end, nsteps, ctypes.byref(done))
    return u, tt.value, done.value, st


def quad_points(p: Problem) -> np.ndarray:
    pc = p.c()
    n = lib().orc_quad_points(ctypes.byref(pc), None)
    xy = np.zeros((n, p.dim))
    lib().orc_quad_points(ctypes.byref(pc), _dp(xy))
    return xy


def project(p: Problem, vals: np.ndarray) -> np.ndarray:
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    u = p.zeros()
    pc = p.c()
    lib().orc_project(ctypes.byref(pc), _dp(vals), _dp(u))
    return u


def project_fn(p: Problem, fn) -> np.ndarray:
    """Project u0 = fn(xy) -> [npts, F] conserved values onto both meshes."""
    xy = quad_points(p)
    vals = np.asarray(fn(xy), dtype=np.float64).reshape(len(xy), p.nfields)
    return project(p, vals)


def eval_cells(p: Problem, u: np.ndarray, mesh: int, xi, eta=None) -> np.ndarray:
    """Field values at reference points of every cell: [ny, nx, nq, F]."""
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    eta = np.zeros_like(xi) if eta is None else np.ascontiguousarray(eta, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros((p.nys, p.nxs, len(xi), p.nfields))
    pc = p.c()
    lib().orc_eval_cells(ctypes.byref(pc), _dp(u), mesh, len(xi), _dp(xi), _dp(eta), _dp(out))
    ny = p.ny if p.dim == 2 else 1
    return out if mesh == 1 else out[:ny, :p.nx]


def eval_points(p: Problem, u: np.ndarray, mesh: int, xy: np.ndarray) -> np.ndarray:
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, p.dim)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros((len(xy), p.nfields))
    pc = p.c()
    lib().orc_eval_points(ctypes.byref(pc), _dp(u), mesh, len(xy), _dp(xy), _dp(out))
    return out


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(n)


# ------------------------------------------------------------- complex step --

_lib_cs_handle = None


def lib_cs():
    """The complex-step build of the oracle (oracle/oecdg_oracle_cs.c)."""
    global _lib_cs_handle
    if _lib_cs_handle is None:
        build()
        L = ctypes.CDLL(_LIB_CS)
        P = ctypes.POINTER(_Problem)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_advance.restype = ctypes.c_int
        L.orc_advance.argtypes = [P, dp, dp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.orc_step_jacobian.restype = ctypes.c_int
        L.orc_step_jacobian.argtypes = [P, dp, ctypes.c_int, ctypes.c_double, dp]
        _lib_cs_handle = L
    return _lib_cs_handle


def step_jvp(p: Problem, u: np.ndarray, v: np.ndarray, nsteps: int = 1, h: float = 1e-30):
    """(step(u), J v) for nsteps steps (tau from the state, no end time) by the
    complex step: the oracle run on u + i h v.  Returns (real part, Im / h,
    status)."""
    z = np.ascontiguousarray(np.asarray(u, dtype=np.float64) + 1j * h * np.asarray(v, dtype=np.float64))
    t = ctypes.c_double(0.0)
    done = ctypes.c_int(0)
    pc = p.c()
    st = lib_cs().orc_advance(ctypes.byref(pc), z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(t),
                              0.0, nsteps, ctypes.byref(done))
    return z.real.copy(), z.imag / h, st


def step_jacobian(p: Problem, u: np.ndarray, nsteps: int = 1, h: float = 1e-30):
    """The oracle's Jacobian of nsteps steps at u, one complex-step run per
    column: J [n, n] with J[r, q] = d step_r / d u_q (flattened state order).
    Returns (J, status)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    n = u.size
    J = np.zeros((n, n))
    pc = p.c()
    st = lib_cs().orc_step_jacobian(ctypes.byref(pc), _dp(u), nsteps, h, _dp(J))
    return J, st


def step_adjoint(p: Problem, u: np.ndarray, lam: np.ndarray, nsteps: int = 1):
    """The oracle's adjoint of nsteps steps at u: J^T lam, shaped like u."""
    J, st = step_jacobian(p, u, nsteps)
    return (J.T @ np.asarray(lam, dtype=np.float64).ravel()).reshape(np.shape(u)), st
