"""ctypes binding of the plain FP64 CPU oracle (``oracle/mprk_oracle.c``).

TEST INFRASTRUCTURE ONLY. The oracle checks the CUDA library; only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may load
it. Nothing in the product package imports this module.

All arrays are float64 numpy arrays in the layout [4][nz][nx] (components
rho, rho*u, rho*w, rho*E; rows bottom to top S | B | F). The 3-D oracle
(``oracle/mprk_oracle3d.c``, functions with a 3 suffix) uses [5][nz][ny][nx]
(rho, rho*u, rho*v, rho*w, rho*E).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mprk_oracle.c")
_SRC3 = os.path.join(_HERE, "mprk_oracle3d.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmprk_oracle.so")

REGION_S, REGION_B, REGION_F = 0, 1, 2
WALL_NOSLIP, WALL_SLIP = 0, 1
RHS_NS, RHS_LINEAR = 0, 1


class Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("nS", C.c_int), ("nB", C.c_int), ("nF", C.c_int),
        ("m", C.c_int), ("wall", C.c_int), ("rhs_mode", C.c_int), ("xwall", C.c_int),
        ("dt", C.c_double), ("dx", C.c_double), ("dz1", C.c_double), ("dz2", C.c_double),
        ("gamma", C.c_double), ("Pr", C.c_double), ("mu1", C.c_double), ("mu2", C.c_double),
        ("G", C.c_double), ("lin_lambda", C.c_double),
    ]

    @property
    def nz(self) -> int:
        return self.nS + self.nB + self.nF

    @property
    def shape(self):
        return (4, self.nz, self.nx)


class Problem3(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nS", C.c_int), ("nB", C.c_int), ("nF", C.c_int),
        ("m", C.c_int), ("wall", C.c_int), ("pad_", C.c_int),
        ("dt", C.c_double), ("dx", C.c_double), ("dy", C.c_double), ("dz1", C.c_double),
        ("dz2", C.c_double), ("gamma", C.c_double), ("Pr", C.c_double), ("mu1", C.c_double),
        ("mu2", C.c_double), ("G", C.c_double),
    ]

    @property
    def nz(self) -> int:
        return self.nS + self.nB + self.nF

    @property
    def shape(self):
        return (5, self.nz, self.ny, self.nx)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    deps = [_SRC, _SRC3] + [os.path.join(_HERE, h) for h in ("mprk_oracle.h", "mprk_oracle3d.h")]
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(d) for d in deps)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-Wall", "-o", tmp, _SRC, _SRC3, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(Problem)
        _lib.or_tableau.argtypes = [C.c_int, C.c_int, dp, dp, dp]
        _lib.or_rhs.argtypes = [pp, dp, dp, C.c_int, C.c_int]
        _lib.or_mprk_step.argtypes = [pp, dp, C.POINTER(C.c_longlong)]
        _lib.or_mprk_step_trace.argtypes = [pp, dp, dp, dp, dp]
        _lib.or_rk2_step.argtypes = [pp, dp, C.c_double]
        _lib.or_rk4_step.argtypes = [pp, dp, C.c_double]
        _lib.or_diagnostics.argtypes = [pp, dp, dp]
        _lib.or_stable_dt.argtypes = [pp, dp, C.c_double]
        _lib.or_stable_dt.restype = C.c_double
        _lib.or_euler_flux.argtypes = [dp, C.c_int, C.c_double, dp]
        _lib.or_euler_flux.restype = None
        _lib.or_lf_flux.argtypes = [dp, dp, C.c_int, C.c_double, dp]
        _lib.or_lf_flux.restype = None
        _lib.or_interface_state.argtypes = [pp, dp, C.c_int, dp]
        _lib.or_set_threads.argtypes = [C.c_int]
        _lib.or_set_threads.restype = None
        _lib.or_get_threads.restype = C.c_int
        _lib.or_rhs_cell_count.restype = C.c_longlong
        _lib.or_tableau_base.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp, dp, dp, dp]
        _lib.or_mprk_step_base.argtypes = [pp, C.c_int, dp, dp, dp, dp]
        _lib.or_rk_step_base.argtypes = [pp, C.c_int, dp, dp, dp, C.c_double]
        p3 = C.POINTER(Problem3)
        _lib.or3_rhs.argtypes = [p3, dp, dp, C.c_int, C.c_int]
        _lib.or3_mprk_step.argtypes = [p3, dp]
        _lib.or3_rk2_step.argtypes = [p3, dp, C.c_double]
        _lib.or3_rk4_step.argtypes = [p3, dp, C.c_double]
        _lib.or3_diagnostics.argtypes = [p3, dp, dp]
        _lib.or3_stable_dt.argtypes = [p3, dp, C.c_double]
        _lib.or3_stable_dt.restype = C.c_double
        _lib.or3_interface_state.argtypes = [p3, dp, C.c_int, C.c_int, dp]
        _lib.or3_lf_flux.argtypes = [dp, dp, C.c_int, C.c_double, dp]
        _lib.or3_lf_flux.restype = None
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_problem(nx, nS, nB, nF, m, dt, dx, dz1=None, dz2=None, gamma=1.4, Pr=0.72,
                 mu1=1.0 / 20000.0, mu2=1.0 / 5000.0, G=0.008140864714, wall=WALL_NOSLIP,
                 rhs_mode=RHS_NS, lin_lambda=0.0, xwall=0) -> Problem:
    dz1 = dx if dz1 is None else dz1
    dz2 = dx if dz2 is None else dz2
    return Problem(nx=nx, nS=nS, nB=nB, nF=nF, m=m, wall=wall, rhs_mode=rhs_mode, xwall=xwall,
                   dt=dt, dx=dx, dz1=dz1, dz2=dz2, gamma=gamma, Pr=Pr, mu1=mu1, mu2=mu2, G=G,
                   lin_lambda=lin_lambda)


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def rhs_cell_count() -> int:
    return int(lib().or_rhs_cell_count())


def get_threads() -> int:
    return int(lib().or_get_threads())


def tableau(m: int, region: int):
    ms = 2 * m
    a = np.zeros((ms, ms))
    b = np.zeros(ms)
    c = np.zeros(ms)
    rc = lib().or_tableau(m, region, _p(a), _p(b), _p(c))
    assert rc == 0
    return a, b, c


def rhs(P: Problem, W: np.ndarray, k_lo: int = 0, k_hi: int | None = None, out=None) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    assert W.shape == P.shape
    R = np.zeros_like(W) if out is None else out
    k_hi = P.nz if k_hi is None else k_hi
    rc = lib().or_rhs(C.byref(P), _p(W), _p(R), k_lo, k_hi)
    assert rc == 0
    return R


def mprk_step(P: Problem, q: np.ndarray, n: int = 1):
    """n slow steps; returns (q_next, cell RHS evaluations of one step)."""
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    assert q.shape == P.shape
    cnt = C.c_longlong(0)
    for _ in range(n):
        rc = lib().or_mprk_step(C.byref(P), _p(q), C.byref(cnt))
        assert rc == 0
    return q, int(cnt.value)


def mprk_trace(P: Problem, q: np.ndarray):
    q = np.ascontiguousarray(q, dtype=np.float64)
    ms = 2 * P.m
    Q = np.zeros((ms,) + P.shape)
    R = np.zeros((ms,) + P.shape)
    qn = np.zeros(P.shape)
    rc = lib().or_mprk_step_trace(C.byref(P), _p(q), _p(Q), _p(R), _p(qn))
    assert rc == 0
    return Q, R, qn


def rk2_step(P: Problem, q: np.ndarray, h: float, n: int = 1) -> np.ndarray:
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    for _ in range(n):
        assert lib().or_rk2_step(C.byref(P), _p(q), h) == 0
    return q


def rk4_step(P: Problem, q: np.ndarray, h: float, n: int = 1) -> np.ndarray:
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    for _ in range(n):
        assert lib().or_rk4_step(C.byref(P), _p(q), h) == 0
    return q


def diagnostics(P: Problem, q: np.ndarray) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(16)
    assert lib().or_diagnostics(C.byref(P), _p(q), _p(out)) == 0
    return out


def stable_dt(P: Problem, q: np.ndarray, cfl: float = 0.4) -> float:
    q = np.ascontiguousarray(q, dtype=np.float64)
    return float(lib().or_stable_dt(C.byref(P), _p(q), cfl))


def euler_flux(q, d: int, gamma: float = 1.4) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    F = np.zeros(4)
    lib().or_euler_flux(_p(q), d, gamma, _p(F))
    return F


def lf_flux(ql, qr, d: int, gamma: float = 1.4) -> np.ndarray:
    ql = np.ascontiguousarray(ql, dtype=np.float64)
    qr = np.ascontiguousarray(qr, dtype=np.float64)
    F = np.zeros(4)
    lib().or_lf_flux(_p(ql), _p(qr), d, gamma, _p(F))
    return F


def interface_state(P: Problem, W: np.ndarray, i: int) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = np.zeros(6)
    assert lib().or_interface_state(C.byref(P), _p(W), i, _p(out)) == 0
    return out


# ---- 3-D (App. B in full) ------------------------------------------------

def make_problem3(nx, ny, nS, nB, nF, m, dt, dx, dy=None, dz1=None, dz2=None, gamma=1.4, Pr=0.72,
                  mu1=1.0 / 20000.0, mu2=1.0 / 5000.0, G=0.008140864714, wall=WALL_NOSLIP) -> Problem3:
    dy = dx if dy is None else dy
    dz1 = dx if dz1 is None else dz1
    dz2 = dx if dz2 is None else dz2
    return Problem3(nx=nx, ny=ny, nS=nS, nB=nB, nF=nF, m=m, wall=wall, pad_=0, dt=dt, dx=dx, dy=dy,
                    dz1=dz1, dz2=dz2, gamma=gamma, Pr=Pr, mu1=mu1, mu2=mu2, G=G)


def rhs3(P: Problem3, W: np.ndarray, k_lo: int = 0, k_hi: int | None = None) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    assert W.shape == P.shape
    R = np.zeros_like(W)
    k_hi = P.nz if k_hi is None else k_hi
    assert lib().or3_rhs(C.byref(P), _p(W), _p(R), k_lo, k_hi) == 0
    return R


def mprk_step3(P: Problem3, q: np.ndarray, n: int = 1) -> np.ndarray:
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    assert q.shape == P.shape
    for _ in range(n):
        assert lib().or3_mprk_step(C.byref(P), _p(q)) == 0
    return q


def rk2_step3(P: Problem3, q: np.ndarray, h: float, n: int = 1) -> np.ndarray:
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    for _ in range(n):
        assert lib().or3_rk2_step(C.byref(P), _p(q), h) == 0
    return q


def rk4_step3(P: Problem3, q: np.ndarray, h: float, n: int = 1) -> np.ndarray:
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    for _ in range(n):
        assert lib().or3_rk4_step(C.byref(P), _p(q), h) == 0
    return q


def diagnostics3(P: Problem3, q: np.ndarray) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(16)
    assert lib().or3_diagnostics(C.byref(P), _p(q), _p(out)) == 0
    return out


def stable_dt3(P: Problem3, q: np.ndarray, cfl: float = 0.4) -> float:
    q = np.ascontiguousarray(q, dtype=np.float64)
    return float(lib().or3_stable_dt(C.byref(P), _p(q), cfl))


def interface_state3(P: Problem3, W: np.ndarray, j: int, i: int) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = np.zeros(9)
    assert lib().or3_interface_state(C.byref(P), _p(W), j, i, _p(out)) == 0
    return out


def lf_flux3(ql, qr, d: int, gamma: float = 1.4) -> np.ndarray:
    ql = np.ascontiguousarray(ql, dtype=np.float64)
    qr = np.ascontiguousarray(qr, dtype=np.float64)
    F = np.zeros(5)
    lib().or3_lf_flux(_p(ql), _p(qr), d, gamma, _p(F))
    return F


# ---- MPRK with a general base method (Sec. 3 remark) ------------------------

# (A, b, c) of the base methods: Heun (the RK2 of Table 1), the third-order
# strong-stability-preserving method of Shu and Osher, classical RK4.
BASES = {
    "rk2": (np.array([[0.0, 0.0], [1.0, 0.0]]), np.array([0.5, 0.5]), np.array([0.0, 1.0])),
    "rk3": (np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.25, 0.25, 0.0]]), np.array([1 / 6, 1 / 6, 2 / 3]),
            np.array([0.0, 1.0, 0.5])),
    "rk4": (np.array([[0.0, 0.0, 0.0, 0.0], [0.5, 0.0, 0.0, 0.0], [0.0, 0.5, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0]]),
            np.array([1 / 6, 1 / 3, 1 / 3, 1 / 6]), np.array([0.0, 0.5, 0.5, 1.0])),
}


def _base(base):
    A, b, c = BASES[base] if isinstance(base, str) else base
    A = np.ascontiguousarray(A, dtype=np.float64)
    return A.shape[0], A, np.ascontiguousarray(b, dtype=np.float64), np.ascontiguousarray(c, dtype=np.float64)


def tableau_base(m: int, region: int, base="rk2"):
    s, A, b, c = _base(base)
    ms = m * s
    a_out, b_out, c_out = np.zeros((ms, ms)), np.zeros(ms), np.zeros(ms)
    assert lib().or_tableau_base(m, region, s, _p(A), _p(b), _p(c), _p(a_out), _p(b_out), _p(c_out)) == 0
    return a_out, b_out, c_out


def mprk_step_base(P: Problem, q: np.ndarray, base="rk2", n: int = 1) -> np.ndarray:
    s, A, b, c = _base(base)
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    for _ in range(n):
        assert lib().or_mprk_step_base(C.byref(P), s, _p(A), _p(b), _p(c), _p(q)) == 0
    return q


def rk_step_base(P: Problem, q: np.ndarray, h: float, base="rk2", n: int = 1) -> np.ndarray:
    s, A, b, c = _base(base)
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    for _ in range(n):
        assert lib().or_rk_step_base(C.byref(P), s, _p(A), _p(b), _p(q), h) == 0
    return q
