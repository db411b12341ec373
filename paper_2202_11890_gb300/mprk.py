"""Thin ctypes binding of libmprk.so (C ABI declared in include/mprk.h).

The functions keep the C names and only marshal arguments; every step of the
computation runs in the library's CUDA kernels. Arrays are numpy float64
(host) or torch CUDA float64 tensors (device), in the layout [4][nz][nx].

The library must be built first (``paper_2202_11890_gb300.build.build()``).
There is no CPU fallback: without the library, or without a GPU, these calls
raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MPRK_OK = 0
MPRK_EINVAL = -1
MPRK_ENOMEM = -2
MPRK_EBUDGET = -3
MPRK_ECUDA = -4
MPRK_ENONFINITE = -5
MPRK_ECFL = -6
MPRK_ETIMEOUT = -7
MPRK_EBUSY = -8
MPRK_ENOTFOUND = -9

MPRK_FP64 = 0
MPRK_FP32FLUX = 1
MPRK_SCHEME_MPRK2 = 0
MPRK_SCHEME_SR_RK2 = 1
MPRK_WALL_NOSLIP = 0
MPRK_WALL_SLIP = 1
MPRK_X_PERIODIC = 0
MPRK_X_WALLS = 1
MPRK_BASE_RK2 = 0
MPRK_BASE_RK3 = 1
MPRK_BASE_RK4 = 2
MPRK_HOST = 0
MPRK_DEVICE = 1

MPRK_SOLO_CELLS_DEFAULT = 262144

MPRK_REQ_PENDING = 1
MPRK_REQ_RUNNING = 2
MPRK_REQ_DONE = 3


class mprk_config(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("nz_S", C.c_int), ("nz_B", C.c_int), ("nz_F", C.c_int),
        ("m", C.c_int), ("precision", C.c_int), ("scheme", C.c_int), ("wall", C.c_int),
        ("diag_every", C.c_int), ("x_walls", C.c_int),
        ("dt", C.c_double), ("cfl", C.c_double), ("dx", C.c_double), ("dz1", C.c_double),
        ("dz2", C.c_double), ("gamma", C.c_double), ("Pr", C.c_double), ("mu1", C.c_double),
        ("mu2", C.c_double), ("G", C.c_double), ("ny", C.c_int), ("base", C.c_int), ("dy", C.c_double),
    ]

    @property
    def nz(self) -> int:
        return self.nz_S + self.nz_B + self.nz_F

    @property
    def shape(self):
        if self.ny > 1:
            return (5, self.nz, self.ny, self.nx)
        return (4, self.nz, self.nx)


class mprk_server_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_longlong), ("max_slots", C.c_int), ("device", C.c_int),
                ("max_queue", C.c_int), ("solo_cells", C.c_int)]


class mprk_stats(C.Structure):
    _fields_ = [("t_submit", C.c_double), ("t_admit", C.c_double), ("t_finish", C.c_double),
                ("cell_stages", C.c_longlong), ("device_bytes", C.c_longlong),
                ("steps_done", C.c_int), ("error", C.c_int)]


class MprkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mprk error {code}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libmprk.so (built in-tree). Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(paper_2202_11890_gb300.build.build())")
    L = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    cfgp = C.POINTER(mprk_config)
    sig = {
        "mprk_config_default": (ip, [cfgp, ip, ip, ip, ip, ip]),
        "mprk_create": (ip, [cfgp, vp, ip, vp, C.POINTER(vp)]),
        "mprk_destroy": (ip, [vp]),
        "mprk_step": (ip, [vp, ip]),
        "mprk_get_state": (ip, [vp, vp, ip]),
        "mprk_set_state": (ip, [vp, vp, ip]),
        "mprk_step_io": (ip, [vp, C.POINTER(vp), C.POINTER(vp), ip]),
        "mprk_diagnostics": (ip, [vp, dp]),
        "mprk_sync": (ip, [vp]),
        "mprk_status": (ip, [vp]),
        "mprk_info": (ip, [vp, dp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                           C.POINTER(vp)]),
        "mprk_rhs": (ip, [vp, vp, vp, ip, ip]),
        "mprk_profile_step": (ip, [vp, dp, C.POINTER(C.c_longlong), ip]),
        "mprk_probe_fp64": (ip, [C.c_longlong, dp, dp, dp, C.POINTER(C.c_int), dp]),
        "mprk_step_static": (ip, [cfgp, vp, ip, vp]),
        "mprk_step_batch": (ip, [C.POINTER(vp), ip, ip]),
        "mprk_batch_test_withhold": (ip, [C.POINTER(vp), ip, ip, ip, C.c_longlong]),
        "mprk_selftest_convert": (ip, [vp, ip, vp, vp, vp, vp]),
        "mprk_selftest_recip": (ip, [vp, ip, vp, vp, vp]),
        "mprk_batch_tune": (ip, [C.POINTER(vp), ip, ip, dp]),
        "mprk_tune_lookup": (ip, [ip, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "mprk_tile_tune": (ip, [C.POINTER(vp), ip, ip, C.POINTER(C.c_int)]),
        "mprk_tile_lookup": (ip, [C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "mprk_tune_save": (ip, [C.c_char_p]),
        "mprk_tune_load": (ip, [C.c_char_p]),
        "mprk_tune_clear": (ip, []),
        "mprk_server_create": (ip, [C.POINTER(mprk_server_config), C.POINTER(vp)]),
        "mprk_submit": (ip, [vp, cfgp, vp, ip, C.POINTER(C.c_uint64)]),
        "mprk_poll": (ip, [vp, C.c_uint64, C.POINTER(C.c_int), vp, C.POINTER(mprk_stats)]),
        "mprk_server_stats": (ip, [vp, dp]),
        "mprk_server_profile": (ip, [vp, dp]),
        "mprk_server_destroy": (ip, [vp]),
        "mprk_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def mprk_last_error() -> str:
    return lib().mprk_last_error().decode()


def _check(rc: int) -> int:
    if rc != MPRK_OK:
        raise MprkError(rc, mprk_last_error())
    return rc


def _ptr(a):
    """(address, location) of a C-contiguous float64 numpy array or torch
    tensor; anything else raises TypeError (the library takes raw pointers)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("state buffers are C-contiguous float64 arrays")
        return a.ctypes.data, MPRK_HOST
    import torch  # device memory comes from torch
    if not (isinstance(a, torch.Tensor) and a.dtype == torch.float64 and a.is_contiguous()):
        raise TypeError("state buffers are contiguous float64 tensors or numpy arrays")
    return a.data_ptr(), (MPRK_DEVICE if a.is_cuda else MPRK_HOST)


def mprk_config_default(nx: int, nz_S: int, nz_B: int, nz_F: int, m: int, **overrides) -> mprk_config:
    cfg = mprk_config()
    _check(lib().mprk_config_default(C.byref(cfg), nx, nz_S, nz_B, nz_F, m))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def mprk_create(cfg: mprk_config, q0, stream=None) -> int:
    addr, loc = _ptr(q0)
    h = C.c_void_p()
    s = None if stream is None else C.c_void_p(int(stream))
    _check(lib().mprk_create(C.byref(cfg), C.c_void_p(addr), loc, s, C.byref(h)))
    return h.value


def mprk_destroy(h: int) -> None:
    _check(lib().mprk_destroy(C.c_void_p(h)))


def mprk_step(h: int, n: int) -> None:
    _check(lib().mprk_step(C.c_void_p(h), int(n)))


def mprk_get_state(h: int, out) -> None:
    addr, loc = _ptr(out)
    _check(lib().mprk_get_state(C.c_void_p(h), C.c_void_p(addr), loc))


def mprk_set_state(h: int, q) -> None:
    addr, loc = _ptr(q)
    _check(lib().mprk_set_state(C.c_void_p(h), C.c_void_p(addr), loc))


def mprk_step_io(h: int, q_in, q_out) -> None:
    """One slow step per input, end to end through host buffers (lists of
    numpy arrays or CPU tensors, pinned for the copy/compute overlap)."""
    if len(q_in) != len(q_out):
        raise ValueError("q_in and q_out differ in length")
    ins, outs = [], []
    for a, b in zip(q_in, q_out):
        (ai, li), (bo, lo) = _ptr(a), _ptr(b)
        if li != MPRK_HOST or lo != MPRK_HOST:
            raise ValueError("mprk_step_io takes host buffers")
        ins.append(ai)
        outs.append(bo)
    n = len(ins)
    arr_in = (C.c_void_p * max(n, 1))(*ins)
    arr_out = (C.c_void_p * max(n, 1))(*outs)
    _check(lib().mprk_step_io(C.c_void_p(h), arr_in, arr_out, n))


def mprk_diagnostics(h: int) -> np.ndarray:
    out = np.zeros(16)
    _check(lib().mprk_diagnostics(C.c_void_p(h), out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def mprk_sync(h: int) -> None:
    _check(lib().mprk_sync(C.c_void_p(h)))


def mprk_status(h: int) -> int:
    return int(lib().mprk_status(C.c_void_p(h)))


def mprk_info(h: int) -> dict:
    dt = C.c_double()
    cs = C.c_longlong()
    nb = C.c_longlong()
    st = C.c_void_p()
    _check(lib().mprk_info(C.c_void_p(h), C.byref(dt), C.byref(cs), C.byref(nb), C.byref(st)))
    return {"dt": dt.value, "cell_stages_per_step": cs.value, "device_bytes": nb.value,
            "stream": st.value or 0}


def mprk_rhs(h: int, W, R, k_lo: int, k_hi: int) -> None:
    wa, wl = _ptr(W)
    ra, rl = _ptr(R)
    if wl != MPRK_DEVICE or rl != MPRK_DEVICE:
        raise ValueError("mprk_rhs takes device tensors")
    _check(lib().mprk_rhs(C.c_void_p(h), C.c_void_p(wa), C.c_void_p(ra), k_lo, k_hi))


def mprk_profile_step(h: int):
    """Per-launch durations (ms) and cell-stages of one slow step, run as a
    graph with an event node after every launch."""
    cap = 4 * 64 + 1
    ms = np.zeros(cap)
    cells = np.zeros(cap, dtype=np.int64)
    n = lib().mprk_profile_step(C.c_void_p(h), ms.ctypes.data_as(C.POINTER(C.c_double)),
                                cells.ctypes.data_as(C.POINTER(C.c_longlong)), cap)
    if n < 0:
        raise MprkError(n, mprk_last_error())
    return ms[:n].copy(), cells[:n].copy()


def mprk_probe_fp64(iters: int = 12000) -> dict:
    """FP64 FMA throughput of the current device (register-only probe)."""
    g, r, mhz, sms, mx = C.c_double(), C.c_double(), C.c_double(), C.c_int(), C.c_double()
    _check(lib().mprk_probe_fp64(int(iters), C.byref(g), C.byref(r), C.byref(mhz), C.byref(sms), C.byref(mx)))
    return {"gflops": g.value, "dfma_per_clk_per_sm": r.value, "sm_mhz": mhz.value, "sms": sms.value,
            "max_mhz": mx.value}


def _handles(hs):
    arr = (C.c_void_p * len(hs))(*[int(h) for h in hs])
    return arr


def mprk_step_batch(handles, n: int) -> None:
    """One graph launch per slow step over all the instances: the persistent
    kernel, or for FP32 flux the per-stage launches (the tuned form)."""
    _check(lib().mprk_step_batch(_handles(handles), len(handles), int(n)))


def mprk_batch_test_withhold(handles, inst_index: int, stage: int, wait_cycles: int) -> int:
    return int(lib().mprk_batch_test_withhold(_handles(handles), len(handles), inst_index, stage,
                                              int(wait_cycles)))


def mprk_selftest_convert(x_dev, narrow, narrow_hw, widen, widen_hw) -> None:
    """Bit-operation vs hardware float/double conversions (device tensors)."""
    _check(lib().mprk_selftest_convert(C.c_void_p(x_dev.data_ptr()), int(x_dev.numel()),
                                       C.c_void_p(narrow.data_ptr()), C.c_void_p(narrow_hw.data_ptr()),
                                       C.c_void_p(widen.data_ptr()), C.c_void_p(widen_hw.data_ptr())))


def mprk_selftest_recip(x_dev, recip, rsqrt, sqrt) -> None:
    """The FP64 tiles' 1/x, 1/sqrt(x), sqrt(x) of a device tensor of doubles."""
    _check(lib().mprk_selftest_recip(C.c_void_p(x_dev.data_ptr()), int(x_dev.numel()),
                                     C.c_void_p(recip.data_ptr()), C.c_void_p(rsqrt.data_ptr()),
                                     C.c_void_p(sqrt.data_ptr())))


def mprk_batch_tune(handles, reps: int = 3) -> dict:
    """Time the batched launch choices (tiles per item, CTAs per SM, FP64
    tile shape) on these instances; the fastest goes to the table and is
    returned."""
    out = (C.c_double * 4)()
    _check(lib().mprk_batch_tune(_handles(handles), len(handles), int(reps), out))
    return {"tiles_per_item": int(out[0]), "ctas_per_sm": int(out[1]), "ms_per_step": float(out[2]),
            "tile_rows": int(out[3])}


def mprk_tune_lookup(precision: int, mean_cells: float):
    g, c, r = C.c_int(), C.c_int(), C.c_int()
    rc = lib().mprk_tune_lookup(int(precision), float(mean_cells), C.byref(g), C.byref(c), C.byref(r))
    if rc < 0:
        raise MprkError(rc, mprk_last_error())
    return {"tiles_per_item": g.value, "ctas_per_sm": c.value, "tile_rows": r.value, "tuned": bool(rc)}


def mprk_tile_tune(handles, reps: int = 3) -> int:
    """Time the six FP64 stage-tile shapes on these instances' launches; the
    fastest per size bucket goes to the table. Returns the buckets written."""
    n = C.c_int()
    _check(lib().mprk_tile_tune(_handles(handles), len(handles), int(reps), C.byref(n)))
    return n.value


def mprk_tile_lookup(cells: float):
    """The table's tile shape for a single-instance FP64 stage launch of
    `cells` cells, or None when the default rule applies."""
    r, t = C.c_int(), C.c_int()
    rc = lib().mprk_tile_lookup(float(cells), C.byref(r), C.byref(t))
    if rc < 0:
        raise MprkError(rc, mprk_last_error())
    return {"tile_rows": r.value, "threads_per_cell": t.value} if rc else None


def mprk_tune_save(path: str) -> None:
    _check(lib().mprk_tune_save(str(path).encode()))


def mprk_tune_load(path: str) -> None:
    _check(lib().mprk_tune_load(str(path).encode()))


def mprk_tune_clear() -> None:
    _check(lib().mprk_tune_clear())


MPRK_STATIC_SCRATCH_BYTES = 32 * 1024 * 1024


def mprk_step_static(cfg: mprk_config, q_dev, n: int, stream=None) -> None:
    """Advance a device tensor in place by n slow steps without allocating
    (scratch lives in the library's fixed device array)."""
    addr, loc = _ptr(q_dev)
    if loc != MPRK_DEVICE:
        raise ValueError("mprk_step_static takes a device tensor")
    s = None if stream is None else C.c_void_p(int(stream))
    _check(lib().mprk_step_static(C.byref(cfg), C.c_void_p(addr), int(n), s))


def mprk_server_create(hbm_budget_bytes: int, max_slots: int = 1024, device: int = 0,
                       max_queue: int = 1 << 20, solo_cells: int = 0) -> int:
    """solo_cells: instances of at least this many cells step alone on side
    streams (0: MPRK_SOLO_CELLS_DEFAULT for FP64 requests, FP32-flux
    requests all batched; -1: every instance in the batch)."""
    cfg = mprk_server_config(hbm_budget_bytes=int(hbm_budget_bytes), max_slots=max_slots, device=device,
                             max_queue=max_queue, solo_cells=int(solo_cells))
    h = C.c_void_p()
    _check(lib().mprk_server_create(C.byref(cfg), C.byref(h)))
    return h.value


def mprk_submit(srv: int, cfg: mprk_config, q0: np.ndarray, n_steps: int) -> int:
    """Queue a solve; returns the ticket. Raises MprkError (EBUDGET, EBUSY, EINVAL)."""
    q0 = np.ascontiguousarray(q0, dtype=np.float64)
    t = C.c_uint64()
    _check(lib().mprk_submit(C.c_void_p(srv), C.byref(cfg), q0.ctypes.data_as(C.c_void_p), int(n_steps),
                             C.byref(t)))
    return t.value


def mprk_poll(srv: int, ticket: int, out: np.ndarray | None = None):
    """(status, error, stats dict). With out given and status DONE, the result
    is copied into out and the ticket is released."""
    st = C.c_int()
    stats = mprk_stats()
    ptr = out.ctypes.data_as(C.c_void_p) if out is not None else None
    rc = lib().mprk_poll(C.c_void_p(srv), C.c_uint64(ticket), C.byref(st), ptr, C.byref(stats))
    if rc == MPRK_ENOTFOUND:
        raise MprkError(rc, mprk_last_error())
    return st.value, rc, {f: getattr(stats, f) for f, _ in mprk_stats._fields_}


def mprk_server_stats(srv: int) -> np.ndarray:
    out = np.zeros(8)
    _check(lib().mprk_server_stats(C.c_void_p(srv), out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def mprk_server_profile(srv: int) -> dict:
    """Where the server thread's time went (seconds) and the GPU seconds of
    its batched steps."""
    out = np.zeros(8)
    _check(lib().mprk_server_profile(C.c_void_p(srv), out.ctypes.data_as(C.POINTER(C.c_double))))
    keys = ("iterations", "admit_s", "step_enqueue_s", "retire_s", "inflight_wait_s", "gpu_busy_s",
            "step_span_s", "admitted")
    return {k: float(v) for k, v in zip(keys, out)}


def mprk_server_destroy(srv: int) -> None:
    _check(lib().mprk_server_destroy(C.c_void_p(srv)))


class Instance:
    """Owning handle: ``Instance(cfg, q0)``; ``step(n)``; ``state()``."""

    def __init__(self, cfg: mprk_config, q0, stream=None):
        self.cfg = cfg
        self.h = mprk_create(cfg, q0, stream)

    def step(self, n: int = 1) -> None:
        mprk_step(self.h, n)

    def state(self) -> np.ndarray:
        out = np.empty(self.cfg.shape)
        mprk_get_state(self.h, out)
        return out

    def set_state(self, q) -> None:
        mprk_set_state(self.h, q)

    def diagnostics(self) -> np.ndarray:
        return mprk_diagnostics(self.h)

    def info(self) -> dict:
        return mprk_info(self.h)

    def sync(self) -> None:
        mprk_sync(self.h)

    def status(self) -> int:
        return mprk_status(self.h)

    def close(self) -> None:
        if self.h:
            mprk_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
