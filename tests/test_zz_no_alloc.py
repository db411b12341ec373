"""The allocation-free entry point mprk_step_static, checked on the GPU
against the ordinary path (mprk_create + mprk_step).

Callers that cannot call cudaMalloc use this entry point. Examples are code
inside another framework's memory pool, processes that reserve all device
memory up front, and real-time loops that must not allocate. It keeps its
scratch in a fixed device array inside the library. The test calls it twice
in a row through the C ABI on a caller-owned device tensor, so the second
call reuses the scratch the first call left behind. The results must match
the ordinary path within the parity tolerance of the other tests (1e-12
relative per component). This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2202_11890_gb300 import workloads as W
from pairs import pair, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_11890_gb300 import build
    build.build()


@pytest.mark.parametrize("dims,m,precision", [((45, 9, 5, 11), 2, 0), ((37, 8, 6, 10), 3, 0),
                                              ((64, 30, 4, 30), 4, 1), ((96, 21, 6, 21), 3, 1)])
def test_static_entry_point_matches_mprk_step(dims, m, precision):
    from paper_2202_11890_gb300 import mprk as M
    g = W.Grid(*dims)
    q = W.gaussian_bumps(g, 41, sigma_cells=3.0)
    cfg, P, dt = pair(g, m, q0=q, precision=precision)
    # the parity tolerances of the other tests: 1e-12 in FP64; in the
    # FP32-flux mode 1e-5, because each call rebuilds that mode's reference
    # rows from the state it is given (the instance keeps those of q0)
    tol = 1e-12 if precision == 0 else 1e-5
    with M.Instance(cfg, q) as inst:
        inst.step(1)
        ref1 = inst.state()
        inst.step(2)
        ref3 = inst.state()
    qd = torch.from_numpy(q.copy()).cuda()
    M.mprk_step_static(cfg, qd, 1)        # first call
    torch.cuda.synchronize()
    out1 = qd.cpu().numpy()
    M.mprk_step_static(cfg, qd, 2)        # second call, scratch left by the first
    torch.cuda.synchronize()
    out3 = qd.cpu().numpy()
    assert np.all(rel_err(out1, ref1) <= tol), rel_err(out1, ref1)
    assert np.all(rel_err(out3, ref3) <= tol), rel_err(out3, ref3)


def test_static_entry_point_rejects_oversize_and_missing_dt():
    from paper_2202_11890_gb300 import mprk as M
    qd = torch.zeros(16, dtype=torch.float64, device="cuda")
    big = M.mprk_config_default(2048, 480, 64, 480, 8, dt=1e-3)
    rc = M.lib().mprk_step_static(C.byref(big), C.c_void_p(qd.data_ptr()), 1, None)
    assert rc == M.MPRK_EINVAL
    assert "static maximum" in M.mprk_last_error()
    nodt = M.mprk_config_default(64, 30, 4, 30, 4)
    rc = M.lib().mprk_step_static(C.byref(nodt), C.c_void_p(qd.data_ptr()), 1, None)
    assert rc == M.MPRK_EINVAL
