"""mprk_step_io: independent one-slow-step solves through host buffers, with
the host copies overlapped with the neighbouring steps' compute. Its results
are checked bitwise against mprk_set_state + mprk_step + mprk_get_state in
turn (FP64, FP32 flux and 3-D; pinned and pageable buffers; an output that
aliases its own input), one result against the oracle's slow step
(Algorithm 1) to 1e-12, and the argument errors."""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_11890_gb300 import workloads as W
from pairs import oracle_threads, pair, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_11890_gb300 import build
    build.build()
    oracle_threads()


def M():
    from paper_2202_11890_gb300 import mprk
    return mprk


def sequential(inst, qs):
    out = []
    for q in qs:
        inst.set_state(q)
        inst.step(1)
        out.append(inst.state())
    return out


def inputs(g, n, seed, bumps=W.gaussian_bumps):
    return [bumps(g, seed + j) for j in range(n)]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("pinned", [True, False])
def test_step_io_equals_set_step_get(precision, pinned):
    """Three different inputs (ragged 70 columns, rows not a tile multiple):
    every result bitwise equal to the sequential calls; the instance is left
    holding the last result."""
    mp = M()
    g = W.Grid(70, 21, 6, 19)
    qs = inputs(g, 3, 40)
    cfg, P, dt = pair(g, 4, q0=qs[0], precision=precision)
    with mp.Instance(cfg, qs[0]) as inst:
        ref = sequential(inst, qs)
        if pinned:
            q_in = [torch.from_numpy(q).pin_memory() for q in qs]
            q_out = [torch.empty_like(t).pin_memory() for t in q_in]
        else:
            q_in = [q.copy() for q in qs]
            q_out = [np.empty_like(q) for q in qs]
        mp.mprk_step_io(inst.h, q_in, q_out)
        for got, want in zip(q_out, ref):
            got = got.numpy() if pinned else got
            assert np.array_equal(got, want)
        assert np.array_equal(inst.state(), ref[-1])


def test_step_io_matches_oracle_and_runs_in_place():
    """Each output written over its own input; one result against the
    oracle's slow step."""
    mp = M()
    g = W.Grid(64, 30, 4, 30)
    qs = inputs(g, 4, 7)
    cfg, P, dt = pair(g, 4, q0=qs[0])
    bufs = [torch.from_numpy(q.copy()).pin_memory() for q in qs]
    with mp.Instance(cfg, qs[0]) as inst:
        ref = sequential(inst, qs)
        mp.mprk_step_io(inst.h, bufs, bufs)
    for b, want in zip(bufs, ref):
        assert np.array_equal(b.numpy(), want)
    q_or, _ = O.mprk_step(P, qs[2])
    assert np.all(rel_err(bufs[2].numpy(), q_or) < 1e-12)


def test_step_io_3d():
    mp = M()
    g = W.Grid3(36, 6, 6, 4, 7)
    qs = inputs(g, 2, 3, bumps=W.gaussian_bumps3)
    cfg = mp.mprk_config_default(g.nx, g.nS, g.nB, g.nF, 2)
    cfg.ny, cfg.dy = g.ny, g.dy
    cfg.dx, cfg.dz1, cfg.dz2 = g.dx, g.dz1, g.dz2
    with mp.Instance(cfg, qs[0]) as inst:
        ref = sequential(inst, qs)
        q_out = [np.empty_like(q) for q in qs]
        mp.mprk_step_io(inst.h, qs, q_out)
    for got, want in zip(q_out, ref):
        assert np.array_equal(got, want)


def test_step_io_errors():
    mp = M()
    g = W.Grid(32, 4, 4, 5)
    q = W.gaussian_bumps(g, 1)
    cfg, P, dt = pair(g, 2, q0=q)
    L = mp.lib()
    with mp.Instance(cfg, q) as inst:
        out = np.empty_like(q)
        arr_in = (C.c_void_p * 2)(q.ctypes.data, None)
        arr_out = (C.c_void_p * 2)(out.ctypes.data, out.ctypes.data)
        assert L.mprk_step_io(C.c_void_p(inst.h), arr_in, arr_out, 2) == mp.MPRK_EINVAL
        assert L.mprk_step_io(C.c_void_p(inst.h), arr_in, arr_out, -1) == mp.MPRK_EINVAL
        assert L.mprk_step_io(C.c_void_p(inst.h), None, arr_out, 1) == mp.MPRK_EINVAL
        assert L.mprk_step_io(C.c_void_p(inst.h), arr_in, arr_out, 0) == mp.MPRK_OK
        with pytest.raises(ValueError):
            mp.mprk_step_io(inst.h, [q], [])
        # the instance still steps after the refusals
        mp.mprk_step_io(inst.h, [q], [out])
        inst.set_state(q)
        inst.step(1)
        assert np.array_equal(out, inst.state())
