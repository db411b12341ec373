"""The benchmark workloads at full size, in the launch configurations the
benchmark times, against the oracle's slow step (Algorithm 1):

* the 4096x2048, m = 8 FP32-flux workload: one slow step and twenty slow
  steps of the stage graph (tensor-copied tiles), every cell within the
  FP32-flux bar (1e-5 relative per component), and the whole 500-step run
  on a 64-column strip of the same rows, m and cell size;
* the 256 uneven instances: one persistent batched step, every instance
  equal to stepping it alone (bitwise in FP64, where both kernels run the
  same non-inlined tile; to 1e-6 in FP32 flux, where the kernels may
  contract float operations differently), and every sixteenth instance
  against the oracle (1e-12 in FP64, 1e-5 in FP32 flux).

The 2048x1024 FP64 workload is covered by test_gpu_parity.py."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_11890_gb300 import workloads as W
from pairs import oracle_threads, pair, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

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


def test_mixed_4096_one_step_full_size():
    mp = M()
    wl = W.mixed_4096()
    q0 = wl.initial_state()
    cfg, P, dt = pair(wl.grid, wl.m, q0=q0, precision=mp.MPRK_FP32FLUX)
    with mp.Instance(cfg, q0) as inst:
        inst.step(1)
        q_gpu = inst.state()
    q_or, _ = O.mprk_step(P, q0)
    err = rel_err(q_gpu, q_or)
    assert np.all(err < 1e-5), err


def _mass_drift(P, q0, q1):
    d0, d1 = O.diagnostics(P, q0), O.diagnostics(P, q1)
    return [float((d1[0] - d0[0]) / d0[0]), float((d1[4] - d0[4]) / d0[4])]


def test_mixed_4096_20_steps_against_oracle():
    """Twenty slow steps of the full-size FP32-flux workload through
    mprk_step against twenty oracle steps from the same state and dt (about
    1.6e9 oracle cell-stages on all host cores)."""
    mp = M()
    wl = W.mixed_4096()
    q0 = wl.initial_state()
    cfg, P, dt = pair(wl.grid, wl.m, q0=q0, precision=mp.MPRK_FP32FLUX)
    steps = 20
    with mp.Instance(cfg, q0) as inst:
        inst.step(steps)
        q_gpu = inst.state()
    q_or, _ = O.mprk_step(P, q0, steps)
    err = rel_err(q_gpu, q_or)
    print(f"mixed_4096 after {steps} slow steps: relative error per component {err.tolist()}; "
          f"mass drift per fluid GPU {_mass_drift(P, q0, q_gpu)} oracle {_mass_drift(P, q0, q_or)}")
    assert np.all(err < 1e-5), err


def test_mixed_strip_whole_run_against_oracle():
    """The FP32-flux workload's whole run (500 slow steps) on a 64-column
    strip: the same rows (960/128/960), m = 8 and cell size (10/4096) as the
    4096x2048 workload, Fourier modes periodic on the strip, dt from the
    Courant rule; against the oracle from the same state and dt."""
    mp = M()
    wl = W.mixed_4096()
    dx = wl.grid.dx
    g = W.Grid(64, wl.grid.nS, wl.grid.nB, wl.grid.nF, dx=dx, dz1=dx, dz2=dx)
    q0 = W.fourier_modes(g, wl.seed, periodic_on_grid=True)
    cfg, P, dt = pair(g, wl.m, q0=q0, precision=mp.MPRK_FP32FLUX)
    with mp.Instance(cfg, q0) as inst:
        inst.step(wl.steps)
        q_gpu = inst.state()
    q_or, _ = O.mprk_step(P, q0, wl.steps)
    err = rel_err(q_gpu, q_or)
    print(f"64-column strip after {wl.steps} slow steps: relative error per component {err.tolist()}; "
          f"mass drift per fluid GPU {_mass_drift(P, q0, q_gpu)} oracle {_mass_drift(P, q0, q_or)}")
    assert np.all(err < 1e-5), err


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_256_one_step_full_size(precision):
    mp = M()
    wls = W.batched_256()
    insts, probs, q0s = [], [], []
    try:
        for wl in wls:
            q0 = wl.initial_state()
            cfg, P, dt = pair(wl.grid, wl.m, q0=q0, precision=precision)
            insts.append(mp.Instance(cfg, q0))
            probs.append(P)
            q0s.append(q0)
        mp.mprk_step_batch([i.h for i in insts], 1)
        batched = [i.state() for i in insts]
        for i, q0, qb in zip(insts, q0s, batched):
            i.set_state(q0)
            i.step(1)
            if precision == 0:
                assert np.array_equal(i.state(), qb)
            else:
                assert np.all(rel_err(i.state(), qb) < 1e-6)
        bar = 1e-12 if precision == 0 else 1e-5
        for j in range(0, len(wls), 16):
            q_or, _ = O.mprk_step(probs[j], q0s[j])
            err = rel_err(batched[j], q_or)
            assert np.all(err < bar), (j, err)
    finally:
        for i in insts:
            i.close()
