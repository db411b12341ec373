"""The benchmark workloads at full size, in the launch configurations the
benchmark times, against the oracle's slow step (Algorithm 1):

* the 4096x2048, m = 8 FP32-flux workload: one slow step of the stage
  graph (tensor-copied tiles), every cell within the FP32-flux bar (1e-5
  relative per component);
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
