"""MPRK with a general base method on the GPU (Sec. 3 remark: the regions'
tableaus built from any s-stage base, here the three-stage SSP method and
classical RK4), through the C ABI, against the oracle's general-base step:
every slow step to 1e-12, the single-rate scheme against the base alone,
the stage count, the batched form, and the rejection of the base where only
Heun runs (the allocation-free entry point, the FP32-flux mode)."""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_11890_gb300 import workloads as W
from pairs import oracle_threads, pair, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BASE = {"rk3": 1, "rk4": 2}


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


@pytest.mark.parametrize("base", ["rk3", "rk4"])
@pytest.mark.parametrize("dims,m,xwall", [((40, 6, 5, 7), 2, 0), ((37, 5, 6, 9), 3, 0), ((40, 6, 5, 7), 1, 0),
                                          ((36, 4, 13, 5), 4, 1)])
def test_general_base_steps_match_oracle(base, dims, m, xwall):
    """Ragged x (37 columns), Gamma inside a tile, m = 1 (the base alone), a
    buffer wider than a tile, walls in x."""
    mp = M()
    g = W.Grid(*dims)
    q = W.gaussian_bumps(g, 5 + m, sigma_cells=2.0, amp=0.03)
    cfg, P, dt = pair(g, m, q0=q, xwall=xwall)
    cfg.base = BASE[base]
    q_or = q.copy()
    with mp.Instance(cfg, q) as inst:
        for _ in range(3):
            inst.step(1)
            q_or = O.mprk_step_base(P, q_or, base)
            err = rel_err(inst.state(), q_or)
            assert np.all(err < 1e-12), err


@pytest.mark.parametrize("base", ["rk3", "rk4"])
def test_single_rate_scheme_is_the_base_alone(base):
    """MPRK_SCHEME_SR_RK2 with a general base: m steps of the base with
    dt/m over the whole grid."""
    mp = M()
    g = W.Grid(40, 6, 5, 7)
    q = W.gaussian_bumps(g, 11, sigma_cells=2.0, amp=0.03)
    cfg, P, dt = pair(g, 3, q0=q, scheme=mp.MPRK_SCHEME_SR_RK2)
    cfg.base = BASE[base]
    with mp.Instance(cfg, q) as inst:
        inst.step(2)
        got = inst.state()
    ref = O.rk_step_base(P, q, dt / 3, base, 6)
    assert np.all(rel_err(got, ref) < 1e-12)


@pytest.mark.parametrize("base,s", [("rk3", 3), ("rk4", 4)])
def test_stage_count_and_profile(base, s):
    mp = M()
    g = W.Grid(40, 6, 5, 7)
    m = 3
    q = W.gaussian_bumps(g, 2, sigma_cells=2.0, amp=0.03)
    cfg, P, dt = pair(g, m, q0=q)
    cfg.base = BASE[base]
    with mp.Instance(cfg, q) as inst:
        info = inst.info()
        assert info["cell_stages_per_step"] == g.nx * (s * g.nS + s * m * (g.nB + g.nF))
        ms, cells = mp.mprk_profile_step(inst.h)
        assert len(ms) == s * m + 1
        assert sum(cells) == info["cell_stages_per_step"]
        got = inst.state()
    ref = O.mprk_step_base(P, q, base)
    assert np.all(rel_err(got, ref) < 1e-12)


def test_batch_with_general_bases_equals_each_alone():
    """One persistent launch over Heun, RK3 and RK4 instances of different
    sizes and m (s m stages each): each instance bitwise equal to stepping
    it alone, the RK4 one against the oracle's general-base step."""
    mp = M()
    cases = []
    for j, (dims, m, base) in enumerate([((40, 6, 5, 7), 2, None), ((37, 5, 6, 9), 3, "rk3"),
                                         ((70, 12, 6, 14), 2, "rk4"), ((36, 4, 13, 5), 4, "rk4")]):
        g = W.Grid(*dims)
        q = W.gaussian_bumps(g, 60 + j, sigma_cells=2.0, amp=0.03)
        cfg, P, dt = pair(g, m, q0=q)
        if base:
            cfg.base = BASE[base]
        cases.append((cfg, P, q, base))
    alone = []
    for cfg, P, q, base in cases:
        with mp.Instance(cfg, q) as inst:
            inst.step(2)
            alone.append(inst.state())
    insts = [mp.Instance(cfg, q) for cfg, P, q, base in cases]
    try:
        mp.mprk_step_batch([i.h for i in insts], 2)
        for i, ref, (cfg, P, q, base) in zip(insts, alone, cases):
            assert np.array_equal(i.state(), ref), (base, rel_err(i.state(), ref))
            assert i.status() == 0
        cfg, P, q, base = cases[2]
        q_or = O.mprk_step_base(P, O.mprk_step_base(P, q, base), base)
        assert np.all(rel_err(insts[2].state(), q_or) < 1e-12)
    finally:
        for i in insts:
            i.close()


def test_general_base_rejected_where_only_heun_runs():
    mp = M()
    g = W.Grid(32, 4, 4, 5)
    q = W.gaussian_bumps(g, 1)
    cfg, P, dt = pair(g, 2, q0=q)
    cfg.base = mp.MPRK_BASE_RK4
    with pytest.raises(mp.MprkError):
        mp.mprk_step_static(cfg, torch.from_numpy(q).cuda(), 1)
    bad = mp.mprk_config()
    C.memmove(C.byref(bad), C.byref(cfg), C.sizeof(cfg))
    bad.precision = mp.MPRK_FP32FLUX
    with pytest.raises(mp.MprkError):
        mp.Instance(bad, q)
