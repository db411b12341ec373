"""The request server (mprk_submit / mprk_poll): continuous batching under
an HBM budget. Each result equals the same solve alone (mprk_step), in any
admission order, and the error paths report codes instead of failing."""
import time

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


def requests(count, seed, precision=1):
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        nx = int(rng.integers(8, 120))
        nB = int(rng.integers(4, 17))
        g = W.Grid(nx, int(rng.integers(2, 30)), nB, int(rng.integers(2, 30)))
        m = int(rng.choice([2, 4, 8]))
        q = W.gaussian_bumps(g, seed * 100 + j, sigma_cells=2.5)
        cfg, P, dt = pair(g, m, q0=q, precision=precision)
        out.append((cfg, q, int(rng.integers(1, 12))))
    return out


def alone(cfg, q, n):
    from paper_2202_11890_gb300 import mprk as M
    with M.Instance(cfg, q) as inst:
        inst.step(n)
        return inst.state()


def drain(M, srv, tickets, timeout=120.0):
    outs = {}
    t0 = time.time()
    while len(outs) < len(tickets):
        assert time.time() - t0 < timeout, "server did not finish"
        for t, shape in tickets.items():
            if t in outs:
                continue
            buf = np.empty(shape)
            st, err, stats = M.mprk_poll(srv, t, buf)
            if st == M.MPRK_REQ_DONE:
                outs[t] = (buf, err, stats)
        time.sleep(0.002)
    return outs


@pytest.mark.parametrize("precision,solo_cells", [(1, 0), (0, 0), (1, 2000), (0, 2000), (1, -1)])
def test_served_results_equal_solo_results(precision, solo_cells):
    """solo_cells 2000: the instances of at least 2000 cells step alone on
    the side streams (bitwise the solve alone in both precisions), the
    others in the batched launch, in the same iterations; -1: all batched."""
    from paper_2202_11890_gb300 import mprk as M
    reqs = requests(24, 5 + precision, precision)
    refs = [alone(cfg, q, n) for cfg, q, n in reqs]
    srv = M.mprk_server_create(hbm_budget_bytes=1 << 30, max_slots=7, solo_cells=solo_cells)
    try:
        tickets = {}
        order = {}
        for j, (cfg, q, n) in enumerate(reqs):
            t = M.mprk_submit(srv, cfg, q, n)
            tickets[t] = q.shape
            order[t] = j
            if j % 5 == 4:
                time.sleep(0.003)  # arrivals while others run
        outs = drain(M, srv, tickets)
        for t, (buf, err, stats) in outs.items():
            j = order[t]
            assert err == 0
            assert stats["steps_done"] == reqs[j][2]
            cfg = reqs[j][0]
            solo = solo_cells > 0 and cfg.nx * (cfg.nz_S + cfg.nz_B + cfg.nz_F) >= solo_cells
            if precision == 0 or solo:
                assert np.array_equal(buf, refs[j]), j
            else:  # FP32 flux: batch and solo kernels agree to float rounding
                assert np.all(rel_err(buf, refs[j]) < 1e-5), (j, rel_err(buf, refs[j]))
        s = M.mprk_server_stats(srv)
        assert s[0] == len(reqs) and s[7] == 0 and s[5] == 0
    finally:
        M.mprk_server_destroy(srv)


@pytest.mark.parametrize("precision", [1, 0])
def test_served_requests_at_full_size_equal_solo_results(precision):
    """Requests drawn like the served workload (sides log-uniform in
    [32, 1024], m in {2, 4, 8}, buffer 4-16 rows) plus a 1024 x 1024 one, a
    few slow steps each: large instances run many waves of tiles, and in
    FP32 flux their interior tiles take the packed pair path. Each result
    equals the solve alone: within 1e-5 in FP32 flux, bitwise in FP64."""
    from paper_2202_11890_gb300 import mprk as M
    _, wls = W.served_stream(7, seed=41 + precision)
    grids = [(wl.grid, wl.m) for wl in wls] + [(W.Grid(1024, 506, 12, 506), 8)]
    rng = np.random.default_rng(43)
    reqs = []
    for j, (g, m) in enumerate(grids):
        q = W.gaussian_bumps(g, 300 + j, sigma_cells=4.0)
        cfg, P, dt = pair(g, m, q0=q, precision=precision)
        reqs.append((cfg, q, int(rng.integers(2, 5))))
    assert max(cfg.nx * (cfg.nz_S + cfg.nz_B + cfg.nz_F) for cfg, _, _ in reqs) >= 1 << 20
    refs = [alone(cfg, q, n) for cfg, q, n in reqs]
    srv = M.mprk_server_create(hbm_budget_bytes=8 << 30, max_slots=8)
    try:
        tickets, order = {}, {}
        for j, (cfg, q, n) in enumerate(reqs):
            t = M.mprk_submit(srv, cfg, q, n)
            tickets[t] = q.shape
            order[t] = j
        outs = drain(M, srv, tickets, timeout=300.0)
        for t, (buf, err, stats) in outs.items():
            j = order[t]
            assert err == 0
            assert stats["steps_done"] == reqs[j][2]
            if precision == 0:
                assert np.array_equal(buf, refs[j]), (j, rel_err(buf, refs[j]))
            else:
                assert np.all(rel_err(buf, refs[j]) < 1e-5), (j, rel_err(buf, refs[j]))
    finally:
        M.mprk_server_destroy(srv)


def test_served_general_base_requests_equal_solo_results():
    """FP64 requests with the Heun, RK3 and RK4 bases mixed in one server:
    each result bitwise equal to the solve alone (every FP64 launch runs the
    same non-inlined tile body), and the cell-stage count of each reports its
    s stages per substep."""
    from paper_2202_11890_gb300 import mprk as M
    reqs = requests(9, 17, precision=0)
    bases = [M.MPRK_BASE_RK2, M.MPRK_BASE_RK3, M.MPRK_BASE_RK4]
    for j, (cfg, q, n) in enumerate(reqs):
        cfg.base = bases[j % 3]
    refs = [alone(cfg, q, n) for cfg, q, n in reqs]
    srv = M.mprk_server_create(hbm_budget_bytes=1 << 30, max_slots=4)
    try:
        tickets, order = {}, {}
        for j, (cfg, q, n) in enumerate(reqs):
            t = M.mprk_submit(srv, cfg, q, n)
            tickets[t] = q.shape
            order[t] = j
        outs = drain(M, srv, tickets)
        for t, (buf, err, stats) in outs.items():
            j = order[t]
            cfg, q, n = reqs[j]
            assert err == 0
            assert np.array_equal(buf, refs[j]), (j, rel_err(buf, refs[j]))
            s = 2 + (j % 3)
            assert stats["cell_stages"] == cfg.nx * (s * cfg.nz_S + s * cfg.m * (cfg.nz_B + cfg.nz_F)) * n
    finally:
        M.mprk_server_destroy(srv)


def test_admission_order_does_not_change_results():
    from paper_2202_11890_gb300 import mprk as M
    reqs = requests(10, 11)
    results = []
    for perm in (np.arange(10), np.random.default_rng(2).permutation(10)):
        srv = M.mprk_server_create(hbm_budget_bytes=1 << 30, max_slots=3)
        try:
            tickets, order = {}, {}
            for j in perm:
                cfg, q, n = reqs[j]
                t = M.mprk_submit(srv, cfg, q, n)
                tickets[t] = q.shape
                order[t] = int(j)
            outs = drain(M, srv, tickets)
            results.append({order[t]: o[0] for t, o in outs.items()})
        finally:
            M.mprk_server_destroy(srv)
    for j in range(10):
        assert np.array_equal(results[0][j], results[1][j])


def test_budget_queue_and_bad_state_errors():
    from paper_2202_11890_gb300 import mprk as M
    cfg, q, n = requests(1, 3)[0]
    srv = M.mprk_server_create(hbm_budget_bytes=1 << 20, max_slots=2, max_queue=2)
    try:
        big = W.Grid(512, 200, 8, 200)
        cbig, _, _ = pair(big, 2, dt=1e-3, precision=1)
        with pytest.raises(M.MprkError) as ei:
            M.mprk_submit(srv, cbig, np.ones((4, big.nz, big.nx)), 1)
        assert ei.value.code == M.MPRK_EBUDGET
        bad = q.copy()
        bad[0, 0, 0] = np.nan
        t_bad = M.mprk_submit(srv, cfg, bad, 2)
        outs = drain(M, srv, {t_bad: q.shape})
        assert outs[t_bad][1] == M.MPRK_ENONFINITE
        with pytest.raises(M.MprkError) as ei:
            M.mprk_poll(srv, 987654321)
        assert ei.value.code == M.MPRK_ENOTFOUND
    finally:
        M.mprk_server_destroy(srv)
    # a full queue answers EBUSY (the server admits nothing: no slot fits)
    srv = M.mprk_server_create(hbm_budget_bytes=1 << 30, max_slots=1, max_queue=1)
    try:
        cfg2, q2, _ = requests(1, 4)[0]
        M.mprk_submit(srv, cfg2, q2, 200)   # occupies the slot
        time.sleep(0.05)
        M.mprk_submit(srv, cfg2, q2, 1)     # queued
        with pytest.raises(M.MprkError) as ei:
            for _ in range(50):
                M.mprk_submit(srv, cfg2, q2, 1)
        assert ei.value.code == M.MPRK_EBUSY
    finally:
        M.mprk_server_destroy(srv)


def test_shutdown_with_requests_in_flight():
    from paper_2202_11890_gb300 import mprk as M
    srv = M.mprk_server_create(hbm_budget_bytes=1 << 30, max_slots=4)
    for cfg, q, n in requests(8, 7):
        M.mprk_submit(srv, cfg, q, 500)
    time.sleep(0.05)
    M.mprk_server_destroy(srv)   # returns; nothing hangs
    cfg, q, n = requests(1, 8)[0]
    assert alone(cfg, q, 1).shape == q.shape  # the device is still usable
