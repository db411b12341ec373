"""The FP64 launcher's tile shapes: a launch with fewer 32x8 tiles than SMs
takes the shortest of 32x2, 32x4, 32x8 that still fits one wave. Grids are
picked from the GPU's SM count so that each shape is chosen; each takes one
slow step against the oracle (1e-12) and equals the batch kernel, whose
tiles are always 32x8, bit for bit."""
import math

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


def tiles(nx, rows, tz):
    return math.ceil(nx / 32) * math.ceil(rows / tz)


def shape(nx, rows, sms):
    for tz in (2, 4, 8):
        if tiles(nx, rows, tz) <= sms:
            return tz
    return 8


def grid_for(tz, sms):
    """A 2-D grid (8 tile columns) whose first stages take tz-row tiles."""
    nx = 256
    for rows in range(24, 4096, 4):
        if shape(nx, rows, sms) == tz and (tz == 8 or tiles(nx, rows, 8) <= sms):
            nB = 8
            nS = (rows - nB) // 2
            return W.Grid(nx, nS, nB, rows - nB - nS)
    raise AssertionError("no grid for this shape")


@pytest.mark.parametrize("tz", [2, 4, 8])
def test_each_tile_shape_matches_oracle_and_batch(tz):
    from paper_2202_11890_gb300 import mprk as M
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    g = grid_for(tz, sms)
    assert shape(g.nx, g.nz, sms) == tz
    q = W.gaussian_bumps(g, 70 + tz, sigma_cells=3.0)
    cfg, P, dt = pair(g, 2, q0=q)
    with M.Instance(cfg, q) as a, M.Instance(cfg, q) as b:
        a.step(1)
        M.mprk_step_batch([b.h], 1)
        qa, qb = a.state(), b.state()
    assert np.array_equal(qa, qb)
    q_or, _ = O.mprk_step(P, q)
    assert np.all(rel_err(qa, q_or) < 1e-12)


# ---- the tuning table's tile shapes ---------------------------------------

SHAPES = [(8, 1), (8, 2), (4, 1), (4, 2), (2, 1), (2, 2)]


def load_table(tmp_path, M, stage_buckets=(), stage_shape=None, batch_bucket=None, batch_rows=None):
    """Load a tuning table that forces a single-instance stage-tile shape on
    the given size buckets and the batch kernel's FP64 tile rows on one."""
    ent = []
    for b in stage_buckets:
        ent.append('{"stage_launch": 1, "bucket": %d, "tile_rows": %d, "threads_per_cell": %d}'
                   % (b, stage_shape[0], stage_shape[1]))
    if batch_bucket is not None:
        ent.append('{"precision": 0, "bucket": %d, "group": 2, "ctas_per_sm": 0, "tile_rows": %d}'
                   % (batch_bucket, batch_rows))
    path = tmp_path / "shapes.json"
    path.write_text('{"gpu": "%s", "entries": [%s]}' % (torch.cuda.get_device_name(0), ", ".join(ent)))
    M.mprk_tune_load(str(path))


def launch_buckets(g, s):
    """Size buckets of an instance's stage launches: every row during the
    first substep, the B and F rows after it."""
    return sorted({int(math.floor(math.log2(g.nx * g.nz))), int(math.floor(math.log2(g.nx * (g.nz - g.nS))))})


@pytest.mark.parametrize("base", [0, 1, 2])
def test_every_tuned_shape_is_bitwise_the_same(base, tmp_path):
    """Each of the six single-instance shapes and both batch shapes, forced
    through the tuning table, give bitwise the same two slow steps as 32x8
    tiles with one thread per cell, for the Heun, RK3 and RK4 bases; the
    32x8 result matches the oracle."""
    from paper_2202_11890_gb300 import mprk as M
    g = W.Grid(100, 20, 6, 22)  # ragged tiles in x and z, Gamma inside a tile
    q = W.gaussian_bumps(g, 90 + base, sigma_cells=3.0)
    cfg, P, dt = pair(g, 3, q0=q)
    cfg.base = base
    bk = launch_buckets(g, 2)
    try:
        results = {}
        for sh in SHAPES:
            load_table(tmp_path, M, bk, sh)
            with M.Instance(cfg, q) as inst:
                inst.step(2)
                results[sh] = inst.state()
        for rows in (8, 4):
            load_table(tmp_path, M, batch_bucket=int(math.floor(math.log2(g.nx * g.nz))), batch_rows=rows)
            assert M.mprk_tune_lookup(0, g.nx * g.nz)["tile_rows"] == rows
            with M.Instance(cfg, q) as inst:
                M.mprk_step_batch([inst.h], 2)
                results[("batch", rows)] = inst.state()
    finally:
        M.mprk_tune_clear()
    ref = results[(8, 1)]
    differ = [k for k, v in results.items() if not np.array_equal(v, ref)]
    assert not differ, differ
    if base == 0:
        q_or, _ = O.mprk_step(P, q, 2)
        assert np.all(rel_err(ref, q_or) < 1e-12)


def test_tile_tuner_records_shapes_and_changes_no_result():
    """mprk_tile_tune times the six shapes on the instances' first-substep
    and later launches, leaves their states untouched, records one shape per
    size bucket, and an instance created afterwards (which captures its step
    with the recorded shapes) steps bitwise like one created before."""
    from paper_2202_11890_gb300 import mprk as M
    M.mprk_tune_clear()
    grids = [W.Grid(256, 30, 8, 34), W.Grid(64, 20, 4, 24)]
    cases = []
    for j, g in enumerate(grids):
        q = W.gaussian_bumps(g, 120 + j, sigma_cells=3.0)
        cfg, P, dt = pair(g, 4, q0=q)
        cases.append((g, cfg, q))
    before = [M.Instance(cfg, q) for g, cfg, q in cases]
    try:
        n = M.mprk_tile_tune([i.h for i in before], reps=2)
        assert n >= 2
        for i, (g, cfg, q) in zip(before, cases):
            assert np.array_equal(i.state(), q)
            for b in launch_buckets(g, 2):
                sh = M.mprk_tile_lookup(2.0 ** b)
                assert sh is not None and (sh["tile_rows"], sh["threads_per_cell"]) in SHAPES
        for i, (g, cfg, q) in zip(before, cases):
            with M.Instance(cfg, q) as after:
                i.step(2)
                after.step(2)
                assert np.array_equal(i.state(), after.state())
    finally:
        for i in before:
            i.close()
        M.mprk_tune_clear()
