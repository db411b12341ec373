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
