"""The 3-D model (App. B in full, ny > 1) on the GPU, through the C ABI,
against the 3-D FP64 oracle: the right-hand side and every slow step to
1e-12 (the 2-D bars), the monitoring sums, and the rejection of 3-D
configurations by the 2-D-only entry points."""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_11890_gb300 import workloads as W
from pairs import oracle_threads, rel_err

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


def pair3(g, m, dt=0.0, wall=0, q0=None, cfl=0.4, **kw):
    mp = M()
    P = O.make_problem3(g.nx, g.ny, g.nS, g.nB, g.nF, m, dt, g.dx, dy=g.dy, dz1=g.dz1, dz2=g.dz2, wall=wall,
                        **kw)
    if dt == 0.0:
        P.dt = dt = O.stable_dt3(P, q0, cfl)
    cfg = mp.mprk_config_default(g.nx, g.nS, g.nB, g.nF, m)
    cfg.ny, cfg.dy = g.ny, g.dy
    cfg.dx, cfg.dz1, cfg.dz2 = g.dx, g.dz1, g.dz2
    cfg.dt, cfg.wall = dt, wall
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg, P, dt


def rel3(a, b):
    scale = np.abs(b).max(axis=(1, 2, 3))
    return np.abs(a - b).max(axis=(1, 2, 3)) / np.where(scale > 0, scale, 1.0)


def gpu_rhs3(cfg, q):
    mp = M()
    with mp.Instance(cfg, q) as inst:
        Wd = torch.from_numpy(q).cuda()
        Rd = torch.zeros_like(Wd)
        mp.mprk_rhs(inst.h, Wd, Rd, 0, cfg.nz_S + cfg.nz_B + cfg.nz_F)
        inst.sync()
        return Rd.cpu().numpy()


@pytest.mark.parametrize("dims,wall", [((37, 6, 5, 4, 6), 0), ((32, 8, 9, 4, 11), 1), ((8, 4, 3, 4, 3), 0),
                                       ((40, 5, 12, 4, 15), 0)])
def test_rhs3_matches_oracle(dims, wall):
    """Ragged x (37, 40 columns), Gamma inside a tile (9 + 4 rows), a grid
    narrower than one tile, no-slip and slip walls."""
    g = W.Grid3(*dims)
    q = W.gaussian_bumps3(g, 13, sigma_cells=2.0, amp=0.03)
    cfg, P, _ = pair3(g, 2, dt=0.01, wall=wall)
    err = rel3(gpu_rhs3(cfg, q), O.rhs3(P, q))
    print("3-D RHS error per component:", err)
    assert np.all(err < 1e-12), err


@pytest.mark.parametrize("m,wall", [(2, 0), (3, 1)])
def test_steps3_match_oracle(m, wall):
    mp = M()
    g = W.Grid3(36, 6, 6, 4, 7)
    q = W.gaussian_bumps3(g, 17 + m, sigma_cells=2.0, amp=0.03)
    cfg, P, dt = pair3(g, m, q0=q, wall=wall)
    q_or = q.copy()
    with mp.Instance(cfg, q) as inst:
        for _ in range(3):
            inst.step(1)
            q_or = O.mprk_step3(P, q_or)
            err = rel3(inst.state(), q_or)
            assert np.all(err < 1e-12), err


def test_diagnostics3_match_oracle():
    mp = M()
    g = W.Grid3(20, 6, 5, 4, 6)
    q = W.gaussian_bumps3(g, 3, sigma_cells=2.0, amp=0.03)
    cfg, P, dt = pair3(g, 2, q0=q)
    with mp.Instance(cfg, q) as inst:
        d = inst.diagnostics()
    ref = O.diagnostics3(P, q)
    assert np.allclose(d[:10], ref[:10], rtol=1e-12, atol=1e-15)
    assert np.allclose(d[10:13], ref[10:13], rtol=1e-12)
    assert d[13] == 0 and np.isclose(d[14], ref[14]) and np.isclose(d[15], ref[15])


def test_3d_rejected_where_2d_only():
    mp = M()
    g = W.Grid3(16, 4, 4, 4, 5)
    q = W.gaussian_bumps3(g, 1)
    cfg, P, dt = pair3(g, 2, q0=q)
    bad = mp.mprk_config()
    C.memmove(C.byref(bad), C.byref(cfg), C.sizeof(cfg))
    bad.precision = mp.MPRK_FP32FLUX
    with pytest.raises(mp.MprkError):
        mp.Instance(bad, q)
    with mp.Instance(cfg, q) as inst:
        with pytest.raises(mp.MprkError):
            mp.mprk_step_batch([inst.h], 1)
    with pytest.raises(mp.MprkError):
        mp.mprk_step_static(cfg, torch.from_numpy(q).cuda(), 1)
