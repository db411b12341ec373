"""x walls (Sec. 5.2: walls on all boundaries) on the GPU, through the C ABI,
against the FP64 oracle: the right-hand side and every slow step to 1e-12
in FP64, a run to 1e-5 in the FP32-flux mode, the batch kernel bitwise
equal to single instances, and the temporal-convergence study of Table 6
(second order against a fine classical RK4 reference)."""
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


def gpu_rhs(cfg, q):
    mp = M()
    with mp.Instance(cfg, q) as inst:
        Wd = torch.from_numpy(q).cuda()
        Rd = torch.zeros_like(Wd)
        mp.mprk_rhs(inst.h, Wd, Rd, 0, cfg.nz_S + cfg.nz_B + cfg.nz_F)
        inst.sync()
        return Rd.cpu().numpy()


@pytest.mark.parametrize("dims,wall", [((37, 9, 5, 11), 0), ((64, 12, 4, 14), 1), ((6, 3, 4, 3), 0),
                                       ((100, 18, 6, 20), 0)])
def test_rhs_with_x_walls(dims, wall):
    """Ragged (37, 100 columns), exact-tile (64) and narrower-than-a-tile (6)
    grids; no-slip and slip walls."""
    g = W.Grid(*dims)
    q = W.gaussian_bumps(g, 31, sigma_cells=2.5, amp=0.03)
    cfg, P, _ = pair(g, 2, dt=0.01, wall=wall, xwall=1)
    err = rel_err(gpu_rhs(cfg, q), O.rhs(P, q))
    assert np.all(err < 1e-12), err


@pytest.mark.parametrize("m,wall", [(2, 0), (3, 1)])
def test_steps_with_x_walls(m, wall):
    mp = M()
    g = W.Grid(45, 9, 5, 12)
    q = W.thermal_convection(g)
    cfg, P, dt = pair(g, m, q0=q, wall=wall, xwall=1)
    q_or = q.copy()
    with mp.Instance(cfg, q) as inst:
        for _ in range(4):
            inst.step(1)
            q_or, _ = O.mprk_step(P, q_or)
            assert np.all(rel_err(inst.state(), q_or) < 1e-12)


def test_fp32_flux_with_x_walls():
    """Tiles at both x walls take the general path; the inner ones the
    packed pair path (with tensor-copied halos)."""
    mp = M()
    g = W.Grid(100, 32, 24, 40)
    q = W.thermal_convection(g)
    cfg, P, dt = pair(g, 4, q0=q, precision=mp.MPRK_FP32FLUX, xwall=1)
    q_or, _ = O.mprk_step(P, q, 20)
    with mp.Instance(cfg, q) as inst:
        inst.step(20)
        err = rel_err(inst.state(), q_or)
    print("fp32flux x-wall error per component:", err)
    assert np.all(err < 1e-5), err


def test_batch_with_x_walls_is_bitwise():
    """Instances with and without x walls in one batch: each equals itself
    stepped alone."""
    mp = M()
    cases = []
    for j, (dims, xw) in enumerate([((40, 8, 4, 9), 1), ((33, 6, 5, 7), 0), ((70, 10, 6, 12), 1)]):
        g = W.Grid(*dims)
        q = W.gaussian_bumps(g, 70 + j, sigma_cells=2.5)
        cfg, _, _ = pair(g, 2 + j, q0=q, xwall=xw)
        cases.append((cfg, q))
    solo = []
    for cfg, q in cases:
        with mp.Instance(cfg, q) as inst:
            inst.step(3)
            solo.append(inst.state())
    insts = [mp.Instance(cfg, q) for cfg, q in cases]
    try:
        mp.mprk_step_batch([i.h for i in insts], 3)
        for inst, ref in zip(insts, solo):
            assert np.array_equal(inst.state(), ref)
    finally:
        for inst in insts:
            inst.close()


@pytest.mark.slow
def test_table6_temporal_convergence():
    """Table 6: MPRK2 (m = 4) on the thermal-convection case (Sec. 5.2,
    second set-up) with dt = 0.025 {1, 1/2, 1/4, 1/8} to t = 2.5, against a
    classical RK4 reference with dt = 0.00125 (the paper's reference is
    RK45). L2 errors of rho, rho u and rho E fall at second order (the paper
    reports 2.04, 2.00, 2.00)."""
    mp = M()
    g = W.convection_grid()
    q0 = W.thermal_convection(g)
    t_end = 2.5
    Pr = O.make_problem(g.nx, g.nS, g.nB, g.nF, 1, 0.0, g.dx, dz1=g.dz1, dz2=g.dz2, xwall=1)
    ref = O.rk4_step(Pr, q0, 0.00125, int(round(t_end / 0.00125)))
    cell = g.dx * np.concatenate([np.full(g.n1, g.dz1), np.full(g.nF, g.dz2)])[:, None]

    def l2(a):
        return np.sqrt((a * a * cell).sum())

    errs = []
    for dt in (0.025, 0.0125, 0.00625, 0.003125):
        cfg, _, _ = pair(g, 4, dt=dt, xwall=1)
        with mp.Instance(cfg, q0) as inst:
            inst.step(int(round(t_end / dt)))
            d = inst.state() - ref
        errs.append([l2(d[0]), l2(np.stack([d[1], d[2]])), l2(d[3])])
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    print("Table 6 errors:", errs.tolist(), "orders:", rates.tolist())
    assert np.all(rates > 1.8), rates
