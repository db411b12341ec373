"""Parity of the CUDA library with the FP64 CPU oracle, through the C ABI.

Bars: the FP64 path matches the oracle to 1e-12 relative (per component,
max norm scaled by the component's max) per slow step and for the
right-hand side alone; the FP32-flux mode to 1e-5 relative after a run.

Why 1e-12 for R as well: R is a difference of face fluxes of order one
(pressure) divided by dx, and cancels to values of order 1e-2, so rounding
differences of a few ulp in the fluxes show up as 1e-14..1e-13 relative to
max |R|. A real mistake in any term shows up at 1e-3 or above."""
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


def gpu_rhs(cfg, W_np, k_lo=0, k_hi=None):
    mp = M()
    k_hi = cfg.nz if k_hi is None else k_hi
    with mp.Instance(cfg, W_np) as inst:
        Wd = torch.from_numpy(W_np).cuda()
        Rd = torch.zeros_like(Wd)
        mp.mprk_rhs(inst.h, Wd, Rd, k_lo, k_hi)
        inst.sync()
        return Rd.cpu().numpy()


RHS_CASES = [
    # grid (nx, nS, nB, nF), kwargs
    ((64, 30, 4, 30), {}),
    ((37, 9, 5, 11), {}),                       # ragged in x and z
    ((5, 2, 4, 2), {}),                         # tiny
    ((40, 7, 6, 9), dict(wall=1)),              # slip walls
    ((33, 6, 4, 7), dict(mu1=0.02, mu2=0.05)),  # strong viscosity
    ((48, 10, 4, 12), dict(dz2=0.07)),          # refined fluid 2
]


@pytest.mark.parametrize("dims,kw", RHS_CASES)
def test_rhs_matches_oracle(dims, kw):
    kw = dict(kw)
    g = W.Grid(*dims)
    if "dz2" in kw:
        g.dz2 = kw.pop("dz2")
    q = W.gaussian_bumps(g, 17, sigma_cells=2.5, amp=0.05)
    cfg, P, _ = pair(g, 2, dt=0.01, **kw)
    R_or = O.rhs(P, q)
    R_gpu = gpu_rhs(cfg, q)
    assert np.all(rel_err(R_gpu, R_or) < 1e-12), rel_err(R_gpu, R_or)


def test_rhs_row_ranges():
    g = W.Grid(45, 10, 6, 13)
    q = W.gaussian_bumps(g, 3, sigma_cells=2.0, amp=0.05)
    cfg, P, _ = pair(g, 2, dt=0.01)
    for lo, hi in [(0, g.nS), (g.nS, g.nz), (g.n1 - 1, g.n1 + 1), (3, 4), (0, g.nz)]:
        R_or = np.zeros_like(q)
        O.rhs(P, q, lo, hi, out=R_or)
        R_gpu = gpu_rhs(cfg, q, lo, hi)
        assert np.all(rel_err(R_gpu[:, lo:hi], R_or[:, lo:hi]) < 1e-12)
        outside = np.ones(g.nz, bool)
        outside[lo:hi] = False
        assert np.all(R_gpu[:, outside] == 0.0)


STEP_CASES = [
    ((64, 30, 4, 30), 4, {}),      # the 64x64 plain workload's grid and rate
    ((37, 9, 5, 11), 1, {}),
    ((37, 9, 5, 11), 2, {}),
    ((50, 12, 16, 14), 8, {}),
    ((29, 6, 4, 9), 3, dict(wall=1)),
    ((40, 8, 4, 8), 4, dict(mu1=0.01, mu2=0.02)),
    ((5, 2, 4, 2), 2, {}),
]


@pytest.mark.parametrize("dims,m,kw", STEP_CASES)
def test_step_matches_oracle_every_step(dims, m, kw):
    """Per slow step from the same q_n: GPU step vs oracle step."""
    mp = M()
    g = W.Grid(*dims)
    q = W.gaussian_bumps(g, 29, sigma_cells=3.0)
    cfg, P, dt = pair(g, m, q0=q, **kw)
    with mp.Instance(cfg, q) as inst:
        for _ in range(3):
            q_or, _ = O.mprk_step(P, q)
            inst.set_state(q)
            inst.step(1)
            q_gpu = inst.state()
            err = rel_err(q_gpu, q_or)
            assert np.all(err < 1e-12), err
            q = q_or


def test_plain_64_whole_run_drift():
    """The 64x64, m = 4 workload for 100 slow steps: the GPU run alone against
    the oracle run alone (drift over the whole run is reported, bar 1e-10)."""
    mp = M()
    wl = W.plain_64()
    q0 = wl.initial_state()
    cfg, P, dt = pair(wl.grid, wl.m, q0=q0)
    q_or, _ = O.mprk_step(P, q0, wl.steps)
    with mp.Instance(cfg, q0) as inst:
        inst.step(wl.steps)
        q_gpu = inst.state()
        d_gpu = inst.diagnostics()
    err = rel_err(q_gpu, q_or)
    print("whole-run drift per component:", err)
    assert np.all(err < 1e-10), err
    d_or = O.diagnostics(P, q_or)
    assert np.allclose(d_gpu[:8], d_or[:8], rtol=1e-13, atol=1e-15)
    assert np.allclose(d_gpu[8:11], d_or[8:11], rtol=1e-12)
    assert d_gpu[11] == 0 and d_gpu[14] == wl.steps
    d0 = O.diagnostics(P, q0)
    assert abs(d_gpu[0] - d0[0]) / d0[0] < 1e-13 and abs(d_gpu[4] - d0[4]) / d0[4] < 1e-13


def test_single_rate_matches_oracle_rk2():
    """The single-rate baseline: m Heun steps of dt/m over the whole grid."""
    mp = M()
    g = W.Grid(41, 10, 4, 12)
    q = W.gaussian_bumps(g, 5, sigma_cells=3.0)
    m = 4
    cfg, P, dt = pair(g, m, q0=q, scheme=mp.MPRK_SCHEME_SR_RK2)
    q_or = O.rk2_step(P, q, dt / m, m)
    with mp.Instance(cfg, q) as inst:
        inst.step(1)
        q_gpu = inst.state()
    assert np.all(rel_err(q_gpu, q_or) < 1e-12)


def test_fp32_flux_mode_error_after_run():
    """FP32 fluxes with FP64 stage values and combinations: <= 1e-5 relative
    after 100 slow steps of the 64x64 workload; mass drift reported."""
    mp = M()
    wl = W.plain_64()
    q0 = wl.initial_state()
    cfg, P, dt = pair(wl.grid, wl.m, q0=q0, precision=mp.MPRK_FP32FLUX)
    q_or, _ = O.mprk_step(P, q0, wl.steps)
    with mp.Instance(cfg, q0) as inst:
        inst.step(wl.steps)
        q_gpu = inst.state()
        d = inst.diagnostics()
    err = rel_err(q_gpu, q_or)
    d0 = O.diagnostics(P, q0)
    print("fp32flux error per component:", err, "mass drift", (d[0] - d0[0]) / d0[0],
          (d[4] - d0[4]) / d0[4])
    assert np.all(err < 1e-5), err


def test_auto_dt_matches_oracle():
    mp = M()
    wl = W.plain_64()
    q0 = wl.initial_state()
    cfg, P, dt = pair(wl.grid, wl.m, q0=q0)
    cfg.dt = 0.0
    with mp.Instance(cfg, q0) as inst:
        assert abs(inst.info()["dt"] - dt) / dt < 1e-14


def test_checkpoint_resume_is_bitwise():
    mp = M()
    g = W.Grid(36, 8, 4, 10)
    q = W.gaussian_bumps(g, 8)
    cfg, P, dt = pair(g, 2, q0=q)
    with mp.Instance(cfg, q) as a:
        a.step(3)
        ck = a.state()
        a.step(2)
        qa = a.state()
    with mp.Instance(cfg, ck) as b:
        b.step(2)
        qb = b.state()
    assert np.array_equal(qa, qb)


def test_runs_are_deterministic():
    mp = M()
    g = W.Grid(70, 12, 6, 15)
    q = W.fourier_modes(g, 4)
    cfg, P, dt = pair(g, 4, q0=q)
    outs = []
    for _ in range(2):
        with mp.Instance(cfg, q) as inst:
            inst.step(5)
            outs.append((inst.state(), inst.diagnostics()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_bad_initial_state_is_rejected():
    mp = M()
    g = W.Grid(16, 4, 4, 4)
    q = W.rest_state(g)
    cfg, P, dt = pair(g, 2, dt=0.01)
    bad = q.copy()
    bad[2, 3, 5] = np.nan
    with pytest.raises(mp.MprkError) as ei:
        mp.Instance(cfg, bad)
    assert ei.value.code == mp.MPRK_ENONFINITE
    bad = q.copy()
    bad[0, 1, 1] = -1.0
    with pytest.raises(mp.MprkError) as ei:
        mp.Instance(cfg, bad)
    assert ei.value.code == mp.MPRK_ENONFINITE


def test_monitoring_flags_a_blow_up():
    """A step far beyond the stability limit makes the state non-finite; the
    in-graph monitoring sets the status word (no device trap)."""
    mp = M()
    g = W.Grid(32, 8, 4, 8)
    q = W.gaussian_bumps(g, 2, amp=0.05)
    cfg, P, dt = pair(g, 2, q0=q, diag_every=1)
    cfg.dt = dt * 40
    with mp.Instance(cfg, q) as inst:
        inst.step(60)
        assert inst.status() in (mp.MPRK_ENONFINITE, mp.MPRK_ECFL)


def test_device_resident_input():
    mp = M()
    g = W.Grid(40, 9, 4, 9)
    q = W.gaussian_bumps(g, 12)
    cfg, P, dt = pair(g, 2, q0=q)
    qd = torch.from_numpy(q).cuda()
    with mp.Instance(cfg, qd) as inst:
        inst.step(1)
        out = torch.empty_like(qd)
        mp.mprk_get_state(inst.h, out)
        q_or, _ = O.mprk_step(P, q)
        assert np.all(rel_err(out.cpu().numpy(), q_or) < 1e-12)


@pytest.mark.slow
def test_large_2048_one_step_full_size():
    """The 2048x1024, m = 8 workload at full size, in the launch configuration
    the benchmark times: one slow step against the oracle over every cell."""
    mp = M()
    wl = W.large_2048()
    q0 = wl.initial_state()
    cfg, P, dt = pair(wl.grid, wl.m, q0=q0)
    q_or, _ = O.mprk_step(P, q0)
    with mp.Instance(cfg, q0) as inst:
        inst.step(1)
        q_gpu = inst.state()
    err = rel_err(q_gpu, q_or)
    assert np.all(err < 1e-12), err


def test_bit_operation_conversions_match_hardware():
    """The FP32-flux mode narrows double -> float (round to nearest, ties to
    even) and widens float -> double with integer bit operations. They must
    agree bit for bit with the hardware conversions, including ties, values
    near the float range limits, zeros, subnormals, Inf and NaN."""
    mp = M()
    rng = np.random.default_rng(5)
    vals = [rng.normal(size=20000), rng.uniform(-1e-30, 1e-30, 2000),
            np.exp(rng.uniform(-80, 80, 4000)) * rng.choice([-1, 1], 4000)]
    # exact ties between two floats: 24-bit mantissa + one half-ulp bit
    m = rng.integers(1 << 23, 1 << 24, 2000).astype(np.float64)
    e = rng.integers(-30, 30, 2000)
    ties = (m + 0.5) * np.exp2(e.astype(np.float64) - 23)
    specials = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-40, -1e-45, 3.4028235677973366e38,
                         3.4028235677973366e38 * 1.0000001, 1.1754943508222875e-38, 2.0 ** -149])
    x = np.concatenate(vals + [ties, -ties, specials])
    xd = torch.from_numpy(x).cuda()
    n = xd.numel()
    nar = torch.empty(n, dtype=torch.float32, device="cuda")
    nar_hw = torch.empty_like(nar)
    wid = torch.empty(n, dtype=torch.float64, device="cuda")
    wid_hw = torch.empty_like(wid)
    mp.mprk_selftest_convert(xd, nar, nar_hw, wid, wid_hw)
    a, b = nar.cpu().numpy().view(np.uint32), nar_hw.cpu().numpy().view(np.uint32)
    assert np.array_equal(a, b), np.count_nonzero(a != b)
    a, b = wid.cpu().numpy().view(np.uint64), wid_hw.cpu().numpy().view(np.uint64)
    assert np.array_equal(a, b)


def test_fp64_reciprocal_and_roots_within_an_ulp():
    """The FP64 tiles compute 1/x, 1/sqrt(x) and sqrt(x) from the hardware's
    approximations and one third-order Householder step. Against references
    in extended precision, over the physical range of densities, pressures
    and sound speeds and far beyond it, each stays within 1.5 units in the
    last place (not correctly rounded: the flux formulas round more than
    that in every step)."""
    mp = M()
    rng = np.random.default_rng(11)
    x = np.concatenate([np.exp2(rng.uniform(-200.0, 200.0, 100000)), rng.uniform(0.5, 2.0, 50000),
                        rng.uniform(1e-3, 1e3, 50000), np.exp2(np.arange(-60.0, 61.0)),
                        np.array([1.0, 4.0, 0.25, 2.0, 3.0, 1.4, 0.4, np.nextafter(1.0, 2.0),
                                  np.nextafter(1.0, 0.0)])])
    xd = torch.from_numpy(x).cuda()
    out = [torch.empty_like(xd) for _ in range(3)]
    mp.mprk_selftest_recip(xd, *out)
    ld = np.longdouble
    xl = x.astype(ld)
    sq = np.sqrt(xl)
    refs = {"recip": ld(1) / xl, "rsqrt": ld(1) / sq, "sqrt": sq}
    for (name, ref), got in zip(refs.items(), out):
        y = got.cpu().numpy()
        ulp = np.spacing(np.abs(ref.astype(np.float64))).astype(ld)
        err = np.abs(y.astype(ld) - ref) / ulp
        print(name, "max ulp error", float(err.max()), "mean", float(err.mean()))
        assert np.all(np.isfinite(y)), name
        assert float(err.max()) <= 1.5, (name, float(err.max()), x[np.argmax(err)])


@pytest.mark.parametrize("dims", [(64, 30, 4, 30), (100, 40, 8, 48)])
def test_fp32_flux_rhs_close_to_oracle(dims):
    """The FP32-flux right-hand side (deviation form) against the FP64
    oracle's. On the 100 x 96 grid, tile rows 16-31 (fluid 1) and 64-79
    (fluid 2) take the packed pair path, the rest the general path. x is
    ragged (100 columns) and wraps at both ends."""
    g = W.Grid(*dims)
    q = W.gaussian_bumps(g, 17, sigma_cells=3.0)
    cfg, P, _ = pair(g, 2, dt=0.01, precision=1)
    R_or = O.rhs(P, q)
    R_gpu = gpu_rhs(cfg, q)
    err = rel_err(R_gpu, R_or)
    print("fp32flux RHS error per component:", err)
    assert np.all(err < 1e-4), err


@pytest.mark.parametrize("m,wall", [(3, 0), (4, 1)])
def test_fp32_flux_pair_path_in_every_band(m, wall):
    """A grid whose 16-row tiles take the packed pair path in the slow band
    (rows 16-31), the buffer (32-47) and the fast band (64-79), next to
    general-path tiles at the walls and at Gamma: 20 slow steps within
    1e-5 of the FP64 oracle."""
    mp = M()
    g = W.Grid(100, 32, 24, 40)
    q0 = W.gaussian_bumps(g, 29 + m, sigma_cells=3.0)
    cfg, P, dt = pair(g, m, q0=q0, precision=mp.MPRK_FP32FLUX, wall=wall)
    q_or, _ = O.mprk_step(P, q0, 20)
    with mp.Instance(cfg, q0) as inst:
        inst.step(20)
        q_gpu = inst.state()
    err = rel_err(q_gpu, q_or)
    print("fp32flux pair-path grid error per component:", err)
    assert np.all(err < 1e-5), err


def test_fp32_flux_pair_path_across_the_slow_buffer_bound():
    """nS = 40: the tile of rows 32-47 holds S rows (32-39) and B rows
    (40-47) and takes the pair path at the two full-row stages, each cell
    combined by its own region. 20 slow steps within 1e-5 of the FP64
    oracle, and the batch kernel (same tile paths) within float rounding
    (1e-6) of the single-instance one."""
    mp = M()
    g = W.Grid(96, 40, 24, 40)
    q0 = W.gaussian_bumps(g, 61, sigma_cells=3.0)
    cfg, P, dt = pair(g, 4, q0=q0, precision=mp.MPRK_FP32FLUX)
    q_or, _ = O.mprk_step(P, q0, 20)
    with mp.Instance(cfg, q0) as a, mp.Instance(cfg, q0) as b:
        a.step(20)
        mp.mprk_step_batch([b.h], 20)
        qa, qb = a.state(), b.state()
    err = rel_err(qa, q_or)
    print("fp32flux S/B-bound tile error per component:", err)
    assert np.all(err < 1e-5), err
    assert np.all(rel_err(qb, qa) < 1e-6)


def test_both_fp64_launch_forms_in_one_step():
    """512 x 96 cells with a thin buffer and fast band: the two full-row
    stages launch 192 tiles (one thread per cell), the later B+F stages 32
    tiles (more SMs than tiles, so two threads per cell). Three slow steps
    within 1e-12 of the oracle, and bitwise equal to the batch kernel's."""
    mp = M()
    g = W.Grid(512, 80, 4, 12)
    q = W.gaussian_bumps(g, 31, sigma_cells=3.0, amp=0.03)
    cfg, P, dt = pair(g, 2, q0=q)
    q_or, _ = O.mprk_step(P, q, 3)
    with mp.Instance(cfg, q) as a, mp.Instance(cfg, q) as b:
        a.step(3)
        mp.mprk_step_batch([b.h], 3)
        qa, qb = a.state(), b.state()
    assert np.all(rel_err(qa, q_or) < 1e-12)
    assert np.array_equal(qa, qb)
