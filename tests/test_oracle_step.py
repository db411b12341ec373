"""Pins of the oracle's MPRK2 slow step (Eq. MRK2, Table 1, Algorithm 1):
m = 1 is the base RK2, closed-form amplification on a linear problem, a
50-digit hand expansion of Table 1, conservation with and without the buffer
condition, the buffer condition itself, and the temporal order."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_11890_gb300 import workloads as W


def small(nx=12, nS=5, nB=4, nF=5, m=2, seed=3, **kw):
    g = W.Grid(nx, nS, nB, nF)
    q = W.gaussian_bumps(g, seed, sigma_cells=2.0, amp=0.02)
    P = O.make_problem(nx, nS, nB, nF, m, 0.0, g.dx, **kw)
    P.dt = O.stable_dt(P, q, 0.4)
    return g, P, q


@pytest.mark.parametrize("wall", [O.WALL_NOSLIP, O.WALL_SLIP])
def test_m1_is_rk2_bitwise(wall):
    g, P, q = small(m=1, wall=wall)
    q1, _ = O.mprk_step(P, q, 3)
    q2 = O.rk2_step(P, q, P.dt, 3)
    assert np.array_equal(q1, q2)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 8])
def test_linear_amplification_closed_form(m):
    """With R = lambda q per cell, each region is a linear RK method: S and B
    give the RK2 factor 1 + z + z^2/2, F gives m RK2 substeps of dt/m."""
    lam, dt = -1.3, 0.37
    z = lam * dt
    g = W.Grid(4, 3, 4, 5)
    P = O.make_problem(4, 3, 4, 5, m, dt, g.dx, rhs_mode=O.RHS_LINEAR, lin_lambda=lam)
    q = np.random.default_rng(0).uniform(0.5, 1.5, P.shape)
    qn, _ = O.mprk_step(P, q)
    slow = 1 + z + z * z / 2
    fast = (1 + z / m + (z / m) ** 2 / 2) ** m
    assert np.allclose(qn[:, :7], slow * q[:, :7], rtol=2e-15, atol=0)
    assert np.allclose(qn[:, 7:], fast * q[:, 7:], rtol=2e-15 * m, atol=0)


def test_linear_rk2_rk4_closed_form():
    lam, h = -0.9, 0.5
    z = lam * h
    g = W.Grid(4, 3, 4, 5)
    P = O.make_problem(4, 3, 4, 5, 1, h, g.dx, rhs_mode=O.RHS_LINEAR, lin_lambda=lam)
    q = np.random.default_rng(1).uniform(0.5, 1.5, P.shape)
    assert np.allclose(O.rk2_step(P, q, h), (1 + z + z * z / 2) * q, rtol=2e-15, atol=0)
    rk4 = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    assert np.allclose(O.rk4_step(P, q, h), rk4 * q, rtol=2e-15, atol=0)


def test_hand_expanded_step_50_digits():
    """Table 1 (m = 2) applied literally, stage by stage, in 50-digit
    arithmetic on a 5x8 grid (S/B/F = 2/4/2). The right-hand side is the
    oracle's, evaluated in double on each composite stage state; Algorithm 1
    fixes which region reads which stage (S stage 3 = S stage 1, S stage 4 =
    S stage 2)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    g, P, q = small(nx=5, nS=2, nB=4, nF=2, m=2, seed=5)
    dt = mp.mpf(P.dt)
    S, B, F = slice(0, 2), slice(2, 6), slice(6, 8)
    tomp = np.vectorize(mp.mpf, otypes=[object])
    tof = np.vectorize(float, otypes=[float])
    qm = tomp(q)

    def rhs(Qm):
        return tomp(O.rhs(P, np.ascontiguousarray(tof(Qm))))

    h, q4 = mp.mpf(1) / 2, mp.mpf(1) / 4
    # stage 1: every region starts from q_n
    Q1 = qm.copy()
    R1 = rhs(Q1)
    # stage 2: F a21 = 1/2; B a21 = 1; S a21 = 1
    Q2 = qm.copy()
    Q2[:, F] = qm[:, F] + dt * (h * R1[:, F])
    Q2[:, B] = qm[:, B] + dt * (1 * R1[:, B])
    Q2[:, S] = qm[:, S] + dt * (1 * R1[:, S])
    R2 = rhs(Q2)
    # stage 3: F a31 = a32 = 1/4; B row zero; S copies stage 1
    Q3 = qm.copy()
    Q3[:, F] = qm[:, F] + dt * (q4 * R1[:, F] + q4 * R2[:, F])
    Q3[:, B] = qm[:, B]
    Q3[:, S] = Q1[:, S]
    R3 = rhs(Q3)
    # stage 4: F a41 = a42 = 1/4, a43 = 1/2; B a43 = 1; S copies stage 2
    Q4 = qm.copy()
    Q4[:, F] = qm[:, F] + dt * (q4 * R1[:, F] + q4 * R2[:, F] + h * R3[:, F])
    Q4[:, B] = qm[:, B] + dt * (1 * R3[:, B])
    Q4[:, S] = Q2[:, S]
    R4 = rhs(Q4)
    # completion: F and B weights 1/4 each; S weights 1/2, 1/2, 0, 0
    qn = qm.copy()
    qn[:, F] = qm[:, F] + dt * (q4 * (R1[:, F] + R2[:, F] + R3[:, F] + R4[:, F]))
    qn[:, B] = qm[:, B] + dt * (q4 * (R1[:, B] + R2[:, B] + R3[:, B] + R4[:, B]))
    qn[:, S] = qm[:, S] + dt * (h * R1[:, S] + h * R2[:, S])
    ref = tof(qn)
    got, _ = O.mprk_step(P, q)
    scale = np.abs(ref).max(axis=(1, 2), keepdims=True)
    assert (np.abs(got - ref) / scale).max() <= 1e-14


def _mass(P, q):
    d = O.diagnostics(P, q)
    return d[0], d[4]


@pytest.mark.parametrize("m", [1, 2, 4, 8])
def test_mass_conservation_per_fluid(m):
    """Sec. 3 remark: with the buffer condition the coupling conserves mass;
    Sec. 5.1 reports a loss bounded by O(1e-13). Walls and the rigid lid carry
    no mass, so each fluid keeps its own mass."""
    g, P, q = small(nx=24, nS=10, nB=4, nF=10, m=m)
    m1, m2 = _mass(P, q)
    qn, _ = O.mprk_step(P, q, 60)
    n1, n2 = _mass(P, qn)
    assert abs(n1 - m1) / m1 < 1e-13 and abs(n2 - m2) / m2 < 1e-13


def test_config_plain_64_conserves_and_stays_bounded():
    wl = W.plain_64()
    g = wl.grid
    q = wl.initial_state()
    P = O.make_problem(g.nx, g.nS, g.nB, g.nF, wl.m, 0.0, g.dx)
    P.dt = O.stable_dt(P, q, 0.4)
    d0 = O.diagnostics(P, q)
    qn, _ = O.mprk_step(P, q, wl.steps)
    d1 = O.diagnostics(P, qn)
    assert abs(d1[0] - d0[0]) / d0[0] < 1e-13
    assert abs(d1[4] - d0[4]) / d0[4] < 1e-13
    assert d1[11] == 0 and d1[12] > 0 and d1[13] > 0
    w0 = np.abs(q[2] / q[0]).max()
    assert np.abs(qn[2] / qn[0]).max() < 2 * w0  # the run stays bounded


def test_energy_and_x_momentum_conservation():
    """Without gravity and with slip walls the outer walls exchange neither
    energy nor x momentum, and the interface passes the same bulk fluxes to
    both fluids, so the totals over both fluids are conserved."""
    g, P, q = small(nx=16, nS=6, nB=4, nF=6, m=4, G=0.0, wall=O.WALL_SLIP, mu1=1e-3, mu2=3e-3)
    d0 = O.diagnostics(P, q)
    qn, _ = O.mprk_step(P, q, 40)
    d1 = O.diagnostics(P, qn)
    E0, E1 = d0[3] + d0[7], d1[3] + d1[7]
    assert abs(E1 - E0) / E0 < 1e-13
    mx0, mx1 = d0[1] + d0[5], d1[1] + d1[5]
    assert abs(mx1 - mx0) / (d0[0] + d0[4]) < 1e-14
    # and they do change per fluid (the interface really exchanges them)
    assert abs(d1[1] - d0[1]) > 1e-10


def test_buffer_condition_bitwise_and_its_failure():
    """Sec. 3: the buffer must be wide enough that the buffer stage values next
    to S repeat with period s = 2. Rows nS and nS+1 feed the S|B face flux."""
    for nB, holds in [(3, True), (4, True), (6, True), (2, False)]:
        g, P, q = small(nx=10, nS=4, nB=nB, nF=6, m=4)
        Q, R, _ = O.mprk_trace(P, q)
        rows = slice(g.nS, g.nS + 2)
        same = all(np.array_equal(Q[i][:, rows], Q[i % 2][:, rows]) for i in range(2 * P.m))
        assert same == holds, nB


@pytest.mark.parametrize("nB,conserves", [(2, False), (3, True), (4, True)])
def test_too_narrow_buffer_breaks_mass_conservation(nB, conserves):
    """The fast region reaches the buffer only through the interface's bulk
    (viscous) fluxes, so the test drives a strong shear and a temperature jump
    across the interface. With two buffer rows fluid 1 then loses mass
    measurably; with three or more it does not (the stencil reaches two rows)."""
    g, P, q = small(nx=24, nS=10, nB=nB, nF=12, m=4, mu1=0.02, mu2=0.02)
    q[1, g.n1:] += 0.2 * q[0, g.n1:]
    q[3, g.n1:] *= 1.1
    P.dt = O.stable_dt(P, q, 0.4)
    m1, _ = _mass(P, q)
    qn, _ = O.mprk_step(P, q, 30)
    n1, _ = _mass(P, qn)
    drift = abs(n1 - m1) / m1
    if conserves:
        assert drift < 1e-13
    else:
        assert drift > 1e-11


@pytest.mark.parametrize("m", [2, 4])
def test_temporal_order_two(m):
    """MPRK2 is second order (Sec. 3 remark; Table 6 reports 2.04/2.00/2.00).
    Reference: classical RK4 with a much smaller step on the same
    semi-discrete system."""
    g, P, q = small(nx=12, nS=5, nB=4, nF=5, m=m, seed=9, mu1=2e-3, mu2=4e-3)
    dt0 = P.dt
    T = 4 * dt0
    Pr = O.make_problem(12, 5, 4, 5, 1, 0.0, g.dx, mu1=2e-3, mu2=4e-3)
    ref = O.rk4_step(Pr, q, dt0 / 64, 4 * 64)
    errs = []
    for k in range(3):
        P.dt = dt0 / 2 ** k
        qn, _ = O.mprk_step(P, q, 4 * 2 ** k)
        errs.append(np.abs(qn - ref).max(axis=(1, 2)))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates[:, [0, 1, 3]] > 1.85), rates
    assert np.all(rates > 1.7), rates


def test_diagnostics_match_plain_sums():
    g, P, q = small(nx=8, nS=3, nB=4, nF=5, m=2)
    P.dz2 = 0.7 * g.dx
    d = O.diagnostics(P, q)
    vol1, vol2 = P.dx * P.dz1, P.dx * P.dz2
    assert np.allclose(d[0:4], q[:, :7].sum(axis=(1, 2)) * vol1, rtol=1e-14)
    assert np.allclose(d[4:8], q[:, 7:].sum(axis=(1, 2)) * vol2, rtol=1e-14)
    assert d[11] == 0
    q2 = q.copy()
    q2[2, 3, 4] = np.nan
    assert O.diagnostics(P, q2)[11] == 1
