"""Pins of the 3-D oracle (App. B, Eq. ns-fv-cartesian-3d in full) against
facts that do not come from the oracle itself:
  * a y-invariant state with v = 0 reduces to the pinned 2-D scheme;
  * swapping x and y (with rho u <-> rho v) swaps R;
  * the interface shear in y has the closed form sigma^_yz = b_v (v2 - v1);
  * mass, energy and horizontal momentum are conserved where the physics
    says so;
  * m = 1 equals Heun bitwise, and MPRK2 converges at second order."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_11890_gb300 import workloads as W

GAM = 1.4


def p3(g, m=2, dt=0.01, **kw):
    return O.make_problem3(g.nx, g.ny, g.nS, g.nB, g.nF, m, dt, g.dx, dy=g.dy, dz1=g.dz1, dz2=g.dz2, **kw)


def lift(q2, ny):
    """A 2-D state [4][nz][nx] as a y-invariant 3-D state with v = 0."""
    nz, nx = q2.shape[1:]
    q3 = np.zeros((5, nz, ny, nx))
    for c3, c2 in ((0, 0), (1, 1), (3, 2), (4, 3)):
        q3[c3] = q2[c2][:, None, :]
    return q3


@pytest.mark.parametrize("wall", [O.WALL_NOSLIP, O.WALL_SLIP])
def test_y_invariant_state_reduces_to_the_2d_scheme(wall):
    """App. B with y dropped is the 2-D scheme (pinned by test_oracle_rhs,
    test_oracle_mms and test_oracle_step): on a y-invariant state with v = 0
    the 3-D R has R(rho v) = 0 and the other four components equal the 2-D R
    in every y column; the same holds for a whole MPRK2 step."""
    g2 = W.Grid(14, 5, 4, 6)
    q2 = W.gaussian_bumps(g2, 21, sigma_cells=2.0, amp=0.03)
    g3 = W.Grid3(14, 5, 5, 4, 6)
    q3 = lift(q2, g3.ny)
    P2 = O.make_problem(g2.nx, g2.nS, g2.nB, g2.nF, 2, 0.01, g2.dx, wall=wall)
    P3 = p3(g3, wall=wall)
    R2, R3 = O.rhs(P2, q2), O.rhs3(P3, q3)
    scale = np.abs(R2).max()
    assert np.abs(R3[2]).max() == 0.0
    for c3, c2 in ((0, 0), (1, 1), (3, 2), (4, 3)):
        assert np.abs(R3[c3] - R2[c2][:, None, :]).max() <= 1e-13 * scale, c3
    P2.dt = P3.dt = O.stable_dt(P2, q2, 0.4)
    s2, _ = O.mprk_step(P2, q2, 2)
    s3 = O.mprk_step3(P3, q3, 2)
    for c3, c2 in ((0, 0), (1, 1), (3, 2), (4, 3)):
        assert np.abs(s3[c3] - s2[c2][:, None, :]).max() <= 1e-13 * np.abs(s2[c2]).max(), c3


@pytest.mark.parametrize("wall", [O.WALL_NOSLIP, O.WALL_SLIP])
def test_swapping_x_and_y_swaps_r(wall):
    """On a square grid (nx = ny, dx = dy), transposing x and y and swapping
    rho u with rho v transposes R the same way: the y faces, y gradients,
    sigma_yz at Gamma and v_w are the x ones rotated."""
    g = W.Grid3(10, 10, 4, 4, 5)
    q = W.gaussian_bumps3(g, 4, sigma_cells=2.0, amp=0.03)
    perm = [0, 2, 1, 3, 4]
    qs = np.ascontiguousarray(q[perm].transpose(0, 1, 3, 2))
    P = p3(g, wall=wall)
    R, Rs = O.rhs3(P, q), O.rhs3(P, qs)
    back = Rs[perm].transpose(0, 1, 3, 2)
    assert np.abs(back - R).max() <= 1e-13 * np.abs(R).max()


def test_interface_y_shear_closed_form():
    """Uniform fluids sliding in y past each other (v1 in fluid 1, v2 in
    fluid 2, same rho and p, no gravity, slip walls): only Gamma acts. The
    rigid lid carries no tangential inviscid flux, and the bulk shear
    sigma^_yz = b_v (v2 - v1) with b_v = 2 mu1 mu2/(dz2 mu1 + dz1 mu2) gives
    R(rho v) = sigma^_yz/dz1 on fluid 1's top row and -sigma^_yz/dz2 on fluid
    2's bottom row; every other row gets 0."""
    g = W.Grid3(6, 5, 3, 4, 5, dz1=0.3, dz2=0.7)
    mu1, mu2, v1, v2 = 2e-3, 5e-3, 0.1, -0.25
    rho, p = 1.1, 0.9
    v = np.where(np.arange(g.nz) < g.n1, v1, v2)[:, None, None] * np.ones((g.nz, g.ny, g.nx))
    q = W.conserved3(rho * np.ones_like(v), 0 * v, v, 0 * v, p * np.ones_like(v))
    P = p3(g, G=0.0, mu1=mu1, mu2=mu2, wall=O.WALL_SLIP)
    R = O.rhs3(P, q)
    bv = 2 * mu1 * mu2 / (g.dz2 * mu1 + g.dz1 * mu2)
    syz = bv * (v2 - v1)
    assert np.allclose(R[2, g.n1 - 1], syz / g.dz1, rtol=1e-12, atol=0)
    assert np.allclose(R[2, g.n1], -syz / g.dz2, rtol=1e-12, atol=0)
    others = [k for k in range(g.nz) if k not in (g.n1 - 1, g.n1)]
    assert np.abs(R[2, others]).max() <= 1e-13 * abs(syz / g.dz1)
    assert np.abs(R[0]).max() <= 1e-14 and np.abs(R[1]).max() <= 1e-14


def test_conservation():
    """Walls and the rigid lid carry no mass: each fluid keeps its mass.
    Without gravity the total energy is conserved (no-slip walls do no
    work). With slip walls the total x and y momentum of both fluids is
    conserved (Gamma's shear is equal and opposite)."""
    g = W.Grid3(8, 8, 4, 4, 5)
    q = W.gaussian_bumps3(g, 11, sigma_cells=2.0, amp=0.05)
    P = p3(g, m=2)
    P.dt = O.stable_dt3(P, q, 0.4)
    d0 = O.diagnostics3(P, q)
    d1 = O.diagnostics3(P, O.mprk_step3(P, q, 10))
    assert abs(d1[0] - d0[0]) / d0[0] < 1e-13 and abs(d1[5] - d0[5]) / d0[5] < 1e-13
    Pg = p3(g, m=2, G=0.0)
    Pg.dt = P.dt
    e0 = O.diagnostics3(Pg, q)
    e1 = O.diagnostics3(Pg, O.mprk_step3(Pg, q, 10))
    assert abs((e1[4] + e1[9]) - (e0[4] + e0[9])) / (e0[4] + e0[9]) < 1e-13
    Ps = p3(g, m=2, wall=O.WALL_SLIP)
    Ps.dt = P.dt
    m0 = O.diagnostics3(Ps, q)
    m1 = O.diagnostics3(Ps, O.mprk_step3(Ps, q, 10))
    scale = m0[0]
    for c in (1, 2):
        assert abs((m1[c] + m1[5 + c]) - (m0[c] + m0[5 + c])) / scale < 1e-13, c


def test_m1_is_heun_bitwise():
    g = W.Grid3(6, 6, 3, 4, 4)
    q = W.gaussian_bumps3(g, 5, sigma_cells=1.5, amp=0.03)
    P = p3(g, m=1)
    P.dt = O.stable_dt3(P, q, 0.4)
    assert np.array_equal(O.mprk_step3(P, q), O.rk2_step3(P, q, P.dt))


def test_temporal_order_two():
    """MPRK2 (m = 2) against classical RK4 with a 64 times smaller step."""
    g = W.Grid3(6, 6, 3, 4, 4)
    q = W.gaussian_bumps3(g, 9, sigma_cells=1.5, amp=0.03)
    kw = dict(mu1=2e-3, mu2=4e-3)
    P = p3(g, m=2, **kw)
    dt0 = O.stable_dt3(P, q, 0.4)
    Pr = p3(g, m=1, **kw)
    ref = O.rk4_step3(Pr, q, dt0 / 64, 4 * 64)
    errs = []
    for k in range(3):
        P.dt = dt0 / 2 ** k
        errs.append(np.abs(O.mprk_step3(P, q, 4 * 2 ** k) - ref).max(axis=(1, 2, 3)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.7), rates
