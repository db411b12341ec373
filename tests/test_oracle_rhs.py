"""Pins of the oracle's right-hand side (Sec. 2.1 and App. B) against facts the
paper or the mathematics fixes: textbook Euler fluxes, consistency and
dissipation of the Lax–Friedrichs flux, states the scheme must keep at rest,
symmetry, closed-form wall and interface shear, and second-order consistency
with the continuous operator (see test_oracle_mms.py)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_11890_gb300 import workloads as W

GAM = 1.4


def cons(rho, u, w, p):
    return np.array([rho, rho * u, rho * w, p / (GAM - 1) + 0.5 * rho * (u * u + w * w)])


def test_euler_flux_is_textbook():
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho, u, w, p = rng.uniform(0.5, 2), rng.normal(), rng.normal(), rng.uniform(0.3, 2)
        E = p / (GAM - 1) / rho + 0.5 * (u * u + w * w)
        H = E + p / rho
        Fx = [rho * u, rho * u * u + p, rho * u * w, rho * u * H]
        Fz = [rho * w, rho * w * u, rho * w * w + p, rho * w * H]
        assert np.allclose(O.euler_flux(cons(rho, u, w, p), 0), Fx, rtol=1e-14, atol=1e-14)
        assert np.allclose(O.euler_flux(cons(rho, u, w, p), 1), Fz, rtol=1e-14, atol=1e-14)


def test_lf_consistency():
    """F*(q, q) = F(q).n exactly: the dissipation vanishes for equal states."""
    rng = np.random.default_rng(2)
    for d in (0, 1):
        for _ in range(20):
            q = cons(rng.uniform(0.5, 2), rng.normal(), rng.normal(), rng.uniform(0.3, 2))
            assert np.array_equal(O.lf_flux(q, q, d), O.euler_flux(q, d))


def test_lf_stationary_contact_dissipation():
    """A resting density jump with equal pressure has equal Euler fluxes
    (0, p, 0, 0). The Lax–Friedrichs flux adds lambda/2 (q_l - q_r). For u = 0
    the Roe sound speed lies between a_l and a_r, so
    lambda = max(a_l, a_r) = max sqrt(gamma p / rho)."""
    p = 0.8
    for rl, rr in [(1.0, 0.5), (0.7, 1.3), (2.0, 1.9)]:
        ql, qr = cons(rl, 0, 0, p), cons(rr, 0, 0, p)
        lam = max(np.sqrt(GAM * p / rl), np.sqrt(GAM * p / rr))
        for d in (0, 1):
            F = O.lf_flux(ql, qr, d)
            assert abs(F[0] - 0.5 * lam * (rl - rr)) < 1e-15
            assert np.sign(F[0]) == np.sign(rl - rr)  # mass diffuses down the jump
            assert abs(F[1 + d] - p) < 1e-15
            assert abs(F[3] - 0.5 * lam * (ql[3] - qr[3])) < 1e-15


def test_lf_mirror_symmetry():
    """Swapping sides and reversing the normal velocity negates the mass and
    energy fluxes: F*(R ql, R qr) with R reflecting the normal direction."""
    rng = np.random.default_rng(3)
    for d in (0, 1):
        for _ in range(10):
            ql = cons(rng.uniform(0.5, 2), rng.normal(), rng.normal(), rng.uniform(0.3, 2))
            qr = cons(rng.uniform(0.5, 2), rng.normal(), rng.normal(), rng.uniform(0.3, 2))
            Rl, Rr = ql.copy(), qr.copy()
            Rl[1 + d] *= -1
            Rr[1 + d] *= -1
            F = O.lf_flux(ql, qr, d)
            Fm = O.lf_flux(Rr, Rl, d)
            assert abs(F[0] + Fm[0]) < 1e-14
            assert abs(F[3] + Fm[3]) < 1e-13
            assert abs(F[1 + d] - Fm[1 + d]) < 1e-13  # normal momentum flux is even


def _problem(nx=8, nS=3, nB=4, nF=3, m=2, **kw):
    return O.make_problem(nx, nS, nB, nF, m, 0.01, 10.0 / nx, **kw)


@pytest.mark.parametrize("wall", [O.WALL_NOSLIP, O.WALL_SLIP])
def test_uniform_rest_is_steady(wall):
    P = _problem(G=0.0, wall=wall, mu1=0.01, mu2=0.03)
    q = np.zeros(P.shape)
    q[0] = 1.3
    q[3] = 0.9 / (GAM - 1)
    assert np.abs(O.rhs(P, q)).max() == 0.0


def test_uniform_x_flow_with_slip_walls_is_steady():
    P = _problem(G=0.0, wall=O.WALL_SLIP, mu1=0.01, mu2=0.03)
    q = np.zeros(P.shape)
    q[:] = cons(1.1, 0.3, 0.0, 0.8)[:, None, None]
    assert np.abs(O.rhs(P, q)).max() < 1e-15


def test_x_invariant_state_stays_x_invariant_bitwise():
    g = W.Grid(6, 4, 4, 5)
    q = W.gaussian_bumps(g, 7)
    q[:] = q[:, :, :1]  # copy column 0 to every column
    P = O.make_problem(6, 4, 4, 5, 2, 0.01, g.dx, mu1=0.01, mu2=0.02)
    R = O.rhs(P, q)
    assert np.array_equal(R, np.broadcast_to(R[:, :, :1], R.shape))


def test_x_reflection_symmetry():
    """Reflecting x (i -> nx-1-i, rho u -> -rho u) reflects R the same way:
    catches index or sign mistakes in the x faces."""
    g = W.Grid(9, 5, 4, 6)
    q = W.gaussian_bumps(g, 11, sigma_cells=1.5, amp=0.05)
    P = O.make_problem(9, 5, 4, 6, 2, 0.01, g.dx, mu1=0.02, mu2=0.05)
    R = O.rhs(P, q)
    qr = q[:, :, ::-1].copy()
    qr[1] *= -1
    Rr = O.rhs(P, qr)
    Rr = Rr[:, :, ::-1].copy()
    Rr[1] *= -1
    scale = np.abs(R).max(axis=(1, 2), keepdims=True)
    assert np.abs(Rr - R).max() / scale.max() < 1e-13


@pytest.mark.parametrize("wall", [O.WALL_NOSLIP, O.WALL_SLIP])
def test_wall_shear_closed_form(wall):
    """Uniform x flow U in both fluids, no gravity. A no-slip wall at distance
    dz/2 from the cell centre exerts the stress mu U / (dz/2), so the wall row
    loses x momentum at the rate 2 mu U / dz^2; a slip wall exerts none.
    Energy is unchanged (the wall does no work, the walls are adiabatic)."""
    mu1, mu2 = 0.01, 0.03
    dz1, dz2 = 0.7, 0.4
    P = O.make_problem(8, 3, 4, 3, 2, 0.01, 1.0, dz1=dz1, dz2=dz2, G=0.0, wall=wall, mu1=mu1,
                       mu2=mu2)
    U = 0.25
    q = np.zeros(P.shape)
    q[:] = cons(1.0, U, 0.0, 0.7)[:, None, None]
    R = O.rhs(P, q)
    want_bot = -2 * mu1 * U / dz1 ** 2 if wall == O.WALL_NOSLIP else 0.0
    want_top = -2 * mu2 * U / dz2 ** 2 if wall == O.WALL_NOSLIP else 0.0
    assert np.allclose(R[1, 0], want_bot, rtol=1e-13, atol=1e-16)
    assert np.allclose(R[1, -1], want_top, rtol=1e-13, atol=1e-16)
    assert np.abs(R[:, 1:-1]).max() < 1e-15  # interior rows and the interface rows
    assert np.abs(R[[0, 2, 3]][:, [0, -1]]).max() < 1e-15


def test_interface_bulk_flux_closed_form():
    """Fluid 1 at rest with temperature T1, fluid 2 moving at u2 with T2, equal
    pressure, no gravity, slip walls. Only the interface rows change, by the
    bulk fluxes. The pins are the physical conditions that define them
    (App. B): the shear stress is continuous through the wall velocity,
    sigma = mu1 (u_w - u1)/(dz1/2) = mu2 (u2 - u_w)/(dz2/2), the heat flux
    likewise through T_w, and u_w and T_w agree from both sides. Fluid 1
    gains sigma/dz1 of x momentum and fluid 2 loses sigma/dz2; the energy
    flux is u_w sigma - Pi_z."""
    mu1, mu2, dz1, dz2, Pr = 0.01, 0.04, 0.5, 0.3, 0.72
    P = O.make_problem(8, 3, 4, 3, 2, 0.01, 1.0, dz1=dz1, dz2=dz2, G=0.0, wall=O.WALL_SLIP,
                       mu1=mu1, mu2=mu2, Pr=Pr)
    p, T1, T2, u1, u2 = 0.7, 1.0, 1.2, 0.0, 0.3
    q = np.zeros(P.shape)
    n1 = 7
    q[:, :n1] = cons(GAM * p / T1, u1, 0.0, p)[:, None, None]
    q[:, n1:] = cons(GAM * p / T2, u2, 0.0, p)[:, None, None]
    st = O.interface_state(P, q, 0)
    sig, Pi, uw1, Tw1, uw2, Tw2 = st
    ka1 = mu1 / (GAM - 1) / Pr
    ka2 = mu2 / (GAM - 1) / Pr
    assert abs(uw1 - uw2) < 1e-15 and abs(Tw1 - Tw2) < 1e-15
    assert abs(sig - mu1 * (uw1 - u1) / (dz1 / 2)) < 1e-15
    assert abs(sig - mu2 * (u2 - uw1) / (dz2 / 2)) < 1e-15
    assert abs(Pi - (-ka1 * (Tw1 - T1) / (dz1 / 2))) < 1e-15
    assert abs(Pi - (-ka2 * (T2 - Tw1) / (dz2 / 2))) < 1e-15
    assert sig > 0 and Pi < 0  # drag toward the faster fluid; heat flows down
    R = O.rhs(P, q)
    assert np.allclose(R[:, n1 - 1], (np.array([0, sig, 0, uw1 * sig - Pi]) / dz1)[:, None],
                       rtol=1e-12, atol=1e-16)
    assert np.allclose(R[:, n1], (-np.array([0, sig, 0, uw2 * sig - Pi]) / dz2)[:, None],
                       rtol=1e-12, atol=1e-16)
    others = [k for k in range(P.nz) if k not in (n1 - 1, n1)]
    assert np.abs(R[:, others]).max() < 1e-15


def test_hydrostatic_rest_is_second_order_steady():
    """The rest state of Sec. 5.2 solves the continuous equations exactly, so
    the discrete R away from walls and the interface shrinks like h^2."""
    errs = []
    for n in (16, 32, 64):
        g = W.Grid(8, n, 4, n)
        g.dx = 10.0 / 64
        g.dz1 = g.dz2 = 2.5 / n
        P = O.make_problem(8, n, 4, n, 2, 0.01, g.dx, dz1=g.dz1, dz2=g.dz2)
        R = O.rhs(P, W.rest_state(g))
        inner = list(range(3, n)) + list(range(n + 7, 2 * n + 1))
        errs.append(np.abs(R[2, inner]).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)
