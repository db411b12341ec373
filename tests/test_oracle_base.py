"""Pins of MPRK with a general base method (the Sec. 3 remark: the base of
the MPRK2 framework can be any Runge–Kutta method, but the coupled method
is second order at most). The region tableaus are built from the base the
way Table 1 builds them from RK2."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_11890_gb300 import workloads as W


def small(nx=10, nS=4, nB=4, nF=5, m=2, seed=3, **kw):
    g = W.Grid(nx, nS, nB, nF)
    q = W.gaussian_bumps(g, seed, sigma_cells=2.0, amp=0.02)
    P = O.make_problem(nx, nS, nB, nF, m, 0.0, g.dx, **kw)
    P.dt = O.stable_dt(P, q, 0.3)
    return g, P, q


@pytest.mark.parametrize("m", [1, 2, 3, 4, 8])
def test_heun_base_gives_table1_tableaus_bitwise(m):
    ms = 2 * m
    for region in (O.REGION_S, O.REGION_B, O.REGION_F):
        a, b, c = O.tableau_base(m, region, "rk2")
        a0, b0, c0 = np.zeros(ms * ms), np.zeros(ms), np.zeros(ms)
        assert O.lib().or_tableau(m, region, O._p(a0), O._p(b0), O._p(c0)) == 0
        assert np.array_equal(a.ravel(), a0) and np.array_equal(b, b0) and np.array_equal(c, c0)


@pytest.mark.parametrize("m", [1, 2, 4])
def test_general_step_with_heun_is_the_rk2_step_bitwise(m):
    g, P, q = small(m=m)
    got = O.mprk_step_base(P, q, "rk2", 2)
    ref, _ = O.mprk_step(P, q, 2)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("base", ["rk3", "rk4"])
def test_m1_is_the_base_method(base):
    """With m = 1 every region runs the base once: the coupled step equals the
    base method alone, bit for bit."""
    g, P, q = small(m=1)
    assert np.array_equal(O.mprk_step_base(P, q, base), O.rk_step_base(P, q, P.dt, base))


def test_generic_single_rate_steps_are_heun_and_rk4():
    g, P, q = small(m=1)
    for base, ref in (("rk2", O.rk2_step(P, q, P.dt)), ("rk4", O.rk4_step(P, q, P.dt))):
        got = O.rk_step_base(P, q, P.dt, base)
        assert np.abs(got - ref).max() <= 1e-15 * np.abs(ref).max(), base


@pytest.mark.parametrize("base,poly", [("rk3", [1, 1, 1 / 2, 1 / 6]), ("rk4", [1, 1, 1 / 2, 1 / 6, 1 / 24])])
@pytest.mark.parametrize("m", [1, 2, 4])
def test_linear_amplification_closed_form(base, poly, m):
    """On R = lambda q, S and B amplify by the base's stability polynomial
    P(z), z = lambda dt (B restarts from q_n with full-step coefficients and
    weights b/m), and F by P(z/m)^m."""
    lam, dt = -1.3, 0.37
    g = W.Grid(6, 3, 4, 3)
    P = O.make_problem(6, 3, 4, 3, m, dt, g.dx, rhs_mode=O.RHS_LINEAR, lin_lambda=lam)
    q = np.ones((4, g.nz, g.nx))
    out = O.mprk_step_base(P, q, base)

    def Pz(z):
        return sum(cf * z ** j for j, cf in enumerate(poly))

    z = lam * dt
    assert np.allclose(out[:, : g.n1], Pz(z), rtol=1e-14, atol=0)
    assert np.allclose(out[:, g.n1:], Pz(z / m) ** m, rtol=1e-14, atol=0)


@pytest.mark.parametrize("base", ["rk3", "rk4"])
def test_mass_conservation_with_a_wide_buffer(base):
    """The buffer condition holds when the buffer is wider than the reach of
    one substep's s stages; then each fluid keeps its mass (Sec. 3 remark)."""
    g, P, q = small(nx=12, nS=5, nB=12, nF=6, m=2)
    P1 = O.diagnostics(P, q)
    qn = O.mprk_step_base(P, q, base, 10)
    P2 = O.diagnostics(P, qn)
    assert abs(P2[0] - P1[0]) / P1[0] < 1e-13 and abs(P2[4] - P1[4]) / P1[4] < 1e-13


def observed_order(base, m):
    g, P, q = small(m=m, seed=9, mu1=2e-3, mu2=4e-3)
    dt0 = P.dt
    Pr = O.make_problem(g.nx, g.nS, g.nB, g.nF, 1, 0.0, g.dx, mu1=2e-3, mu2=4e-3)
    ref = O.rk4_step(Pr, q, dt0 / 128, 4 * 128)
    errs = []
    for k in range(3):
        P.dt = dt0 / 2 ** k
        errs.append(np.abs(O.mprk_step_base(P, q, base, 4 * 2 ** k) - ref).max())
    return np.log2(np.array(errs[:-1]) / np.array(errs[1:]))


def test_the_bases_alone_keep_their_orders():
    """m = 1: the RK3 and RK4 bases converge at orders 3 and 4."""
    r3, r4 = observed_order("rk3", 1), observed_order("rk4", 1)
    assert np.all(r3 > 2.7) and np.all(r4 > 3.5), (r3, r4)


def test_the_coupled_method_is_second_order_at_most():
    """The Sec. 3 remark. The multirate part of the error is D(dt) = MPRK(m =
    2) - MPRK(m = 1) at equal dt: the coupled step minus the base alone. With
    the RK4 base and a disturbance moving across the S/B boundary, D first
    falls at fourth order (the fast band's own truncation error), then at
    second order once the coupling error takes over, about 1e-9 here."""
    g = W.Grid(10, 4, 4, 5)
    rho0, p0 = W.rest_primitives(g)
    x, z = g.x_centres()[None, :], g.z_centres()[:, None]
    zc = z[g.nS, 0] - 0.5 * g.dz1
    env = np.exp(-(x ** 2 + (z - zc) ** 2) / (2 * (1.5 * g.dx) ** 2))
    q = W.conserved(rho0 * (1 + 0.1 * env), 0 * env, 0.3 * env, p0)
    P2 = O.make_problem(g.nx, g.nS, g.nB, g.nF, 2, 0.0, g.dx, mu1=2e-3, mu2=4e-3)
    P1 = O.make_problem(g.nx, g.nS, g.nB, g.nF, 1, 0.0, g.dx, mu1=2e-3, mu2=4e-3)
    dt0 = O.stable_dt(P2, q, 0.3)
    D = []
    for k in range(5):
        P2.dt = P1.dt = dt0 / 2 ** k
        n = 2 * 2 ** k
        D.append(np.abs(O.mprk_step_base(P2, q, "rk4", n) - O.mprk_step_base(P1, q, "rk4", n)).max())
    rates = np.log2(np.array(D[:-1]) / np.array(D[1:]))
    assert rates[0] > 3.8 and rates[1] > 3.8, rates
    assert 1.4 < rates[-1] < 2.5, rates
