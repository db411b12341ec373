"""Pins of the oracle's x walls (xwall = 1). Sec. 5.2 puts adiabatic no-slip
walls on every boundary of the thermal-convection domain; the x walls follow
the z-wall rules with x as the normal. The pins are closed forms (a
pressure ramp at rest, a uniform flow along the walls), a checkerboard flow
whose wall ghosts equal its periodic image, conservation, the left-right
mirror image, the unchanged interior and the temporal order."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_11890_gb300 import workloads as W

GAM = 1.4


def problem(g, m=2, **kw):
    return O.make_problem(g.nx, g.nS, g.nB, g.nF, m, 0.01, g.dx, dz1=g.dz1, dz2=g.dz2, **kw)


def uniform(g, rho, u, w, p):
    q = np.empty((4, g.nz, g.nx))
    q[0], q[1], q[2] = rho, rho * u, rho * w
    q[3] = p / (GAM - 1) + 0.5 * rho * (u * u + w * w)
    return q


@pytest.mark.parametrize("wall", [O.WALL_NOSLIP, O.WALL_SLIP])
def test_checkerboard_normal_flow_sees_the_wall_as_its_periodic_image(wall):
    """u(i) = +u0, -u0, +u0, ... with nx even, w = 0, uniform rho and p, no
    gravity. Every central slope vanishes, and the x-wall ghosts (rho u
    flipped; u flipped) equal the periodic neighbours of the two edge columns.
    So R with x walls equals R with periodic x exactly. Flipping the wrong
    component, or not flipping, breaks the equality at the edge columns."""
    g = W.Grid(10, 5, 4, 6)
    u = np.where(np.arange(g.nx) % 2 == 0, 0.3, -0.3)[None, :] * np.ones((g.nz, 1))
    q = uniform(g, 1.3, 0.0, 0.0, 0.9)
    q[1] = 1.3 * u
    q[3] = 0.9 / (GAM - 1) + 0.5 * 1.3 * u * u
    kw = dict(G=0.0, mu1=2e-3, mu2=5e-3, wall=wall)
    Rw, Rp = O.rhs(problem(g, xwall=1, **kw), q), O.rhs(problem(g, xwall=0, **kw), q)
    scale = np.abs(Rp).max()
    assert np.abs(Rw - Rp).max() <= 1e-14 * scale
    assert np.abs(Rp[1]).max() > 0.1  # the flow does feel its faces


def test_pressure_ramp_at_rest_closed_form():
    """At rest with uniform rho, p linear in x, no gravity: only rho E has a
    slope. The wall cell's slope uses its mirror ghost, (E_1 - E_0)/(2 dx), so
    the wall state is E_0 - (E_1 - E_0)/4. The inner face averages
    (3E_0 + E_1)/4 and (E_0 + E_1)/2. The x-momentum flux is the pressure
    (gamma - 1) E on both faces, so R(rho u) in column 0 is
    -(5/8)(p_1 - p_0)/dx, and -(5/8)(p_{nx-1} - p_{nx-2})/dx in the last
    column. Extrapolating the wall state the wrong way gives -(1/8)."""
    g = W.Grid(10, 5, 4, 6)
    rho = 1.2
    p = 0.8 + 0.05 * np.arange(g.nx)[None, :] * np.ones((g.nz, 1))
    q = uniform(g, rho, 0.0, 0.0, 1.0)
    q[3] = p / (GAM - 1)
    R = O.rhs(problem(g, G=0.0, xwall=1), q)
    for k in range(g.nz):
        for i, (pa, pb) in ((0, (p[k, 0], p[k, 1])), (g.nx - 1, (p[k, -2], p[k, -1]))):
            want = -(5.0 / 8.0) * (pb - pa) / g.dx
            assert abs(R[1, k, i] - want) <= 1e-12 * abs(want), (k, i, R[1, k, i], want)


@pytest.mark.parametrize("wall,factor", [(O.WALL_NOSLIP, -2.0), (O.WALL_SLIP, 0.0)])
def test_uniform_tangential_flow_wall_shear(wall, factor):
    """A uniform flow (0, w0) along the x walls, without gravity: the mirror
    ghost keeps rho w, so the inviscid tangential flux vanishes. No-slip
    ghost -w0 gives sigma_xz = 2 mu w0/dx, so R(rho w) = -2 mu w0/dx^2 in
    both edge columns. The slip ghost +w0 gives 0. Rows next to the z walls
    and Gamma, where the vertical flow meets a wall, are left out."""
    g = W.Grid(10, 6, 4, 7)
    mu1, mu2 = 3e-3, 1e-3
    P = problem(g, G=0.0, mu1=mu1, mu2=mu2, wall=wall, xwall=1)
    w0 = 0.2
    q = uniform(g, 1.1, 0.0, w0, 0.8)
    R = O.rhs(P, q)
    rows = [k for k in range(2, g.nz - 2) if abs(k - g.n1) > 2 and abs(k - (g.n1 - 1)) > 2]
    assert rows
    for k in rows:
        mu = mu1 if k < g.n1 else mu2
        want = factor * mu * w0 / g.dx ** 2
        for i in (0, g.nx - 1):
            assert abs(R[2, k, i] - want) <= 1e-12 * max(abs(want), mu * w0 / g.dx ** 2), (k, i)
        assert np.all(np.abs(R[2, k, 1:-1]) <= 1e-13)


def test_walls_conserve_mass_and_keep_the_interior():
    """The sum of R(rho) dV over each fluid vanishes with x walls (no face
    carries mass out). Columns 2 .. nx-3, whose stencil does not reach a
    wall, get the periodic R bit for bit."""
    g = W.Grid(16, 6, 4, 7)
    q = W.gaussian_bumps(g, 5, sigma_cells=2.0, amp=0.03)
    Pw = problem(g, xwall=1)
    Pp = problem(g, xwall=0)
    Rw, Rp = O.rhs(Pw, q), O.rhs(Pp, q)
    for rows, dz in ((slice(0, g.n1), g.dz1), (slice(g.n1, g.nz), g.dz2)):
        tot = Rw[0, rows].sum() * g.dx * dz
        scale = np.abs(Rw[0, rows]).sum() * g.dx * dz
        assert abs(tot) <= 1e-13 * scale
    assert np.array_equal(Rw[:, :, 2:-2], Rp[:, :, 2:-2])
    assert np.abs(Rw[:, :, :2] - Rp[:, :, :2]).max() > 1e-6  # the walls do act


def test_rest_state_is_the_same_with_x_walls():
    """The hydrostatic rest state is x-invariant with u = 0: the mirror ghost
    equals the cell, so x walls change nothing."""
    g = W.Grid(12, 6, 4, 6)
    q = W.rest_state(g)
    assert np.allclose(O.rhs(problem(g, xwall=1), q), O.rhs(problem(g, xwall=0), q), rtol=0, atol=1e-15)


@pytest.mark.parametrize("wall", [O.WALL_NOSLIP, O.WALL_SLIP])
def test_left_right_mirror_image(wall):
    """Reflecting the state in x (columns reversed, rho u negated) reflects R
    the same way: the two walls are mirror images of each other."""
    g = W.Grid(14, 5, 4, 6)
    q = W.gaussian_bumps(g, 8, sigma_cells=2.0, amp=0.03)
    P = problem(g, wall=wall, xwall=1)
    flip = np.array([1.0, -1.0, 1.0, 1.0])[:, None, None]
    qm = flip * q[:, :, ::-1]
    R, Rm = O.rhs(P, q), O.rhs(P, qm)
    scale = np.abs(R).max(axis=(1, 2), keepdims=True)
    assert np.abs(Rm - flip * R[:, :, ::-1]).max(axis=(1, 2)).max() <= 1e-13 * scale.max()


def test_x_walls_keep_mass_over_a_run_and_order_two():
    """With walls on all sides, 40 MPRK2 steps keep each fluid's mass to
    1e-13. The error against a fine classical RK4 run falls at second order
    as the step halves (Table 6: 2.04, 2.00, 2.00)."""
    g = W.Grid(12, 5, 4, 6)
    q = W.thermal_convection(g)
    P = problem(g, m=4, mu1=2e-3, mu2=4e-3, xwall=1)
    P.dt = O.stable_dt(P, q, 0.4)
    d0 = O.diagnostics(P, q)
    qn, _ = O.mprk_step(P, q, 40)
    d1 = O.diagnostics(P, qn)
    assert abs(d1[0] - d0[0]) / d0[0] < 1e-13 and abs(d1[4] - d0[4]) / d0[4] < 1e-13
    dt0 = P.dt
    Pr = problem(g, m=1, mu1=2e-3, mu2=4e-3, xwall=1)
    ref = O.rk4_step(Pr, q, dt0 / 64, 4 * 64)
    errs = []
    for k in range(3):
        P.dt = dt0 / 2 ** k
        qk, _ = O.mprk_step(P, q, 4 * 2 ** k)
        errs.append(np.abs(qk - ref).max(axis=(1, 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.7), rates
