"""Second-order consistency of the oracle's right-hand side with the continuous
Navier–Stokes operator of Sec. 2 (Eq. cns-gov, nondimensional form of App. A).

The continuous operator is derived here symbolically (sympy) from the PDE, not
from the oracle's discrete formulas. For a smooth manufactured state sampled
at cell centres, the discrete R must approach it like h^2 at cells away from
the walls and the interface. The inviscid part, the viscous part and the
gravity source are checked separately, so that a dropped term, a wrong sign or
a wrong coefficient in any of them fails."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_11890_gb300 import workloads as W

sp = pytest.importorskip("sympy")

GAM, PR = 1.4, 0.72


def _continuous_operator():
    x, z, mu, G = sp.symbols("x z mu G", real=True)
    kx = 2 * sp.pi / 10
    rho = 1 + sp.Rational(1, 10) * sp.sin(kx * x) * sp.cos(sp.Rational(7, 10) * z)
    u = sp.Rational(1, 10) * sp.cos(kx * x + sp.Rational(3, 10)) + sp.Rational(1, 20) * sp.sin(z / 2)
    w = sp.Rational(1, 20) * sp.sin(kx * x) * sp.sin(sp.Rational(3, 5) * z + sp.Rational(1, 2))
    p = sp.Rational(7, 10) + sp.Rational(1, 20) * sp.cos(sp.Rational(4, 5) * z) * sp.sin(kx * x + 1)
    rE = p / (GAM - 1) + rho * (u ** 2 + w ** 2) / 2
    T = GAM * p / rho
    kap = mu / ((GAM - 1) * PR)
    ux, uz, wx, wz = sp.diff(u, x), sp.diff(u, z), sp.diff(w, x), sp.diff(w, z)
    div = ux + wz
    sxx = mu * (2 * ux - sp.Rational(2, 3) * div)
    szz = mu * (2 * wz - sp.Rational(2, 3) * div)
    sxz = mu * (uz + wx)
    FI = [rho * u, rho * u * u + p, rho * u * w, u * (rE + p)]
    HI = [rho * w, rho * w * u, rho * w * w + p, w * (rE + p)]
    FV = [0, sxx, sxz, u * sxx + w * sxz + kap * sp.diff(T, x)]
    HV = [0, sxz, szz, u * sxz + w * szz + kap * sp.diff(T, z)]
    src = [0, 0, -rho * G, -rho * w * G]
    state = [rho, u, w, p]
    inv = [-sp.diff(FI[c], x) - sp.diff(HI[c], z) for c in range(4)]
    vis = [sp.diff(FV[c], x) + sp.diff(HV[c], z) for c in range(4)]
    f_state = sp.lambdify((x, z), state, "numpy")
    f_inv = sp.lambdify((x, z), inv, "numpy")
    f_vis = sp.lambdify((x, z, mu), vis, "numpy")
    f_src = sp.lambdify((x, z, G), src, "numpy")
    return f_state, f_inv, f_vis, f_src


@pytest.fixture(scope="module")
def operator():
    return _continuous_operator()


def _grid_and_state(f_state, nx):
    n1 = nx // 2
    g = W.Grid(nx, n1 - 4, 4, n1)
    X = g.x_centres()[None, :] * np.ones((g.nz, 1))
    Z = g.z_centres()[:, None] * np.ones((1, nx))
    rho, u, w, p = [np.broadcast_to(np.asarray(a, dtype=float), X.shape) for a in f_state(X, Z)]
    return g, X, Z, W.conserved(rho, u, w, p)


def _interior(g):
    """Rows whose centres lie at least 1.5 from the walls and the interface (a
    fixed physical region, so that refinement compares like with like)."""
    z = g.z_centres()
    zlo, zhi = -g.n1 * g.dz1, (g.nz - g.n1) * g.dz2
    d = np.minimum(np.minimum(z - zlo, zhi - z), np.abs(z))
    return np.nonzero(d >= 1.5)[0]


def _err(g, R, L):
    rows = _interior(g)
    return np.abs(R[:, rows] - np.asarray([np.broadcast_to(l, R.shape[1:]) for l in L])[:, rows])


@pytest.mark.parametrize("part", ["inviscid", "viscous", "source"])
def test_second_order_consistency(operator, part):
    f_state, f_inv, f_vis, f_src = operator
    mu1, mu2, Gv = 0.02, 0.05, 0.1
    errs = []
    for nx in (20, 40, 80):
        g, X, Z, q = _grid_and_state(f_state, nx)
        def R(mu1_, mu2_, G_):
            P = O.make_problem(nx, g.nS, g.nB, g.nF, 2, 0.01, g.dx, mu1=mu1_, mu2=mu2_, G=G_)
            return O.rhs(P, q)
        if part == "inviscid":
            Rd = R(0.0, 0.0, 0.0)
            L = f_inv(X, Z)
        elif part == "viscous":
            Rd = R(mu1, mu2, 0.0) - R(0.0, 0.0, 0.0)
            mu = np.where(np.arange(g.nz)[:, None] < g.n1, mu1, mu2) * np.ones((1, nx))
            L = f_vis(X, Z, mu)
        else:
            Rd = R(0.0, 0.0, Gv) - R(0.0, 0.0, 0.0)
            L = f_src(X, Z, Gv)
        e = _err(g, Rd, L)
        errs.append(e.max(axis=(1, 2)))
    errs = np.array(errs)  # [refinement][component]
    if part == "source":
        # point values of the source are sampled exactly: equal to round-off
        assert errs.max() < 1e-15, errs
        return
    comps = [c for c in range(4) if errs[0, c] > 1e-13]
    assert comps, errs
    rates = np.log2(errs[:-1, comps] / errs[1:, comps])
    assert np.all(rates > 1.7), (part, errs, rates)
    # the discrete operator is close to the continuous one in absolute terms
    Lscale = max(np.abs(np.asarray(l)).max() for l in L)
    assert errs[-1, comps].max() < 0.05 * Lscale
