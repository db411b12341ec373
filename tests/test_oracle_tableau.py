"""Pins of the oracle's Butcher tableaus (Table 1; Eq. MRK2; Eq. speedup)."""
import os
from fractions import Fraction

import numpy as np
import pytest

from conftest import GOLDEN
from oracle import oracle as O


def _read_table1():
    blocks, cur = {}, None
    for line in open(os.path.join(GOLDEN, "table1_mprk2_m2.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = line.strip("[]")
            blocks[cur] = {"c": [], "a": [], "b": None}
            continue
        left, right = line.split("|")
        vals = [float(Fraction(v)) for v in right.split()]
        if left.strip() == "b":
            blocks[cur]["b"] = vals
        else:
            blocks[cur]["c"].append(float(Fraction(left.strip())))
            blocks[cur]["a"].append(vals)
    out = {}
    for name, blk in blocks.items():
        n = len(blk["c"])
        a = np.zeros((n, n))
        for i, row in enumerate(blk["a"]):
            a[i, : len(row)] = row
        out[name] = (a, np.array(blk["b"]), np.array(blk["c"]))
    return out


TABLE1 = _read_table1()
REGIONS = {"S": O.REGION_S, "B": O.REGION_B, "F": O.REGION_F}


@pytest.mark.parametrize("name", ["F", "B", "S"])
def test_m2_equals_table1(name):
    a, b, c = O.tableau(2, REGIONS[name])
    ga, gb, gc = TABLE1[name]
    assert np.array_equal(a, ga)
    assert np.array_equal(b, gb)
    assert np.array_equal(c, gc)


@pytest.mark.parametrize("name", ["F", "B", "S"])
def test_m1_is_base_rk2(name):
    a, b, c = O.tableau(1, REGIONS[name])
    ga, gb, gc = TABLE1["RK2"]
    assert np.array_equal(a, ga) and np.array_equal(b, gb) and np.array_equal(c, gc)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 8, 16])
@pytest.mark.parametrize("name", ["F", "B", "S"])
def test_consistency_conditions(m, name):
    """Row sums equal c (internal consistency), weights sum to 1 (first order),
    sum b c = 1/2 (second order), strictly lower triangular (explicit)."""
    a, b, c = O.tableau(m, REGIONS[name])
    assert np.allclose(a.sum(axis=1), c, rtol=0, atol=1e-15)
    assert abs(b.sum() - 1.0) < 1e-15
    assert abs(b @ c - 0.5) < 1e-15
    assert np.all(np.triu(a) == 0.0)


@pytest.mark.parametrize("m", [1, 2, 4, 8])
def test_slow_stages_collapse(m):
    """Algorithm 1: slow stages past s = 2 repeat stage mod(i-1,2)+1, and the
    slow weights vanish past stage 2; the buffer restarts at every odd stage."""
    aS, bS, cS = O.tableau(m, O.REGION_S)
    aB, bB, cB = O.tableau(m, O.REGION_B)
    for i in range(2, 2 * m):
        assert np.array_equal(aS[i], aS[i % 2])
        assert bS[i] == 0.0
        if i % 2 == 0:
            assert np.all(aB[i] == 0.0)
    # the buffer and the slow region see the same stage times
    assert np.array_equal(cS, cB)


def test_partitioned_pairs_share_stage_times_of_fast():
    """The fast tableau is m Heun substeps of dt/m: stage times k/m, (k+1)/m."""
    for m in [1, 2, 4, 8]:
        _, _, c = O.tableau(m, O.REGION_F)
        want = np.array([[k / m, (k + 1) / m] for k in range(m)]).ravel()
        assert np.allclose(c, want, rtol=0, atol=1e-15)


def test_speedup_counter_matches_table2():
    """Cell RHS evaluations counted inside one oracle step reproduce Eq. speedup
    and the spd column of Table 2 (N_B = 6, N_total = 100 rows)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table2_spd.txt")) if not l.startswith("#")]
    from paper_2202_11890_gb300 import workloads as W
    for r in rows:
        nS, ntot = int(r[0]), int(r[1])
        nB = 6
        nF = ntot - nS - nB
        for j, m in enumerate([2, 4, 8]):
            nx = 4
            g = W.Grid(nx, nS, nB, nF)
            P = O.make_problem(nx, nS, nB, nF, m, 1e-4, g.dx)
            q = W.rest_state(g)
            _, n_mprk = O.mprk_step(P, q)
            before = O.rhs_cell_count()
            for _ in range(m):
                O.rk2_step(P, q, 1e-4 / m)
            n_sr = O.rhs_cell_count() - before
            assert n_mprk == nx * (2 * nS + 2 * m * (nB + nF))
            assert n_sr == 2 * m * nx * ntot
            spd = n_sr / n_mprk
            formula = 1.0 / (1.0 + (1.0 / m - 1.0) * nS / ntot)
            assert abs(spd - formula) < 1e-12
            assert f"{spd + 1e-9:.1f}" == r[2 + j]
