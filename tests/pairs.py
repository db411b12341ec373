"""Matched problem descriptions for the CUDA library and the CPU oracle."""
import os

import numpy as np

from oracle import oracle as O
from paper_2202_11890_gb300 import workloads as W


def oracle_threads():
    O.set_threads(max(1, min(os.cpu_count() or 1, 32)))


def pair(grid: W.Grid, m: int, dt: float = 0.0, precision: int = 0, scheme: int = 0, wall: int = 0,
         mu1=W.MU1, mu2=W.MU2, G=-W.G_SIGNED, diag_every: int = 0, q0=None, cfl=0.4, xwall: int = 0):
    """(mprk_config, oracle Problem, dt) for the same problem. dt == 0 picks
    the oracle's Courant-number step for q0."""
    from paper_2202_11890_gb300 import mprk as M
    P = O.make_problem(grid.nx, grid.nS, grid.nB, grid.nF, m, dt, grid.dx, dz1=grid.dz1,
                       dz2=grid.dz2, mu1=mu1, mu2=mu2, G=G, wall=wall, xwall=xwall)
    if dt == 0.0:
        assert q0 is not None
        dt = O.stable_dt(P, q0, cfl)
        P.dt = dt
    cfg = M.mprk_config_default(grid.nx, grid.nS, grid.nB, grid.nF, m)
    cfg.dt = dt
    cfg.dx, cfg.dz1, cfg.dz2 = grid.dx, grid.dz1, grid.dz2
    cfg.mu1, cfg.mu2, cfg.G = mu1, mu2, G
    cfg.precision, cfg.scheme, cfg.wall, cfg.diag_every = precision, scheme, wall, diag_every
    cfg.x_walls = xwall
    return cfg, P, dt


def rel_err(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Per-component max |a - b| / max |b| (the parity norm)."""
    scale = np.abs(b).max(axis=(-2, -1))
    scale = np.where(scale > 0, scale, 1.0)
    return np.abs(a - b).max(axis=(-2, -1)) / scale
