"""Oracle for the compute-plus-communication demonstration: Jacobi sweeps on a grid whose
rows are split into subdomains arranged in a ring (the paper's application study, Sec. 5.4:
each rank exchanges boundary rows with its two neighbours).

Splitting the grid and exchanging halo rows must not change the result (the paper reports
that Jacobi's convergence is unaffected by pipelined multi-path transfers), so the oracle
is the undivided grid: rows wrap around (the ring), columns 0 and W-1 stay fixed, and every
interior point becomes ((up + down) + (left + right)) * 0.25, each operation rounded to
fp32 in that order.

This module is test infrastructure (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def step(grid: np.ndarray) -> np.ndarray:
    """One sweep of the periodic-in-rows grid (float32, shape rows x cols)."""
    g = np.asarray(grid, dtype=np.float32)
    up = np.roll(g, 1, axis=0)
    down = np.roll(g, -1, axis=0)
    out = g.copy()
    vert = (up[:, 1:-1] + down[:, 1:-1]).astype(np.float32)
    horiz = (g[:, :-2] + g[:, 2:]).astype(np.float32)
    out[:, 1:-1] = ((vert + horiz).astype(np.float32) * np.float32(0.25)).astype(np.float32)
    return out


def run(grid: np.ndarray, iterations: int) -> np.ndarray:
    g = np.asarray(grid, dtype=np.float32)
    for _ in range(iterations):
        g = step(g)
    return g
