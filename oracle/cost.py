"""Oracle cost model and exhaustive split search.

The paper tunes the number of paths and chunks per path offline by exhaustive search
over link bandwidths, latencies and message sizes, separately for graph and non-graph
execution (Sec. 4.4), but prints no model.  This project states one, in integer
picoseconds so that every implementation evaluates it bit-identically:

* path p with ``b_p`` bytes in ``k_p = ceil(b_p / C)`` chunks, issue latency ``alpha_p``
  per chunk and bandwidth ``beta_p`` (bytes/s):
      T_p = alpha_p * k_p + ceil(b_p * 1e12 / beta_p)
* the two-hop staged path (Sec. 4.3: one stream per hop, hop two of a chunk after its
  hop one) pipelines its chunks, so it pays one extra issue latency and one chunk at
  the faster hop on top of streaming everything at the slower hop:
      T_HS = alpha * (k + 1) + ceil(b * 1e12 / min(beta1, beta2))
             + ceil(min(C, b) * 1e12 / max(beta1, beta2))
* a path with no bytes costs 0;
* shared resources: HBM, ``T_HBM = ceil(sum_p h_p * b_p * 1e12 / B_HBM)``, and each
  direction of the host link, ``T_link = ceil(sum_p l_p * b_p * 1e12 / B_link)``, where
  ``h`` and ``l`` count how many times a path's byte crosses HBM or the link;
* total: ``T = alpha_launch + max(max_p T_p, T_HBM, T_link_h2d, T_link_d2h)``.

The exhaustive search (tiny messages only) tries every split in which paths
0..P-2 carry multiples of A and the last path the remainder, for every chunk size
``A * 2**k <= max(N, A)`` shared by all paths, and keeps the minimum under the
canonical tie-break: lowest T, then fewest non-empty paths, then the
lexicographically largest (b_0, b_1, ...), then the largest chunk.

This module is test infrastructure (see the package docstring).
"""
from __future__ import annotations

from typing import NamedTuple

from .planner import ALLOWED_KINDS, CE, D2D, D2H, H2D, HS, SM, ZC

PS_PER_S = 10 ** 12

# h: HBM crossings per payload byte; (l_h2d, l_d2h): host-link crossings per byte.
# Device-to-device: read source + write destination.  Staged device-to-device goes
# out over the link to pinned host memory and back.  Host-to-device and
# device-to-host touch HBM once directly and three times through a device stage
# (write stage, read stage, write destination / read source, write stage, read stage).
HBM_CROSSINGS = {
    (D2D, CE): 2, (D2D, SM): 2, (D2D, HS): 2,
    (H2D, CE): 1, (H2D, ZC): 1, (H2D, HS): 3,
    (D2H, CE): 1, (D2H, ZC): 1, (D2H, HS): 3,
}
LINK_CROSSINGS = {
    (D2D, CE): (0, 0), (D2D, SM): (0, 0), (D2D, HS): (1, 1),
    (H2D, CE): (1, 0), (H2D, ZC): (1, 0), (H2D, HS): (1, 0),
    (D2H, CE): (0, 1), (D2H, ZC): (0, 1), (D2H, HS): (0, 1),
}


class PathModel(NamedTuple):
    alpha_ps: int    # issue latency per chunk
    beta_Bps: int    # bandwidth (first hop for the staged path)
    beta2_Bps: int   # second hop of the staged path; ignored by other kinds


class Model(NamedTuple):
    launch_ps: int
    hbm_Bps: int
    link_h2d_Bps: int
    link_d2h_Bps: int
    paths: dict      # kind -> PathModel


def ceil_div(a: int, b: int) -> int:
    return -(-a // b)


def path_time(kind: int, nbytes: int, chunk: int, pm: PathModel) -> int:
    if nbytes == 0:
        return 0
    k = ceil_div(nbytes, chunk)
    if kind == HS:
        slow = min(pm.beta_Bps, pm.beta2_Bps)
        fast = max(pm.beta_Bps, pm.beta2_Bps)
        return (pm.alpha_ps * (k + 1) + ceil_div(nbytes * PS_PER_S, slow)
                + ceil_div(min(chunk, nbytes) * PS_PER_S, fast))
    return pm.alpha_ps * k + ceil_div(nbytes * PS_PER_S, pm.beta_Bps)


def plan_time(direction: int, kinds, bytes_per_path, chunk: int, model: Model) -> int:
    """Modelled time in picoseconds of one transfer split as ``bytes_per_path``."""
    for k in kinds:
        if k not in ALLOWED_KINDS[direction]:
            raise ValueError("path kind cannot carry this direction")
    worst_path = max(path_time(k, b, chunk, model.paths[k]) for k, b in zip(kinds, bytes_per_path))
    hbm = ceil_div(sum(HBM_CROSSINGS[(direction, k)] * b for k, b in zip(kinds, bytes_per_path)) * PS_PER_S,
                   model.hbm_Bps)
    up = ceil_div(sum(LINK_CROSSINGS[(direction, k)][0] * b for k, b in zip(kinds, bytes_per_path)) * PS_PER_S,
                  model.link_h2d_Bps)
    down = ceil_div(sum(LINK_CROSSINGS[(direction, k)][1] * b for k, b in zip(kinds, bytes_per_path)) * PS_PER_S,
                    model.link_d2h_Bps)
    return model.launch_ps + max(worst_path, hbm, up, down)


def chunk_candidates(nbytes: int, align: int) -> list[int]:
    out = []
    c = align
    while c <= max(nbytes, align):
        out.append(c)
        c *= 2
    return out


def _splits(nbytes: int, paths: int, align: int):
    """Every split: paths 0..P-2 take multiples of A, the last takes the rest."""
    if paths == 1:
        yield (nbytes,)
        return
    for b0 in range(0, nbytes + 1, align):
        for rest in _splits(nbytes - b0, paths - 1, align):
            yield (b0,) + rest


def brute_force(nbytes: int, direction: int, kinds, model: Model, align: int = 16):
    """Optimal (bytes_per_path, chunk, time_ps) by exhaustive search; tiny N only."""
    if nbytes > 4096 or len(kinds) > 3:
        raise ValueError("exhaustive search is for N <= 4096 and at most 3 paths")
    best_key, best = None, None
    for chunk in chunk_candidates(nbytes, align):
        for split in _splits(nbytes, len(kinds), align):
            t = plan_time(direction, kinds, split, chunk, model)
            key = (t, sum(1 for b in split if b > 0), tuple(-b for b in split), -chunk)
            if best_key is None or key < best_key:
                best_key, best = key, (split, chunk, t)
    return best


def shares_for_split(nbytes: int, split) -> list[int]:
    """Integer shares (out of 65536) whose horizontal split reproduces ``split``.

    Valid when N <= 65536 and paths 0..P-2 carry multiples of A: then
    ``w_p = ceil(65536 * b_p / N)`` gives ``floor(N * w_p / 65536) == b_p``.  A path
    with zero bytes cannot be listed (shares must be positive), so the caller drops it.
    """
    if nbytes == 0:
        raise ValueError("no split of an empty message")
    w = [ceil_div(65536 * b, nbytes) for b in split[:-1]]
    w.append(65536 - sum(w))
    return w
