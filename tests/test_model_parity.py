"""The library's cost model and split search (host code, no GPU) agree exactly with the
oracle's model and exhaustive search."""
import random

import pytest

import paper_2604_22228_gb300 as mpt
from oracle import cost as C
from oracle import planner as P
from paper_2604_22228_gb300 import build


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def random_model(rng):
    def bw():
        return rng.choice([10 ** 12, 3 * 10 ** 12, 10 ** 11, rng.randrange(10 ** 9, 10 ** 13)])
    paths = {k: C.PathModel(rng.choice([0, 100, 1000, rng.randrange(0, 10 ** 6)]), bw(), bw())
             for k in (P.CE, P.SM, P.HS, P.ZC)}
    return C.Model(rng.choice([0, 5000, rng.randrange(0, 10 ** 7)]), bw(), bw(), bw(), paths)


def as_lib(m: C.Model):
    return {"launch_ps": m.launch_ps, "hbm_Bps": m.hbm_Bps, "link_h2d_Bps": m.link_h2d_Bps,
            "link_d2h_Bps": m.link_d2h_Bps, "ce": tuple(m.paths[P.CE]), "sm": tuple(m.paths[P.SM]),
            "hs": tuple(m.paths[P.HS]), "zc": tuple(m.paths[P.ZC])}


def test_model_time_identical():
    rng = random.Random(11)
    for _ in range(3000):
        m = random_model(rng)
        d = rng.choice([P.D2D, P.H2D, P.D2H])
        kinds = [rng.choice(P.ALLOWED_KINDS[d]) for _ in range(rng.randrange(1, 5))]
        bytes_ = [rng.choice([0, rng.randrange(1, 10 ** 4), rng.randrange(0, 1 << 40)]) for _ in kinds]
        chunk = rng.choice([16, 4096, 1 << 20, rng.randrange(1, 1 << 30)])
        assert mpt.mpt_model_time(as_lib(m), d, kinds, bytes_, chunk) == C.plan_time(d, kinds, bytes_, chunk, m)


def test_optimizer_matches_exhaustive_search_on_tiny_messages():
    rng = random.Random(12)
    for trial in range(120):
        m = random_model(rng)
        d = rng.choice([P.D2D, P.H2D, P.D2H])
        kinds = [rng.choice(P.ALLOWED_KINDS[d]) for _ in range(rng.randrange(1, 4))]
        n = rng.choice([0, 1, 15, 16, 100, rng.randrange(0, 4097), 4096])
        if len(kinds) == 3 and n > 1500:
            n = rng.randrange(0, 1500)  # keep the Python search quick
        split, chunk, t = C.brute_force(n, d, kinds, m)
        got = mpt.mpt_model_optimize(as_lib(m), n, d, kinds)
        assert got == (tuple(split), chunk, t), (trial, n, d, kinds, m)


def test_optimizer_closed_forms():
    one = 10 ** 12
    m = C.Model(0, 10 ** 18, 10 ** 18, 10 ** 18, {k: C.PathModel(0, one, one) for k in (P.CE, P.SM, P.HS, P.ZC)})
    m = m._replace(paths={**m.paths, P.CE: C.PathModel(0, 3 * one, one)})
    assert mpt.mpt_model_optimize(as_lib(m), 4096, P.D2D, [P.CE, P.SM]) == ((3072, 1024), 4096, 1024)
    # large messages: shares on a 1/64 grid
    b, chunk, t = mpt.mpt_model_optimize(as_lib(m), 64 << 20, P.D2D, [P.CE, P.SM])
    assert b == (48 << 20, 16 << 20)


def test_invalid_model_rejected():
    m = C.Model(0, 0, 1, 1, {k: C.PathModel(0, 1, 1) for k in (P.CE, P.SM, P.HS, P.ZC)})
    with pytest.raises(mpt.MptError):
        mpt.mpt_model_time(as_lib(m), P.D2D, [P.CE], [10], 16)
    m = m._replace(hbm_Bps=1)
    with pytest.raises(mpt.MptError):
        mpt.mpt_model_optimize(as_lib(m), 100, P.D2D, [P.ZC])
