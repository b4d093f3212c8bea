"""Pins for the oracle cost model and its exhaustive search (CPU only): closed forms
of the stated model on cases whose optimum can be worked out by hand."""
import random

import pytest

from oracle import cost as C
from oracle import planner as P

ONE_B_PER_PS = 10 ** 12  # bandwidth at which T in ps equals the byte count


def model(alpha=0, beta=ONE_B_PER_PS, beta2=ONE_B_PER_PS, launch=0, hbm=10 ** 18, link=10 ** 18, override=None):
    paths = {k: C.PathModel(alpha, beta, beta2) for k in (P.CE, P.SM, P.HS, P.ZC)}
    paths.update(override or {})
    return C.Model(launch, hbm, link, link, paths)


def test_single_path_closed_form():
    m = model(alpha=700, beta=3 * 10 ** 11, launch=5000)
    for n, c in [(1, 16), (1000, 64), (4096, 512), (10 ** 6, 4096)]:
        k = -(-n // c)
        want = 5000 + 700 * k + -(-n * 10 ** 12 // (3 * 10 ** 11))
        assert C.plan_time(P.D2D, [P.CE], [n], c, m) == want


def test_equal_paths_split_evenly():
    split, chunk, t = C.brute_force(4096, P.D2D, [P.CE, P.SM], model())
    assert split == (2048, 2048) and t == 2048 and chunk == 4096  # all chunks tie: largest wins


def test_three_to_one_bandwidth_split():
    # copy engine at 3 bytes/ps, SM kernel at 1 byte/ps: T = max(ceil(b0/3), b1)
    m = model(override={P.CE: C.PathModel(0, 3 * ONE_B_PER_PS, ONE_B_PER_PS)})
    split, _, t = C.brute_force(4096, P.D2D, [P.CE, P.SM], m)
    assert split == (3072, 1024) and t == 1024


def test_shared_hbm_bound_tie_break():
    # HBM at 1 byte/ps makes every split cost 2N: the tie-break picks one path (the
    # first, carrying everything) and the largest chunk.
    m = model(hbm=ONE_B_PER_PS)
    split, chunk, t = C.brute_force(4096, P.D2D, [P.CE, P.SM], m)
    assert (split, chunk, t) == ((4096, 0), 4096, 8192)


def test_staged_pipeline_closed_form():
    # one staged path, both hops at 1 byte/ps, 100 ps per chunk:
    # T = 100*(N/C + 1) + N + C, minimised over powers of two at C = 512.
    m = model(alpha=100)
    split, chunk, t = C.brute_force(4096, P.D2D, [P.HS], m)
    assert chunk == 512 and t == 100 * (8 + 1) + 4096 + 512 and split == (4096,)


def test_staged_h2d_crosses_hbm_three_times():
    m = model(hbm=ONE_B_PER_PS)
    assert C.plan_time(P.H2D, [P.HS], [1000], 1024, m) == 3000
    assert C.plan_time(P.H2D, [P.CE], [1000], 1024, m) == 1000
    assert C.plan_time(P.D2D, [P.HS], [1000], 1024, model(link=ONE_B_PER_PS // 2)) == 2000


def test_host_link_shared_by_host_paths():
    m = model(link=ONE_B_PER_PS)
    # copy engine and zero-copy kernel share the link: splitting cannot beat N
    split, _, t = C.brute_force(2048, P.H2D, [P.CE, P.ZC], m)
    assert t == 2048 and split == (2048, 0)


def test_launch_latency_is_additive():
    a = C.brute_force(1024, P.D2D, [P.CE, P.SM], model())
    b = C.brute_force(1024, P.D2D, [P.CE, P.SM], model(launch=12345))
    assert a[0] == b[0] and b[2] == a[2] + 12345


def test_shares_reproduce_split():
    rng = random.Random(7)
    for _ in range(300):
        n = rng.randrange(1, 4097)
        npaths = rng.randrange(2, 4)
        split, rest = [], n
        for _ in range(npaths - 1):
            b = 16 * rng.randrange(0, rest // 16 + 1)
            split.append(b)
            rest -= b
        split.append(rest)
        if any(b == 0 for b in split[:-1]) or split[-1] == 0:
            continue
        w = C.shares_for_split(n, split)
        specs = [P.PathSpec(P.CE, s, 16) for s in w]
        assert P.path_bytes(n, specs, 16) == split


def test_shares_for_split_closed_forms():
    # N = 65536: a share is a byte count
    assert C.shares_for_split(65536, [16384, 4096, 45056]) == [16384, 4096, 45056]
    # halves of 32 KiB
    assert C.shares_for_split(32768, [16384, 16384]) == [32768, 32768]
    # thirds of 48 bytes: 65536 * 16 / 48 = 21845.33 rounds up to 21846 (floor(48 * 21846 /
    # 65536) = 16), and the last path takes the rest of 65536
    assert C.shares_for_split(48, [16, 16, 16]) == [21846, 21846, 21844]


def test_shares_for_split_are_the_smallest_that_work():
    # each listed share is the least w with floor(N * w / 65536) == b_p: one less falls short
    rng = random.Random(11)
    for _ in range(200):
        n = rng.randrange(32, 4097)
        b0 = 16 * rng.randrange(1, n // 16)
        if b0 >= n:
            continue
        w0 = C.shares_for_split(n, [b0, n - b0])[0]
        assert (n * w0) // 65536 == b0
        assert (n * (w0 - 1)) // 65536 < b0


def test_exhaustive_search_rejects_large_inputs():
    with pytest.raises(ValueError):
        C.brute_force(4097, P.D2D, [P.CE], model())
