"""Host logic of the benchmark that decides what a serving measurement may claim, checked
on the CPU against brute force."""
import random

import bench


def _lay_out(sizes, kinds, ring_bytes):
    """Destinations filled in order into per-kind rings, wrapping to 0 when a request does
    not fit (the layout the native replay uses)."""
    heads, laps, place = {}, {}, []
    for nb, kind in zip(sizes, kinds):
        step = (nb + 255) // 256 * 256
        if heads.get(kind, 0) + step > ring_bytes[kind]:
            heads[kind] = 0
            laps[kind] = laps.get(kind, 0) + 1
        a = heads.get(kind, 0)
        heads[kind] = a + step
        place.append((kind, laps.get(kind, 0), a, a + nb))
    return place


def test_ring_next_overwrite_matches_brute_force():
    rng = random.Random(5)
    for trial in range(30):
        n = rng.randint(1, 300)
        sizes = [rng.choice([16, 100, 4096, 70000, 300000]) for _ in range(n)]
        kinds = [rng.choice(["dev", "host"]) for _ in range(n)]
        place = _lay_out(sizes, kinds, {"dev": 1 << 20, "host": 1 << 19})
        got = bench.ring_next_overwrite(place)
        for k, (kind, lap, a, b) in enumerate(place):
            want = -1
            for j in range(k + 1, n):
                kj, lj, aj, bj = place[j]
                if kj == kind and lj == lap + 1 and aj < b and bj > a:
                    want = j
                    break
            assert got[k] == want, (trial, k)


def test_ring_next_overwrite_edges():
    # touching ranges do not overlap; a later lap two rings ahead is not "next"
    place = [("dev", 0, 0, 100), ("dev", 0, 256, 356), ("dev", 1, 100, 256), ("dev", 1, 256, 300),
             ("dev", 2, 0, 50)]
    assert bench.ring_next_overwrite(place) == [-1, 3, -1, -1, -1]
