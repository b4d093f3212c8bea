"""Pins for the oracle planner (CPU only).

Each test checks the oracle against something other than itself: plans derived by hand
from the rules of Sec. 4.3 / Algorithm 1, special cases with closed forms, and an
invariant checker that must reject planted mistakes.
"""
import os
import random

import pytest

from oracle import planner as P

HERE = os.path.dirname(os.path.abspath(__file__))
MiB = 1 << 20


def load_golden(name):
    cases, cur = [], None
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "case":
                cur = {"N": int(tok[1]), "A": int(tok[2]), "paths": [], "chunks": []}
            elif tok[0] == "path":
                cur["paths"].append(tuple(int(t) for t in tok[1:]))
            elif tok[0] == "chunk":
                cur["chunks"].append(P.Chunk(*(int(t) for t in tok[1:])))
            elif tok[0] == "end":
                cases.append(cur)
    return cases


def test_copy64_worked_plan():
    # 64 MiB over {copy engine, SM kernel} at 50/50 with 4 MiB chunks: the copy engine
    # owns [0, 32 MiB) and the SM kernel [32 MiB, 64 MiB), eight 4 MiB chunks each.
    specs = [(P.CE, 32768, 4 * MiB), (P.SM, 32768, 4 * MiB)]
    got = P.plan(64 * MiB, P.D2D, specs)
    want = [P.Chunk(k * 4 * MiB, 4 * MiB, 0, k) for k in range(8)] + \
           [P.Chunk(32 * MiB + k * 4 * MiB, 4 * MiB, 1, k) for k in range(8)]
    assert got == want


@pytest.mark.parametrize("case", load_golden("interleave_plans.txt"), ids=lambda c: f"N{c['N']}")
def test_interleave_golden(case):
    got = P.plan(case["N"], P.D2D, case["paths"], case["A"], P.INTERLEAVE)
    assert got == case["chunks"]
    P.check_invariants(case["N"], case["paths"], case["A"], got)


def test_empty_message_has_no_chunks():
    for layout in (P.CONTIG, P.INTERLEAVE):
        assert P.plan(0, P.D2D, [(P.CE, 40000, 16), (P.SM, 25536, 16)], 16, layout) == []


def test_message_below_alignment_is_one_chunk_on_last_path():
    for n in range(1, 16):
        for layout in (P.CONTIG, P.INTERLEAVE):
            got = P.plan(n, P.D2D, [(P.CE, 30000, 64), (P.SM, 35536, 64)], 16, layout)
            assert got == [P.Chunk(0, n, 1, 0)]


def test_single_path_closed_form():
    for n, c in [(1000, 64), (4096, 4096), (4097, 4096), (10 * MiB + 3, MiB)]:
        got = P.plan(n, P.H2D, [(P.CE, 65536, c)], 16)
        k = -(-n // c)
        assert len(got) == k
        assert [x.offset for x in got] == [j * c for j in range(k)]
        assert all(x.nbytes == c for x in got[:-1]) and got[-1].nbytes == n - (k - 1) * c


def test_horizontal_split_closed_form():
    # 1000 bytes at 1/3, 1/3, 1/3 (21845, 21845, 21846), A = 16:
    # floor(1000*21845/65536) = 333 -> 320; 320; remainder 360.
    assert P.path_bytes(1000, [P.PathSpec(1, 21845, 16), P.PathSpec(2, 21845, 16),
                               P.PathSpec(4, 21846, 16)], 16) == [320, 320, 360]


def test_invariants_hold_on_random_plans():
    rng = random.Random(1234)
    for _ in range(400):
        A = 1 << rng.randrange(0, 7)
        npaths = rng.randrange(1, 5)
        cuts = sorted(rng.sample(range(1, 65536), npaths - 1))
        shares = [b - a for a, b in zip([0] + cuts, cuts + [65536])]
        kinds = [rng.choice(P.ALLOWED_KINDS[P.D2D]) for _ in range(npaths)]
        specs = [(k, s, A * rng.randrange(1, 40)) for k, s in zip(kinds, shares)]
        n = rng.choice([0, 1, A - 1, A, rng.randrange(0, 5000), rng.randrange(0, 1 << 22)])
        n = max(n, 0)
        for layout in (P.CONTIG, P.INTERLEAVE):
            chunks = P.plan(n, P.D2D, specs, A, layout)
            P.check_invariants(n, specs, A, chunks)
            if layout == P.CONTIG:
                # regions in path order: every chunk of path p precedes every chunk of p+1
                ends = {}
                for c in chunks:
                    ends.setdefault(c.path_index, []).append(c.offset)
                order = [min(v) for _, v in sorted(ends.items())]
                assert order == sorted(order)


def _valid_plan():
    specs = [(P.CE, 32768, 64), (P.SM, 32768, 64)]
    return specs, P.plan(1024, P.D2D, specs, 16)


@pytest.mark.parametrize("mutate", [
    "overlap", "gap", "misalign", "bad_index", "short_inner", "drop_last", "empty", "path_swap"])
def test_checker_rejects_planted_mistakes(mutate):
    specs, chunks = _valid_plan()
    chunks = list(chunks)
    if mutate == "overlap":
        chunks[1] = chunks[1]._replace(offset=chunks[1].offset - 16)
    elif mutate == "gap":
        chunks[1] = chunks[1]._replace(offset=chunks[1].offset + 16)
    elif mutate == "misalign":
        chunks[0] = chunks[0]._replace(nbytes=chunks[0].nbytes - 8)
        chunks[1] = chunks[1]._replace(offset=chunks[1].offset - 8, nbytes=chunks[1].nbytes + 8)
    elif mutate == "bad_index":
        chunks[2] = chunks[2]._replace(chunk_index=5)
    elif mutate == "short_inner":
        chunks[0] = chunks[0]._replace(nbytes=48)
        chunks.insert(1, P.Chunk(48, 16, 0, 1))
        chunks = [c if c.path_index != 0 or c.offset < 64 else c._replace(chunk_index=c.chunk_index + 1)
                  for c in chunks]
    elif mutate == "drop_last":
        chunks.pop()
    elif mutate == "empty":
        chunks.append(P.Chunk(1024, 0, 1, 8))
    elif mutate == "path_swap":
        # move one of path 0's chunks to path 1: shares no longer respected
        c = chunks.pop(7)
        chunks.append(c._replace(path_index=1, chunk_index=8))
    with pytest.raises(AssertionError):
        P.check_invariants(1024, specs, 16, chunks)


@pytest.mark.parametrize("n,direction,specs,align,layout", [
    (-1, P.D2D, [(P.CE, 65536, 16)], 16, P.CONTIG),
    (10, 7, [(P.CE, 65536, 16)], 16, P.CONTIG),
    (10, P.D2D, [(P.CE, 65536, 16)], 16, 3),
    (10, P.D2D, [(P.CE, 65536, 16)], 24, P.CONTIG),
    (10, P.D2D, [(P.CE, 65536, 16)], 8192, P.CONTIG),
    (10, P.D2D, [], 16, P.CONTIG),
    (10, P.D2D, [(P.CE, 8192, 16)] * 9, 16, P.CONTIG),
    (10, P.D2D, [(P.ZC, 65536, 16)], 16, P.CONTIG),
    (10, P.H2D, [(P.SM, 65536, 16)], 16, P.CONTIG),
    (10, P.D2D, [(P.CE, 0, 16), (P.SM, 65536, 16)], 16, P.CONTIG),
    (10, P.D2D, [(P.CE, 30000, 16), (P.SM, 30000, 16)], 16, P.CONTIG),
    (10, P.D2D, [(P.CE, 65536, 0)], 16, P.CONTIG),
    (10, P.D2D, [(P.CE, 65536, 24)], 16, P.CONTIG),
])
def test_invalid_requests_rejected(n, direction, specs, align, layout):
    with pytest.raises(ValueError):
        P.plan(n, direction, specs, align, layout)
