"""The library's planner (mpt_plan, host code, no GPU) produces exactly the oracle's plan,
and rejects exactly the requests the oracle rejects."""
import random

import pytest

import paper_2604_22228_gb300 as mpt
from oracle import planner as P
from paper_2604_22228_gb300 import build

from test_oracle_planner import load_golden

MiB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def lib_plan(n, direction, specs, align=16, layout=P.CONTIG):
    h = mpt.mpt_plan(None, n, direction, specs, align, layout)
    try:
        return [P.Chunk(*c) for c in mpt.mpt_plan_chunks(h)], mpt.mpt_plan_paths(h)
    finally:
        mpt.mpt_plan_destroy(h)


def test_copy64_plan_identical():
    specs = [(P.CE, 32768, 4 * MiB), (P.SM, 32768, 4 * MiB)]
    got, paths = lib_plan(64 * MiB, P.D2D, specs)
    assert got == P.plan(64 * MiB, P.D2D, specs)
    assert [(p["kind"], p["share"], p["chunk_bytes"]) for p in paths] == specs


@pytest.mark.parametrize("case", load_golden("interleave_plans.txt"), ids=lambda c: f"N{c['N']}")
def test_golden_interleave_identical(case):
    got, _ = lib_plan(case["N"], P.D2D, case["paths"], case["A"], P.INTERLEAVE)
    assert got == case["chunks"]


def test_random_plans_identical():
    rng = random.Random(20260)
    for trial in range(1500):
        A = 1 << rng.randrange(0, 13)
        direction = rng.choice([P.D2D, P.H2D, P.D2H])
        npaths = rng.randrange(1, 9)
        cuts = sorted(rng.sample(range(1, 65536), npaths - 1))
        shares = [b - a for a, b in zip([0] + cuts, cuts + [65536])]
        specs = [(rng.choice(P.ALLOWED_KINDS[direction]), s, A * rng.randrange(1, 64)) for s in shares]
        n = rng.choice([0, 1, A - 1, A, A + 1, rng.randrange(0, 1 << 16), rng.randrange(0, 1 << 26),
                        rng.randrange(0, 1 << 44)])
        want_chunks = sum(-(-b // s[2]) for b, s in zip(P.path_bytes(n, [P.PathSpec(*s) for s in specs], A), specs))
        if want_chunks > 200000:
            continue
        layout = rng.choice([P.CONTIG, P.INTERLEAVE])
        got, _ = lib_plan(n, direction, specs, A, layout)
        assert got == P.plan(n, direction, specs, A, layout), (trial, n, direction, specs, A, layout)


@pytest.mark.parametrize("n,direction,specs,align,layout", [
    (10, 7, [(P.CE, 65536, 16)], 16, P.CONTIG),
    (10, P.D2D, [(P.CE, 65536, 16)], 16, 3),
    (10, P.D2D, [(P.CE, 65536, 16)], 24, P.CONTIG),
    (10, P.D2D, [(P.CE, 65536, 16)], 8192, P.CONTIG),
    (10, P.D2D, [(P.CE, 8192, 16)] * 9, 16, P.CONTIG),
    (10, P.D2D, [(P.ZC, 65536, 16)], 16, P.CONTIG),
    (10, P.H2D, [(P.SM, 65536, 16)], 16, P.CONTIG),
    (10, P.D2H, [(P.SM, 65536, 16)], 16, P.CONTIG),
    (10, P.D2D, [(P.CE, 0, 16), (P.SM, 65536, 16)], 16, P.CONTIG),
    (10, P.D2D, [(P.CE, 30000, 16), (P.SM, 30000, 16)], 16, P.CONTIG),
    (10, P.D2D, [(P.CE, 65536, 24)], 16, P.CONTIG),
    (10, P.D2D, [(3, 65536, 16)], 16, P.CONTIG),
])
def test_invalid_requests_rejected_by_both(n, direction, specs, align, layout):
    with pytest.raises(ValueError):
        P.plan(n, direction, specs, align, layout)
    with pytest.raises(mpt.MptError) as e:
        lib_plan(n, direction, specs, align, layout)
    assert e.value.status == mpt.MPT_EINVAL


def test_zero_chunk_needs_context():
    with pytest.raises(mpt.MptError):
        lib_plan(1000, P.D2D, [(P.SM, 65536, 0)])


def test_chunk_count_limit():
    with pytest.raises(mpt.MptError) as e:
        lib_plan((mpt.MPT_MAX_CHUNKS + 1) * 16, P.D2D, [(P.SM, 65536, 16)])
    assert "limit" in str(e.value)
    got, _ = lib_plan(mpt.MPT_MAX_CHUNKS * 16, P.D2D, [(P.SM, 65536, 16)])
    assert len(got) == mpt.MPT_MAX_CHUNKS


def test_host_thread_staging_is_host_link_only():
    """MPT_HS_HOST_THREADS has a CPU hop between a host buffer and a page-locked slot: it
    carries H2D and D2H transfers, and the plan's chunks are those of the oracle (flags do not
    change the split)."""
    for direction in (P.H2D, P.D2H):
        specs = [(P.ZC, 40000, 4096), (P.HS, 25536, 1024, 0, mpt.MPT_HS_HOST_THREADS)]
        got, _ = lib_plan(100_000 + 7, direction, specs)
        assert got == P.plan(100_000 + 7, direction, [s[:3] for s in specs], 16, P.CONTIG)
    with pytest.raises(mpt.MptError) as e:
        lib_plan(4096, P.D2D, [(P.HS, 65536, 1024, 0, mpt.MPT_HS_HOST_THREADS)])
    assert e.value.status == mpt.MPT_EINVAL


def test_duplex_flag_needs_a_host_side_and_a_context():
    import paper_2604_22228_gb300 as mpt
    with pytest.raises(mpt.MptError) as e:  # device-to-device has no link direction to share
        mpt.mpt_plan(None, 1 << 20, mpt.MPT_D2D, None, 16, mpt.MPT_PLAN_DUPLEX)
    assert e.value.status == mpt.MPT_EINVAL
    with pytest.raises(mpt.MptError) as e:  # pageable memory is not the duplex case
        mpt.mpt_plan(None, 1 << 20, mpt.MPT_H2D, None, 16, mpt.MPT_PLAN_DUPLEX | mpt.MPT_PLAN_PAGEABLE)
    assert e.value.status == mpt.MPT_EINVAL
    with pytest.raises(mpt.MptError) as e:  # the tuned choice needs a context
        mpt.mpt_plan(None, 1 << 20, mpt.MPT_H2D, None, 16, mpt.MPT_PLAN_DUPLEX)
    assert e.value.status == mpt.MPT_EINVAL


def _shipped_entries():
    import json
    import os
    import re
    root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2604_22228_gb300", "tuned")
    out = []
    for name in sorted(os.listdir(root)) if os.path.isdir(root) else []:
        if not name.endswith(".jsonl"):
            continue
        with open(os.path.join(root, name)) as f:
            for line in f:
                if line.strip() and not line.startswith("#"):
                    out.append((re.sub(r"\.jsonl$", "", name), json.loads(line)))
    return out


def test_shipped_tuned_tables_give_oracle_plans():
    """Every entry of the shipped offline-tuned tables is a path set the oracle accepts for its
    direction, and at both ends of the entry's size bucket (2^b and 2^(b+1) - 1 bytes) the
    library's plan equals the oracle's plan, which passes the oracle's invariant checker."""
    entries = _shipped_entries()
    assert entries, "no shipped table"
    for dev, e in entries:
        specs = [(p[0], p[1], p[2]) for p in e["paths"]]
        assert sum(s[1] for s in specs) == P.SHARE_ONE, (dev, e)
        assert all(s[0] in P.ALLOWED_KINDS[e["dir"]] for s in specs), (dev, e)
        assert e["us"] > 0, (dev, e)
        for n in (1 << e["bucket"], (2 << e["bucket"]) - 1):
            want = P.plan(n, e["dir"], specs)
            P.check_invariants(n, specs, 16, want)
            got, paths = lib_plan(n, e["dir"], specs)
            assert got == want, (dev, e, n)
            assert [(p["kind"], p["share"], p["chunk_bytes"]) for p in paths] == specs
