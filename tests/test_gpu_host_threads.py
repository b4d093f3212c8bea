"""GPU parity of host-thread staging (MPT_HS_HOST_THREADS): the host-staged path with a CPU
hop -- host buffer <-> page-locked slot by the context's host threads, slot <-> device by a
copy engine (Algorithm 2 StageHostCopy).  Bytes are compared with the oracle's copy, guard
bytes around every destination must survive, and host buffers may be pageable."""
import numpy as np
import pytest

import paper_2604_22228_gb300 as mpt
from oracle import planner as P
from oracle import transfer as T

from gpu_util import Buf, seeded

pytestmark = pytest.mark.gpu
MiB = 1 << 20
HT = mpt.MPT_HS_HOST_THREADS


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    from paper_2604_22228_gb300 import build
    build.build()
    c = mpt.mpt_ctx_create(0)
    yield c
    st, site = mpt.mpt_ctx_status(c)
    mpt.mpt_ctx_destroy(c)
    assert st == mpt.MPT_OK, f"device status {st} at site {site}"


def _pageable_zc(ctx):
    return bool(mpt.mpt_ctx_info(ctx)["pageable_access"])


def _move(ctx, n, direction, specs, host_kind, mode, seed, src_off=0, dst_off=0, replays=2):
    import torch
    src = Buf(n, host_kind if direction == P.H2D else "dev", src_off)
    dst = Buf(n, host_kind if direction == P.D2H else "dev", dst_off)
    data = seeded("u32", seed, n)
    src.fill(data)
    plan = mpt.mpt_plan(ctx, n, direction, specs)
    try:
        resolved = [(p["kind"], p["share"], p["chunk_bytes"]) for p in mpt.mpt_plan_paths(plan)]
        assert [P.Chunk(*c) for c in mpt.mpt_plan_chunks(plan)] == P.plan(n, direction, resolved, 16, P.CONTIG)
        s = torch.cuda.current_stream()
        info = None
        for _ in range(replays):
            h = mpt.mpt_prepare(ctx, plan, dst.ptr, src.ptr,
                                mpt.MPT_PREPARE_GRAPH if mode == "graph" else mpt.MPT_PREPARE_EAGER)
            info = mpt.mpt_graph_get_info(h)
            mpt.mpt_launch(h, s)
            mpt.mpt_graph_release(h)
        torch.cuda.synchronize()
    finally:
        mpt.mpt_plan_destroy(plan)
    out = dst.numpy()
    expect = T.copy(data)
    assert np.array_equal(out, expect), f"first mismatch at {int(np.argmax(out != expect))}"
    assert dst.guards_intact(), "bytes outside the destination were written"
    return info


@pytest.mark.parametrize("mode", ["graph", "eager"])
@pytest.mark.parametrize("direction", [P.H2D, P.D2H])
@pytest.mark.parametrize("host_kind", ["pinned", "pageable"])
def test_host_threads_alone(ctx, mode, direction, host_kind):
    for n, cb in ((1, 16), (4096 + 3, 1024), (3 * MiB + 7, MiB), (17 * MiB + 5, 4 * MiB)):
        info = _move(ctx, n, direction, [(P.HS, 65536, cb, 0, HT)], host_kind, mode, 31 + n, 3, 5)
        if mode == "graph":
            k = -(-n // cb)
            assert info["host_nodes"] == k and info["memcpy_nodes"] == k


@pytest.mark.parametrize("mode", ["graph", "eager"])
@pytest.mark.parametrize("direction", [P.H2D, P.D2H])
def test_host_threads_with_zero_copy_pageable(ctx, mode, direction):
    """The multi-path for ordinary host memory: zero-copy kernel + host-thread staging."""
    if not _pageable_zc(ctx):
        pytest.skip("device cannot reach pageable host memory")
    n = 24 * MiB + 11
    specs = [(P.ZC, 40000, 4 * MiB), (P.HS, 25536, 2 * MiB, 0, HT)]
    _move(ctx, n, direction, specs, "pageable", mode, 77, 1, 9)


@pytest.mark.parametrize("direction", [P.H2D, P.D2H])
def test_host_threads_with_copy_engine_pinned(ctx, direction):
    specs = [(P.CE, 30000, 2 * MiB), (P.HS, 20000, MiB, 0, HT), (P.ZC, 15536, MiB)]
    _move(ctx, 9 * MiB + 48, direction, specs, "pinned", "graph", 91)


def test_pageable_needs_host_side_paths(ctx):
    """A copy-engine path may not touch pageable memory: such plans are refused."""
    n = 2 * MiB
    src, dev = Buf(n, "pageable"), Buf(n, "dev")
    plan = mpt.mpt_plan(ctx, n, P.H2D, [(P.CE, 32768, MiB), (P.HS, 32768, MiB, 0, HT)])
    try:
        for mode in (mpt.MPT_PREPARE_GRAPH, mpt.MPT_PREPARE_EAGER):
            with pytest.raises(mpt.MptError) as e:
                mpt.mpt_prepare(ctx, plan, dev.ptr, src.ptr, mode)
            assert e.value.status == mpt.MPT_EINVAL
    finally:
        mpt.mpt_plan_destroy(plan)


def test_rebind_refused_and_capture_rebuilds(ctx):
    import torch
    n = 3 * MiB
    a, b = Buf(n, "pageable"), Buf(n, "pageable")
    dev = Buf(n, "dev")
    da, db = seeded("u32", 5, n), seeded("u32", 6, n)
    a.fill(da)
    b.fill(db)
    plan = mpt.mpt_plan(ctx, n, P.H2D, [(P.HS, 65536, MiB, 0, HT)])
    try:
        g = mpt.mpt_capture(ctx, plan, dev.ptr, a.ptr)
        with pytest.raises(mpt.MptError) as e:
            mpt.mpt_graph_rebind(g, plan, dev.ptr, b.ptr)
        assert e.value.status == mpt.MPT_ENOTSUP
        mpt.mpt_launch(g, torch.cuda.current_stream())
        assert np.array_equal(dev.numpy(), da)
        g2 = mpt.mpt_capture(ctx, plan, dev.ptr, b.ptr)  # a new graph, not a retargeted one
        assert mpt.mpt_graph_get_info(g2)["rebinds"] == 0
        mpt.mpt_launch(g2, torch.cuda.current_stream())
        assert np.array_equal(dev.numpy(), db)
        for h in (g, g2):
            mpt.mpt_graph_release(h)
    finally:
        mpt.mpt_plan_destroy(plan)


def test_eager_refused_inside_stream_capture(ctx):
    import torch
    n = MiB
    src, dev = Buf(n, "pinned"), Buf(n, "dev")
    plan = mpt.mpt_plan(ctx, n, P.H2D, [(P.HS, 65536, 256 * 1024, 0, HT)])
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    try:
        with torch.cuda.graph(graph, stream=s):
            with pytest.raises(mpt.MptError) as e:
                mpt.mpt_launch_eager(ctx, plan, dev.ptr, src.ptr, s)
            assert e.value.status == mpt.MPT_EINVAL
    finally:
        mpt.mpt_plan_destroy(plan)


def test_concurrent_transfers_share_the_pool(ctx):
    """Two streams, each replaying its own host-thread graph several times: CPU hops of both
    run on the one pool at once."""
    import torch
    n = 12 * MiB + 3
    bufs = []
    for k in range(2):
        src, dst = Buf(n, "pageable"), Buf(n, "dev")
        data = seeded("u32", 200 + k, n)
        src.fill(data)
        bufs.append((src, dst, data))
    plan = mpt.mpt_plan(ctx, n, P.H2D, [(P.HS, 65536, 2 * MiB, 0, HT)])
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    try:
        gs = [mpt.mpt_capture(ctx, plan, d.ptr, s.ptr) for s, d, _ in bufs]
        for _ in range(4):
            for g, st in zip(gs, streams):
                mpt.mpt_launch(g, st)
        torch.cuda.synchronize()
        for (s, d, data) in bufs:
            assert np.array_equal(d.numpy(), T.copy(data)) and d.guards_intact()
        for g in gs:
            mpt.mpt_graph_release(g)
    finally:
        mpt.mpt_plan_destroy(plan)


def _pageable_safe(paths):
    return all(p["kind"] == P.ZC or (p["kind"] == P.HS and p["flags"] & HT) for p in paths)


@pytest.mark.parametrize("direction", [P.H2D, P.D2H])
def test_pageable_plans_from_the_tuner(monkeypatch, direction):
    """mpt_plan(..., MPT_PLAN_PAGEABLE) gives a plan whose every path accepts pageable host
    memory, untuned (default) and after mpt_tune(mode | MPT_MODE_PAGEABLE); both move a
    pageable buffer bit-exactly."""
    import torch
    monkeypatch.setenv("MPT_TUNE_DEFAULTS", "0")
    c = mpt.mpt_ctx_create(0)
    try:
        for n in (300_000 + 3, 16 * MiB + 5):
            untuned = mpt.mpt_plan(c, n, direction, None, 16, mpt.MPT_PLAN_PAGEABLE)
            assert _pageable_safe(mpt.mpt_plan_paths(untuned))
            mpt.mpt_plan_destroy(untuned)
            specs, us = mpt.mpt_tune(c, direction, n, mpt.MPT_MODE_GRAPH | mpt.MPT_MODE_PAGEABLE)
            assert us > 0 and _pageable_safe(specs)
            got, _ = mpt.mpt_tune_get(c, direction, n, mpt.MPT_MODE_GRAPH | mpt.MPT_MODE_PAGEABLE)
            assert got == specs
            with pytest.raises(mpt.MptError):  # the page-locked entry of this bucket is separate
                mpt.mpt_tune_get(c, direction, n, mpt.MPT_MODE_GRAPH)
            plan = mpt.mpt_plan(c, n, direction, None, 16, mpt.MPT_PLAN_PAGEABLE)
            assert mpt.mpt_plan_paths(plan) == specs
            host, dev = Buf(n, "pageable"), Buf(n, "dev")
            data = seeded("u32", 300 + n, n)
            (host if direction == P.H2D else dev).fill(data)
            dst, src = (dev, host) if direction == P.H2D else (host, dev)
            g = mpt.mpt_capture(c, plan, dst.ptr, src.ptr)
            mpt.mpt_launch(g, torch.cuda.current_stream())
            torch.cuda.synchronize()
            assert np.array_equal(dst.numpy(), T.copy(data)) and dst.guards_intact()
            mpt.mpt_graph_release(g)
            mpt.mpt_plan_destroy(plan)
        with pytest.raises(mpt.MptError) as e:
            mpt.mpt_plan(c, 4096, P.D2D, None, 16, mpt.MPT_PLAN_PAGEABLE)
        assert e.value.status == mpt.MPT_EINVAL
    finally:
        mpt.mpt_ctx_destroy(c)
