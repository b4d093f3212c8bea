"""Windows of concurrent multi-path transfers, and both host-link directions at once, against
the oracle byte for byte.

The paper's bandwidth tests post a window of 1, 4 or 16 messages before waiting for any, and
its bidirectional test runs both directions together (Sec. 5.3).  Here W prepared handles
(tuned plans or explicit multi-path plans; CUDA graph or direct issue) are launched at once on
W streams, and an H2D plan and a D2H plan over copy engine + zero-copy kernel + staged path
run at the same time.  Every window moves its own seeded payload, so a transfer that read or
wrote another window's buffer shows up as wrong bytes.
"""
import numpy as np
import pytest

import paper_2604_22228_gb300 as mpt
from oracle import transfer as T

from gpu_util import Buf, seeded

pytestmark = pytest.mark.gpu
MiB = 1 << 20
CE, SM, HS, ZC = mpt.MPT_PATH_CE, mpt.MPT_PATH_SM, mpt.MPT_PATH_HS, mpt.MPT_PATH_ZC


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


MULTI = {
    mpt.MPT_D2D: [(CE, 32768, MiB), (SM, 32768, MiB)],
    mpt.MPT_H2D: [(CE, 21846, MiB), (ZC, 21845, MiB), (HS, 21845, MiB)],
    mpt.MPT_D2H: [(CE, 21846, MiB), (ZC, 21845, MiB), (HS, 21845, MiB)],
}
WHERE = {mpt.MPT_D2D: ("dev", "dev"), mpt.MPT_H2D: ("host", "dev"), mpt.MPT_D2H: ("dev", "host")}


def _launch_together(handles, streams):
    """Launch handles[w] on streams[w], all released by one event on the current stream."""
    import torch
    main = torch.cuda.current_stream()
    go = torch.cuda.Event()
    go.record(main)
    for h, s in zip(handles, streams):
        s.wait_event(go)
        mpt.mpt_launch(h, s)
    for s in streams:
        main.wait_stream(s)
    torch.cuda.synchronize()


@pytest.mark.parametrize("direction", [mpt.MPT_D2D, mpt.MPT_H2D, mpt.MPT_D2H], ids=["d2d", "h2d", "d2h"])
@pytest.mark.parametrize("pathset", ["tuned", "multi"])
@pytest.mark.parametrize("mode", [mpt.MPT_PREPARE_GRAPH, mpt.MPT_PREPARE_EAGER], ids=["graph", "eager"])
def test_window_of_concurrent_transfers(ctx, direction, pathset, mode):
    import torch
    n = 4 * MiB + 4096 + 5
    wmax = 16
    s_where, d_where = WHERE[direction]
    srcs = [Buf(n, s_where, w % 16) for w in range(wmax)]
    dsts = [Buf(n, d_where, (3 * w) % 16) for w in range(wmax)]
    plan = mpt.mpt_plan(ctx, n, direction, None if pathset == "tuned" else MULTI[direction])
    handles = [mpt.mpt_prepare(ctx, plan, dsts[w].ptr, srcs[w].ptr, mode) for w in range(wmax)]
    streams = [torch.cuda.Stream() for _ in range(wmax)]
    try:
        for rnd, win in enumerate((1, 4, 16)):
            datas = [seeded("u8", 0x77000 + 100 * rnd + w, n) for w in range(win)]
            for w in range(win):
                srcs[w].fill(datas[w])
                dsts[w].view.zero_()
            torch.cuda.synchronize()
            _launch_together(handles[:win], streams[:win])
            for w in range(win):
                out = dsts[w].numpy()
                want = T.copy(datas[w])
                assert np.array_equal(out, want), (win, w, int(np.argmax(out != want)))
                assert dsts[w].guards_intact(), (win, w)
    finally:
        for h in handles:
            mpt.mpt_graph_release(h)
        mpt.mpt_plan_destroy(plan)
    st, site = mpt.mpt_ctx_status(ctx)
    assert st == mpt.MPT_OK, f"status {st} site {site}"


@pytest.mark.parametrize("pathset", ["tuned", "multi"])
@pytest.mark.parametrize("mode", [mpt.MPT_PREPARE_GRAPH, mpt.MPT_PREPARE_EAGER], ids=["graph", "eager"])
def test_host_to_device_and_device_to_host_at_once(ctx, pathset, mode):
    import torch
    n = 24 * MiB + 333
    h_src, d_dst = Buf(n, "host", 1), Buf(n, "dev", 2)
    d_src, h_dst = Buf(n, "dev", 3), Buf(n, "host", 4)
    up = mpt.mpt_plan(ctx, n, mpt.MPT_H2D, None if pathset == "tuned" else MULTI[mpt.MPT_H2D])
    down = mpt.mpt_plan(ctx, n, mpt.MPT_D2H, None if pathset == "tuned" else MULTI[mpt.MPT_D2H])
    hu = mpt.mpt_prepare(ctx, up, d_dst.ptr, h_src.ptr, mode)
    hd = mpt.mpt_prepare(ctx, down, h_dst.ptr, d_src.ptr, mode)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    try:
        for rnd in range(3):  # fresh bytes each round: a stale replay would show
            a, b = seeded("u32", 0x88000 + 2 * rnd, n), seeded("u32", 0x88001 + 2 * rnd, n)
            h_src.fill(a)
            d_src.fill(b)
            _launch_together([hu, hd], streams)
            assert np.array_equal(d_dst.numpy(), T.copy(a)), rnd
            assert np.array_equal(h_dst.numpy(), T.copy(b)), rnd
            assert d_dst.guards_intact() and h_dst.guards_intact()
    finally:
        for h in (hu, hd):
            mpt.mpt_graph_release(h)
        for p in (up, down):
            mpt.mpt_plan_destroy(p)
    st, site = mpt.mpt_ctx_status(ctx)
    assert st == mpt.MPT_OK, f"status {st} site {site}"


def test_duplex_plans_tuned_under_opposite_traffic(ctx):
    """Plans tuned while the other link direction is busy (MPT_MODE_DUPLEX), used for an H2D and
    a D2H transfer at once: the plan flag picks the tuned entry, an untuned size falls back to
    one copy-engine chunk, and both destinations equal the oracle's copies."""
    import torch
    n = 32 * MiB + 48
    # an untuned bucket: one copy-engine chunk covering the message
    try:
        mpt.mpt_tune_get(ctx, mpt.MPT_H2D, 3 * MiB, mpt.MPT_MODE_GRAPH | mpt.MPT_MODE_DUPLEX)
        untuned = False
    except mpt.MptError as e:
        untuned = e.status == mpt.MPT_EAGAIN
    if untuned:
        p = mpt.mpt_plan(ctx, 3 * MiB, mpt.MPT_H2D, None, 16, mpt.MPT_PLAN_DUPLEX)
        assert [(q["kind"], q["share"]) for q in mpt.mpt_plan_paths(p)] == [(CE, 65536)]
        assert len(mpt.mpt_plan_chunks(p)) == 1
        mpt.mpt_plan_destroy(p)
    tuned = {}
    for direction in (mpt.MPT_H2D, mpt.MPT_D2H):
        paths, us = mpt.mpt_tune(ctx, direction, n, mpt.MPT_MODE_GRAPH | mpt.MPT_MODE_DUPLEX, 3)
        assert paths and us > 0
        got, _ = mpt.mpt_tune_get(ctx, direction, n, mpt.MPT_MODE_GRAPH | mpt.MPT_MODE_DUPLEX)
        assert [tuple(x.values())[:2] for x in got] == [tuple(x.values())[:2] for x in paths]
        tuned[direction] = paths
    h_src, d_dst = Buf(n, "host"), Buf(n, "dev")
    d_src, h_dst = Buf(n, "dev"), Buf(n, "host")
    up = mpt.mpt_plan(ctx, n, mpt.MPT_H2D, None, 16, mpt.MPT_PLAN_DUPLEX)
    down = mpt.mpt_plan(ctx, n, mpt.MPT_D2H, None, 16, mpt.MPT_PLAN_DUPLEX)
    assert [q["kind"] for q in mpt.mpt_plan_paths(up)] == [q["kind"] for q in tuned[mpt.MPT_H2D]]
    hu = mpt.mpt_capture(ctx, up, d_dst.ptr, h_src.ptr)
    hd = mpt.mpt_capture(ctx, down, h_dst.ptr, d_src.ptr)
    try:
        a, b = seeded("u32", 0x99001, n), seeded("u32", 0x99002, n)
        h_src.fill(a)
        d_src.fill(b)
        _launch_together([hu, hd], [torch.cuda.Stream(), torch.cuda.Stream()])
        assert np.array_equal(d_dst.numpy(), T.copy(a))
        assert np.array_equal(h_dst.numpy(), T.copy(b))
        assert d_dst.guards_intact() and h_dst.guards_intact()
    finally:
        for h in (hu, hd):
            mpt.mpt_graph_release(h)
        for q in (up, down):
            mpt.mpt_plan_destroy(q)
