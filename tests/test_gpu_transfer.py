"""GPU parity: every transfer path, graph and eager, against the oracle (bit-exact bytes,
identical plans, identical digests).  Calls go through the C ABI via the binding."""
import numpy as np
import pytest

import paper_2604_22228_gb300 as mpt
import payload
from oracle import planner as P
from oracle import transfer as T

from gpu_util import Buf, seeded

pytestmark = pytest.mark.gpu
MiB = 1 << 20


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


def run_transfer(ctx, n, direction, specs, kind="u8", seed=1, src_off=0, dst_off=0, layout=P.CONTIG, align=16,
                 mode="graph", replays=2):
    src_where = "host" if direction == P.H2D else "dev"
    dst_where = "host" if direction == P.D2H else "dev"
    src = Buf(n, src_where, src_off)
    dst = Buf(n, dst_where, dst_off)
    data = seeded(kind, seed, n)
    src.fill(data)
    plan = mpt.mpt_plan(ctx, n, direction, specs, align, layout)
    try:
        got_plan = [P.Chunk(*c) for c in mpt.mpt_plan_chunks(plan)]
        resolved = [(p["kind"], p["share"], p["chunk_bytes"]) for p in mpt.mpt_plan_paths(plan)]
        assert got_plan == P.plan(n, direction, resolved, align, layout)
        import torch
        s = torch.cuda.current_stream()
        info = None
        for _ in range(replays):
            if mode == "graph":
                g = mpt.mpt_capture(ctx, plan, dst.ptr, src.ptr)
                info = mpt.mpt_graph_get_info(g)
                mpt.mpt_launch(g, s)
                mpt.mpt_graph_release(g)
            else:
                mpt.mpt_launch_eager(ctx, plan, dst.ptr, src.ptr, s)
        torch.cuda.synchronize()
    finally:
        mpt.mpt_plan_destroy(plan)
    expect = T.copy(data)
    out = dst.numpy()
    assert np.array_equal(out, expect), f"first mismatch at {int(np.argmax(out != expect))}"
    assert dst.guards_intact(), "bytes outside the destination were written"
    st, site = mpt.mpt_ctx_status(ctx)
    assert st == mpt.MPT_OK, f"device status {st} site {site}"
    return info, dst


SIZES = [1, 15, 16, 17, 255, 4096, 65536 + 3, MiB + 5, 3 * 48 * 1024 + 7, 5 * MiB + 11]
OFFSETS = [(0, 0), (1, 1), (3, 3), (8, 8), (15, 15), (0, 1), (5, 9), (16, 0)]


@pytest.mark.parametrize("variant", [mpt.MPT_SM_VEC128, mpt.MPT_SM_BULK, mpt.MPT_SM_TILE8K])
def test_sm_copy_kernel_sizes_and_alignment(ctx, variant):
    import torch
    for n in SIZES:
        for so, do in OFFSETS:
            src, dst = Buf(n, "dev", so), Buf(n, "dev", do)
            data = seeded("u8", n * 31 + so, n)
            src.fill(data)
            mpt.mpt_sm_copy(ctx, dst.ptr, src.ptr, n, variant, 0, torch.cuda.current_stream())
            out = dst.numpy()
            assert np.array_equal(out, data), (variant, n, so, do, int(np.argmax(out != data)))
            assert dst.guards_intact(), (variant, n, so, do)
    assert mpt.mpt_ctx_status(ctx)[0] == mpt.MPT_OK


@pytest.mark.parametrize("ctas", [1, 3, 152, 1000])
def test_sm_copy_kernel_grid_sizes(ctx, ctas):
    import torch
    n = 7 * MiB + 333
    for variant in (mpt.MPT_SM_VEC128, mpt.MPT_SM_BULK, mpt.MPT_SM_TILE8K):
        src, dst = Buf(n, "dev"), Buf(n, "dev")
        data = seeded("f32", 9, n)
        src.fill(data)
        mpt.mpt_sm_copy(ctx, dst.ptr, src.ptr, n, variant, ctas, torch.cuda.current_stream())
        assert np.array_equal(dst.numpy(), data) and dst.guards_intact()


def test_copy64_graph_two_paths(ctx):
    # 64 MiB u8 payload, copy engine + SM kernel at 50/50, 4 MiB chunks, one graph.
    specs = [(P.CE, 32768, 4 * MiB), (P.SM, 32768, 4 * MiB)]
    info, dst = run_transfer(ctx, 64 * MiB, P.D2D, specs, "u8", payload.SEED_COPY64)
    assert info["memcpy_nodes"] == 8 and info["kernel_nodes"] == 1 and info["nodes"] == 9
    assert mpt.mpt_hash_device(ctx, dst.ptr, dst.n) == T.hash64(seeded("u8", payload.SEED_COPY64, 64 * MiB))


@pytest.mark.parametrize("mode", ["graph", "eager"])
@pytest.mark.parametrize("pathset", ["ce", "sm", "sm_bulk", "sm_8k", "ce+sm", "ce+sm_8k", "hs", "ce+sm+hs"])
def test_d2d_paths(ctx, mode, pathset):
    sets = {
        "ce": [(P.CE, 65536, MiB)],
        "sm": [(P.SM, 65536, MiB)],
        "sm_bulk": [(P.SM, 65536, MiB, 0, mpt.MPT_SM_BULK)],
        "sm_8k": [(P.SM, 65536, MiB, 0, mpt.MPT_SM_TILE8K)],
        "ce+sm": [(P.CE, 20000, MiB), (P.SM, 45536, 256 * 1024)],
        "ce+sm_8k": [(P.CE, 20000, MiB), (P.SM, 45536, 256 * 1024, 7, mpt.MPT_SM_TILE8K)],
        "hs": [(P.HS, 65536, MiB)],
        "ce+sm+hs": [(P.CE, 30000, MiB), (P.SM, 30000, MiB, 0, mpt.MPT_SM_BULK), (P.HS, 5536, 512 * 1024)],
    }
    for n in (8, 4096, 3 * MiB + 48, 9 * MiB + 5):
        run_transfer(ctx, n, P.D2D, sets[pathset], "f32", payload.SEED_D2D_SWEEP + n, mode=mode)


@pytest.mark.parametrize("mode", ["graph", "eager"])
@pytest.mark.parametrize("direction", [P.H2D, P.D2H])
@pytest.mark.parametrize("pathset", ["ce", "zc", "hs", "all"])
def test_host_paths(ctx, mode, direction, pathset):
    sets = {
        "ce": [(P.CE, 65536, MiB)],
        "zc": [(P.ZC, 65536, MiB)],
        "hs": [(P.HS, 65536, MiB)],
        "all": [(P.CE, 30000, MiB), (P.ZC, 20000, 2 * MiB), (P.HS, 15536, 512 * 1024)],
    }
    for n in (4096, 5 * MiB + 4, 11 * MiB + 7):
        run_transfer(ctx, n, direction, sets[pathset], "u32", payload.SEED_HOST_SWEEP + n, mode=mode)


@pytest.mark.parametrize("mode", ["graph", "eager"])
def test_interleave_layout(ctx, mode):
    specs = [(P.CE, 21845, 64 * 1024), (P.SM, 21845, 128 * 1024), (P.HS, 21846, 64 * 1024)]
    for n in (100, 1 << 20, 5 * MiB + 13):
        run_transfer(ctx, n, P.D2D, specs, "bf16", 77 + n, layout=P.INTERLEAVE, mode=mode)
    specs = [(P.CE, 30000, 64 * 1024), (P.ZC, 35536, 32 * 1024)]
    run_transfer(ctx, 3 * MiB + 9, P.H2D, specs, "u32", 5, layout=P.INTERLEAVE, mode=mode)


def test_unaligned_buffers_multipath(ctx):
    specs = [(P.CE, 32768, MiB), (P.SM, 32768, MiB, 0, mpt.MPT_SM_BULK)]
    for so, do in [(1, 1), (3, 7), (8, 0)]:
        run_transfer(ctx, 4 * MiB + 3, P.D2D, specs, "u8", so * 10 + do, src_off=so, dst_off=do)
    run_transfer(ctx, 2 * MiB + 3, P.H2D, [(P.CE, 32768, MiB), (P.ZC, 32768, MiB)], "u8", 3, src_off=5, dst_off=9)


def test_empty_and_tiny_messages(ctx):
    for n in (0, 1, 7):
        run_transfer(ctx, n, P.D2D, [(P.CE, 32768, 16), (P.SM, 32768, 16)], "u8", n)
    plan = mpt.mpt_plan(ctx, 0, P.D2D, [(P.SM, 65536, 16)])
    g = mpt.mpt_capture(ctx, plan, 0, 0)
    assert mpt.mpt_graph_get_info(g)["nodes"] == 0
    mpt.mpt_launch(g, None)
    mpt.mpt_graph_release(g)
    mpt.mpt_plan_destroy(plan)


def test_hash_matches_oracle(ctx):
    for n in (0, 1, 7, 8, 9, 4096, MiB + 3):
        for off in (0, 1, 8):
            b = Buf(n, "dev", off)
            data = seeded("u8", 1000 + n + off, n)
            b.fill(data)
            assert mpt.mpt_hash_device(ctx, b.ptr, n) == T.hash64(data), (n, off)


def test_graph_cache_hits_and_eviction(ctx):
    # a context of its own: the shared one caches graphs of earlier tests whose freed
    # addresses the allocator may hand out again
    import torch
    ctx = mpt.mpt_ctx_create(0)
    n = MiB
    src, dst = Buf(n, "dev"), Buf(n, "dev")
    plan = mpt.mpt_plan(ctx, n, P.D2D, [(P.CE, 32768, 256 * 1024), (P.SM, 32768, 256 * 1024)])
    g1 = mpt.mpt_capture(ctx, plan, dst.ptr, src.ptr)
    g2 = mpt.mpt_capture(ctx, plan, dst.ptr, src.ptr)
    assert g1 == g2
    g3 = mpt.mpt_capture(ctx, plan, dst.ptr + 16, src.ptr)  # different address: new graph
    assert g3 != g1
    assert mpt.mpt_graph_evict(ctx, dst.ptr + 100) == 2
    # held references survive eviction
    src.fill(seeded("u8", 4, n))
    mpt.mpt_launch(g1, torch.cuda.current_stream())
    assert np.array_equal(dst.numpy(), seeded("u8", 4, n))
    for g in (g1, g2, g3):
        mpt.mpt_graph_release(g)
    mpt.mpt_plan_destroy(plan)
    assert mpt.mpt_ctx_status(ctx)[0] == mpt.MPT_OK
    mpt.mpt_ctx_destroy(ctx)


def test_graph_cache_lru_capacity(monkeypatch):
    import torch
    monkeypatch.setenv("MPT_GRAPH_CACHE", "3")
    ctx = mpt.mpt_ctx_create(0)
    n = 64 * 1024
    src, dst = Buf(n, "dev"), Buf(8 * n, "dev")
    data = seeded("u8", 17, n)
    src.fill(data)
    plan = mpt.mpt_plan(ctx, n, P.D2D, [(P.SM, 65536, n)])
    graphs = [mpt.mpt_capture(ctx, plan, dst.ptr + i * n, src.ptr) for i in range(5)]
    assert len(set(graphs)) == 5
    # only the three most recent stay cached; capturing the first again builds a new graph
    assert mpt.mpt_capture(ctx, plan, dst.ptr + 4 * n, src.ptr) == graphs[4]
    again = mpt.mpt_capture(ctx, plan, dst.ptr, src.ptr)
    assert again != graphs[0]
    for g in graphs:  # evicted graphs still run while referenced
        mpt.mpt_launch(g, torch.cuda.current_stream())
    out = dst.numpy()
    for i in range(5):
        assert np.array_equal(out[i * n:(i + 1) * n], data)
    for g in graphs + [again, graphs[4]]:
        mpt.mpt_graph_release(g)
    mpt.mpt_plan_destroy(plan)
    mpt.mpt_ctx_destroy(ctx)


def test_pointer_kind_checked(ctx):
    n = 4096
    host, dev = Buf(n, "host"), Buf(n, "dev")
    plan = mpt.mpt_plan(ctx, n, P.D2D, [(P.SM, 65536, 4096)])
    with pytest.raises(mpt.MptError) as e:
        mpt.mpt_capture(ctx, plan, dev.ptr, host.ptr)
    assert e.value.status == mpt.MPT_EINVAL
    mpt.mpt_plan_destroy(plan)
    plan = mpt.mpt_plan(ctx, n, P.H2D, [(P.CE, 65536, 4096)])
    with pytest.raises(mpt.MptError):
        mpt.mpt_capture(ctx, plan, dev.ptr, dev.ptr)
    mpt.mpt_plan_destroy(plan)


def test_overlapping_source_and_destination_rejected(ctx):
    """The paths copy their chunks at the same time, so a message whose source and
    destination ranges share bytes has no defined result: every entry point refuses it with
    MPT_EINVAL and moves nothing.  Ranges that only touch are fine."""
    import torch
    n = 64 * 1024
    buf = Buf(3 * n, "dev")
    data = seeded("u8", 77, 3 * n)
    buf.fill(data)
    base = buf.ptr
    plan = mpt.mpt_plan(ctx, n, P.D2D, [(P.CE, 32768, 16384), (P.SM, 32768, 16384)])
    try:
        for dst, src in ((base + 16, base), (base, base + n - 16), (base, base)):
            for call in (lambda: mpt.mpt_capture(ctx, plan, dst, src),
                         lambda: mpt.mpt_prepare(ctx, plan, dst, src, mpt.MPT_PREPARE_EAGER),
                         lambda: mpt.mpt_launch_eager(ctx, plan, dst, src),
                         lambda: mpt.mpt_sm_copy(ctx, dst, src, n)):
                with pytest.raises(mpt.MptError) as e:
                    call()
                assert e.value.status == mpt.MPT_EINVAL and "overlap" in str(e.value)
        torch.cuda.synchronize()
        assert np.array_equal(buf.numpy(), data), "a refused copy moved bytes"
        # adjacent ranges [base, base+n) -> [base+n, base+2n) are a valid copy
        g = mpt.mpt_capture(ctx, plan, base + n, base)
        mpt.mpt_launch(g)
        mpt.mpt_graph_release(g)
        out = buf.numpy()
        assert np.array_equal(out[n:2 * n], T.copy(data[:n]))
        assert np.array_equal(out[:n], data[:n]) and np.array_equal(out[2 * n:], data[2 * n:])
    finally:
        mpt.mpt_plan_destroy(plan)


def test_batch_source_overlapping_a_destination_rejected(ctx):
    """A batch's transfers run at the same time: a source that overlaps any destination of
    the same batch (its own or another transfer's) is refused."""
    n = 4096
    buf = Buf(4 * n, "dev")
    data = seeded("u8", 78, 4 * n)
    buf.fill(data)
    b = buf.ptr
    for xf in ([(b, b + n // 2, n, P.D2D)],                                 # its own destination
               [(b, b + 2 * n, n, P.D2D), (b + 3 * n, b + n // 2, n, P.D2D)]):  # another's
        with pytest.raises(mpt.MptError) as e:
            mpt.mpt_batch_submit(ctx, xf)
        assert e.value.status == mpt.MPT_EINVAL and "overlaps a destination" in str(e.value)
    # sources may overlap one another
    h = mpt.mpt_batch_submit(ctx, [(b, b + 2 * n, n, P.D2D), (b, b + 3 * n, n, P.D2D)])
    mpt.mpt_batch_wait(h)
    mpt.mpt_batch_release(h)
    out = buf.numpy()
    assert np.array_equal(out[:2 * n], data[:2 * n]), "a refused batch moved bytes"
    assert np.array_equal(out[2 * n:3 * n], data[:n]) and np.array_equal(out[3 * n:], data[:n])


def test_staged_chunk_above_stage_size_rejected(ctx):
    n = 32 * MiB
    src, dst = Buf(n, "dev"), Buf(n, "dev")
    plan = mpt.mpt_plan(ctx, n, P.D2D, [(P.HS, 65536, 16 * MiB)])
    with pytest.raises(mpt.MptError) as e:
        mpt.mpt_capture(ctx, plan, dst.ptr, src.ptr)
    assert e.value.status == mpt.MPT_EINVAL
    mpt.mpt_plan_destroy(plan)


@pytest.mark.parametrize("specs,direction", [
    ([(P.CE, 32768, 256 * 1024), (P.SM, 32768, 256 * 1024)], P.D2D),
    ([(P.CE, 30000, 256 * 1024), (P.SM, 30000, 512 * 1024, 0, mpt.MPT_SM_BULK), (P.HS, 5536, 256 * 1024)], P.D2D),
    ([(P.CE, 20000, 256 * 1024), (P.ZC, 25536, 256 * 1024), (P.HS, 20000, 128 * 1024)], P.H2D),
    ([(P.CE, 20000, 256 * 1024), (P.ZC, 25536, 256 * 1024), (P.HS, 20000, 128 * 1024)], P.D2H),
])
def test_graph_rebind_in_place(specs, direction):
    """A captured graph retargeted at new addresses (cudaGraphExecUpdate, no new
    instantiation) moves the new message exactly, and the capture fast path reuses an
    idle cached graph of the same plan."""
    import torch
    ctx = mpt.mpt_ctx_create(0)
    n = 3 * MiB + 32
    sw, dw = ("host" if direction == P.H2D else "dev"), ("host" if direction == P.D2H else "dev")
    bufs = [(Buf(n, sw), Buf(n, dw)) for _ in range(3)]
    datas = [seeded("u32", 40 + i, n) for i in range(3)]
    for (s, _), d in zip(bufs, datas):
        s.fill(d)
    plan = mpt.mpt_plan(ctx, n, direction, specs)
    g = mpt.mpt_capture(ctx, plan, bufs[0][1].ptr, bufs[0][0].ptr)
    mpt.mpt_launch(g, torch.cuda.current_stream())
    assert np.array_equal(bufs[0][1].numpy(), datas[0])
    mpt.mpt_graph_rebind(g, plan, bufs[1][1].ptr, bufs[1][0].ptr)
    info = mpt.mpt_graph_get_info(g)
    assert info["rebinds"] == 1 and info["update_us"] > 0
    mpt.mpt_launch(g, torch.cuda.current_stream())
    assert np.array_equal(bufs[1][1].numpy(), datas[1]) and bufs[1][1].guards_intact()
    mpt.mpt_graph_release(g)  # now only the cache holds it
    g2 = mpt.mpt_capture(ctx, plan, bufs[2][1].ptr, bufs[2][0].ptr)  # fast path: retarget, no instantiate
    assert g2 == g and mpt.mpt_graph_get_info(g2)["rebinds"] == 2
    mpt.mpt_launch(g2, torch.cuda.current_stream())
    assert np.array_equal(bufs[2][1].numpy(), datas[2])
    other = mpt.mpt_plan(ctx, n, direction, [(specs[0][0], 65536, 64 * 1024)])
    with pytest.raises(mpt.MptError) as e:
        mpt.mpt_graph_rebind(g2, other, bufs[0][1].ptr, bufs[0][0].ptr)
    assert e.value.status == mpt.MPT_EINVAL
    mpt.mpt_graph_release(g2)
    mpt.mpt_plan_destroy(other)
    mpt.mpt_plan_destroy(plan)
    assert mpt.mpt_ctx_status(ctx)[0] == mpt.MPT_OK
    mpt.mpt_ctx_destroy(ctx)


def test_prepare_eager_and_auto_modes(monkeypatch):
    """mpt_prepare: direct issue (no graph, no fork/join for one path) and AUTO move the
    message exactly like a graph."""
    import torch
    monkeypatch.setenv("MPT_TUNE_DEFAULTS", "0")  # empty tuner table: AUTO falls back to a graph
    ctx = mpt.mpt_ctx_create(0)
    n = 2 * MiB + 48
    for specs in ([(P.SM, 65536, MiB)], [(P.CE, 65536, 512 * 1024)], [(P.CE, 32768, MiB), (P.SM, 32768, MiB)],
                  [(P.HS, 65536, MiB)]):
        plan = mpt.mpt_plan(ctx, n, P.D2D, specs)
        for mode in (mpt.MPT_PREPARE_EAGER, mpt.MPT_PREPARE_AUTO, mpt.MPT_PREPARE_GRAPH):
            src, dst = Buf(n, "dev", 3), Buf(n, "dev", 3)
            data = seeded("u8", 11 + mode, n)
            src.fill(data)
            h = mpt.mpt_prepare(ctx, plan, dst.ptr, src.ptr, mode)
            assert mpt.mpt_graph_get_info(h)["mode"] == (1 if mode == mpt.MPT_PREPARE_EAGER else 0)
            mpt.mpt_launch(h, torch.cuda.current_stream())
            mpt.mpt_launch(h, torch.cuda.current_stream())
            assert np.array_equal(dst.numpy(), data) and dst.guards_intact()
            mpt.mpt_graph_release(h)
        mpt.mpt_plan_destroy(plan)
    # AUTO follows the tuner: after tuning both modes the choice is the faster one
    mpt.mpt_tune(ctx, P.D2D, 4096, mpt.MPT_MODE_GRAPH)
    mpt.mpt_tune(ctx, P.D2D, 4096, mpt.MPT_MODE_EAGER)
    g_us = mpt.mpt_tune_get(ctx, P.D2D, 4096, mpt.MPT_MODE_GRAPH)[1]
    e_us = mpt.mpt_tune_get(ctx, P.D2D, 4096, mpt.MPT_MODE_EAGER)[1]
    plan = mpt.mpt_plan(ctx, 4096, P.D2D, [(P.SM, 65536, 4096)])
    src, dst = Buf(4096, "dev"), Buf(4096, "dev")
    h = mpt.mpt_prepare(ctx, plan, dst.ptr, src.ptr, mpt.MPT_PREPARE_AUTO)
    assert mpt.mpt_graph_get_info(h)["mode"] == (1 if e_us < g_us else 0)
    mpt.mpt_graph_release(h)
    mpt.mpt_plan_destroy(plan)
    assert mpt.mpt_ctx_status(ctx)[0] == mpt.MPT_OK
    mpt.mpt_ctx_destroy(ctx)


def test_device_info(ctx):
    info = mpt.mpt_ctx_info(ctx)
    import torch
    p = torch.cuda.get_device_properties(0)
    assert info["sms"] == p.multi_processor_count and info["name"] == p.name
    assert info["copy_engines"] >= 1 and info["l2_bytes"] > 0 and info["memory_bytes"] > 0


def test_pageable_host_memory_through_zero_copy(ctx):
    """On a device that reaches pageable host memory (a coherent Grace host), zero-copy-only
    plans, batches and mpt_sm_copy move ordinary (not page-locked) host buffers; plans with
    copy-engine or staged paths still require page-locked memory."""
    import torch
    if not mpt.mpt_ctx_info(ctx)["pageable_access"]:
        pytest.skip("device cannot reach pageable host memory")
    n = 5 * MiB + 7
    host_src = seeded("u32", 71, n).copy()          # numpy: pageable
    host_dst = np.zeros(n + 64, dtype=np.uint8)
    dev = Buf(n, "dev")
    zc = mpt.mpt_plan(ctx, n, P.H2D, [(P.ZC, 65536, MiB)])
    for mode in (mpt.MPT_PREPARE_GRAPH, mpt.MPT_PREPARE_EAGER):
        h = mpt.mpt_prepare(ctx, zc, dev.ptr, host_src.ctypes.data, mode)
        mpt.mpt_launch(h, torch.cuda.current_stream())
        assert np.array_equal(dev.numpy(), host_src)
        mpt.mpt_graph_release(h)
    back = mpt.mpt_plan(ctx, n, P.D2H, [(P.ZC, 65536, MiB)])
    g = mpt.mpt_capture(ctx, back, host_dst.ctypes.data + 3, dev.ptr)
    mpt.mpt_launch(g, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert np.array_equal(host_dst[3:3 + n], host_src) and not host_dst[:3].any() and not host_dst[3 + n:].any()
    mpt.mpt_graph_release(g)
    ce = mpt.mpt_plan(ctx, n, P.H2D, [(P.CE, 32768, MiB), (P.ZC, 32768, MiB)])
    with pytest.raises(mpt.MptError) as e:
        mpt.mpt_capture(ctx, ce, dev.ptr, host_src.ctypes.data)
    assert e.value.status == mpt.MPT_EINVAL
    # a batch reading pageable memory
    out = torch.zeros(2 * MiB, dtype=torch.uint8, device="cuda")
    b = mpt.mpt_batch_submit(ctx, [(host_src.ctypes.data + 16, out.data_ptr(), MiB, mpt.MPT_H2D),
                                   (host_src.ctypes.data + 5, out.data_ptr() + MiB, 1000, mpt.MPT_H2D)],
                             torch.cuda.current_stream())
    mpt.mpt_batch_wait(b)
    mpt.mpt_batch_release(b)
    o = out.cpu().numpy()
    assert np.array_equal(o[:MiB], host_src[16:16 + MiB]) and np.array_equal(o[MiB:MiB + 1000], host_src[5:1005])
    for p in (zc, back, ce):
        mpt.mpt_plan_destroy(p)


def test_lane_timers():
    """Lane timers report one duration per path of a traced multi-path eager launch, and a
    large share on a slow path (the staged route over the host link) shows up as the
    longest lane."""
    import torch
    ctx = mpt.mpt_ctx_create(0)
    n = 32 * MiB
    src, dst = Buf(n, "dev"), Buf(n, "dev")
    src.fill(seeded("u8", 5, n))
    plan = mpt.mpt_plan(ctx, n, P.D2D, [(P.CE, 21845, 4 * MiB), (P.SM, 21845, 4 * MiB), (P.HS, 21846, 4 * MiB)])
    mpt.mpt_launch_eager(ctx, plan, dst.ptr, src.ptr, torch.cuda.current_stream())
    assert mpt.mpt_lane_times(ctx) == []  # not traced yet
    mpt.mpt_trace_lanes(ctx, True)
    mpt.mpt_launch_eager(ctx, plan, dst.ptr, src.ptr, torch.cuda.current_stream())
    t = mpt.mpt_lane_times(ctx)
    assert len(t) == 3 and all(x > 0 for x in t)
    assert t[2] == max(t)  # ~11 MB through host memory twice, far slower than HBM paths
    assert np.array_equal(dst.numpy(), seeded("u8", 5, n))
    mpt.mpt_trace_lanes(ctx, False)
    mpt.mpt_plan_destroy(plan)
    mpt.mpt_ctx_destroy(ctx)
