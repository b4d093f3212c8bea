"""mpt_host_alloc: page-locked, device-mapped host buffers and their device alias, used by the
zero-copy kernel and by copy-engine graphs, against the oracle; and mpt_host_free dropping the
context's cached graphs on the buffer, so that none is ever launched or retargeted on freed
memory.  A buffer allocated without a context is freed after mpt_graph_evict, as the header
asks of every buffer a cached graph refers to."""
import ctypes

import numpy as np
import pytest

import paper_2604_22228_gb300 as mpt
from oracle import transfer as T

from gpu_util import seeded

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
    assert st == mpt.MPT_OK, (st, site)


@pytest.mark.parametrize("with_ctx", [True, False])
def test_host_buffer_reaches_the_device_through_either_address(ctx, with_ctx):
    import torch
    n = 3 * MiB + 5
    host, alias = mpt.mpt_host_alloc(ctx if with_ctx else None, n)
    try:
        assert host and alias
        data = seeded("u8", 0xA11C, n)
        ctypes.memmove(host, data.ctypes.data, n)
        s = torch.cuda.current_stream()
        for src in (host, alias):
            dst = torch.zeros(n, dtype=torch.uint8, device="cuda")
            mpt.mpt_sm_copy(ctx, dst.data_ptr(), src, n, mpt.MPT_SM_VEC128, 0, s)  # zero-copy kernel
            torch.cuda.synchronize()
            assert np.array_equal(dst.cpu().numpy(), T.copy(data))
        dst = torch.zeros(n, dtype=torch.uint8, device="cuda")
        plan = mpt.mpt_plan(ctx, n, mpt.MPT_H2D, [(mpt.MPT_PATH_CE, 65536, MiB)])
        g = mpt.mpt_capture(ctx, plan, dst.data_ptr(), host)
        mpt.mpt_launch(g, s)
        torch.cuda.synchronize()
        mpt.mpt_graph_release(g)  # the cache still holds the graph, bound to `host`
        mpt.mpt_plan_destroy(plan)
        assert np.array_equal(dst.cpu().numpy(), T.copy(data))
        # and back: device -> the host buffer
        back = seeded("u8", 0xA11D, n)
        dev = torch.from_numpy(back).cuda()
        mpt.mpt_sm_copy(ctx, alias, dev.data_ptr(), n, mpt.MPT_SM_VEC128, 0, s)
        torch.cuda.synchronize()
        got = np.ctypeslib.as_array((ctypes.c_uint8 * n).from_address(host)).copy()
        assert np.array_equal(got, T.copy(back))
    finally:
        if with_ctx:
            mpt.mpt_host_free(ctx, host)  # drops the cached graph on the buffer, then frees it
        else:
            mpt.mpt_graph_evict(ctx, host)
            mpt.mpt_host_free(None, host)
    assert mpt.mpt_graph_evict(ctx, host) == 0  # nothing cached on the freed buffer


def test_freeing_drops_only_the_graphs_on_the_buffer(ctx):
    import torch
    n = 2 * MiB
    a, _ = mpt.mpt_host_alloc(ctx, n)
    b, _ = mpt.mpt_host_alloc(ctx, n)
    dev = torch.zeros(2 * n, dtype=torch.uint8, device="cuda")
    plan = mpt.mpt_plan(ctx, n, mpt.MPT_H2D, [(mpt.MPT_PATH_CE, 65536, MiB)])
    held = []
    try:
        # two graphs of the same plan, both held, so that neither is retargeted to the other
        for h, off in ((a, 0), (b, n)):
            held.append(mpt.mpt_capture(ctx, plan, dev.data_ptr() + off, h))
        mpt.mpt_host_free(ctx, a)
        assert mpt.mpt_graph_evict(ctx, a) == 0   # a's graph left the cache with the buffer
        assert mpt.mpt_graph_evict(ctx, b) == 1   # b's graph was still cached
        mpt.mpt_launch(held[1], torch.cuda.current_stream())  # b is still allocated
        torch.cuda.synchronize()
    finally:
        for g in held:
            mpt.mpt_graph_release(g)
        mpt.mpt_plan_destroy(plan)
        mpt.mpt_host_free(ctx, b)


def test_host_alloc_refuses_a_null_output():
    lib = mpt.lib()
    assert lib.mpt_host_alloc(None, 64, None, None) == mpt.MPT_EINVAL
