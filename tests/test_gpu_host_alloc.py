"""mpt_host_alloc: page-locked, device-mapped host buffers and their device alias, used by the
zero-copy kernel and by copy-engine graphs, against the oracle."""
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
        mpt.mpt_graph_release(g)
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
        mpt.mpt_host_free(host)


def test_host_alloc_refuses_a_null_output():
    lib = mpt.lib()
    assert lib.mpt_host_alloc(None, 64, None, None) == mpt.MPT_EINVAL
