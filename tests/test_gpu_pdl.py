"""GPU: stream order under programmatic dependent launch.  Single-path eager transfers launch
their copy kernels with programmatic stream serialization, so a kernel may start while the
one before it on the stream is still running; these tests chain copies whose source is the
previous copy's destination (read after write) or whose destination is the previous copy's
source (write after read), on one stream, and compare every byte with the oracle's copy."""
import numpy as np
import pytest

import paper_2604_22228_gb300 as mpt
from oracle import planner as P
from oracle import transfer as T

from gpu_util import seeded

pytestmark = pytest.mark.gpu
MiB = 1 << 20


@pytest.fixture(scope="module", params=[1, 0], ids=["pdl", "nopdl"])
def ctx(request):
    import os
    import torch
    torch.cuda.init()
    from paper_2604_22228_gb300 import build
    build.build()
    old = os.environ.get("MPT_PDL")
    os.environ["MPT_PDL"] = str(request.param)
    try:
        c = mpt.mpt_ctx_create(0)
    finally:
        if old is None:
            os.environ.pop("MPT_PDL", None)
        else:
            os.environ["MPT_PDL"] = old
    yield c
    st, site = mpt.mpt_ctx_status(c)
    mpt.mpt_ctx_destroy(c)
    assert st == mpt.MPT_OK, f"device status {st} at site {site}"


def _plan(ctx, n, kind, ctas=0, flags=0):
    chunk = max(16, (n + 15) // 16 * 16)
    return mpt.mpt_plan(ctx, n, P.D2D, [(kind, 65536, chunk, ctas, flags)], 16, mpt.MPT_PLAN_EAGER)


@pytest.mark.parametrize("n", [1, 16, 1000, 65536 + 3, 3 * MiB + 7])
def test_read_after_write_chain(ctx, n):
    """b0 -> b1 -> ... -> b63 on one stream, each hop a direct launch; a hop that read its
    source before the previous hop finished would carry zeros forward."""
    import torch
    hops = 63
    data = seeded("u8", 11, n)
    bufs = [torch.zeros(n + 16, dtype=torch.uint8, device="cuda") for _ in range(hops + 1)]
    bufs[0][:n].copy_(torch.from_numpy(data))
    # kernel->kernel (64 KiB and 8 KiB tiles) and copy-engine edges
    kinds = [(mpt.MPT_PATH_SM, 0), (mpt.MPT_PATH_SM, mpt.MPT_SM_TILE8K), (mpt.MPT_PATH_CE, 0), (mpt.MPT_PATH_SM, 0)]
    plans = {k: _plan(ctx, n, k[0], 0, k[1]) for k in set(kinds)}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    try:
        for i in range(hops):
            mpt.mpt_launch_eager(ctx, plans[kinds[i % len(kinds)]], bufs[i + 1].data_ptr(), bufs[i].data_ptr(), s)
        s.synchronize()
    finally:
        for p in plans.values():
            mpt.mpt_plan_destroy(p)
    expect = T.copy(data)
    for i in (1, hops // 2, hops):
        out = bufs[i][:n].cpu().numpy()
        assert np.array_equal(out, expect), f"hop {i}: first mismatch at {int(np.argmax(out != expect))}"
        assert not bufs[i][n:].any(), f"hop {i} wrote past the message"


@pytest.mark.parametrize("variant", [mpt.MPT_SM_VEC128, mpt.MPT_SM_BULK, mpt.MPT_SM_TILE8K])
def test_write_after_read(ctx, variant):
    """copy x -> y, then z -> x: the second kernel must not overwrite x before the first has
    read all of it (64 MiB, several waves of CTAs)."""
    import torch
    n = 64 * MiB + 48
    p_data, q_data = seeded("u8", 21, n), seeded("u8", 22, n)
    x = torch.from_numpy(p_data).cuda()
    z = torch.from_numpy(q_data).cuda()
    y = torch.zeros(n, dtype=torch.uint8, device="cuda")
    plan = _plan(ctx, n, mpt.MPT_PATH_SM, 0, variant)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    try:
        for _ in range(3):
            mpt.mpt_launch_eager(ctx, plan, y.data_ptr(), x.data_ptr(), s)
            mpt.mpt_launch_eager(ctx, plan, x.data_ptr(), z.data_ptr(), s)
            mpt.mpt_launch_eager(ctx, plan, z.data_ptr(), y.data_ptr(), s)
        s.synchronize()
    finally:
        mpt.mpt_plan_destroy(plan)
    # each round: y <- x, x <- z, z <- y (the new y)
    xs, zs = p_data, q_data
    for _ in range(3):
        ys = xs
        xs, zs = zs, ys
    assert np.array_equal(y.cpu().numpy(), T.copy(ys))
    assert np.array_equal(x.cpu().numpy(), T.copy(xs))
    assert np.array_equal(z.cpu().numpy(), T.copy(zs))


def test_many_tiny_hops_with_foreign_kernels(ctx):
    """2000 8-byte hops ping-ponging between two buffers, a torch kernel adding 1 between
    every pair: the final value counts the hops that saw their predecessor's result."""
    import torch
    a = torch.zeros(2, dtype=torch.int32, device="cuda")
    b = torch.zeros(2, dtype=torch.int32, device="cuda")
    plan = _plan(ctx, 8, mpt.MPT_PATH_SM)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    rounds = 1000
    try:
        with torch.cuda.stream(s):
            for _ in range(rounds):
                mpt.mpt_launch_eager(ctx, plan, b.data_ptr(), a.data_ptr(), s)
                b.add_(1)
                mpt.mpt_launch_eager(ctx, plan, a.data_ptr(), b.data_ptr(), s)
        s.synchronize()
    finally:
        mpt.mpt_plan_destroy(plan)
    assert a.tolist() == [rounds, rounds] and b.tolist() == [rounds, rounds]
