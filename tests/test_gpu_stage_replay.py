"""A staged host-to-device graph stays correct after a replay whose device-side waits ran out.

The staged route's second hop waits on a per-chunk ready flag raised after the chunk's first
hop (Algorithm 2 StageHostCopy, Sec. 4.5 dependency handling).  When such a wait gives up,
its CTA stops, so flags raised later in that replay stay raised.  The next replay of the same
graph must not take them for its own: with fresh source bytes it has to deliver exactly those
bytes.  The waits are made to run out without any fault: the context's wait limit is set to
1 ns, so a wait gives up unless its chunk's copy has already landed.
"""
import numpy as np
import pytest

import paper_2604_22228_gb300 as mpt
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
    mpt.mpt_ctx_set_wait_limit(c, 0)
    st, site = mpt.mpt_ctx_status(c)
    mpt.mpt_ctx_destroy(c)
    assert st == mpt.MPT_OK, f"device status {st} at site {site}"


@pytest.mark.parametrize("specs", [
    [(mpt.MPT_PATH_HS, 65536, 8 * MiB)],
    [(mpt.MPT_PATH_CE, 16384, 4 * MiB), (mpt.MPT_PATH_HS, 32768, 4 * MiB), (mpt.MPT_PATH_ZC, 16384, 4 * MiB)],
], ids=["hs", "ce+hs+zc"])
def test_replay_after_timed_out_waits_moves_fresh_bytes(ctx, specs):
    import torch
    n = 48 * MiB + 4096 + 7  # several chunks and a ragged last one
    src, dst = Buf(n, "host"), Buf(n, "dev")
    first, second = seeded("u32", 0x51, n), seeded("u32", 0x52, n)
    plan = mpt.mpt_plan(ctx, n, mpt.MPT_H2D, specs)
    g = mpt.mpt_capture(ctx, plan, dst.ptr, src.ptr)
    s = torch.cuda.current_stream()
    try:
        src.fill(first)
        mpt.mpt_ctx_set_wait_limit(ctx, 1)
        timed_out = 0
        for _ in range(3):
            mpt.mpt_launch(g, s)
            torch.cuda.synchronize()
            st, site = mpt.mpt_ctx_status(ctx)
            if st == mpt.MPT_ETIMEDOUT:
                timed_out += 1
            else:  # every chunk happened to be ready when its wait began: then it is complete
                assert st == mpt.MPT_OK
                assert np.array_equal(dst.numpy(), first)
        assert timed_out >= 1, "a 1 ns wait limit never ran out"

        # fresh source bytes and the default limit: a consumer that trusted a flag left raised
        # by the replays above would copy the stage before this replay refilled it
        mpt.mpt_ctx_set_wait_limit(ctx, 0)
        src.fill(second)
        want = T.copy(second)
        for _ in range(2):
            mpt.mpt_launch(g, s)
            torch.cuda.synchronize()
            st, site = mpt.mpt_ctx_status(ctx)
            assert st == mpt.MPT_OK, f"status {st} site {site}"
            out = dst.numpy()
            assert np.array_equal(out, want), f"first mismatch at {int(np.argmax(out != want))}"
            assert dst.guards_intact()
    finally:
        mpt.mpt_ctx_set_wait_limit(ctx, 0)
        mpt.mpt_graph_release(g)
        mpt.mpt_plan_destroy(plan)


def test_wait_limit_bounds(ctx):
    with pytest.raises(mpt.MptError) as e:
        mpt.mpt_ctx_set_wait_limit(ctx, 10 * 10 ** 9 + 1)
    assert e.value.status == mpt.MPT_EINVAL
    mpt.mpt_ctx_set_wait_limit(ctx, 10 * 10 ** 9)
    mpt.mpt_ctx_set_wait_limit(ctx, 0)
