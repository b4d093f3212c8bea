"""Every ring configuration of the bulk-copy SM kernel (cp.async.bulk through shared memory)
against the oracle: sizes from one byte to several waves of tiles with ragged tails, source and
destination offsets (equal modulo 16, the bulk body; different, the vec128 fallback), grid
sizes below and above the resident CTAs, and plans whose SM path is cut into many ranges."""
import numpy as np
import pytest

import paper_2604_22228_gb300 as mpt
from oracle import planner as P
from oracle import transfer as T

from gpu_util import Buf, seeded

pytestmark = pytest.mark.gpu
MiB = 1 << 20


@pytest.fixture(params=range(mpt.MPT_BULK_CONFIGS))
def bulk_ctx(request, monkeypatch):
    import torch
    torch.cuda.init()
    from paper_2604_22228_gb300 import build
    build.build()
    monkeypatch.setenv("MPT_BULK_CONFIG", str(request.param))
    c = mpt.mpt_ctx_create(0)
    yield c
    st, site = mpt.mpt_ctx_status(c)
    mpt.mpt_ctx_destroy(c)
    assert st == mpt.MPT_OK, f"device status {st} at site {site}"


def test_bulk_sizes_offsets_and_grids(bulk_ctx):
    import torch
    s = torch.cuda.current_stream()
    cases = [(n, so, do, 0) for n in (1, 17, 4096, 65536 + 3, 3 * 48 * 1024 + 7, 5 * MiB + 11, 37 * MiB + 5)
             for so, do in ((0, 0), (3, 3), (15, 15), (16, 0))]
    cases += [(9 * MiB + 1, 5, 9, 0)]  # differ modulo 16: the vec128 fallback
    cases += [(7 * MiB + 333, 0, 0, g) for g in (1, 3, 152, 1000)]
    for n, so, do, ctas in cases:
        src, dst = Buf(n, "dev", so), Buf(n, "dev", do)
        data = seeded("u8", n * 7 + so + 13 * ctas, n)
        src.fill(data)
        mpt.mpt_sm_copy(bulk_ctx, dst.ptr, src.ptr, n, mpt.MPT_SM_BULK, ctas, s)
        out = dst.numpy()
        want = T.copy(data)
        assert np.array_equal(out, want), (n, so, do, ctas, int(np.argmax(out != want)))
        assert dst.guards_intact(), (n, so, do, ctas)


@pytest.mark.parametrize("mode", ["graph", "eager"])
def test_bulk_in_multi_range_plans(bulk_ctx, mode):
    """Round-robin plans give the SM path one range per chunk (16 ranges per launch)."""
    import torch
    n = 41 * MiB + 4096 + 3
    specs = [(P.CE, 16384, MiB), (P.SM, 49152, 512 * 1024, 0, mpt.MPT_SM_BULK)]
    src, dst = Buf(n, "dev", 4), Buf(n, "dev", 4)
    data = seeded("f32", 0xB01C, n)
    src.fill(data)
    plan = mpt.mpt_plan(bulk_ctx, n, P.D2D, specs, 16, P.INTERLEAVE)
    try:
        if mode == "graph":
            g = mpt.mpt_capture(bulk_ctx, plan, dst.ptr, src.ptr)
            mpt.mpt_launch(g, torch.cuda.current_stream())
            mpt.mpt_graph_release(g)
        else:
            mpt.mpt_launch_eager(bulk_ctx, plan, dst.ptr, src.ptr, torch.cuda.current_stream())
        torch.cuda.synchronize()
    finally:
        mpt.mpt_plan_destroy(plan)
    out = dst.numpy()
    want = T.copy(data)
    assert np.array_equal(out, want), int(np.argmax(out != want))
    assert dst.guards_intact()


def test_bulk_config_out_of_range_is_refused(monkeypatch):
    import torch
    torch.cuda.init()
    monkeypatch.setenv("MPT_BULK_CONFIG", str(mpt.MPT_BULK_CONFIGS))
    with pytest.raises(mpt.MptError) as e:
        mpt.mpt_ctx_create(0)
    assert e.value.status == mpt.MPT_EINVAL
