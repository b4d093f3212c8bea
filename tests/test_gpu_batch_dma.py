"""GPU parity of the batch's DMA lanes (the persistent kernel plus copy-engine lanes that take
the large entries): bytes against the oracle, every entry's completion flag and time, lanes
switched on and off between batches, pageable entries kept with the kernel."""
import numpy as np
import pytest

import paper_2604_22228_gb300 as mpt
import payload

from test_gpu_batch import Workload

pytestmark = pytest.mark.gpu
MiB = 1 << 20


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    from paper_2604_22228_gb300 import build
    build.build()
    c = mpt.mpt_ctx_create(0)
    mpt.mpt_batch_configure_dma(c, 2, 4, 256 * 1024)
    yield c
    st, site = mpt.mpt_ctx_status(c)
    mpt.mpt_ctx_destroy(c)
    assert st == mpt.MPT_OK, (st, site)


def _run(ctx, w, n):
    import torch
    b = mpt.mpt_batch_submit(ctx, w.xfers, torch.cuda.current_stream())
    mpt.mpt_batch_wait(b)
    done, flags = mpt.mpt_batch_poll(b, n)
    times = mpt.mpt_batch_times(b, n)
    mpt.mpt_batch_release(b)
    assert done == n and all(flags)
    assert all(0 <= t < 10 ** 10 for t in times)
    assert np.array_equal(w.result(), w.expected())


@pytest.mark.parametrize("align", [16, 1])
@pytest.mark.parametrize("n,max_bytes", [(8, 2 * MiB), (300, MiB), (1000, 4 * MiB)])
def test_dma_lanes_match_oracle(ctx, n, max_bytes, align):
    _run(ctx, Workload(n, payload.SEED_BATCH + 7 * n, max_bytes, align=align), n)


def test_dma_lanes_device_to_host(ctx):
    _run(ctx, Workload(200, 78, 2 * MiB, kind="u8", d2h=True), 200)


def test_dma_lanes_switch_between_batches(ctx):
    """Batches with and without lane-sized entries alternate on the same slots: lane nodes
    are retargeted, switched off and on again."""
    for rep in range(8):
        big = rep % 3 != 1
        n = 40 if big else 100
        w = Workload(n, 1200 + rep, 3 * MiB if big else 64 * 1024, kind="u32", align=16 if rep % 2 else 1)
        _run(ctx, w, n)


def test_pageable_entries_stay_with_the_kernel(ctx):
    import torch
    if not mpt.mpt_ctx_info(ctx)["pageable_access"]:
        pytest.skip("device cannot reach pageable host memory")
    n = 3 * MiB
    src = payload.fill("u32", 91, 2 * n).copy()                # pageable numpy buffer
    pinned = torch.from_numpy(payload.fill("u32", 92, n)).pin_memory()
    out = torch.zeros(4 * n, dtype=torch.uint8, device="cuda")
    xf = [(src.ctypes.data, out.data_ptr(), n, mpt.MPT_H2D),                   # pageable: kernel
          (pinned.data_ptr(), out.data_ptr() + n, n, mpt.MPT_H2D),             # pinned: a lane
          (src.ctypes.data + n + 16, out.data_ptr() + 2 * n, n - 32, mpt.MPT_H2D)]
    b = mpt.mpt_batch_submit(ctx, xf, torch.cuda.current_stream())
    mpt.mpt_batch_wait(b)
    done, _ = mpt.mpt_batch_poll(b, 3)
    mpt.mpt_batch_release(b)
    o = out.cpu().numpy()
    assert done == 3
    assert np.array_equal(o[:n], src[:n]) and np.array_equal(o[n:2 * n], pinned.numpy())
    assert np.array_equal(o[2 * n:3 * n - 32], src[n + 16:2 * n - 16]) and not o[3 * n - 32:].any()


def test_configure_dma_rejects_bad_values():
    c = mpt.mpt_ctx_create(0)
    try:
        for args in ((9, 4, MiB), (1, 0, MiB), (1, 65, MiB), (1, 4, 8)):
            with pytest.raises(mpt.MptError) as e:
                mpt.mpt_batch_configure_dma(c, *args)
            assert e.value.status == mpt.MPT_EINVAL
        mpt.mpt_batch_configure_dma(c, 0, 0, 0)  # lanes off
    finally:
        mpt.mpt_ctx_destroy(c)


@pytest.mark.parametrize("objective", [mpt.MPT_BATCH_TUNE_TIME, mpt.MPT_BATCH_TUNE_P99])
def test_batch_tune_applies_a_measured_setting(objective):
    """mpt_batch_tune measures every candidate setting on the given batch, applies the best,
    and later batches under it stay bit-exact."""
    import torch
    c = mpt.mpt_ctx_create(0)
    try:
        w = Workload(300, 4242, 4 * MiB, kind="u32")
        r = mpt.mpt_batch_tune(c, w.xfers, objective, 1, torch.cuda.current_stream())
        sms = mpt.mpt_ctx_info(c)["sms"]
        assert r["candidates"] == 30 and r["ctas"] in (sms, 2 * sms, 3 * sms)
        assert r["tile_bytes"] in [k << 10 for k in (64, 128, 256, 512, 1024)]
        assert r["dma_lanes"] in (0, 2) and r["batch_us"] > 0 and r["p99_us"] > 0
        w2 = Workload(300, 4243, 4 * MiB, kind="u32")
        _run(c, w2, 300)
    finally:
        mpt.mpt_ctx_destroy(c)
