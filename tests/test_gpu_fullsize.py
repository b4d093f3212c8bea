"""Parity at the benchmark's largest sizes, in the launch configuration bench.py times:
the 1 GiB device-to-device message through the tuned handle (graph or direct issue), and
2 GiB host-to-device and device-to-host through the tuned plans.  Every destination byte is
compared with the oracle's (the payload stream regenerated on the host, since a transfer's
result is its source) in 64 MiB pieces; the GPU digest is a second check.  Messages above
4 GiB are checked by digest against the oracle's digest of the same bytes, plus windows at
the 4 GiB boundary."""
import numpy as np
import pytest

import paper_2604_22228_gb300 as mpt
import payload
from oracle import transfer as T

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
MiB, GiB = 1 << 20, 1 << 30


def _handle(ctx, n, direction, dst, src):
    """The bench's choice: graph or direct issue, as the tuner measured faster."""
    mode = mpt.MPT_PREPARE_GRAPH
    try:
        g_us = mpt.mpt_tune_get(ctx, direction, n, mpt.MPT_MODE_GRAPH)[1]
        e_us = mpt.mpt_tune_get(ctx, direction, n, mpt.MPT_MODE_EAGER)[1]
        mode = mpt.MPT_PREPARE_EAGER if e_us < g_us else mpt.MPT_PREPARE_GRAPH
    except mpt.MptError:
        pass
    plan = mpt.mpt_plan(ctx, n, direction, None, 16,
                        mpt.MPT_PLAN_EAGER if mode == mpt.MPT_PREPARE_EAGER else mpt.MPT_LAYOUT_CONTIG)
    return plan, mpt.mpt_prepare(ctx, plan, dst, src, mode)


def _check_all(got_at, kind, seed, n, piece=64 * MiB):
    """Compare the whole destination with the oracle copy of the payload, piece by piece."""
    for off in range(0, n, piece):
        w = min(piece, n - off)
        want = T.copy(payload.fill_window(kind, seed, off, w))
        got = got_at(off, w)
        assert np.array_equal(got, want), f"first mismatch at {off + int(np.argmax(got != want))}"


def _check_windows(got_at, kind, seed, n, rng, count=24, width=4096):
    for off in [0, n - width] + list(rng.integers(0, n - width, count)):
        off = int(off)
        assert np.array_equal(got_at(off, width), payload.fill_window(kind, seed, off, width)), off


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = mpt.mpt_ctx_create(0)
    yield c
    assert mpt.mpt_ctx_status(c)[0] == mpt.MPT_OK
    mpt.mpt_ctx_destroy(c)


def test_d2d_1gib_tuned(ctx):
    import torch
    n = GiB
    host = torch.empty(n, dtype=torch.uint8).pin_memory()
    payload.fill("f32", payload.SEED_D2D_SWEEP, n, out=host.numpy())
    src = host.cuda()
    dst = torch.zeros(n + 4096, dtype=torch.uint8, device="cuda")
    plan, h = _handle(ctx, n, mpt.MPT_D2D, dst.data_ptr(), src.data_ptr())
    for _ in range(2):
        mpt.mpt_launch(h, torch.cuda.current_stream())
    torch.cuda.synchronize()
    _check_all(lambda o, w: dst[o:o + w].cpu().numpy(), "f32", payload.SEED_D2D_SWEEP, n)
    assert int(dst[n:].sum()) == 0  # nothing written past the message
    assert mpt.mpt_hash_device(ctx, dst.data_ptr(), n) == mpt.mpt_hash_device(ctx, src.data_ptr(), n)
    mpt.mpt_graph_release(h)
    mpt.mpt_plan_destroy(plan)


@pytest.mark.parametrize("direction", [mpt.MPT_H2D, mpt.MPT_D2H])
def test_host_2gib_tuned(ctx, direction):
    import torch
    n = 2 * GiB
    host = torch.empty(n, dtype=torch.uint8).pin_memory()
    dev = torch.empty(n, dtype=torch.uint8, device="cuda")
    if direction == mpt.MPT_H2D:
        payload.fill("u32", payload.SEED_HOST_SWEEP, n, out=host.numpy())
        src, dst = host, dev
    else:
        dev.copy_(torch.from_numpy(payload.fill("u32", payload.SEED_HOST_SWEEP, n)))
        host.zero_()
        src, dst = dev, host
    plan, h = _handle(ctx, n, direction, dst.data_ptr(), src.data_ptr())
    mpt.mpt_launch(h, torch.cuda.current_stream())
    torch.cuda.synchronize()
    view = (lambda o, w: dst[o:o + w].cpu().numpy()) if direction == mpt.MPT_H2D else \
        (lambda o, w: dst.numpy()[o:o + w])
    _check_all(view, "u32", payload.SEED_HOST_SWEEP, n)
    assert mpt.mpt_hash_device(ctx, dst.data_ptr(), n) == mpt.mpt_hash_device(ctx, src.data_ptr(), n)
    mpt.mpt_graph_release(h)
    mpt.mpt_plan_destroy(plan)


def test_digest_of_full_message_matches_oracle(ctx):
    """The GPU digest used above equals the oracle's digest on a 256 MiB payload."""
    import torch
    n = 256 * MiB
    data = payload.fill("f32", payload.SEED_D2D_SWEEP, n)
    t = torch.from_numpy(data).cuda()
    assert mpt.mpt_hash_device(ctx, t.data_ptr(), n) == T.hash64(data)


BEYOND_N = 4 * GiB + 4096 + 13
BEYOND_SEED = payload.SEED_D2D_SWEEP + 5
BEYOND_PERIOD = GiB - 28672


@pytest.fixture(scope="module")
def beyond_oracle():
    """The tiled message above 4 GiB built on the host, and the oracle's digest of it."""
    base_np = payload.fill("u32", BEYOND_SEED, BEYOND_PERIOD)
    host = np.empty(BEYOND_N, dtype=np.uint8)
    for o in range(0, BEYOND_N, BEYOND_PERIOD):
        m = min(BEYOND_PERIOD, BEYOND_N - o)
        host[o:o + m] = base_np[:m]
    digest = T.hash64(host)
    del host
    return base_np, digest


def _tiled_source(n, base_np, period):
    """n bytes on the device: the seeded u32 payload repeated with a period that does not
    divide 2^32, so a 64-bit offset truncated to 32 bits reads different bytes."""
    import torch
    base = torch.from_numpy(base_np).cuda()
    src = torch.empty(n, dtype=torch.uint8, device="cuda")
    for o in range(0, n, period):
        m = min(period, n - o)
        src[o:o + m].copy_(base[:m])
    return src


@pytest.mark.parametrize("case", ["sm_eager", "sm_graph", "sm8k_graph", "bulk_graph", "ce_sm_graph", "batch"])
def test_d2d_beyond_4gib(ctx, case, beyond_oracle):
    """A message above 4 GiB: 64-bit offsets in every path (kernel tile offsets, copy-engine
    chunk offsets, batch descriptors).  Whole-buffer digest against the oracle's digest of
    the same bytes, untouched tail, and windows at the 4 GiB boundary against the oracle's
    bytes."""
    import torch
    n, period = BEYOND_N, BEYOND_PERIOD
    base_np, want_digest = beyond_oracle
    src = _tiled_source(n, base_np, period)
    dst = torch.zeros(n + 4096, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    if case == "batch":
        xf = [(src.data_ptr(), dst.data_ptr(), n, mpt.MPT_D2D)]
        b = mpt.mpt_batch_submit(ctx, xf, s)
        mpt.mpt_batch_wait(b)
        done, _ = mpt.mpt_batch_poll(b, 1)
        mpt.mpt_batch_release(b)
        assert done == 1
    else:
        specs = {
            "sm_eager": [(mpt.MPT_PATH_SM, 65536, n // 16 * 16 + 16)],
            "sm_graph": [(mpt.MPT_PATH_SM, 65536, GiB)],
            "sm8k_graph": [(mpt.MPT_PATH_SM, 65536, GiB, 0, mpt.MPT_SM_TILE8K)],
            "bulk_graph": [(mpt.MPT_PATH_SM, 65536, GiB, 0, mpt.MPT_SM_BULK)],
            "ce_sm_graph": [(mpt.MPT_PATH_CE, 32768, GiB), (mpt.MPT_PATH_SM, 32768, 512 * MiB)],
        }[case]
        plan = mpt.mpt_plan(ctx, n, mpt.MPT_D2D, specs)
        mode = mpt.MPT_PREPARE_EAGER if case.endswith("eager") else mpt.MPT_PREPARE_GRAPH
        h = mpt.mpt_prepare(ctx, plan, dst.data_ptr(), src.data_ptr(), mode)
        mpt.mpt_launch(h, s)
        mpt.mpt_graph_release(h)
        mpt.mpt_plan_destroy(plan)
    torch.cuda.synchronize()
    assert mpt.mpt_hash_device(ctx, dst.data_ptr(), n) == want_digest
    assert int(dst[n:].sum()) == 0
    for off in (0, (1 << 32) - 2048, 1 << 32, n - 4096):
        p = off % period
        want = base_np[p:p + 4096] if p + 4096 <= period else np.concatenate([base_np[p:], base_np[:p + 4096 - period]])
        assert np.array_equal(dst[off:off + 4096].cpu().numpy(), T.copy(want)), off
