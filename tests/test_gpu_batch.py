"""GPU parity of the batched path (persistent descriptor-table kernel) against the oracle,
plus its host-visible completion flags, slot ring, bounded waits and validation."""
import numpy as np
import pytest

import paper_2604_22228_gb300 as mpt
import payload
from oracle import transfer as T

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


class Workload:
    """Transfers of the batched workload's shape (log-uniform sizes, 70% device-to-device,
    30% host-to-device, 16-byte gaps) packed into a device source arena, a page-locked host
    source arena and a device destination arena."""

    def __init__(self, n, seed, max_bytes, kind="bf16", d2h=False, align=16):
        import torch
        sizes, d2d, gaps = payload.batch_workload(n, seed, 256, max_bytes)
        self.items, offs = payload.batch_layout(sizes, [x or d2h for x in d2d], gaps, align=align)
        self.src_np = {a: payload.fill(kind, seed + i + 1, max(16, offs[a] + 64)) for i, a in enumerate(("dev", "host"))}
        self.src = {"dev": torch.from_numpy(self.src_np["dev"]).cuda(),
                    "host": torch.from_numpy(self.src_np["host"]).pin_memory()}
        dst_bytes = offs["dst"] + 64
        self.d2h = d2h
        if d2h:
            self.dst = torch.full((dst_bytes,), 0x5A, dtype=torch.uint8).pin_memory()
        else:
            self.dst = torch.full((dst_bytes,), 0x5A, dtype=torch.uint8, device="cuda")
        self.dst_init = np.full(dst_bytes, 0x5A, dtype=np.uint8)
        direction = lambda a: (mpt.MPT_D2H if d2h else (mpt.MPT_D2D if a == "dev" else mpt.MPT_H2D))
        self.xfers = [(self.src[a].data_ptr() + s, self.dst.data_ptr() + d, sz, direction(a))
                      for a, s, d, sz in self.items]

    def expected(self):
        return T.batch_expected(self.dst_init, self.src_np, self.items)

    def result(self):
        import torch
        torch.cuda.synchronize()
        return self.dst.cpu().numpy() if not self.d2h else self.dst.numpy().copy()


@pytest.mark.parametrize("align", [16, 1])
@pytest.mark.parametrize("n,max_bytes", [(1, 4096), (37, 64 * 1024), (300, MiB), (1000, 4 * MiB)])
def test_batch_matches_oracle(ctx, n, max_bytes, align):
    """align 16: offsets on 16-byte multiples (the aligned kernel); align 1: transfers packed
    back to back, sources and destinations differing modulo 16 (the general kernel)."""
    import torch
    w = Workload(n, payload.SEED_BATCH + n, max_bytes, align=align)
    b = mpt.mpt_batch_submit(ctx, w.xfers, torch.cuda.current_stream())
    mpt.mpt_batch_wait(b)
    done, flags = mpt.mpt_batch_poll(b, n)
    times = mpt.mpt_batch_times(b, n)
    mpt.mpt_batch_release(b)
    assert done == n and all(flags)
    assert all(0 <= t < 10 ** 10 for t in times)
    assert np.array_equal(w.result(), w.expected())


def test_batch_slots_replay_and_reuse(ctx):
    import torch
    s = torch.cuda.current_stream()
    for rep in range(10):
        w = Workload(64, 900 + rep, 256 * 1024, kind="u32")
        b = mpt.mpt_batch_submit(ctx, w.xfers, s)
        mpt.mpt_batch_wait(b)
        mpt.mpt_batch_release(b)
        assert np.array_equal(w.result(), w.expected()), rep


def test_batch_device_to_host_flags_publish_data(ctx):
    """Once a transfer's host flag reads done, its destination bytes in page-locked host
    memory are already there -- no stream synchronisation needed."""
    import time
    import torch
    w = Workload(200, 77, MiB, kind="u8", d2h=True)
    b = mpt.mpt_batch_submit(ctx, w.xfers, torch.cuda.current_stream())
    exp = w.expected()
    host = w.dst.numpy()
    seen = set()
    t0 = time.time()
    while len(seen) < len(w.items) and time.time() - t0 < 30:
        _, flags = mpt.mpt_batch_poll(b, len(w.items))
        for i, f in enumerate(flags):
            if f and i not in seen:
                _, _, d, sz = w.items[i]
                assert np.array_equal(host[d:d + sz], exp[d:d + sz]), i
                seen.add(i)
    mpt.mpt_batch_wait(b)
    mpt.mpt_batch_release(b)
    assert len(seen) == len(w.items)


def test_batch_ring_full_then_free(ctx):
    import torch
    w = Workload(8, 5, 4096)
    held = [mpt.mpt_batch_submit(ctx, w.xfers[i:i + 1], torch.cuda.current_stream()) for i in range(4)]
    with pytest.raises(mpt.MptError) as e:
        mpt.mpt_batch_submit(ctx, w.xfers[4:5])
    assert e.value.status == mpt.MPT_EAGAIN
    mpt.mpt_batch_release(held.pop(0))
    held.append(mpt.mpt_batch_submit(ctx, w.xfers[4:5], torch.cuda.current_stream()))
    for b in held:
        mpt.mpt_batch_wait(b)
        mpt.mpt_batch_release(b)


def test_batch_bounded_host_wait(ctx):
    import torch
    src = torch.empty(512 * MiB, dtype=torch.uint8).pin_memory()
    dst = torch.empty(512 * MiB, dtype=torch.uint8, device="cuda")
    xfers = [(src.data_ptr() + i * 16 * MiB, dst.data_ptr() + i * 16 * MiB, 16 * MiB, mpt.MPT_H2D) for i in range(32)]
    b = mpt.mpt_batch_submit(ctx, xfers, torch.cuda.current_stream())
    with pytest.raises(mpt.MptError) as e:
        mpt.mpt_batch_wait(b, 1000)  # 1 us: the 512 MiB host-to-device batch is still running
    assert e.value.status == mpt.MPT_ETIMEDOUT
    mpt.mpt_batch_wait(b)  # and it completes when waited for again
    mpt.mpt_batch_release(b)
    torch.cuda.synchronize()
    assert torch.equal(src[:MiB].cuda(), dst[:MiB]) and torch.equal(src[-MiB:].cuda(), dst[-MiB:])


def test_batch_rejects_bad_descriptors(ctx):
    import torch
    a = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    h = torch.zeros(1 << 16, dtype=torch.uint8).pin_memory()
    p, q = a.data_ptr(), h.data_ptr()
    bad = [
        [(p, p + 4096, 100, mpt.MPT_D2D), (p + 8192, p + 4096 + 50, 100, mpt.MPT_D2D)],  # overlapping dst
        [(p, p + 4096, 100, mpt.MPT_H2D)],  # host-to-device from device memory
        [(q, p, 100, mpt.MPT_D2D)],         # device-to-device from host memory
        [(p, 0, 100, mpt.MPT_D2D)],         # NULL destination
        [(p, p + 4096, 100, 7)],            # unknown direction
    ]
    for xf in bad:
        with pytest.raises(mpt.MptError) as e:
            mpt.mpt_batch_submit(ctx, xf)
        assert e.value.status == mpt.MPT_EINVAL, xf
    with pytest.raises(mpt.MptError):
        mpt.mpt_batch_submit(ctx, [])


def test_device_wait_gives_up_and_reports(ctx):
    """Failure detection without a fault: a flag nothing raises makes the bounded device
    wait give up, record MPT_ETIMEDOUT, and leave the GPU usable."""
    import torch
    st, site = mpt.mpt_selftest_flag_timeout(ctx, 50_000_000)
    assert st == mpt.MPT_ETIMEDOUT and site == 2
    assert mpt.mpt_ctx_status(ctx)[0] == mpt.MPT_OK  # reset after being read
    x = torch.arange(4096, dtype=torch.int32, device="cuda")
    y = torch.zeros_like(x)
    mpt.mpt_sm_copy(ctx, y.data_ptr(), x.data_ptr(), x.numel() * 4)
    torch.cuda.synchronize()
    assert torch.equal(x, y)


def test_copy_each_and_batch_watch(ctx):
    """The per-transfer baseline (one copy per transfer, a stream per direction) and the
    batched path's host-observed completion times: both move the oracle's bytes; every time
    lies within the call; copies on one stream complete in issue order."""
    import torch
    w = Workload(300, 4242, MiB)
    streams = [torch.cuda.Stream() for _ in range(3)]
    t0 = mpt.mpt_now_ns()
    ts = mpt.mpt_copy_each(ctx, w.xfers, streams)
    wall = mpt.mpt_now_ns() - t0
    assert np.array_equal(w.result(), w.expected())
    assert len(ts) == 300 and all(0 <= t <= wall for t in ts)
    for d in (mpt.MPT_D2D, mpt.MPT_H2D):
        seq = [t for t, x in zip(ts, w.xfers) if x[3] == d]
        assert seq and seq == sorted(seq), d

    w2 = Workload(300, 4243, MiB)
    t0 = mpt.mpt_now_ns()
    b = mpt.mpt_batch_submit(ctx, w2.xfers, torch.cuda.current_stream())
    ts2 = mpt.mpt_batch_watch(b, t0, 300)
    wall = mpt.mpt_now_ns() - t0
    assert mpt.mpt_batch_poll(b)[0] == 300
    mpt.mpt_batch_release(b)
    assert len(ts2) == 300 and all(0 <= t <= wall for t in ts2)
    assert np.array_equal(w2.result(), w2.expected())

    with pytest.raises(mpt.MptError) as e:
        mpt.mpt_copy_each(ctx, [(w.xfers[0][0], w.xfers[0][1], 16, 9)], streams)
    assert e.value.status == mpt.MPT_EINVAL


@pytest.mark.slow
def test_batch_full_size_workload(ctx):
    """4096 transfers of 256 B..16 MiB (about 5.9 GiB), 70% device-to-device, 30% host-to-
    device: every transfer's destination equals the oracle's copy of its source bytes."""
    import torch
    period = 64 * MiB
    sizes, d2d, gaps = payload.batch_workload(4096)
    items, offs = payload.batch_layout(sizes, d2d, gaps)
    base = payload.fill("bf16", payload.SEED_BATCH, period)
    base_t = torch.from_numpy(base)

    def arena(nbytes, pinned):
        t = torch.empty(nbytes, dtype=torch.uint8).pin_memory() if pinned else \
            torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        src = base_t.to(t.device)
        for o in range(0, nbytes, period):
            m = min(period, nbytes - o)
            t[o:o + m].copy_(src[:m])
        return t

    src = {"dev": arena(offs["dev"] + 64, False), "host": arena(offs["host"] + 64, True)}
    dst = torch.zeros(offs["dst"] + 64, dtype=torch.uint8, device="cuda")
    mpt.mpt_batch_register(ctx, src["dev"].data_ptr(), src["dev"].numel())
    mpt.mpt_batch_register(ctx, src["host"].data_ptr(), src["host"].numel())
    mpt.mpt_batch_register(ctx, dst.data_ptr(), dst.numel())
    xfers = [(src[a].data_ptr() + s, dst.data_ptr() + d, sz, mpt.MPT_D2D if a == "dev" else mpt.MPT_H2D)
             for a, s, d, sz in items]
    b = mpt.mpt_batch_submit(ctx, xfers, torch.cuda.current_stream())
    mpt.mpt_batch_wait(b, 60 * 10 ** 9)
    assert mpt.mpt_batch_poll(b)[0] == 4096
    mpt.mpt_batch_release(b)
    out = dst.cpu().numpy()
    # both source arenas repeat `base`: arena byte s is base[s mod period]
    ext = np.concatenate([base, base[:16 * MiB]])
    assert max(sz for _, _, _, sz in items) <= 16 * MiB
    for i, (a, s, d, sz) in enumerate(items):
        p = s % period
        assert np.array_equal(out[d:d + sz], T.copy(ext[p:p + sz])), (i, a, s, d, sz)


# one transfer per batch around the tile boundaries: below the configured 256 KiB tile a
# batch is cut into power-of-two tiles of at least 32 KiB spread over the grid (456 CTAs
# aligned, 304 for the general kernel), above it into the configured tile
TILE_EDGE_SIZES = [1, 15, 16, 17, 32 * 1024 - 1, 32 * 1024, 32 * 1024 + 1, 456 * 32 * 1024 - 16,
                   456 * 32 * 1024 + 16, 304 * 64 * 1024 + 7, 456 * 256 * 1024 + 48, 8 * MiB + 3, 64 * MiB + 5]


@pytest.mark.parametrize("direction", [mpt.MPT_D2D, mpt.MPT_H2D, mpt.MPT_D2H], ids=["d2d", "h2d", "d2h"])
@pytest.mark.parametrize("offsets", [(0, 0), (3, 11)], ids=["aligned", "shifted"])
def test_batch_tile_sizes_follow_the_batch(ctx, direction, offsets):
    """A lone transfer of every size around the tile boundaries, its source and destination
    aligned or not, equals the oracle's copy with the guard bytes untouched."""
    from gpu_util import Buf, seeded
    where = {mpt.MPT_D2D: ("dev", "dev"), mpt.MPT_H2D: ("host", "dev"), mpt.MPT_D2H: ("dev", "host")}[direction]
    for k, n in enumerate(TILE_EDGE_SIZES):
        src, dst = Buf(n, where[0], offsets[0]), Buf(n, where[1], offsets[1])
        data = seeded("u8", 0xB0000 + 32 * k + direction, n)
        src.fill(data)
        b = mpt.mpt_batch_submit(ctx, [(src.ptr, dst.ptr, n, direction)])
        mpt.mpt_batch_wait(b)
        done, _ = mpt.mpt_batch_poll(b, 1)
        mpt.mpt_batch_release(b)
        assert done == 1, n
        assert np.array_equal(dst.numpy(), T.copy(data)), n
        assert dst.guards_intact(), n
    st, site = mpt.mpt_ctx_status(ctx)
    assert st == mpt.MPT_OK, (st, site)


def test_batch_counters_reset_across_replays(ctx):
    """The kernel leaves its cursors and tile counts at zero for the next replay of its slot
    (no reset node runs between replays): batches of one to three transfers and batches of
    hundreds alternate on the same slot, aligned and packed, and every one of them equals
    the oracle with every flag raised and a completion time from its own launch."""
    import torch
    s = torch.cuda.current_stream()
    for rep in range(12):
        small = rep % 2 == 0
        n = 1 + rep % 3 if small else 200 + 50 * (rep % 3)
        w = Workload(n, 0xC000 + rep, MiB if small else 2 * MiB, align=16 if rep % 4 < 2 else 1)
        b = mpt.mpt_batch_submit(ctx, w.xfers, s)
        mpt.mpt_batch_wait(b)
        done, flags = mpt.mpt_batch_poll(b, n)
        times = mpt.mpt_batch_times(b, n)
        mpt.mpt_batch_release(b)
        assert done == n and all(flags), rep
        # times count from this launch's start: a start left over from another launch would
        # put them far off (or clamp them all to 0)
        assert all(0 <= t < 10 ** 9 for t in times) and max(times) > 0, (rep, times[:4])
        assert np.array_equal(w.result(), w.expected()), rep
    st, site = mpt.mpt_ctx_status(ctx)
    assert st == mpt.MPT_OK, (st, site)


@pytest.mark.parametrize("split", [True, False], ids=["two_cursors", "one_cursor"])
@pytest.mark.parametrize("link_ctas", [1, 7, 32, 10 ** 6], ids=["1", "7", "32", "all"])
@pytest.mark.parametrize("align", [16, 1])
def test_batch_link_ctas_and_cursors(ctx, split, link_ctas, align):
    """However few CTAs may take host-link tiles (one, a handful, the default 32, every CTA),
    with two cursors or one, a mixed batch (device-to-device and host-to-device transfers,
    sizes from 256 B to 4 MiB) equals the oracle and raises every flag: CTAs outside the link
    group stop when the device tiles run out, and the link group finishes the rest."""
    import os
    import torch
    env = {"MPT_BATCH_LINK_CTAS": str(link_ctas), "MPT_BATCH_SPLIT": "1" if split else "0"}
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        mpt.mpt_batch_configure(ctx, 0, 0, 0, 0)  # rebuilt: the batch ring reads both here
        w = Workload(300, 0xD000 + link_ctas % 97 + 7 * split + align, 4 * MiB, align=align)
        b = mpt.mpt_batch_submit(ctx, w.xfers, torch.cuda.current_stream())
        mpt.mpt_batch_wait(b)
        done, flags = mpt.mpt_batch_poll(b, len(w.xfers))
        mpt.mpt_batch_release(b)
        assert done == len(w.xfers) and all(flags)
        assert np.array_equal(w.result(), w.expected())
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
        mpt.mpt_batch_configure(ctx, 0, 0, 0, 0)
    st, site = mpt.mpt_ctx_status(ctx)
    assert st == mpt.MPT_OK, (st, site)
