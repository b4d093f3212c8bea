"""The allocation-free digest entry point against the regular one and the oracle.

mpt_hash_ranges_noalloc is for callers that cannot allocate device memory when they need a
digest; its scratch accumulators live in a static device array shared by every call.  It
must give exactly what mpt_hash_device gives, call after call (the array keeps the previous
call's contents, so stale sums would show up on the second call), and both must equal the
oracle's digest of the same host bytes (ranges starting off an 8-byte boundary included).
This file is collected last so that a run stopping at the first failure has run every other
test first.
"""
import pytest

import paper_2604_22228_gb300 as mpt
import payload
from oracle import transfer as T
from paper_2604_22228_gb300 import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    build.build()
    c = mpt.mpt_ctx_create(0)
    yield c
    mpt.mpt_ctx_destroy(c)


def _ranges(seed, sizes):
    """Device copies of seeded payloads; range i starts i mod 8 bytes into its buffer.
    Returns (tensor, device pointer, size, the range's host bytes)."""
    import torch
    bufs = []
    for i, n in enumerate(sizes):
        host = payload.fill("u8", seed + i, n + 8)
        t = torch.from_numpy(host).cuda()
        off = i % 8  # some ranges start off an 8-byte boundary
        bufs.append((t, t.data_ptr() + off, n, host[off:off + n]))
    return bufs


def test_noalloc_digest_matches_context_digest_twice(ctx):
    import torch
    sizes = [0, 1, 7, 8, 4096, 65536 + 5, (3 << 20) + 11, 9, 15, 17]
    for call, seed in enumerate((101, 202)):  # two calls in a row, different data
        bufs = _ranges(seed, sizes)
        got = mpt.mpt_hash_ranges_noalloc([(p, n) for _, p, n, _ in bufs], torch.cuda.current_stream())
        assert got == [mpt.mpt_hash_device(ctx, p, n) for _, p, n, _ in bufs], f"call {call}"
        assert got == [T.hash64(h) for _, _, _, h in bufs], f"call {call} against the oracle"


def test_noalloc_digest_limits(ctx):
    import torch
    assert mpt.mpt_hash_ranges_noalloc([]) == []
    t = torch.zeros(64, dtype=torch.uint8, device="cuda")
    full = [(t.data_ptr(), 64)] * mpt.MPT_NOALLOC_MAX_RANGES
    got = mpt.mpt_hash_ranges_noalloc(full)
    assert len(got) == mpt.MPT_NOALLOC_MAX_RANGES and len(set(got)) == 1
    assert got[0] == mpt.mpt_hash_device(ctx, t.data_ptr(), 64)
    with pytest.raises(mpt.MptError) as e:
        mpt.mpt_hash_ranges_noalloc(full + [(t.data_ptr(), 64)])
    assert e.value.status == mpt.MPT_EINVAL and "maximum" in str(e.value)
