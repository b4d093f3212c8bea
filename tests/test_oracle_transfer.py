"""Pins for the oracle's copy and digest, and for the seeded payload generator (CPU only)."""
import numpy as np
import pytest

import payload
from oracle import transfer as T

# splitmix64 started at state 1234567: the first five outputs, as published with the
# reference C implementation of splitmix64 (Vigna) and widely reproduced.
SPLITMIX_1234567 = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                    4593380528125082431, 16408922859458223821]
GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def test_mix64_matches_published_splitmix64():
    states = np.array([(1234567 + (i + 1) * GAMMA) & M64 for i in range(5)], dtype=np.uint64)
    assert [int(v) for v in T.mix64(states)] == SPLITMIX_1234567


def test_payload_generator_matches_published_splitmix64():
    assert [payload.splitmix64_scalar(1234567, i) for i in range(5)] == SPLITMIX_1234567
    assert [int(v) for v in payload.splitmix64_words(1234567, 0, 5)] == SPLITMIX_1234567
    assert [int(v) for v in payload.splitmix64_words(1234567, 2, 3)] == SPLITMIX_1234567[2:]


def test_digest_closed_forms():
    assert T.hash64(b"") == 0                                   # mix64(0) = 0
    m1 = int(T.mix64(np.array([1], dtype=np.uint64))[0])
    assert T.hash64(b"\x01") == (2 * m1) & M64                  # mix64(1) + mix64(1 ^ 0)
    m8 = int(T.mix64(np.array([8], dtype=np.uint64))[0])
    assert T.hash64(bytes(8)) == m8                             # mix64(8) + mix64(0)
    m16 = int(T.mix64(np.array([16], dtype=np.uint64))[0])
    mg = int(T.mix64(np.array([GAMMA], dtype=np.uint64))[0])
    assert T.hash64(bytes(16)) == (m16 + mg) & M64               # word 1 is 0 ^ GAMMA


def test_digest_single_word_change():
    rng = np.random.default_rng(3)
    a = rng.integers(0, 256, 4096 + 5, dtype=np.uint8)
    b = a.copy()
    j = 300
    b[8 * j + 3] ^= 0x40
    wa = int(a[8 * j:8 * j + 8].view("<u8")[0])
    wb = int(b[8 * j:8 * j + 8].view("<u8")[0])
    ta = int(T.mix64(np.array([wa ^ ((j * GAMMA) & M64)], dtype=np.uint64))[0])
    tb = int(T.mix64(np.array([wb ^ ((j * GAMMA) & M64)], dtype=np.uint64))[0])
    assert (T.hash64(a) - T.hash64(b)) & M64 == (ta - tb) & M64


def test_digest_is_position_sensitive_and_pads_with_zeros():
    a = np.arange(64, dtype=np.uint8)
    b = a.copy()
    b[[0, 8]] = b[[8, 0]]
    assert T.hash64(a) != T.hash64(b)
    # 9 bytes: the tail word is the 9th byte zero-padded
    nine = np.arange(1, 10, dtype=np.uint8)
    w0 = int(nine[:8].view("<u8")[0])
    m = lambda v: int(T.mix64(np.array([v & M64], dtype=np.uint64))[0])
    assert T.hash64(nine) == (m(9) + m(w0) + m(9 ^ GAMMA)) & M64


def test_digest_block_boundaries():
    # the oracle digests in 4 Mi-word blocks; a buffer spanning two blocks equals the
    # sum of its two halves' word terms.
    n = (1 << 22) * 8 + 24
    buf = payload.fill("u8", 99, n)
    whole = T.hash64(buf)
    lo = buf[: (1 << 22) * 8]
    hi_terms = (T.hash64(buf) - T.hash64(lo)) & M64
    m = lambda v: int(T.mix64(np.array([v & M64], dtype=np.uint64))[0])
    words = buf[(1 << 22) * 8:].view("<u8")
    expect = sum(m(int(w) ^ ((((1 << 22) + i) * GAMMA) & M64)) for i, w in enumerate(words))
    assert hi_terms == (expect + m(n) - m((1 << 22) * 8)) & M64
    assert whole != T.hash64(buf[:-1])


def test_copy_is_identity():
    buf = payload.fill("u32", 5, 12345)
    out = T.copy(buf)
    assert out.tobytes() == buf.tobytes() and out is not buf


def test_batch_expected():
    dev = np.arange(100, dtype=np.uint8)
    host = np.arange(100, 200, dtype=np.uint8)
    dst = np.zeros(64, dtype=np.uint8)
    out = T.batch_expected(dst, {"dev": dev, "host": host}, [("dev", 10, 0, 16), ("host", 5, 32, 8)])
    assert list(out[:16]) == list(range(10, 26))
    assert list(out[32:40]) == list(range(105, 113))
    assert not out[16:32].any() and not out[40:].any()
    with pytest.raises(ValueError):
        T.batch_expected(dst, {"dev": dev}, [("dev", 0, 0, 16), ("dev", 0, 8, 16)])


def test_payload_encodings():
    n = 1000
    f = payload.fill("f32", 11, 4 * n).view("<f4")
    assert f.min() >= -1.0 and f.max() < 1.0
    x = payload.splitmix64_words(11, 0, n)
    assert np.array_equal(f.astype(np.float64), (x >> np.uint64(40)).astype(np.float64) * 2.0 ** -23 - 1.0)
    bf = payload.fill("bf16", 11, 2 * n).view("<u2")
    assert np.array_equal(bf, (f.view("<u4") >> 16).astype(np.uint16))
    u = payload.fill("u32", 11, 4 * n).view("<u4")
    assert np.array_equal(u, (x & np.uint64(0xFFFFFFFF)).astype(np.uint32))
    b = payload.fill("u8", 11, 8 * n).view("<u8")
    assert np.array_equal(b, x)


def test_payload_prefix_property():
    for kind in ("u8", "u32", "f32", "bf16"):
        full = payload.fill(kind, 21, 4099)
        for n in (0, 1, 3, 7, 64, 4098):
            assert np.array_equal(payload.fill(kind, 21, n), full[:n])


def test_batch_and_serving_workloads_shape():
    sizes, d2d, gaps = payload.batch_workload(4096)
    assert len(sizes) == 4096 and min(sizes) >= 256 and max(sizes) <= 16 << 20
    assert all(s % 2 == 0 for s in sizes) and all(g % 16 == 0 and 16 <= g <= 112 for g in gaps)
    frac = sum(d2d) / len(d2d)
    assert 0.66 < frac < 0.74
    sched = payload.serving_schedule(1000.0, 2.0)
    assert 1800 < len(sched) < 2200
    assert all(16 <= nb <= 256 << 20 and nb % 16 == 0 for _, nb, _ in sched)
    med = sorted(nb for _, nb, _ in sched)[len(sched) // 2]
    assert (1 << 20) * 0.8 < med < (1 << 20) * 1.25


def test_serving_schedule_request_cap():
    assert len(payload.serving_schedule(1e6, 1e9, max_requests=25)) == 25
    capped = payload.serving_schedule(1000.0, 0.5, max_requests=10 ** 9)
    assert 400 < len(capped) < 600 and capped[-1][0] < 0.5


def test_batch_layout_offsets():
    sizes, d2d, gaps = [10, 33, 16], [True, False, True], [16, 32, 48]
    items, offs = payload.batch_layout(sizes, d2d, gaps)
    # dev: 0+16=16 (10 B, ends 26) -> up16(26)=32 +48 = 80; host: 0+32 = 32; dst: 16, up16(26)+32=64, up16(97)+48=160
    assert items == [("dev", 16, 16, 10), ("host", 32, 64, 33), ("dev", 80, 160, 16)]
    assert all(s % 16 == 0 and d % 16 == 0 for _, s, d, _ in items)
    packed, _ = payload.batch_layout(sizes, d2d, gaps, align=1)
    assert packed == [("dev", 16, 16, 10), ("host", 32, 58, 33), ("dev", 74, 139, 16)]


def test_fill_window_matches_prefix_stream():
    for kind in ("u8", "u32", "f32", "bf16"):
        full = payload.fill(kind, 33, 5000)
        for off, n in [(0, 10), (1, 7), (3, 100), (4095, 905), (17, 0)]:
            assert np.array_equal(payload.fill_window(kind, 33, off, n), full[off:off + n]), (kind, off, n)


def test_workload_generators_follow_their_stated_distributions():
    """The synthetic inputs stand in for the paper's workloads, so their distributions are
    pinned: batch sizes log-uniform on [256 B, 16 MiB] (quartiles at 4 KiB, 64 KiB and
    1 MiB); serving arrivals Poisson (exponential gaps with mean 1/rate, coefficient of
    variation 1), sizes lognormal around 1 MiB with sigma 1.5, directions 50/25/25."""
    import math
    sizes, _, _ = payload.batch_workload(4096)
    s = sorted(sizes)
    for q, want in ((0.25, 4096), (0.5, 65536), (0.75, 1 << 20)):
        got = s[int(q * len(s))]
        assert abs(math.log(got / want)) < 0.35, (q, got)   # 1/8 of the log range is 1.39
    sched = payload.serving_schedule(10000.0, 2.0)
    n = len(sched)
    gaps = [b[0] - a[0] for a, b in zip(sched, sched[1:])]
    mean = sum(gaps) / len(gaps)
    sd = math.sqrt(sum((g - mean) ** 2 for g in gaps) / len(gaps))
    assert abs(mean * 10000.0 - 1.0) < 0.03 and abs(sd / mean - 1.0) < 0.05
    logs = [math.log(nb / (1 << 20)) for _, nb, _ in sched if 1 << 10 < nb < 200 << 20]
    mu = sum(logs) / len(logs)
    sigma = math.sqrt(sum((x - mu) ** 2 for x in logs) / len(logs))
    assert abs(mu) < 0.05 and abs(sigma - 1.5) < 0.06, (mu, sigma)
    mix = [sum(1 for _, _, d in sched if d == k) / n for k in (0, 1, 2)]
    assert abs(mix[0] - 0.5) < 0.02 and abs(mix[1] - 0.25) < 0.02 and abs(mix[2] - 0.25) < 0.02
