"""Serving loop: continuous batching.  Each request's result is the same alone and in the
mix (bit-exact digests, and equal to its source per the oracle's definition of a transfer),
admission respects the staging budget, and refused requests do not stop the server."""
import math
import time

import numpy as np
import pytest

import paper_2604_22228_gb300 as mpt
import payload

pytestmark = pytest.mark.gpu
KiB, MiB = 1 << 10, 1 << 20


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    from paper_2604_22228_gb300 import build
    build.build()
    c = mpt.mpt_ctx_create(0)
    yield c
    mpt.mpt_ctx_destroy(c)


class Arenas:
    """Requests of the serving workload's shape (lognormal sizes, 50/25/25 directions) with
    their own source windows and destination regions."""

    def __init__(self, n, seed, median=64 * KiB, cap=4 * MiB):
        import torch
        sched = payload.serving_schedule(1e6, 1e9, seed=seed, median_bytes=median, cap_bytes=cap, max_requests=n)
        self.reqs = []
        offs = {"dsrc": 0, "hsrc": 0, "ddst": 0, "hdst": 0}
        for k, (_, nb, d) in enumerate(sched):
            s_ar = "hsrc" if d == mpt.MPT_H2D else "dsrc"
            d_ar = "hdst" if d == mpt.MPT_D2H else "ddst"
            self.reqs.append((k, s_ar, offs[s_ar], d_ar, offs[d_ar], nb, d))
            offs[s_ar] += nb + 16
            offs[d_ar] += nb + 16
        self.src_np = {a: payload.fill("u32", seed + i, offs[a] + 64) for i, a in enumerate(("dsrc", "hsrc"))}
        self.t = {"dsrc": torch.from_numpy(self.src_np["dsrc"]).cuda(),
                  "hsrc": torch.from_numpy(self.src_np["hsrc"]).pin_memory(),
                  "ddst": torch.zeros(offs["ddst"] + 64, dtype=torch.uint8, device="cuda"),
                  "hdst": torch.zeros(offs["hdst"] + 64, dtype=torch.uint8).pin_memory()}

    def ptr(self, arena, off):
        return self.t[arena].data_ptr() + off

    def clear_dst(self):
        import torch
        self.t["ddst"].zero_()
        self.t["hdst"].zero_()
        torch.cuda.synchronize()

    def digests(self, which):
        out = []
        for i in range(0, len(self.reqs), mpt.MPT_NOALLOC_MAX_RANGES):
            chunk = self.reqs[i:i + mpt.MPT_NOALLOC_MAX_RANGES]
            if which == "dst":
                rng = [(self.ptr(d_ar, d_off), nb) for _, _, _, d_ar, d_off, nb, _ in chunk]
            else:
                rng = [(self.ptr(s_ar, s_off), nb) for _, s_ar, s_off, _, _, nb, _ in chunk]
            out += mpt.mpt_hash_ranges_noalloc(rng)
        return out


def run(server, ar, order, one_at_a_time, timeout=60):
    done = {}
    t0 = time.time()
    pending = list(order)
    while (pending or len(done) < len(order)) and time.time() - t0 < timeout:
        if pending and (not one_at_a_time or len(done) == len(order) - len(pending)):
            k, s_ar, s_off, d_ar, d_off, nb, d = ar.reqs[pending.pop(0)]
            mpt.mpt_serve_submit(server, ar.ptr(s_ar, s_off), ar.ptr(d_ar, d_off), nb, d, k, mpt.mpt_now_ns())
        for c in mpt.mpt_serve_poll(server):
            done[c[0]] = c
    return done


@pytest.mark.parametrize("streams,ctas", [(1, -3), (0, 0)], ids=["in_order", "concurrent"])
def test_results_same_alone_and_in_the_mix(ctx, streams, ctas):
    """Each request's result is the same alone and in the mix -- with batches in submission
    order on one stream (three CTAs per SM), and with batches in flight on streams of their
    own (the default: one CTA per SM, batch kernels sharing the SMs)."""
    ar = Arenas(400, payload.SEED_SERVE)
    if ctas < 0:  # -k: k CTAs per SM
        ctas = -ctas * mpt.mpt_ctx_info(ctx)["sms"]
    server = mpt.mpt_serve_start(ctx, streams=streams, batch_ctas=ctas)
    alone = run(server, ar, range(len(ar.reqs)), one_at_a_time=True)
    assert len(alone) == len(ar.reqs) and all(c[5] == mpt.MPT_OK for c in alone.values())
    h_alone = ar.digests("dst")
    ar.clear_dst()
    rng = np.random.default_rng(1)
    mix = run(server, ar, list(rng.permutation(len(ar.reqs))), one_at_a_time=False)
    stats = mpt.mpt_serve_stats(server)
    mpt.mpt_serve_stop(server)
    assert len(mix) == len(ar.reqs) and all(c[5] == mpt.MPT_OK for c in mix.values())
    h_mix = ar.digests("dst")
    assert h_mix == h_alone
    assert h_mix == ar.digests("src")  # a transfer's result is its source (the oracle's copy)
    assert stats["batches"] < len(ar.reqs) + len(ar.reqs)  # the mix shared batches
    assert all(c[3] >= c[2] >= c[1] for c in mix.values())  # arrival <= admit <= complete
    # oracle byte check on a sample of destinations
    for k in rng.choice(len(ar.reqs), 20, replace=False):
        _, s_ar, s_off, d_ar, d_off, nb, _ = ar.reqs[k]
        got = ar.t[d_ar][d_off:d_off + nb].cpu().numpy()
        assert np.array_equal(got, ar.src_np[s_ar][s_off:s_off + nb])


def test_admission_respects_budget(ctx):
    ar = Arenas(120, 17, median=256 * KiB, cap=512 * KiB)
    budget = 2 * MiB
    server = mpt.mpt_serve_start(ctx, staging_budget_bytes=budget)
    done = run(server, ar, range(len(ar.reqs)), one_at_a_time=False)
    stats = mpt.mpt_serve_stats(server)
    mpt.mpt_serve_stop(server)
    assert len(done) == len(ar.reqs)
    assert 0 < stats["max_inflight_bytes"] <= budget
    assert ar.digests("dst") == ar.digests("src")


def test_oversized_request_runs_alone(ctx):
    import torch
    a = torch.arange(8 * MiB, dtype=torch.uint8, device="cuda")
    b = torch.zeros_like(a)
    server = mpt.mpt_serve_start(ctx, staging_budget_bytes=MiB)
    mpt.mpt_serve_submit(server, a.data_ptr(), b.data_ptr(), a.numel(), mpt.MPT_D2D, 7)
    got = []
    t0 = time.time()
    while not got and time.time() - t0 < 30:
        got = mpt.mpt_serve_poll(server)
    mpt.mpt_serve_stop(server)
    assert got and got[0][0] == 7 and got[0][5] == mpt.MPT_OK
    assert torch.equal(a, b)


def test_refused_request_reported_and_server_continues(ctx):
    import torch
    d = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    h = torch.ones(1 << 20, dtype=torch.uint8).pin_memory()
    server = mpt.mpt_serve_start(ctx)
    # device-to-device from host memory: the batch path refuses it
    mpt.mpt_serve_submit(server, h.data_ptr(), d.data_ptr(), 4096, mpt.MPT_D2D, 1)
    got = {}
    t0 = time.time()
    while 1 not in got and time.time() - t0 < 30:
        for c in mpt.mpt_serve_poll(server):
            got[c[0]] = c
    mpt.mpt_serve_submit(server, h.data_ptr(), d.data_ptr(), 4096, mpt.MPT_H2D, 2)
    while 2 not in got and time.time() - t0 < 30:
        for c in mpt.mpt_serve_poll(server):
            got[c[0]] = c
    mpt.mpt_serve_stop(server)
    assert got[1][5] == mpt.MPT_EINVAL and got[2][5] == mpt.MPT_OK
    assert int(d[:4096].sum()) == 4096


def test_replay_keeps_the_schedule_and_results(ctx):
    """mpt_serve_replay submits a trace at its scheduled times from a native loop; every
    request completes, after its scheduled arrival, with the same bytes as alone (digests),
    and a trace with decreasing times is refused."""
    import threading
    ar = Arenas(300, payload.SEED_SERVE + 9)
    server = mpt.mpt_serve_start(ctx)
    n = len(ar.reqs)
    xf = [(ar.ptr(s_ar, s_off), ar.ptr(d_ar, d_off), nb, d) for _, s_ar, s_off, d_ar, d_off, nb, d in ar.reqs]
    t0 = mpt.mpt_now_ns() + 5_000_000
    due = [t0 + 50_000 * k for k in range(n)]  # 20k requests/s
    import ctypes
    late = (ctypes.c_uint64 * n)()
    th = threading.Thread(target=mpt.mpt_serve_replay, args=(server, xf, list(range(n)), due, late))
    th.start()
    done = {}
    t_end = time.time() + 60
    while len(done) < n and time.time() < t_end:
        for c in mpt.mpt_serve_poll(server):
            done[c[0]] = c
    th.join()
    with pytest.raises(mpt.MptError) as e:
        mpt.mpt_serve_replay(server, xf[:2], [0, 1], [due[1], due[0]])
    assert e.value.status == mpt.MPT_EINVAL
    mpt.mpt_serve_stop(server)
    assert len(done) == n and all(c[5] == mpt.MPT_OK for c in done.values())
    assert all(done[k][1] == due[k] and done[k][3] >= due[k] for k in range(n))  # arrival = schedule
    assert sorted(late)[n // 2] < 1_000_000  # the native loop keeps the schedule (median < 1 ms)
    assert ar.digests("dst") == ar.digests("src")


def test_bad_request_among_good_ones_refused_alone(ctx):
    """Requests are checked one by one at admission: a request with the wrong memory kinds,
    submitted amid valid ones that share its batch, is refused on its own and the others
    complete with their sources' bytes."""
    import torch
    ar = Arenas(200, payload.SEED_SERVE + 3)
    h = torch.ones(1 << 16, dtype=torch.uint8).pin_memory()
    d = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    server = mpt.mpt_serve_start(ctx)
    bad_tag = 10 ** 6
    for i, (k, s_ar, s_off, d_ar, d_off, nb, dr) in enumerate(ar.reqs):
        if i == len(ar.reqs) // 2:  # device-to-device from page-locked host memory
            mpt.mpt_serve_submit(server, h.data_ptr(), d.data_ptr(), 4096, mpt.MPT_D2D, bad_tag)
        mpt.mpt_serve_submit(server, ar.ptr(s_ar, s_off), ar.ptr(d_ar, d_off), nb, dr, k)
    done = {}
    t0 = time.time()
    while len(done) < len(ar.reqs) + 1 and time.time() - t0 < 60:
        for c in mpt.mpt_serve_poll(server):
            done[c[0]] = c
    stats = mpt.mpt_serve_stats(server)
    mpt.mpt_serve_stop(server)
    assert done[bad_tag][5] == mpt.MPT_EINVAL and stats["rejected"] == 1
    assert all(done[k][5] == mpt.MPT_OK for k in range(len(ar.reqs)))
    assert ar.digests("dst") == ar.digests("src")
    assert int(d.sum()) == 0


def test_backlog_of_a_slow_client_drains_in_order(ctx):
    """A client that stops polling leaves finished requests waiting in the server; polling
    later hands each out once, oldest first, in pieces of any size, and the counters
    record the backlog, the longest worker turn and the admission queue."""
    ar = Arenas(3000, payload.SEED_SERVE + 4, median=16 * KiB, cap=256 * KiB)
    n = len(ar.reqs)
    server = mpt.mpt_serve_start(ctx)
    for k, s_ar, s_off, d_ar, d_off, nb, dr in ar.reqs:
        mpt.mpt_serve_submit(server, ar.ptr(s_ar, s_off), ar.ptr(d_ar, d_off), nb, dr, k)
    t0 = time.time()
    while mpt.mpt_serve_stats(server)["completed"] < n and time.time() - t0 < 60:
        time.sleep(0.01)
    stats = mpt.mpt_serve_stats(server)
    got = []
    while len(got) < n and time.time() - t0 < 60:
        got += mpt.mpt_serve_poll(server, cap=97)
    mpt.mpt_serve_reset_stats(server)  # high-water marks to zero, running counts kept
    after = mpt.mpt_serve_stats(server)
    mpt.mpt_serve_stop(server)
    assert all(v == 0 for k, v in after.items() if k.startswith("max_"))
    assert after["completed"] == n and after["submitted"] == n and after["batches"] == stats["batches"]
    assert stats["completed"] == n and stats["max_pending_completions"] == n
    assert stats["max_turn_ns"] > 0 and stats["max_waiting"] >= 1
    assert sorted(c[0] for c in got) == list(range(n))
    assert all(c[5] == mpt.MPT_OK for c in got)
    assert all(a[3] <= b[3] for a, b in zip(got, got[1:]))  # oldest completion first
    assert ar.digests("dst") == ar.digests("src")


@pytest.mark.parametrize("spin_us", ["0", "50"], ids=["blocking", "short_spin"])
def test_worker_that_blocks_between_requests(ctx, spin_us):
    """With the idle worker blocking at once (MPT_SERVE_SPIN_US=0) or after a short spin,
    requests that arrive after gaps longer than the spin (so the worker has gone to sleep)
    still complete, each equal to its source per the oracle's definition of a transfer."""
    import os
    ar = Arenas(40, payload.SEED_SERVE + 7)
    old = os.environ.get("MPT_SERVE_SPIN_US")
    os.environ["MPT_SERVE_SPIN_US"] = spin_us
    try:
        server = mpt.mpt_serve_start(ctx)
    finally:
        if old is None:
            os.environ.pop("MPT_SERVE_SPIN_US", None)
        else:
            os.environ["MPT_SERVE_SPIN_US"] = old
    done = {}
    for k, s_ar, s_off, d_ar, d_off, nb, d in ar.reqs:
        time.sleep(0.0005 if k % 2 else 0.003)  # half the gaps outlast a 2 ms spin as well
        mpt.mpt_serve_submit(server, ar.ptr(s_ar, s_off), ar.ptr(d_ar, d_off), nb, d, k, mpt.mpt_now_ns())
        t0 = time.time()
        while k not in done and time.time() - t0 < 10:
            for c in mpt.mpt_serve_poll(server):
                done[c[0]] = c
    mpt.mpt_serve_stop(server)
    assert len(done) == len(ar.reqs) and all(c[5] == mpt.MPT_OK for c in done.values())
    assert ar.digests("dst") == ar.digests("src")
    for k in range(0, len(ar.reqs), 7):
        _, s_ar, s_off, d_ar, d_off, nb, _ = ar.reqs[k]
        got = ar.t[d_ar][d_off:d_off + nb].cpu().numpy()
        assert np.array_equal(got, ar.src_np[s_ar][s_off:s_off + nb])
