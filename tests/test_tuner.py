"""Autotuner: environment overrides (host logic, CPU) and measured tuning, persistence and
tuned plans on the GPU."""
import os

import numpy as np
import pytest

import paper_2604_22228_gb300 as mpt
from oracle import planner as P
from oracle import transfer as T
from paper_2604_22228_gb300 import build

MiB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def test_env_path_set(monkeypatch):
    monkeypatch.setenv("MPT_PATHS", "ce,sm")
    monkeypatch.setenv("MPT_SHARES", "16384,49152")
    monkeypatch.setenv("MPT_CHUNK_BYTES", "65536")
    monkeypatch.setenv("MPT_CTAS", "77")
    monkeypatch.setenv("MPT_SM_VARIANT", "bulk")
    h = mpt.mpt_plan(None, 10 * MiB, mpt.MPT_D2D, None)
    paths = mpt.mpt_plan_paths(h)
    chunks = mpt.mpt_plan_chunks(h)
    mpt.mpt_plan_destroy(h)
    assert [(p["kind"], p["share"], p["chunk_bytes"], p["ctas"], p["flags"]) for p in paths] == \
        [(P.CE, 16384, 65536, 77, 0), (P.SM, 49152, 65536, 77, mpt.MPT_SM_BULK)]
    assert [P.Chunk(*c) for c in chunks] == P.plan(10 * MiB, P.D2D, [(P.CE, 16384, 65536), (P.SM, 49152, 65536)])


def test_env_chunks_per_path(monkeypatch):
    # Sec. 4.4: the number of chunks per path set through the environment
    monkeypatch.setenv("MPT_PATHS", "ce,sm")
    monkeypatch.setenv("MPT_CHUNKS", "4")
    h = mpt.mpt_plan(None, 8 * MiB, mpt.MPT_D2D, None)
    chunks = mpt.mpt_plan_chunks(h)
    mpt.mpt_plan_destroy(h)
    assert len(chunks) == 8 and all(c[1] == MiB for c in chunks)


@pytest.mark.parametrize("paths,shares", [("ce,xx", None), ("ce,sm", "1,2,3"), ("ce,sm,hs,zc,ce", None),
                                          ("zc", None)])
def test_env_invalid(monkeypatch, paths, shares):
    monkeypatch.setenv("MPT_PATHS", paths)
    if shares:
        monkeypatch.setenv("MPT_SHARES", shares)
    with pytest.raises(mpt.MptError) as e:
        mpt.mpt_plan(None, MiB, mpt.MPT_D2D, None)
    assert e.value.status == mpt.MPT_EINVAL


def test_tuner_needs_context_without_env(monkeypatch):
    monkeypatch.delenv("MPT_PATHS", raising=False)
    with pytest.raises(mpt.MptError):
        mpt.mpt_plan(None, MiB, mpt.MPT_D2D, None)


@pytest.mark.gpu
def test_tune_persist_and_use(tmp_path, monkeypatch):
    import torch
    monkeypatch.delenv("MPT_PATHS", raising=False)
    monkeypatch.setenv("MPT_TUNE_DEFAULTS", "0")  # start from an empty table
    ctx = mpt.mpt_ctx_create(0)
    try:
        results = {}
        for d, n in [(P.D2D, 4 * MiB), (P.D2D, 4096), (P.H2D, 8 * MiB), (P.D2H, 3 * MiB)]:
            paths, us = mpt.mpt_tune(ctx, d, n, mpt.MPT_MODE_GRAPH)
            assert 1 <= len(paths) <= 4 and us > 0
            results[(d, n)] = paths
            h = mpt.mpt_plan(ctx, n + 16, d, None)  # same log2 bucket
            assert mpt.mpt_plan_paths(h) == [dict(p, chunk_bytes=max(16, (p["chunk_bytes"] + 15) // 16 * 16))
                                            for p in paths]
            mpt.mpt_plan_destroy(h)
        paths, us = mpt.mpt_tune(ctx, P.D2D, 4 * MiB, mpt.MPT_MODE_EAGER)
        f = str(tmp_path / "tune.jsonl")
        mpt.mpt_tune_save(ctx, f)
        lines = open(f).read().splitlines()
        assert len(lines) == 5
        ctx2 = mpt.mpt_ctx_create(0, f)
        for (d, n), paths in results.items():
            assert mpt.mpt_tune_get(ctx2, d, n)[0] == paths
        mpt.mpt_ctx_destroy(ctx2)
        # a transfer through the tuned plan is still an exact copy
        n = 4 * MiB + 48
        src = torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda")
        dst = torch.zeros_like(src)
        h = mpt.mpt_plan(ctx, n, P.D2D, None)
        g = mpt.mpt_capture(ctx, h, dst.data_ptr(), src.data_ptr())
        mpt.mpt_launch(g, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert torch.equal(src, dst)
        mpt.mpt_graph_release(g)
        mpt.mpt_plan_destroy(h)
        assert mpt.mpt_ctx_status(ctx)[0] == mpt.MPT_OK
    finally:
        mpt.mpt_ctx_destroy(ctx)


@pytest.mark.gpu
def test_tune_file_rejects_garbage(tmp_path):
    f = tmp_path / "bad.jsonl"
    f.write_text('{"dir": 0, "mode": 0, "bucket": 20, "layout": 0, "us": 1.0, "paths": [[3, 65536, 16, 0, 0]]}\n')
    with pytest.raises(mpt.MptError):
        mpt.mpt_ctx_create(0, str(f))


@pytest.mark.gpu
def test_model_fallback_plans_are_valid(monkeypatch):
    import torch
    monkeypatch.delenv("MPT_PATHS", raising=False)
    ctx = mpt.mpt_ctx_create(0)
    try:
        for d in (P.D2D, P.H2D, P.D2H):
            for n in (1, 1000, MiB, 64 * MiB + 3):
                h = mpt.mpt_plan(ctx, n, d, None)
                paths = [(p["kind"], p["share"], p["chunk_bytes"]) for p in mpt.mpt_plan_paths(h)]
                chunks = [P.Chunk(*c) for c in mpt.mpt_plan_chunks(h)]
                assert chunks == P.plan(n, d, paths)
                mpt.mpt_plan_destroy(h)
    finally:
        mpt.mpt_ctx_destroy(ctx)


@pytest.mark.gpu
def test_shipped_defaults_load(monkeypatch):
    """The offline-tuned table for this device model (tuned/<device>.jsonl next to the
    library) is loaded by a new context, and every entry in it is a valid path set."""
    import os
    import re

    import torch
    name = re.sub(r"[^0-9A-Za-z]", "_", torch.cuda.get_device_name(0))
    path = os.path.join(os.path.dirname(mpt._ffi.LIB_PATH), "tuned", name + ".jsonl")
    if not os.path.exists(path):
        pytest.skip(f"no shipped table for {name}")
    monkeypatch.delenv("MPT_TUNE_FILE", raising=False)
    ctx = mpt.mpt_ctx_create(0)
    try:
        paths, us = mpt.mpt_tune_get(ctx, P.D2D, 1 << 30, mpt.MPT_MODE_GRAPH)
        assert paths and us > 0
    finally:
        mpt.mpt_ctx_destroy(ctx)
    monkeypatch.setenv("MPT_TUNE_DEFAULTS", "0")
    ctx = mpt.mpt_ctx_create(0)
    try:
        with pytest.raises(mpt.MptError):
            mpt.mpt_tune_get(ctx, P.D2D, 1 << 30, mpt.MPT_MODE_GRAPH)
    finally:
        mpt.mpt_ctx_destroy(ctx)


def _verbose_lines(err, tag):
    """Parse MPT_TUNE_VERBOSE lines: (median us, [(kind, share, chunk, ctas, flags), ...])."""
    import re
    out = []
    for line in err.splitlines():
        if not line.startswith(tag + " dir="):
            continue
        us = float(re.search(r" us=([0-9.]+)", line).group(1))
        paths = [tuple(int(x) for x in m.split()) for m in re.findall(r"\[([0-9 ]+)\]", line)]
        out.append((us, paths))
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("direction,n,kinds", [(P.D2D, 4 * MiB, {P.CE, P.SM}),
                                               (P.H2D, 8 * MiB, {P.CE, P.ZC, P.HS})])
def test_tune_confirms_leaders_against_single_paths(capfd, monkeypatch, direction, n, kinds):
    """mpt_tune re-times its leaders together with the fastest single-path candidate of each
    path kind in interleaved rounds, and keeps the lowest median of those rounds: the rounds
    hold a single-path candidate of every kind that was measured, the three first-pass
    leaders, and the stored choice is the confirmed minimum."""
    monkeypatch.delenv("MPT_PATHS", raising=False)
    monkeypatch.setenv("MPT_TUNE_VERBOSE", "1")
    ctx = mpt.mpt_ctx_create(0)
    try:
        capfd.readouterr()
        paths, us = mpt.mpt_tune(ctx, direction, n, mpt.MPT_MODE_GRAPH)
        err = capfd.readouterr().err
        assert mpt.mpt_ctx_status(ctx)[0] == mpt.MPT_OK
    finally:
        mpt.mpt_ctx_destroy(ctx)
    first = _verbose_lines(err, "mpt_tune")
    confirm = _verbose_lines(err, "mpt_tune confirm")
    assert len(first) >= 10 and 3 <= len(confirm) <= 3 + len(kinds)
    assert {p[0][0] for _, p in confirm if len(p) == 1} >= kinds
    # the three first-pass leaders were confirmed; medians print rounded to 0.01 us, so ties
    # at the third place are allowed either way
    confirmed = [q for _, q in confirm]
    ranked = sorted(first, key=lambda r: r[0])
    cut = ranked[2][0]
    for u, p in ranked:
        if u < cut:
            assert p in confirmed, p
    assert sum(1 for u, p in ranked if u <= cut and p in confirmed) >= 3
    best_us = min(u for u, _ in confirm)
    chosen = [tuple(q[k] for k in ("kind", "share", "chunk_bytes", "ctas", "flags")) for q in paths]
    assert chosen in [p for u, p in confirm if u == best_us]
    assert abs(us - best_us) < 0.006
