"""Single-GPU multi-path transfers with CUDA graphs, on GB300 (sm_103a).

A message of N bytes is split over several transfer paths by share (horizontal split),
each path's part is cut into chunks (vertical split), and the paths run concurrently
inside one cached CUDA graph (Sec. 4.2-4.3 of the paper).  On one GPU the paths are the
copy engines, an SM copy kernel, a two-hop staged route and a zero-copy kernel over
mapped page-locked host memory.

This module is a thin binding over the C ABI of ``include/mpt.h``: the functions carry
the C names and only marshal arguments (pointers may be ints or anything with
``data_ptr()``; streams may be ints, ``None`` or objects with ``cuda_stream``).  Every
byte moves inside libmpt.so; a missing library raises instead of falling back.
"""
from __future__ import annotations

import ctypes as C

from . import _ffi
from ._ffi import (MPT_D2D, MPT_D2H, MPT_H2D, MPT_LAYOUT_CONTIG, MPT_LAYOUT_INTERLEAVE, MPT_MAX_CHUNKS,  # noqa: F401
                   MPT_NOALLOC_MAX_RANGES, MPT_BULK_CONFIGS, MPT_MAX_PATHS, MPT_PATH_CE, MPT_PATH_HS, MPT_PATH_SM, MPT_PATH_ZC, MPT_SHARE_ONE, MPT_SM_BULK, MPT_SM_TILE8K, MPT_HS_HOST_THREADS, MPT_PLAN_PAGEABLE, MPT_MODE_PAGEABLE, MPT_PLAN_DUPLEX, MPT_MODE_DUPLEX, MPT_BATCH_TUNE_TIME, MPT_BATCH_TUNE_P99,
                   MPT_SM_VEC128, MPT_PLAN_EAGER, MPT_MODE_GRAPH, MPT_MODE_EAGER, MPT_PREPARE_GRAPH,
                   MPT_PREPARE_EAGER, MPT_PREPARE_AUTO, STATUS_NAMES)
from ._ffi import MPT_EAGAIN, MPT_ECUDA, MPT_EINVAL, MPT_ENOMEM, MPT_ENOTSUP, MPT_ETIMEDOUT, MPT_OK  # noqa: F401


class MptError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def lib():
    return _ffi.load()


def _check(st: int, where: str) -> None:
    if st != MPT_OK:
        raise MptError(st, where, lib().mpt_last_error().decode(errors="replace"))


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x).__name__}")


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _specs(paths):
    arr = (_ffi.mpt_path_spec * len(paths))()
    for i, p in enumerate(paths):
        if isinstance(p, dict):
            p = (p["kind"], p["share"], p.get("chunk_bytes", 0), p.get("ctas", 0), p.get("flags", 0))
        p = tuple(p) + (0,) * (5 - len(p))
        arr[i] = _ffi.mpt_path_spec(*p)
    return arr


def mpt_version() -> str:
    return lib().mpt_version().decode()


def mpt_last_error() -> str:
    return lib().mpt_last_error().decode(errors="replace")


def mpt_ctx_create(device: int = 0, tune_file: str | None = None) -> int:
    h = C.c_void_p()
    _check(lib().mpt_ctx_create(device, tune_file.encode() if tune_file else None, C.byref(h)), "mpt_ctx_create")
    return h.value


def mpt_ctx_destroy(ctx: int) -> None:
    _check(lib().mpt_ctx_destroy(ctx), "mpt_ctx_destroy")


def mpt_ctx_info(ctx: int) -> dict:
    info = _ffi.mpt_device_info()
    _check(lib().mpt_ctx_info(ctx, C.byref(info)), "mpt_ctx_info")
    out = {name: getattr(info, name) for name, _ in _ffi.mpt_device_info._fields_}
    out["name"] = info.name.decode(errors="replace")
    return out


def mpt_trace_lanes(ctx: int, enable: bool = True) -> None:
    _check(lib().mpt_trace_lanes(ctx, 1 if enable else 0), "mpt_trace_lanes")


def mpt_lane_times(ctx: int) -> list[float]:
    """Per-path lane durations (ms) of the last traced multi-path eager launch (-1: not timed)."""
    out = (C.c_float * MPT_MAX_PATHS)()
    n = C.c_uint32()
    _check(lib().mpt_lane_times(ctx, out, MPT_MAX_PATHS, C.byref(n)), "mpt_lane_times")
    return [round(v, 6) for v in out[: n.value]]


def mpt_ctx_status(ctx: int) -> tuple[int, int]:
    """(status, site) of the context's device status word, which is then reset."""
    site = C.c_uint32()
    st = lib().mpt_ctx_status(ctx, C.byref(site))
    return st, site.value


def mpt_ctx_set_wait_limit(ctx: int, ns: int) -> None:
    """Wait limit of the staged host-to-device path's device-side flag waits (0 = default)."""
    _check(lib().mpt_ctx_set_wait_limit(ctx, ns), "mpt_ctx_set_wait_limit")


def mpt_plan(ctx, nbytes: int, direction: int, paths, align: int = 16, layout: int = MPT_LAYOUT_CONTIG) -> int:
    h = C.c_void_p()
    if paths is None:
        st = lib().mpt_plan(ctx, nbytes, direction, None, 0, align, layout, C.byref(h))
    else:
        arr = _specs(paths)
        st = lib().mpt_plan(ctx, nbytes, direction, arr, len(paths), align, layout, C.byref(h))
    _check(st, "mpt_plan")
    return h.value


def mpt_plan_chunks(plan: int) -> list[tuple[int, int, int, int]]:
    n = C.c_size_t()
    _check(lib().mpt_plan_chunks(plan, None, 0, C.byref(n)), "mpt_plan_chunks")
    arr = (_ffi.mpt_chunk * max(1, n.value))()
    _check(lib().mpt_plan_chunks(plan, arr, n.value, C.byref(n)), "mpt_plan_chunks")
    return [(c.offset, c.bytes, c.path_index, c.chunk_index) for c in arr[: n.value]]


def mpt_plan_paths(plan: int) -> list[dict]:
    arr = (_ffi.mpt_path_spec * MPT_MAX_PATHS)()
    n = C.c_uint32()
    _check(lib().mpt_plan_paths(plan, arr, MPT_MAX_PATHS, C.byref(n)), "mpt_plan_paths")
    return [dict(kind=s.kind, share=s.share, chunk_bytes=s.chunk_bytes, ctas=s.ctas, flags=s.flags)
            for s in arr[: n.value]]


def mpt_plan_destroy(plan: int) -> None:
    _check(lib().mpt_plan_destroy(plan), "mpt_plan_destroy")


def mpt_capture(ctx: int, plan: int, dst, src) -> int:
    h = C.c_void_p()
    _check(lib().mpt_capture(ctx, plan, _ptr(dst), _ptr(src), C.byref(h)), "mpt_capture")
    return h.value


def mpt_prepare(ctx: int, plan: int, dst, src, mode: int = MPT_PREPARE_AUTO) -> int:
    h = C.c_void_p()
    _check(lib().mpt_prepare(ctx, plan, _ptr(dst), _ptr(src), mode, C.byref(h)), "mpt_prepare")
    return h.value


def mpt_launch(graph: int, stream=None) -> None:
    _check(lib().mpt_launch(graph, _stream(stream)), "mpt_launch")


def mpt_graph_get_info(graph: int) -> dict:
    info = _ffi.mpt_graph_info()
    _check(lib().mpt_graph_get_info(graph, C.byref(info)), "mpt_graph_get_info")
    return {name: getattr(info, name) for name, _ in _ffi.mpt_graph_info._fields_}


def mpt_graph_rebind(graph: int, plan: int, dst, src) -> None:
    _check(lib().mpt_graph_rebind(graph, plan, _ptr(dst), _ptr(src)), "mpt_graph_rebind")


def mpt_graph_release(graph: int) -> None:
    _check(lib().mpt_graph_release(graph), "mpt_graph_release")


def mpt_graph_evict(ctx: int, ptr) -> int:
    n = C.c_uint32()
    _check(lib().mpt_graph_evict(ctx, _ptr(ptr), C.byref(n)), "mpt_graph_evict")
    return n.value


def mpt_launch_eager(ctx: int, plan: int, dst, src, stream=None) -> None:
    _check(lib().mpt_launch_eager(ctx, plan, _ptr(dst), _ptr(src), _stream(stream)), "mpt_launch_eager")


def mpt_sm_copy(ctx: int, dst, src, nbytes: int, variant: int = MPT_SM_VEC128, ctas: int = 0, stream=None) -> None:
    _check(lib().mpt_sm_copy(ctx, _ptr(dst), _ptr(src), nbytes, variant, ctas, _stream(stream)), "mpt_sm_copy")


def mpt_hash_device(ctx: int, ptr, nbytes: int, stream=None) -> int:
    out = C.c_uint64()
    _check(lib().mpt_hash_device(ctx, _ptr(ptr), nbytes, _stream(stream), C.byref(out)), "mpt_hash_device")
    return out.value


def _model(m):
    if isinstance(m, _ffi.mpt_model):
        return m
    out = _ffi.mpt_model(m["launch_ps"], m["hbm_Bps"], m["link_h2d_Bps"], m["link_d2h_Bps"])
    for name in ("ce", "sm", "hs", "zc"):
        setattr(out, name, _ffi.mpt_path_model(*m[name]))
    return out


def mpt_model_time(model, direction: int, kinds, nbytes_per_path, chunk: int) -> int:
    n = len(kinds)
    k = (C.c_uint32 * n)(*kinds)
    b = (C.c_uint64 * n)(*nbytes_per_path)
    out = C.c_uint64()
    _check(lib().mpt_model_time(C.byref(_model(model)), direction, k, b, n, chunk, C.byref(out)), "mpt_model_time")
    return out.value


def mpt_model_optimize(model, nbytes: int, direction: int, kinds, align: int = 16):
    """(bytes per path, chunk, modelled ps) of the best split under the model."""
    n = len(kinds)
    k = (C.c_uint32 * n)(*kinds)
    b = (C.c_uint64 * n)()
    chunk, ps = C.c_uint64(), C.c_uint64()
    _check(lib().mpt_model_optimize(C.byref(_model(model)), nbytes, direction, k, n, align, b, C.byref(chunk),
                                    C.byref(ps)), "mpt_model_optimize")
    return tuple(b), chunk.value, ps.value


def _paths_out(arr, n):
    return [dict(kind=s.kind, share=s.share, chunk_bytes=s.chunk_bytes, ctas=s.ctas, flags=s.flags)
            for s in arr[:n]]


def mpt_tune(ctx: int, direction: int, nbytes: int, mode: int = MPT_MODE_GRAPH, reps: int = 0):
    """Measure and store the best path set for this bucket; returns (paths, microseconds)."""
    arr = (_ffi.mpt_path_spec * 4)()
    n, us = C.c_uint32(), C.c_double()
    _check(lib().mpt_tune(ctx, direction, nbytes, mode, reps, arr, C.byref(n), C.byref(us)), "mpt_tune")
    return _paths_out(arr, n.value), us.value


def mpt_tune_save(ctx: int, path: str) -> None:
    _check(lib().mpt_tune_save(ctx, path.encode()), "mpt_tune_save")


def mpt_tune_load(ctx: int, path: str) -> None:
    _check(lib().mpt_tune_load(ctx, path.encode()), "mpt_tune_load")


def mpt_tune_get(ctx: int, direction: int, nbytes: int, mode: int = MPT_MODE_GRAPH):
    arr = (_ffi.mpt_path_spec * 4)()
    n, us = C.c_uint32(), C.c_double()
    _check(lib().mpt_tune_get(ctx, direction, nbytes, mode, arr, C.byref(n), C.byref(us)), "mpt_tune_get")
    return _paths_out(arr, n.value), us.value


def mpt_batch_configure(ctx: int, slots: int = 0, max_xfers: int = 0, ctas: int = 0, tile_bytes: int = 0) -> None:
    _check(lib().mpt_batch_configure(ctx, slots, max_xfers, ctas, tile_bytes), "mpt_batch_configure")


def mpt_batch_configure_dma(ctx: int, lanes: int, items_per_lane: int = 8, min_bytes: int = 4 << 20) -> None:
    _check(lib().mpt_batch_configure_dma(ctx, lanes, items_per_lane, min_bytes), "mpt_batch_configure_dma")


def mpt_batch_register(ctx: int, base, nbytes: int) -> None:
    _check(lib().mpt_batch_register(ctx, _ptr(base), nbytes), "mpt_batch_register")


def make_xfers(xfers):
    """ctypes array of mpt_xfer from (src, dst, nbytes, direction) tuples."""
    arr = (_ffi.mpt_xfer * max(1, len(xfers)))()
    for i, (s, d, n, direction) in enumerate(xfers):
        arr[i] = _ffi.mpt_xfer(_ptr(s), _ptr(d), n, direction, 0)
    return arr


def mpt_batch_submit(ctx: int, xfers, stream=None) -> int:
    """xfers: a ctypes mpt_xfer array from make_xfers, or a list of (src, dst, nbytes, dir)."""
    n = len(xfers)
    arr = xfers if isinstance(xfers, C.Array) else make_xfers(xfers)
    h = C.c_void_p()
    _check(lib().mpt_batch_submit(ctx, arr, n, _stream(stream), C.byref(h)), "mpt_batch_submit")
    return h.value


def mpt_batch_tune(ctx: int, xfers, objective: int = 0, reps: int = 0, stream=None) -> dict:
    """Measure batch settings on a representative batch, apply the best; returns it."""
    n = len(xfers)
    arr = xfers if isinstance(xfers, C.Array) else make_xfers(xfers)
    out = _ffi.mpt_batch_tuning()
    _check(lib().mpt_batch_tune(ctx, arr, n, objective, reps, _stream(stream), C.byref(out)), "mpt_batch_tune")
    return {name: getattr(out, name) for name, _ in _ffi.mpt_batch_tuning._fields_ if name != "reserved"}


def mpt_batch_poll(batch: int, n: int | None = None):
    """(completed count, per-transfer flags or None)."""
    done = C.c_size_t()
    flags = (C.c_uint8 * n)() if n else None
    _check(lib().mpt_batch_poll(batch, C.byref(done), flags), "mpt_batch_poll")
    return done.value, (list(flags) if flags is not None else None)


def mpt_batch_wait(batch: int, timeout_ns: int = 10 ** 10) -> None:
    _check(lib().mpt_batch_wait(batch, timeout_ns), "mpt_batch_wait")


def mpt_batch_times(batch: int, n: int) -> list[int]:
    out = (C.c_uint64 * n)()
    _check(lib().mpt_batch_times(batch, out), "mpt_batch_times")
    return list(out)


def mpt_batch_watch(batch: int, t0_ns: int, n: int, timeout_ns: int = 60 * 10 ** 9) -> list[int]:
    """Per-transfer completion times (ns after t0_ns) as first seen from the host; waits."""
    out = (C.c_uint64 * max(1, n))()
    _check(lib().mpt_batch_watch(batch, t0_ns, out, timeout_ns), "mpt_batch_watch")
    return list(out[:n])


def mpt_copy_each(ctx: int, xfers, streams, wait: bool = True, timeout_ns: int = 60 * 10 ** 9):
    """Every transfer as its own cudaMemcpyAsync on streams[dir] (three streams: D2D, H2D,
    D2H).  wait: block and return each completion time in ns after the call began."""
    n = len(xfers)
    arr = xfers if isinstance(xfers, C.Array) else make_xfers(xfers)
    ss = (C.c_void_p * 3)(*[_stream(s) for s in streams])
    out = (C.c_uint64 * max(1, n))() if wait else None
    _check(lib().mpt_copy_each(ctx, arr, n, ss, out, timeout_ns), "mpt_copy_each")
    return list(out[:n]) if wait else None


def mpt_batch_release(batch: int) -> None:
    _check(lib().mpt_batch_release(batch), "mpt_batch_release")


def mpt_now_ns() -> int:
    return lib().mpt_now_ns()


def mpt_serve_start(ctx: int, staging_budget_bytes: int = 0, max_batch: int = 0, max_inflight_batches: int = 0,
                    streams: int = 0, batch_ctas: int = 0) -> int:
    cfg = _ffi.mpt_serve_config(staging_budget_bytes, max_batch, max_inflight_batches, streams, batch_ctas)
    h = C.c_void_p()
    _check(lib().mpt_serve_start(ctx, C.byref(cfg), C.byref(h)), "mpt_serve_start")
    return h.value


def mpt_serve_submit(server: int, src, dst, nbytes: int, direction: int, tag: int, arrival_ns: int = 0) -> None:
    x = _ffi.mpt_xfer(_ptr(src), _ptr(dst), nbytes, direction, 0)
    _check(lib().mpt_serve_submit(server, C.byref(x), tag, arrival_ns), "mpt_serve_submit")


_COMPLETION_BUF = None


def mpt_serve_replay(server: int, xfers, tags, due_ns, late_out=None) -> None:
    """Submit xfers[i] at due_ns[i] from a native loop (see the C API).  xfers: a ctypes
    mpt_xfer array (make_xfers) or (src, dst, nbytes, dir) tuples; tags, due_ns: sequences
    of ints or ctypes uint64 arrays; late_out: optional ctypes uint64 array for the delays."""
    n = len(xfers)
    arr = xfers if isinstance(xfers, C.Array) else make_xfers(xfers)
    t = tags if isinstance(tags, C.Array) else (C.c_uint64 * max(1, n))(*tags)
    d = due_ns if isinstance(due_ns, C.Array) else (C.c_uint64 * max(1, n))(*due_ns)
    _check(lib().mpt_serve_replay(server, arr, t, d, n, late_out), "mpt_serve_replay")


def mpt_serve_poll(server: int, cap: int = 4096) -> list[tuple]:
    """Finished requests as (tag, arrival_ns, admit_ns, complete_ns, bytes, status)."""
    global _COMPLETION_BUF
    if _COMPLETION_BUF is None or len(_COMPLETION_BUF) < cap:
        _COMPLETION_BUF = (_ffi.mpt_completion * cap)()
    n = C.c_size_t()
    _check(lib().mpt_serve_poll(server, _COMPLETION_BUF, cap, C.byref(n)), "mpt_serve_poll")
    return [(c.tag, c.arrival_ns, c.admit_ns, c.complete_ns, c.bytes, c.status) for c in _COMPLETION_BUF[:n.value]]


def mpt_serve_stats(server: int) -> dict:
    st = _ffi.mpt_serve_stats_t()
    _check(lib().mpt_serve_stats(server, C.byref(st)), "mpt_serve_stats")
    return {name: getattr(st, name) for name, _ in _ffi.mpt_serve_stats_t._fields_}


def mpt_serve_reset_stats(server: int) -> None:
    _check(lib().mpt_serve_reset_stats(server), "mpt_serve_reset_stats")


def mpt_serve_stop(server: int) -> None:
    _check(lib().mpt_serve_stop(server), "mpt_serve_stop")


def mpt_demo_jacobi_step(inp, out, rows: int, cols: int, stream=None) -> None:
    _check(lib().mpt_demo_jacobi_step(_ptr(inp), _ptr(out), rows, cols, _stream(stream)), "mpt_demo_jacobi_step")


def mpt_selftest_flag_timeout(ctx: int, timeout_ns: int):
    """(status, site) left by a bounded device wait on a flag nothing raises."""
    site = C.c_uint32()
    st = lib().mpt_selftest_flag_timeout(ctx, timeout_ns, C.byref(site))
    return st, site.value


def mpt_hash_ranges_noalloc(ranges, stream=None) -> list[int]:
    """Digests of [(pointer, nbytes), ...] without any allocation (see include/mpt.h)."""
    n = len(ranges)
    ptrs = (C.c_void_p * max(1, n))(*[_ptr(p) for p, _ in ranges])
    sizes = (C.c_uint64 * max(1, n))(*[b for _, b in ranges])
    out = (C.c_uint64 * max(1, n))()
    _check(lib().mpt_hash_ranges_noalloc(ptrs, sizes, n, _stream(stream), out), "mpt_hash_ranges_noalloc")
    return list(out[:n])


def mpt_host_alloc(ctx, nbytes: int) -> tuple[int, int]:
    """(host address, device alias) of a new page-locked, device-mapped host buffer."""
    p, d = C.c_void_p(), C.c_void_p()
    _check(lib().mpt_host_alloc(ctx, nbytes, C.byref(p), C.byref(d)), "mpt_host_alloc")
    return p.value, d.value


def mpt_host_free(ctx, ptr) -> None:
    """Free an mpt_host_alloc buffer; with its context, cached graphs on it are dropped first."""
    _check(lib().mpt_host_free(ctx, _ptr(ptr)), "mpt_host_free")


def mpt_host_bandwidth(ptr, nbytes: int, threads: int, op: int, reps: int = 3) -> float:
    """Host-memory GB/s of `threads` CPU threads streaming over [ptr, ptr+nbytes): op 0 read,
    1 write, 2 copy (first half into the second half)."""
    out = C.c_double()
    _check(lib().mpt_host_bandwidth(_ptr(ptr), nbytes, threads, op, reps, C.byref(out)), "mpt_host_bandwidth")
    return out.value
