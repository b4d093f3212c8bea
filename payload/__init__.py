"""Seeded synthetic inputs for the multi-path transfer library and its oracle.

This module is the one piece of code that both the CUDA path's tests/benchmarks
and the CPU oracle use.  It holds no arithmetic of the transfer method itself:
it only manufactures message payloads, message sizes and arrival schedules from
a seed, so that both sides see identical inputs.

Generator: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; the 64-bit finaliser constants are Stafford's "Mix13").
Word ``i`` of a stream seeded with ``s`` is the ``i``-th output (0-based) of the
sequential generator whose state starts at ``s``::

    z = s + (i + 1) * GAMMA            (mod 2**64)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    x_i = z ^ (z >> 31)

Payload encodings (a message of ``n`` bytes is the first ``n`` bytes of the
element stream, so a size that is not a multiple of the element size takes a
prefix of the last element's bytes):

* ``u8``   word ``i`` supplies bytes ``8i .. 8i+7`` little-endian;
* ``u32``  element ``j`` is the low 32 bits of ``x_j``;
* ``f32``  element ``j`` is ``(x_j >> 40) * 2**-23 - 1``, uniform on [-1, 1) and
  exact in binary32;
* ``bf16`` element ``j`` is the upper 16 bits of that binary32 value (truncation).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Seeds of the five workloads: 64 MiB copy, device sweep, host sweep, batched, serving.
SEED_COPY64 = 0x5EED0001
SEED_D2D_SWEEP = 0x5EED0002
SEED_HOST_SWEEP = 0x5EED0003
SEED_BATCH = 0x5EED0004
SEED_SERVE = 0x5EED0005

ELEM_BYTES = {"u8": 8, "u32": 4, "f32": 4, "bf16": 2}
_BLOCK_WORDS = 1 << 22  # generate in 32 MiB blocks to bound temporaries


def splitmix64_scalar(seed: int, i: int) -> int:
    """Output ``i`` (0-based) of splitmix64 started at state ``seed`` (Python ints)."""
    z = (seed + (i + 1) * GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64_words(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of splitmix64 at ``seed`` as uint64."""
    out = np.empty(count, dtype=np.uint64)
    g = np.uint64(GAMMA)
    base = np.uint64((seed + (start + 1) * GAMMA) & MASK64)
    with np.errstate(over="ignore"):
        for b0 in range(0, count, _BLOCK_WORDS):
            m = min(_BLOCK_WORDS, count - b0)
            z = np.arange(b0, b0 + m, dtype=np.uint64)
            z *= g
            z += base
            z ^= z >> np.uint64(30)
            z *= _M1
            z ^= z >> np.uint64(27)
            z *= _M2
            z ^= z >> np.uint64(31)
            out[b0:b0 + m] = z
    return out


def fill(kind: str, seed: int, nbytes: int, out: np.ndarray | None = None) -> np.ndarray:
    """Payload of ``nbytes`` bytes of element type ``kind`` as a uint8 array.

    ``out`` (uint8, length >= nbytes) receives the bytes when given, so a pinned
    host tensor's numpy view can be filled in place.
    """
    if kind not in ELEM_BYTES:
        raise ValueError(f"unknown payload kind {kind!r}")
    if out is None:
        out = np.empty(nbytes, dtype=np.uint8)
    dst = out[:nbytes]
    eb = {"u8": 8, "u32": 4, "f32": 4, "bf16": 2}[kind]
    nelem = (nbytes + eb - 1) // eb
    step = _BLOCK_WORDS
    for e0 in range(0, nelem, step):
        m = min(step, nelem - e0)
        x = splitmix64_words(seed, e0, m)
        if kind == "u8":
            raw = x.astype("<u8").view(np.uint8)
        elif kind == "u32":
            raw = (x & np.uint64(0xFFFFFFFF)).astype("<u4").view(np.uint8)
        else:
            u = (x >> np.uint64(40)).astype(np.float64)
            f = (u * (2.0 ** -23) - 1.0).astype("<f4")
            if kind == "f32":
                raw = f.view(np.uint8)
            else:
                raw = (f.view("<u4") >> np.uint32(16)).astype("<u2").view(np.uint8)
        b0 = e0 * eb
        b1 = min(nbytes, b0 + raw.size)
        dst[b0:b1] = raw[: b1 - b0]
    return dst


def fill_window(kind: str, seed: int, offset: int, nbytes: int) -> np.ndarray:
    """Bytes [offset, offset + nbytes) of the payload stream (what ``fill`` would give for a
    message of offset + nbytes bytes), generated without the bytes before ``offset``."""
    eb = ELEM_BYTES[kind]
    first = offset // eb
    lead = offset - first * eb
    x = splitmix64_words(seed, first, (lead + nbytes + eb - 1) // eb)
    if kind == "u8":
        raw = x.astype("<u8").view(np.uint8)
    elif kind == "u32":
        raw = (x & np.uint64(0xFFFFFFFF)).astype("<u4").view(np.uint8)
    else:
        f = ((x >> np.uint64(40)).astype(np.float64) * (2.0 ** -23) - 1.0).astype("<f4")
        raw = f.view(np.uint8) if kind == "f32" else (f.view("<u4") >> np.uint32(16)).astype("<u2").view(np.uint8)
    return raw[lead:lead + nbytes].copy()


def request_seed(seed: int, request_id: int) -> int:
    """Per-request payload seed: splitmix64 output ``request_id`` of stream ``seed``."""
    return splitmix64_scalar(seed, request_id)


def unit_double(x: int) -> float:
    """Map a 64-bit word to [0, 1) using its top 53 bits."""
    return (x >> 11) * (2.0 ** -53)


def batch_workload(n: int = 4096, seed: int = SEED_BATCH, min_bytes: int = 256,
                   max_bytes: int = 16 << 20, d2d_fraction: float = 0.7):
    """Sizes, directions and 16-byte gaps of the batched workload.

    Sizes are log-uniform on [min_bytes, max_bytes]: ``2*floor(exp(ln(min) + u*ln(max/min))/2)``
    with ``u`` from the top 53 bits of word ``3k``; transfer ``k`` is device-to-device when
    word ``3k+1`` maps below ``d2d_fraction``, else host-to-device; the gap placed before it in
    its arenas is ``16*(1 + (word 3k+2 mod 7))`` bytes, so every address is a multiple of 16.
    Returns (sizes, is_d2d, gaps) as Python lists.
    """
    lo, hi = math.log(min_bytes), math.log(max_bytes / min_bytes)
    sizes, d2d, gaps = [], [], []
    for k in range(n):
        u = unit_double(splitmix64_scalar(seed, 3 * k))
        sizes.append(2 * int(math.floor(math.exp(lo + u * hi) / 2)))
        d2d.append(unit_double(splitmix64_scalar(seed, 3 * k + 1)) < d2d_fraction)
        gaps.append(16 * (1 + splitmix64_scalar(seed, 3 * k + 2) % 7))
    return sizes, d2d, gaps


def batch_layout(sizes, d2d, gaps, align: int = 16, host_name: str = "host", dev_name: str = "dev"):
    """Pack the batched workload into arenas: transfer k sits ``gaps[k]`` bytes after the
    previous transfer's end rounded up to ``align`` (16: offsets on 16-byte multiples, in
    general not on larger boundaries), in the device source arena when ``d2d[k]`` else the
    host one, and at the same rule in the destination arena.  Returns (items, arena_bytes)
    with items (arena, src_offset, dst_offset, nbytes)."""
    up = lambda x: (x + align - 1) // align * align
    offs = {dev_name: 0, host_name: 0, "dst": 0}
    items = []
    for sz, is_d2d, gap in zip(sizes, d2d, gaps):
        a = dev_name if is_d2d else host_name
        offs[a] = up(offs[a]) + gap
        offs["dst"] = up(offs["dst"]) + gap
        items.append((a, offs[a], offs["dst"], sz))
        offs[a] += sz
        offs["dst"] += sz
    return items, offs


def serving_schedule(rate_per_s: float, duration_s: float, seed: int = SEED_SERVE,
                     median_bytes: int = 1 << 20, sigma: float = 1.5,
                     cap_bytes: int = 256 << 20, mix=(0.5, 0.25, 0.25), max_requests: int | None = None):
    """Open-loop Poisson arrivals with lognormal sizes and a direction mix.

    Inter-arrival gaps are ``-ln(1-u)/rate``; sizes are
    ``min(cap, max(16, round(median*exp(sigma*z))))`` rounded up to a multiple of 16,
    with ``z`` standard normal from Box-Muller on two splitmix doubles; the direction is
    0 (device-to-device), 1 (host-to-device) or 2 (device-to-host) by ``mix``.
    Stops at ``duration_s`` or after ``max_requests`` requests, whichever comes first.
    Returns a list of (arrival_s, nbytes, direction).
    """
    out = []
    t = 0.0
    k = 0
    while max_requests is None or k < max_requests:
        u = unit_double(splitmix64_scalar(seed, 4 * k))
        t += -math.log(1.0 - u) / rate_per_s
        if t >= duration_s:
            break
        u1 = unit_double(splitmix64_scalar(seed, 4 * k + 1))
        u2 = unit_double(splitmix64_scalar(seed, 4 * k + 2))
        z = math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)
        nb = min(cap_bytes, max(16, int(round(median_bytes * math.exp(sigma * z)))))
        nb = (nb + 15) & ~15
        nb = min(nb, cap_bytes)
        ud = unit_double(splitmix64_scalar(seed, 4 * k + 3))
        d = 0 if ud < mix[0] else (1 if ud < mix[0] + mix[1] else 2)
        out.append((t, nb, d))
        k += 1
    return out
