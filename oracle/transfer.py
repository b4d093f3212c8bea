"""Oracle for what a transfer produces, plus the digest used to compare buffers.

Whatever paths, chunks and pipelining carry a message, the destination must end up
holding exactly the source bytes (Sec. 4.5: pre-assigned, non-overlapping chunk
regions; completion only after every chunk has arrived).  So the expected result
of every transfer is ``memcpy(dst, src, N)`` and the oracle is that copy.

Digest (stated by this project; order-independent so that a parallel reduction
computes it exactly): with ``w_i`` the i-th little-endian 8-byte word of the buffer,
zero-padded at the end, GAMMA the splitmix64 increment and mix64 the splitmix64
output finaliser,

    H(buf) = mix64(N) + sum_i mix64(w_i XOR (i * GAMMA))      (mod 2**64).

This module is test infrastructure (see the package docstring).
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_G = np.uint64(GAMMA)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_BLOCK = 1 << 22


def mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64's output finaliser applied elementwise to uint64 values."""
    z = np.asarray(z, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def copy(src: np.ndarray) -> np.ndarray:
    """The expected destination of a transfer of ``src``: the same bytes."""
    src = np.ascontiguousarray(src).view(np.uint8).reshape(-1)
    dst = np.empty_like(src)
    dst[:] = src
    return dst


def hash64(buf) -> int:
    """Digest of a byte buffer (see the module docstring)."""
    b = np.ascontiguousarray(np.frombuffer(buf, dtype=np.uint8) if isinstance(buf, (bytes, bytearray))
                             else buf).view(np.uint8).reshape(-1)
    n = b.size
    nw = (n + 7) // 8
    total = np.uint64(0)
    with np.errstate(over="ignore"):
        for w0 in range(0, nw, _BLOCK):
            m = min(_BLOCK, nw - w0)
            lo, hi = w0 * 8, min(n, (w0 + m) * 8)
            part = np.zeros(m * 8, dtype=np.uint8)
            part[: hi - lo] = b[lo:hi]
            words = part.view("<u8").astype(np.uint64)
            idx = np.arange(w0, w0 + m, dtype=np.uint64) * _G
            total = total + np.sum(mix64(words ^ idx), dtype=np.uint64)
        total = total + mix64(np.array([n], dtype=np.uint64))[0]
    return int(total)


def batch_expected(dst_arena: np.ndarray, sources: dict, xfers) -> np.ndarray:
    """Expected destination arena after a batch of transfers.

    ``sources`` maps an arena name to its bytes; each transfer is
    ``(src_arena, src_offset, dst_offset, nbytes)`` and copies those bytes into the
    destination arena.  Destination regions must not overlap (each transfer owns its
    region, Sec. 4.5), which is checked.
    """
    out = copy(dst_arena)
    spans = sorted((d, d + n) for (_, _, d, n) in xfers if n > 0)
    for (a0, a1), (b0, _) in zip(spans, spans[1:]):
        if b0 < a1:
            raise ValueError("destination regions overlap")
    for arena, s, d, n in xfers:
        out[d:d + n] = np.asarray(sources[arena]).view(np.uint8)[s:s + n]
    return out
