"""Oracle planner: the 2-D split of one message over a path set.

Sec. 4.3 ("2-D Pipelining Engine"): a message is first divided among the selected
paths (horizontal split), then each path's part is cut into smaller chunks that are
sent in a pipeline (vertical split).  Algorithm 1 (CreateGraph) walks the paths in
order, giving path p a byte count derived from ``share[p]`` and advancing a running
offset ``sent_data``; the text after Algorithm 2 says the production code deals the
chunks to the paths one at a time (round robin) instead.  Sec. 4.5 requires every
chunk to write its own pre-assigned, non-overlapping destination region.

Readings taken where the paper is silent or inconsistent (Algorithm 1's chunk
formula advances ``sent_data`` once per path, so it cannot describe a multi-chunk
path):

* shares are integers out of 65536 that sum to 65536;
* path p < P-1 receives ``b_p = floor_A(floor(N * w_p / 65536))`` bytes and the last
  path receives the remainder, so every region but the last starts and ends on a
  multiple of the alignment A;
* chunk size ``C_p`` is explicit per path and a multiple of A;
* CONTIG layout: path p owns one contiguous region, regions in path order, each cut
  into chunks of ``C_p`` with a short final chunk;
* INTERLEAVE layout: chunks are dealt in rounds, path 0..P-1 each emitting one chunk
  of ``min(C_p, remaining_p)`` per round, laid back to back; the single chunk whose
  length may not be a multiple of A (the last path's final chunk when N mod A != 0)
  is held back and placed at the very end so that every offset stays A-aligned.

This module is test infrastructure (see the package docstring).
"""
from __future__ import annotations

from typing import NamedTuple

SHARE_ONE = 65536
MAX_PATHS = 8
MAX_ALIGN = 4096

D2D, H2D, D2H = 0, 1, 2
CE, SM, HS, ZC = 1, 2, 4, 8
CONTIG, INTERLEAVE = 0, 1

# Which path kinds can carry which direction on one GPU: the SM copy kernel moves
# device memory, the zero-copy kernel moves between mapped host memory and the
# device, copy engines and the two-hop staged route serve every direction.
ALLOWED_KINDS = {
    D2D: (CE, SM, HS),
    H2D: (CE, ZC, HS),
    D2H: (CE, ZC, HS),
}


class PathSpec(NamedTuple):
    kind: int
    share: int        # parts of 65536
    chunk_bytes: int  # C_p, a positive multiple of the alignment


class Chunk(NamedTuple):
    offset: int
    nbytes: int
    path_index: int
    chunk_index: int


def _is_pow2(x: int) -> bool:
    return x > 0 and (x & (x - 1)) == 0


def validate(nbytes: int, direction: int, specs, align: int, layout: int) -> None:
    """Raise ValueError when the request is not a plan the library must accept."""
    if not isinstance(nbytes, int) or nbytes < 0:
        raise ValueError("message size must be a non-negative integer")
    if direction not in ALLOWED_KINDS:
        raise ValueError("unknown direction")
    if layout not in (CONTIG, INTERLEAVE):
        raise ValueError("unknown layout")
    if not _is_pow2(align) or align > MAX_ALIGN:
        raise ValueError("alignment must be a power of two no larger than 4096")
    if not 1 <= len(specs) <= MAX_PATHS:
        raise ValueError("between 1 and 8 paths")
    total = 0
    for s in specs:
        if s.kind not in ALLOWED_KINDS[direction]:
            raise ValueError("path kind cannot carry this direction")
        if s.share <= 0:
            raise ValueError("every listed path needs a positive share")
        if s.chunk_bytes <= 0 or s.chunk_bytes % align != 0:
            raise ValueError("chunk size must be a positive multiple of the alignment")
        total += s.share
    if total != SHARE_ONE:
        raise ValueError("shares must sum to 65536")


def path_bytes(nbytes: int, specs, align: int) -> list[int]:
    """Horizontal split: bytes per path (Sec. 4.3; Algorithm 1's share[p])."""
    out = []
    given = 0
    for p, s in enumerate(specs):
        if p < len(specs) - 1:
            exact_floor = (nbytes * s.share) // SHARE_ONE
            b = (exact_floor // align) * align
        else:
            b = nbytes - given
        out.append(b)
        given += b
    return out


def plan(nbytes: int, direction: int, specs, align: int = 16, layout: int = CONTIG) -> list[Chunk]:
    """All chunks of the plan, sorted by (path_index, chunk_index)."""
    specs = [PathSpec(*s) for s in specs]
    validate(nbytes, direction, specs, align, layout)
    b = path_bytes(nbytes, specs, align)
    chunks: list[Chunk] = []
    if layout == CONTIG:
        start = 0
        for p, s in enumerate(specs):
            j = 0
            pos = 0
            while pos < b[p]:
                n = min(s.chunk_bytes, b[p] - pos)
                chunks.append(Chunk(start + pos, n, p, j))
                pos += n
                j += 1
            start += b[p]
    else:
        remaining = list(b)
        emitted = [0] * len(specs)
        last = len(specs) - 1
        held = None  # the one chunk whose length is not a multiple of A
        offset = 0
        while any(r > 0 for r in remaining):
            for p, s in enumerate(specs):
                if remaining[p] == 0:
                    continue
                n = min(s.chunk_bytes, remaining[p])
                remaining[p] -= n
                if p == last and remaining[p] == 0 and n % align != 0:
                    held = (n, p, emitted[p])
                else:
                    chunks.append(Chunk(offset, n, p, emitted[p]))
                    offset += n
                emitted[p] += 1
        if held is not None:
            n, p, j = held
            chunks.append(Chunk(offset, n, p, j))
            offset += n
        assert offset == nbytes
    chunks.sort(key=lambda c: (c.path_index, c.chunk_index))
    return chunks


def check_invariants(nbytes: int, specs, align: int, chunks) -> None:
    """Raise AssertionError unless the chunk list is a valid plan for these inputs.

    The checks restate Sec. 4.5's ordering guarantee (pre-assigned, non-overlapping
    regions that together make up the whole message) and the share/chunk contract:
    * every chunk is non-empty and starts on a multiple of A;
    * sorted by offset, the chunks tile [0, N) exactly: no gap, no overlap;
    * a path's chunk indices run 0..k-1 and every chunk but its last has C_p bytes;
    * path p < P-1 carries between its exact share minus A (exclusive) and its exact
      share; the last path carries its exact share plus less than (P-1)*A -- so each
      path is within one chunk of its share whenever C_p >= (P-1)*A.
    """
    specs = [PathSpec(*s) for s in specs]
    P = len(specs)
    for c in chunks:
        assert c.nbytes > 0, f"empty chunk {c}"
        assert c.offset % align == 0, f"misaligned chunk {c}"
        assert 0 <= c.path_index < P, f"bad path index {c}"
    pos = 0
    for c in sorted(chunks, key=lambda c: c.offset):
        assert c.offset == pos, f"gap or overlap at offset {pos}: {c}"
        pos += c.nbytes
    assert pos == nbytes, f"chunks end at {pos}, message has {nbytes} bytes"
    for p, s in enumerate(specs):
        mine = sorted((c for c in chunks if c.path_index == p), key=lambda c: c.chunk_index)
        assert [c.chunk_index for c in mine] == list(range(len(mine))), f"path {p} chunk indices"
        for c in mine[:-1]:
            assert c.nbytes == s.chunk_bytes, f"path {p}: inner chunk {c} is not C_p"
        got = sum(c.nbytes for c in mine)
        # compare 65536*got with N*w_p to stay in integers
        scaled_exact = nbytes * s.share
        scaled_got = got * SHARE_ONE
        if p < P - 1:
            assert scaled_got <= scaled_exact, f"path {p} exceeds its share"
            assert scaled_exact - scaled_got < align * SHARE_ONE, f"path {p} short by >= A"
        else:
            assert scaled_got >= scaled_exact, f"last path below its share"
            assert scaled_got - scaled_exact < max(1, P - 1) * align * SHARE_ONE or P == 1, \
                f"last path over its share by >= (P-1)*A"
            if P == 1:
                assert got == nbytes
        if s.chunk_bytes >= (P - 1) * align:
            assert abs(scaled_got - scaled_exact) <= s.chunk_bytes * SHARE_ONE, \
                f"path {p} not within one chunk of its share"
