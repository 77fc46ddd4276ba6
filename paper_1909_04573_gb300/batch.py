"""Host-side planning for multi-camera workloads larger than device memory.

The fingerprint sums of Sec. III-A / III-B run over independent SDA groups, so a
camera's frames can be processed in several calls as long as no group is split
(each call accumulates whole groups into the camera's num/den).  plan_chunks
packs the cameras' groups, in order, into chunks of at most ``budget`` bytes of
frames; every chunk becomes one prnu_fingerprint_accumulate_multi call over
views of one reusable frame buffer.
"""
from __future__ import annotations

from dataclasses import dataclass

ALIGN = 256  # byte alignment of every piece inside the chunk buffer


@dataclass(frozen=True)
class Piece:
    """Frames f0..f1-1 of camera ``cam`` at byte ``offset`` of the chunk buffer."""
    cam: int
    f0: int
    f1: int
    offset: int


def _align(x: int) -> int:
    return (x + ALIGN - 1) // ALIGN * ALIGN


def plan_chunks(cams, budget: int):
    """cams: [(frame_bytes, m, d)].  Returns [[Piece]]: consecutive chunks,
    each holding runs of whole groups (a run starts at a multiple of d; the
    ragged last group ends at m) whose aligned sizes add up to at most
    ``budget`` bytes.  Every frame of every camera appears exactly once, in
    order.  Raises ValueError when one group does not fit the budget."""
    chunks, cur, used = [], [], 0
    for ci, (fb, m, d) in enumerate(cams):
        if fb < 1 or m < 1 or d < 1 or d > m:
            raise ValueError(f"camera {ci}: need frame_bytes, m, d >= 1 and d <= m")
        if _align(min(d, m) * fb) > budget:
            raise ValueError(f"camera {ci}: one group of {d} frames ({d * fb} B) exceeds the budget {budget} B")
        f = 0
        while f < m:
            room = budget - used
            # whole groups that fit, then the ragged tail if it is the last group
            f1 = min(m, f + max(0, room // (fb * d)) * d)
            if f1 == f and m - f < d and _align((m - f) * fb) <= room:
                f1 = m
            while f1 > f and _align((f1 - f) * fb) > room:  # alignment slack: drop one group
                f1 = f + ((f1 - f - 1) // d) * d
            if f1 == f:
                if not cur:
                    raise ValueError(f"camera {ci}: no group fits an empty chunk")
                chunks.append(cur)
                cur, used = [], 0
                continue
            cur.append(Piece(ci, f, f1, used))
            used += _align((f1 - f) * fb)
            f = f1
    if cur:
        chunks.append(cur)
    return chunks
