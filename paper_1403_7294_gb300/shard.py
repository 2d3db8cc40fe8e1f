"""Splitting one text across ranks (host logic, no GPU needed).

A text of n bases is cut into `world` contiguous owned ranges of end
positions, aligned to 64 bases. A rank that owns [begin, end) needs the bases
[max(0, begin - (L_max - 1)), end): the state after reading position i only
depends on the last L_max bases (the deepest state has depth L_max), so
starting L_max - 1 bases early reproduces every occurrence ending in the
range. Occurrences are attributed to the rank that owns their end position,
so concatenating the ranks' results gives each occurrence exactly once and
summing their counts gives the counts of one scan. No exchange is needed
during the scan: the only collective is the final gather.
"""
from __future__ import annotations


def owned_range(n: int, world: int, rank: int, align: int = 64) -> tuple[int, int]:
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    units = (n + align - 1) // align
    lo_u = units * rank // world
    hi_u = units * (rank + 1) // world
    return min(n, lo_u * align), min(n, hi_u * align)


def read_window(begin: int, end: int, max_len: int) -> tuple[int, int]:
    """Bases a rank must hold to own end positions [begin, end)."""
    return max(0, begin - (max_len - 1)), end


def gather_occurrences(parts):
    """Concatenate per-rank (k, 3) [text_id, pos, pid] arrays into the canonical order."""
    import numpy as np

    parts = [p for p in parts if len(p)]
    if not parts:
        return np.zeros((0, 3), dtype=np.int64)
    a = np.concatenate(parts)
    return a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))]
