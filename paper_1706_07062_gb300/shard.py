"""Splitting one image's rays across processes (one per GPU) and putting the
outputs back together.

Geodesics are independent (Sec. 2.3: the paper's rays are trivially
parallel), so a multi-GPU run is a set of replicas that each trace their own
share of the pixels; the only exchange is the host-side concatenation of the
outputs.  Shares are whole image rows: row q goes to rank q mod world
("interleaved": every rank gets rows from the top, the shadow and the bottom
of the image, so the expensive rays near the critical curve are spread
evenly) or rows come in contiguous blocks ("contiguous").  Host logic only;
the tracing itself is the library's kerr_trace_camera_pixels.
"""
from __future__ import annotations

import numpy as np


def row_partition(nx: int, ny: int, world: int, rank: int,
                  mode: str = "interleaved") -> np.ndarray:
    """Flat pixel indices (q * nx + p, ascending) of rank `rank`'s rows."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    if mode == "interleaved":
        rows = np.arange(rank, ny, world, dtype=np.int64)
    elif mode == "contiguous":
        bounds = np.linspace(0, ny, world + 1).round().astype(np.int64)
        rows = np.arange(bounds[rank], bounds[rank + 1], dtype=np.int64)
    else:
        raise ValueError(f"unknown partition mode {mode!r}")
    return (rows[:, None] * nx + np.arange(nx, dtype=np.int64)[None, :]).ravel()


def concat(parts, indices, n: int) -> np.ndarray:
    """Reassemble per-rank outputs: parts[r] holds, along its last axis, the
    values of the pixels indices[r]; returns the image-ordered array with
    last axis n.  Raises unless the indices tile 0 .. n-1 exactly once."""
    idx = np.concatenate([np.asarray(i, dtype=np.int64) for i in indices])
    if idx.size != n or not np.array_equal(np.sort(idx), np.arange(n)):
        raise ValueError("the shares do not tile the image exactly once")
    first = np.asarray(parts[0])
    out = np.empty(first.shape[:-1] + (n,), dtype=first.dtype)
    for part, i in zip(parts, indices):
        out[..., np.asarray(i, dtype=np.int64)] = np.asarray(part)
    return out
