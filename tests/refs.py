"""Independent test-side derivations used to pin the oracle (no code shared with oracle/ or the CUDA path).

``closed_schedule`` enumerates the retained points of the quasi-logarithmic history grid (Sec. III of
arXiv:1504.06123) from closed-form block counts instead of simulating the block-merge rule, so that a
mistake in the oracle's recursive insertion shows up as a mismatch.
"""
from __future__ import annotations

import numpy as np


def block_counts(C: int, B: int, t: int) -> dict:
    """Points held by block b (1 = coarsest .. B = finest) after step t >= 0.

    Blocks start full.  Block B receives a point every step, block b < B every 2^(B-b) steps (each
    time block b+1 merges); a receiving block b >= 2 that is full hands its two oldest points on, so
    its count alternates C-1 (after an even-numbered receipt) and C.  Block 1 stays full.
    """
    counts = {}
    for b in range(1, B + 1):
        if b == 1:
            counts[b] = C
        else:
            r = t >> (B - b)          # index of the latest receipt
            counts[b] = C - 1 if r % 2 == 0 else C
    return counts


def closed_schedule(C: int, B: int, t: int):
    """(t', span, block, weight) of every retained point after step t, newest first.

    Within block b the points are 2^(B-b) apart, and the gap from the oldest point of block b+1 to the
    newest of block b is 2^(B-b) as well.  The trapezoidal weight is the mean of the two neighbouring
    gaps (one-sided at both ends of the grid).
    """
    counts = block_counts(C, B, t)
    pts = []
    age = 0
    for b in range(B, 0, -1):
        sp = 1 << (B - b)
        for k in range(counts[b]):
            if pts:
                age += sp
            pts.append([t - age, sp, b])
    ages = np.array([t - p[0] for p in pts], dtype=float)
    n = len(pts)
    out = []
    for k in range(n):
        gap_lo = ages[k] - ages[k - 1] if k > 0 else 0.0
        gap_hi = ages[k + 1] - ages[k] if k < n - 1 else 0.0
        out.append((pts[k][0], pts[k][1], pts[k][2], 0.5 * (gap_lo + gap_hi)))
    return out
