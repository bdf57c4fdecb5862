"""Sampled pivoting for the oracle.  Test infrastructure only.

Sec. 3.2 (after Algorithm 1) and Sec. 4: instead of locating the largest
magnitude of the whole vector (a global reduction), the pivot is the entry of
largest magnitude in a small random sample of the candidate entries; the
experiments use samples of 5 and 25 entries.

Reading (the paper gives no sampling rule): for pivot choice number c of a
basis (c = 0 at the initialisation, c = j + 1 when step j picks p_{j+1}) and
sampling seed s, draw t = 0, 1, 2, ... is SplitMix64 output number
c * 4096 + t of the generator started at s (the same counter hash as the
sketch, see sketch.py), and its index is floor(out * n / 2^64).  A draw that
hits a pivot row or an index already drawn for this choice is discarded; the
first `size` accepted indices form the sample.  If no more than `size`
candidates remain, the sample is all of them; draws stop after 4096.  The
pivot is the sampled index of largest |value|, lowest index on ties; if every
sampled value is zero (or nothing was accepted) the full maximum over the
candidates is used, so a nonzero vector always gives a nonzero pivot.
"""
from __future__ import annotations

import numpy as np

from .sketch import splitmix64_at

SAMPLE_SEED_XOR = 0xA5A5A5A5A5A5A5A5
MAX_DRAWS = 4096


def sample_indices(seed: int, choice: int, n: int, size: int, is_piv: np.ndarray) -> list:
    """The accepted sample of pivot choice `choice` (list of row indices)."""
    remaining = int(n - np.count_nonzero(is_piv))
    if remaining <= size:
        return [int(i) for i in np.flatnonzero(~is_piv)]
    outs = splitmix64_at(seed, np.arange(MAX_DRAWS, dtype=np.uint64) + np.uint64(choice * MAX_DRAWS))
    taken = []
    seen = set()
    for out in outs:
        idx = (int(out) * n) >> 64
        if is_piv[idx] or idx in seen:
            continue
        seen.add(idx)
        taken.append(idx)
        if len(taken) == size:
            break
    return taken


def sampled_pivot(vec: np.ndarray, is_piv: np.ndarray, seed: int, choice: int, size: int) -> int:
    """Pivot row under sampled pivoting (see the module docstring)."""
    cand = sample_indices(seed, choice, vec.size, size, is_piv)
    best, best_abs = -1, 0.0
    for idx in sorted(cand):                       # ascending: lowest index wins ties
        a = abs(float(vec[idx]))
        if a > best_abs:
            best, best_abs = idx, a
    if best >= 0:
        return best
    a = np.where(is_piv, -1.0, np.abs(vec))
    return int(np.argmax(a))
