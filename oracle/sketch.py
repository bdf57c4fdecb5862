"""Sketching matrices S (l x n) for the oracle.

Sec. 2 of the paper introduces oblivious subspace embeddings S with
(1-eps)||a|| <= ||S a|| <= (1+eps)||a|| (Eq. 3) and names sparse sign
embeddings among the structured choices; the experiments use Gaussian
embeddings with entries N(0, 1/l).

SparseSignSketch is the block sparse-sign embedding used by the library:
column i of S has exactly one nonzero, +-1/sqrt(zeta), in each of zeta
disjoint row blocks (so zeta distinct rows), row and sign drawn from a
SplitMix64 counter hash (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014):

    SM(seed, c) = mix(seed + GAMMA * (c + 1))     (mod 2^64)
    mix(z):  z = (z ^ (z >> 30)) * C1;  z = (z ^ (z >> 27)) * C2;  z ^ (z >> 31)

i.e. output number c of the SplitMix64 sequence started from state ``seed``.
Column i reads W = ceil(24*zeta/64) consecutive outputs, c = W*i .. W*i+W-1,
as one little-endian bit string; bits [24t, 24t+24) are chunk t:
    sign_t = chunk & 1 (1 means negative),  r = chunk >> 1  (23 bits)
    block t = rows [lo_t, hi_t), lo_t = floor(t*l/zeta)
    row_t   = lo_t + floor(r * (hi_t - lo_t) / 2^23)

IdentitySketch (S = I) and DenseSketch (any explicit matrix, e.g. a Gaussian
embedding drawn by a test) let the same oracle reduce to GMRES and to the
Gaussian sketch-and-solve statements of Sec. 3.2.
"""
from __future__ import annotations

import numpy as np

from .storage import round_to  # noqa: F401  (S is kept in the basis storage type)

GAMMA = 0x9E3779B97F4A7C15
C1 = 0xBF58476D1CE4E5B9
C2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1


def splitmix64_mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(C1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(C2)
        return z ^ (z >> np.uint64(31))


def splitmix64_at(seed: int, counters: np.ndarray) -> np.ndarray:
    """Output number ``counters`` (0-based) of SplitMix64 started at ``seed``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & MASK64) + np.uint64(GAMMA) * (c + np.uint64(1))
    return splitmix64_mix(state)


def words_per_column(zeta: int) -> int:
    return (24 * zeta + 63) // 64


def block_bounds(m_s: int, zeta: int):
    t = np.arange(zeta + 1, dtype=np.int64)
    edges = (t * m_s) // zeta
    return edges[:-1], edges[1:] - edges[:-1]


def sparse_sign_structure(seed: int, cols: np.ndarray, m_s: int, zeta: int):
    """Rows (len(cols), zeta) int64 and signs (len(cols), zeta) in {+1, -1}."""
    if not (1 <= zeta <= 16) or m_s < zeta:
        raise ValueError("need 1 <= zeta <= 16 and m_s >= zeta")
    cols = np.asarray(cols, dtype=np.uint64)
    W = words_per_column(zeta)
    ctr = cols[:, None] * np.uint64(W) + np.arange(W, dtype=np.uint64)[None, :]
    words = splitmix64_at(seed, ctr)                      # (ncol, W) uint64
    lo, size = block_bounds(m_s, zeta)
    rows = np.empty((cols.size, zeta), dtype=np.int64)
    signs = np.empty((cols.size, zeta), dtype=np.float64)
    for t in range(zeta):
        bit = 24 * t
        w0, off = bit // 64, bit % 64
        chunk = words[:, w0] >> np.uint64(off)
        if off + 24 > 64:                                  # straddles two words
            chunk = chunk | (words[:, w0 + 1] << np.uint64(64 - off))
        chunk = chunk & np.uint64(0xFFFFFF)
        neg = (chunk & np.uint64(1)).astype(bool)
        r = (chunk >> np.uint64(1)).astype(np.int64)
        rows[:, t] = lo[t] + ((r * size[t]) >> 23)
        signs[:, t] = np.where(neg, -1.0, 1.0)
    return rows, signs


class SparseSignSketch:
    """Block sparse-sign embedding S (m_s x n), never stored densely."""

    def __init__(self, seed: int, n: int, m_s: int, zeta: int = 8, chunk: int = 1 << 20):
        self.seed, self.n, self.m, self.zeta, self.chunk = int(seed), int(n), int(m_s), int(zeta), chunk

    def apply(self, x: np.ndarray) -> np.ndarray:
        """S @ x for a length-n vector (float64 sums)."""
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros(self.m)
        for s in range(0, self.n, self.chunk):
            e = min(self.n, s + self.chunk)
            rows, signs = sparse_sign_structure(self.seed, np.arange(s, e), self.m, self.zeta)
            out += np.bincount(rows.ravel(), weights=(signs * x[s:e, None]).ravel(),
                               minlength=self.m)
        return out / np.sqrt(self.zeta)

    def matrix(self) -> np.ndarray:
        """Dense S (tiny n only)."""
        S = np.zeros((self.m, self.n))
        rows, signs = sparse_sign_structure(self.seed, np.arange(self.n), self.m, self.zeta)
        for t in range(self.zeta):
            S[rows[:, t], np.arange(self.n)] = signs[:, t] / np.sqrt(self.zeta)
        return S


class GaussianSketch:
    """Gaussian embedding S (l x n) with N(0, 1/l) entries (Sec. 2; the
    experiments of Sec. 4 use it), drawn from the SplitMix64 counter hash by
    the Box-Muller transform (Box & Muller, Ann. Math. Stat. 1958): entry
    (r, i) takes outputs 2c and 2c + 1, c = r*n + i, of the generator started
    at ``seed``; u = ((out >> 11) + 1) * 2^-53 lies in (0, 1];
    z = sqrt(-2 ln u_1) cos(2 pi u_2); S[r, i] = z / sqrt(l).  ``storage``
    rounds the entries to the type the library keeps S in."""

    def __init__(self, seed: int, n: int, m_s: int, storage: str = "f64"):
        self.seed, self.n, self.m = int(seed), int(n), int(m_s)
        c = np.arange(self.m * self.n, dtype=np.uint64)
        o1 = splitmix64_at(self.seed, 2 * c)
        o2 = splitmix64_at(self.seed, 2 * c + np.uint64(1))
        u1 = ((o1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        u2 = ((o2 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
        self.S = round_to((z / np.sqrt(self.m)).reshape(self.m, self.n), storage)

    @staticmethod
    def entries(seed: int, n: int, m_s: int, rows, cols, storage: str = "f64") -> np.ndarray:
        """S[rows[t], cols[t]] by the same definition, for a few entries of a
        sketch too large to form."""
        r = np.asarray(rows, dtype=np.uint64)
        i = np.asarray(cols, dtype=np.uint64)
        c = r * np.uint64(n) + i
        o1 = splitmix64_at(int(seed), 2 * c)
        o2 = splitmix64_at(int(seed), 2 * c + np.uint64(1))
        u1 = ((o1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        u2 = ((o2 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
        return round_to(z / np.sqrt(int(m_s)), storage)

    def apply(self, x):
        return self.S @ np.asarray(x, dtype=np.float64)

    def matrix(self):
        return self.S


class IdentitySketch:
    """S = I: the sketched problem is the unsketched one."""

    def __init__(self, n: int):
        self.n = self.m = int(n)

    def apply(self, x):
        return np.array(x, dtype=np.float64, copy=True)

    def matrix(self):
        return np.eye(self.n)


class DenseSketch:
    """An explicit sketch matrix supplied by the caller (e.g. Gaussian N(0, 1/l))."""

    def __init__(self, S: np.ndarray):
        self.S = np.asarray(S, dtype=np.float64)
        self.m, self.n = self.S.shape

    def apply(self, x):
        return self.S @ np.asarray(x, dtype=np.float64)

    def matrix(self):
        return self.S
