"""Pins for the oracle's sketch (Sec. 2: subspace embeddings, sparse sign
embeddings) against things other than itself: the published SplitMix64
check values, a scalar re-derivation of the bit layout with Python integers,
structural properties of the block sparse-sign matrix, and the embedding's
expected norm E||S x||^2 = ||x||^2."""
import os

import numpy as np
import pytest

from oracle import sketch as sk

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_ints(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [int(l) for l in f if l.strip() and not l.startswith("#")]


def test_splitmix64_published_check_values():
    want = _golden_ints("splitmix64_seed1234567.txt")
    got = sk.splitmix64_at(1234567, np.arange(len(want)))
    assert [int(v) for v in got] == want


def _scalar_rows_signs(seed, i, m_s, zeta):
    """Python-int restatement of the column layout (no numpy wrapping)."""
    M = (1 << 64) - 1
    W = (24 * zeta + 63) // 64
    bits = 0
    for w in range(W):
        z = (seed + 0x9E3779B97F4A7C15 * (W * i + w + 1)) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        z = z ^ (z >> 31)
        bits |= z << (64 * w)
    rows, signs = [], []
    for t in range(zeta):
        ch = (bits >> (24 * t)) & 0xFFFFFF
        lo = t * m_s // zeta
        hi = (t + 1) * m_s // zeta
        rows.append(lo + ((ch >> 1) * (hi - lo) >> 23))
        signs.append(-1.0 if ch & 1 else 1.0)
    return rows, signs


@pytest.mark.parametrize("zeta,m_s", [(8, 200), (8, 124), (3, 7), (16, 600), (1, 5)])
def test_sparse_sign_layout_matches_scalar_derivation(zeta, m_s):
    seed = 0xDEADBEEF12345
    cols = np.array([0, 1, 2, 77, 4095, 65535, 4194303, 2 ** 31 + 5], dtype=np.uint64)
    rows, signs = sk.sparse_sign_structure(seed, cols, m_s, zeta)
    for r, c in enumerate(cols):
        rr, ss = _scalar_rows_signs(seed, int(c), m_s, zeta)
        assert list(rows[r]) == rr
        assert list(signs[r]) == ss


def test_sparse_sign_structure_one_entry_per_block():
    m_s, zeta, n = 124, 8, 5000
    rows, signs = sk.sparse_sign_structure(99, np.arange(n), m_s, zeta)
    lo, size = sk.block_bounds(m_s, zeta)
    assert size.min() >= 1 and size.sum() == m_s
    for t in range(zeta):
        assert np.all(rows[:, t] >= lo[t]) and np.all(rows[:, t] < lo[t] + size[t])
    # distinct rows per column, unit column norm
    assert all(len(set(r)) == zeta for r in rows[:200])
    S = sk.SparseSignSketch(99, 300, m_s, zeta).matrix()
    assert np.allclose(np.linalg.norm(S, axis=0), 1.0, atol=1e-15)
    assert set(np.unique(np.abs(S[S != 0]))) == {1.0 / np.sqrt(zeta)}


def test_sparse_sign_rows_uniform_within_blocks():
    # chi-square on block 0: rows ~ uniform over its size
    m_s, zeta, n = 200, 8, 200000
    rows, signs = sk.sparse_sign_structure(7, np.arange(n), m_s, zeta)
    counts = np.bincount(rows[:, 0], minlength=25)[:25]
    expected = n / 25
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 70  # 24 dof; p ~ 3e-6 tail
    assert abs(signs.mean()) < 0.01


def test_sketch_apply_equals_dense_product():
    n, m_s = 257, 40
    S = sk.SparseSignSketch(12345, n, m_s, 8)
    x = np.random.default_rng(0).standard_normal(n)
    assert np.allclose(S.apply(x), S.matrix() @ x, rtol=0, atol=1e-13)
    # chunked application gives the same sums
    S2 = sk.SparseSignSketch(12345, n, m_s, 8, chunk=50)
    assert np.allclose(S2.apply(x), S.apply(x), rtol=0, atol=1e-13)


def test_sparse_sign_preserves_norm_in_expectation():
    """E ||S x||^2 = ||x||^2 for a sparse-sign embedding with +-1/sqrt(zeta)
    entries and independent signs (Sec. 2, Eq. 3 in expectation)."""
    n, m_s = 400, 64
    x = np.random.default_rng(1).standard_normal(n)
    ratios = [np.sum(sk.SparseSignSketch(s, n, m_s, 8).apply(x) ** 2) / np.sum(x ** 2)
              for s in range(400)]
    mean, sd = np.mean(ratios), np.std(ratios) / np.sqrt(len(ratios))
    assert abs(mean - 1.0) < 4 * sd + 1e-3


def test_gaussian_sketch_entries_are_n01_over_l():
    """Box-Muller on the counter hash: entries N(0, 1/l) — mean, variance,
    kurtosis within CLT bands and a Kolmogorov-Smirnov test on l * n = 400k
    entries; a different seed gives an uncorrelated matrix."""
    from scipy import stats
    l, n = 100, 4000
    S = sk.GaussianSketch(2024, n, l).matrix()
    z = S.ravel() * np.sqrt(l)
    N = z.size
    assert abs(z.mean()) < 5 / np.sqrt(N)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / N)
    assert abs(stats.kurtosis(z)) < 5 * np.sqrt(24.0 / N)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    z2 = sk.GaussianSketch(2025, n, l).matrix().ravel() * np.sqrt(l)
    assert abs(np.corrcoef(z, z2)[0, 1]) < 5 / np.sqrt(N)


def test_gaussian_sketch_is_an_embedding_in_expectation():
    """E||S x||^2 = ||x||^2 (Eq. 3 in expectation) over seeds."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal(300)
    vals = [np.linalg.norm(sk.GaussianSketch(s, 300, 40).apply(x)) ** 2 for s in range(300)]
    # ||Sx||^2 / ||x||^2 ~ chi^2_l / l: mean 1, sd sqrt(2/l)
    ratio = np.array(vals) / np.dot(x, x)
    assert abs(ratio.mean() - 1.0) < 4 * np.sqrt(2.0 / 40) / np.sqrt(300)


def test_gaussian_sketch_entries_match_matrix():
    """The per-entry evaluation gives the matrix's entries (same definition,
    used to check samples of sketches too large to form)."""
    l, n = 30, 500
    rng = np.random.default_rng(4)
    rows, cols = rng.integers(0, l, 300), rng.integers(0, n, 300)
    for storage in ("f64", "bf16", "f16"):
        S = sk.GaussianSketch(77, n, l, storage).matrix()
        e = sk.GaussianSketch.entries(77, n, l, rows, cols, storage)
        assert np.array_equal(e, S[rows, cols])


def test_round_to_bf16_is_rne():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.140625, 1e-30])
    r = sk.round_to(v, "bf16")
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7 and r[3] == -3.140625
    assert abs(r[4] - 1e-30) <= 2 ** -8 * 1e-30
