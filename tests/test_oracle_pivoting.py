"""Pins for sampled pivoting (Sec. 3.2 and Sec. 4; oracle/pivoting.py):

* a sample that covers every candidate reduces to full max-|.| pivoting, so
  the whole run equals the full-pivoting run;
* samples are distinct, never pivot rows, and their first draws are uniform
  over the rows (chi-square over many choices);
* the processes keep their defining relations (Eq. Hessenberg_s and Eq.
  Hessenberg_r, unit lower trapezoidal bases) under sampled pivots, and the
  pivot is the largest sampled magnitude;
* a sampled pivot is never zero while the vector is nonzero.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import pivoting, scmrh, slslu, sketch as sk


def _rand_system(n, seed):
    rng = np.random.default_rng(seed)
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    return A, rng.standard_normal(n)


def test_full_sample_is_full_pivoting():
    A, b = _rand_system(24, 1)
    S = sk.SparseSignSketch(3, 24, 20, 8)
    full = scmrh.run(lambda v: A @ v, b, S, 12)
    smp = scmrh.run(lambda v: A @ v, b, S, 12, pivot_sample=24, pivot_seed=99)
    assert smp.piv == full.piv
    assert np.array_equal(smp.V, full.V)


def test_samples_distinct_exclude_pivots_and_uniform():
    n, size = 50, 5
    is_piv = np.zeros(n, dtype=bool)
    is_piv[[3, 17, 40]] = True
    firsts = []
    for c in range(4000):
        smp = pivoting.sample_indices(12345, c, n, size, is_piv)
        assert len(smp) == size and len(set(smp)) == size
        assert not any(is_piv[i] for i in smp)
        firsts.append(smp[0])
    counts = np.bincount(firsts, minlength=n)[~is_piv]
    _, pval = stats.chisquare(counts)
    assert pval > 1e-4


def test_sampled_scmrh_keeps_relation_and_picks_sampled_max():
    A, b = _rand_system(60, 2)
    S = sk.SparseSignSketch(5, 60, 40, 8)
    seed, size = 777, 5
    st = scmrh.run(lambda v: A @ v, b, S, 20, pivot_sample=size, pivot_seed=seed)
    k = st.k_done
    V, H = st.V, st.H
    res = np.linalg.norm(A @ V[:, :k] - V @ H) / (np.linalg.norm(A, 2) * np.linalg.norm(V[:, :k], 2))
    assert res < 1e-13
    for i, p in enumerate(st.piv):
        assert V[p, i] == 1.0 and np.all(V[p, i + 1:] == 0.0)
    # replay: each pivot is the largest magnitude of its sample
    full = scmrh.run(lambda v: A @ v, b, S, 20, forced_pivots=st.piv)
    assert full.piv == st.piv
    is_piv = np.zeros(60, dtype=bool)
    u0 = b.copy()
    cand = pivoting.sample_indices(seed, 0, 60, size, is_piv)
    assert st.piv[0] == max(sorted(cand), key=lambda i: abs(u0[i]))
    # with only 5 of 60 entries sampled the run differs from full pivoting
    assert st.piv != scmrh.run(lambda v: A @ v, b, S, 20).piv


def test_sampled_slslu_keeps_relations():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((50, 30)) / np.sqrt(50)
    A[:30, :30] += np.eye(30)
    b = rng.standard_normal(50)
    st = slslu.run(lambda v: A @ v, lambda v: A.T @ v, b, sk.SparseSignSketch(1, 30, 40, 8),
                   sk.SparseSignSketch(2, 50, 40, 8), 12, pivot_sample=25, pivot_seeds=(31, 32))
    k = st.k_done
    nA = np.linalg.norm(A, 2)
    assert np.linalg.norm(A @ st.L[:, :k] - st.D @ st.H) / (nA * np.linalg.norm(st.L[:, :k], 2)) < 1e-13
    assert np.linalg.norm(A.T @ st.D - st.L @ st.W) / (nA * np.linalg.norm(st.D, 2)) < 1e-13


def test_sampled_pivot_is_nonzero_for_nonzero_vector():
    n = 100
    v = np.zeros(n)
    v[37] = 1e-3                                 # one nonzero, almost surely outside a 5-sample
    is_piv = np.zeros(n, dtype=bool)
    hits = 0
    for c in range(50):
        p = pivoting.sampled_pivot(v, is_piv, 4242, c, 5)
        assert v[p] != 0.0
        hits += 37 in pivoting.sample_indices(4242, c, n, 5, is_piv)
    assert hits < 50                             # the full-max fallback was exercised
