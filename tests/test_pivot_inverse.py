"""The pivot-block solve's inverse form, checked on the CPU against the
oracle's own L_p (no GPU, no library code):

* appending row j of L_p appends row j of M = L_p^{-1} by
  M(j, c) = -( L(j, c) + sum_{c < i < j} L(j, i) M(i, c) ), the block inverse
  of [L 0; l^T 1]; built row by row this equals numpy's inverse of the whole
  L_p, and h = M u(p) equals the forward substitution L_p h = u(p) (scipy),
  which in turn equals the oracle's H columns (the sequential elimination of
  Algorithm 1);
* with max-|.| pivots every |L(i, c)| <= 1, and on the deblurring workloads
  (FP64 and BF16 storage) max |M| stays small, far below the 2^20 at which
  the solve switches to forward substitution.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from gen import problems as P
from oracle import operators as ops, scmrh, sketch as sk

GROWTH_SWITCH = 2.0 ** 20


def _inverse_by_rows(L):
    """M = L^{-1} for unit lower triangular L, one appended row at a time."""
    k1 = L.shape[0]
    M = np.eye(k1)
    for j in range(1, k1):
        for c in range(j):
            M[j, c] = -(L[j, c] + sum(L[j, i] * M[i, c] for i in range(c + 1, j)))
    return M


def _state(name, storage):
    p = P.make(name)
    A = ops.make_apply(p)
    S = sk.SparseSignSketch(p.sketch_seed, p.n, p.m_s, p.zeta)
    st = scmrh.run(A, p.b[0].astype(np.float64), S, p.k, storage=storage)
    return p, A, st


@pytest.mark.parametrize("storage", ["f64", "bf16"])
def test_rows_of_the_inverse_and_the_product(storage):
    p, A, st = _state("deblur64", storage)
    k = st.k_done
    piv = st.piv[:k + 1]
    L = st.V[piv, :k + 1]
    assert np.array_equal(np.diag(L), np.ones(k + 1)) and not np.triu(L, 1).any()
    M = _inverse_by_rows(L)
    assert np.allclose(M, np.linalg.inv(L), rtol=0, atol=1e-13)
    for j in (1, 5, 20, k - 1):
        u = A(st.V[:, j])[piv[:j + 1]]
        h_fwd = sla.solve_triangular(L[:j + 1, :j + 1], u, lower=True, unit_diagonal=True)
        h_inv = M[:j + 1, :j + 1] @ u
        assert np.allclose(h_inv, h_fwd, rtol=0, atol=1e-13 * np.abs(h_fwd).max())
        assert np.allclose(h_fwd, st.H[:j + 1, j], rtol=0, atol=1e-12 * np.abs(h_fwd).max())


@pytest.mark.parametrize("name,storage", [("deblur64", "f64"), ("deblur64", "bf16"), ("deblur256", "bf16")])
def test_inverse_stays_small_on_the_workloads(name, storage):
    p, A, st = _state(name, storage)
    k = st.k_done
    L = st.V[st.piv[:k + 1], :k + 1]
    assert np.abs(L).max() <= 1.0
    growth = np.abs(np.linalg.inv(L)).max()
    assert growth < 4.0 < GROWTH_SWITCH, growth
