"""Pins for the oracle's sLSLU (Sec. 3, Algorithm 1 and Algorithm 2) against
facts fixed by the paper and by mathematics:

* Eq. (Hessenberg_r): A L_k = D_{k+1} H_{k+1,k} and A^T D_{k+1} = L_{k+1} W_{k+1}
  with W upper triangular; D and L unit lower trapezoidal under their pivot
  orders, |D|, |L| <= 1 under max-|.| pivoting.
* Sec. 3.1: range(L_k) = K_k(A^T A, A^T b).  With S_1 = S_2 = I the sketched
  problem is the minimal-residual (and Tikhonov) problem over that space, i.e.
  the LSQR iterate; checked against an orthonormal basis of the Krylov space
  built independently (power matrix + QR) and against Golub-Kahan
  bidiagonalisation.
* k = n, S = I: the dense least-squares / Tikhonov solutions.
* Eq. (eqthm) with M = D_{k+1}: ||r_LS|| <= ||r_LSLU|| <= kappa(D_{k+1}) ||r_LS||,
  and ||r_LS|| <= ||r_S|| for any sketch.
"""
import numpy as np
import pytest

from oracle import slslu, sketch as sk


def _rand_rect(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) / np.sqrt(m)
    A[:n, :n] += np.eye(n)
    b = rng.standard_normal(m)
    return A, b


def _run(A, b, k, S1=None, S2=None):
    m, n = A.shape
    S1 = S1 or sk.IdentitySketch(n)
    S2 = S2 or sk.IdentitySketch(m)
    return slslu.run(lambda v: A @ v, lambda v: A.T @ v, b, S1, S2, k)


def _krylov_basis(A, b, k):
    """Orthonormal basis of K_k(A^T A, A^T b): power vectors, each scaled, then QR."""
    v = A.T @ b
    cols = []
    for _ in range(k):
        cols.append(v / np.linalg.norm(v))
        v = A.T @ (A @ cols[-1])
    Q, _ = np.linalg.qr(np.stack(cols, axis=1))
    return Q


def _golub_kahan(A, b, k):
    """k steps of Golub-Kahan bidiagonalisation with full reorthogonalisation;
    returns the LSQR iterate x_k = V_k argmin ||beta e_1 - B_k y||."""
    m, n = A.shape
    U = np.zeros((m, k + 1))
    V = np.zeros((n, k))
    B = np.zeros((k + 1, k))
    beta = np.linalg.norm(b)
    U[:, 0] = b / beta
    for j in range(k):
        v = A.T @ U[:, j] - (B[j, j - 1] * V[:, j - 1] if j > 0 else 0.0)
        v -= V[:, :j] @ (V[:, :j].T @ v)
        B[j, j] = np.linalg.norm(v)
        V[:, j] = v / B[j, j]
        u = A @ V[:, j] - B[j, j] * U[:, j]
        u -= U[:, :j + 1] @ (U[:, :j + 1].T @ u)
        B[j + 1, j] = np.linalg.norm(u)
        U[:, j + 1] = u / B[j + 1, j]
    rhs = np.zeros(k + 1)
    rhs[0] = beta
    y = np.linalg.lstsq(B, rhs, rcond=None)[0]
    return V @ y


def test_generalized_hessenberg_relations_and_trapezoids():
    A, b = _rand_rect(50, 30, 3)
    st = _run(A, b, 12, sk.SparseSignSketch(7, 30, 40, 8), sk.SparseSignSketch(8, 50, 40, 8))
    k = st.k_done
    assert k == 12 and not st.breakdown and st.l_done == 13
    D, L, H, W = st.D, st.L, st.H, st.W
    nA = np.linalg.norm(A, 2)
    r1 = np.linalg.norm(A @ L[:, :k] - D @ H) / (nA * np.linalg.norm(L[:, :k], 2))
    r2 = np.linalg.norm(A.T @ D - L @ W) / (nA * np.linalg.norm(D, 2))
    assert r1 < 1e-13 and r2 < 1e-13, (r1, r2)
    assert np.all(np.tril(W, -1) == 0.0)
    assert np.all(np.tril(H, -2) == 0.0)
    for M, piv in ((D, st.pt), (L, st.pg)):
        for i, p in enumerate(piv):
            assert M[p, i] == 1.0 and np.all(M[p, i + 1:] == 0.0)
        assert np.max(np.abs(M)) <= 1.0
        assert len(set(piv)) == len(piv)
    # the first column of W is the pivot entry of A^T d_1, i.e. alpha / beta
    assert abs(W[0, 0] - st.alpha / st.beta) <= 1e-14 * abs(W[0, 0])


@pytest.mark.parametrize("k", [1, 3, 7, 12])
def test_identity_sketches_give_lsqr(k):
    A, b = _rand_rect(40, 25, 11)
    st = _run(A, b, 12)
    x = slslu.solve(st, k)
    Q = _krylov_basis(A, b, k)
    x_ref = Q @ np.linalg.lstsq(A @ Q, b, rcond=None)[0]
    x_gk = _golub_kahan(A, b, k)
    assert np.linalg.norm(x_ref - x_gk) <= 1e-8 * np.linalg.norm(x_gk)
    assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref), k


@pytest.mark.parametrize("lam", [0.05, 0.5])
def test_identity_sketches_give_projected_tikhonov(lam):
    A, b = _rand_rect(40, 25, 12)
    k = 9
    st = _run(A, b, k)
    x = slslu.solve(st, k, lam)
    Q = _krylov_basis(A, b, k)
    M = np.vstack([A @ Q, lam * Q])
    y = np.linalg.lstsq(M, np.concatenate([b, np.zeros(Q.shape[0])]), rcond=None)[0]
    x_ref = Q @ y
    assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)


@pytest.mark.parametrize("shape", [(20, 20), (30, 20)])
@pytest.mark.parametrize("lam", [0.0, 0.3])
def test_full_dimension_is_dense_solution(shape, lam):
    m, n = shape
    A, b = _rand_rect(m, n, 21)
    st = _run(A, b, n)
    assert st.k_done == n or st.breakdown
    k = min(st.k_done, st.l_done)
    x = slslu.solve(st, k, lam)
    x_ref = np.linalg.solve(A.T @ A + lam ** 2 * np.eye(n), A.T @ b)
    assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)


def test_residual_inequalities():
    A, b = _rand_rect(60, 40, 5)
    S1, S2 = sk.SparseSignSketch(31, 40, 48, 8), sk.SparseSignSketch(32, 60, 48, 8)
    st = _run(A, b, 10, S1, S2)
    for k in (2, 5, 10):
        Q = _krylov_basis(A, b, k)
        r_ls = np.linalg.norm(A @ (Q @ np.linalg.lstsq(A @ Q, b, rcond=None)[0]) - b)
        r_s = np.linalg.norm(A @ slslu.solve(st, k) - b)
        r_lslu = np.linalg.norm(A @ slslu.lslu_solve(st, k) - b)
        kappa = np.linalg.cond(st.D[:, :k + 1])
        assert r_ls <= r_s * (1 + 1e-12)
        assert r_ls <= r_lslu * (1 + 1e-12) and r_lslu <= kappa * r_ls * (1 + 1e-12)


def test_breakdown_gives_exact_solution():
    # A block diagonal and b supported on its 3 x 3 block: after three steps
    # every row of that block is a pivot row, so the elimination leaves u = 0
    # exactly, H(4,3) = 0 (the algorithm's stopping branch) and the iterate
    # solves the system
    rng = np.random.default_rng(4)
    A = np.zeros((12, 12))
    A[:3, :3] = rng.standard_normal((3, 3)) + 2 * np.eye(3)
    A[3:, 3:] = rng.standard_normal((9, 9)) + 2 * np.eye(9)
    b = np.zeros(12)
    b[:3] = rng.standard_normal(3)
    st = _run(A, b, 8)
    assert st.breakdown and st.k_done == 3 and st.H[3, 2] == 0.0
    x = slslu.solve(st, 3)
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)
