"""Pins for the oracle's sCMRH (Sec. 3) against facts fixed by the paper and
by mathematics, none of them a retyping of the oracle's own formulas:

* Eq. (Hessenberg_s): A V_k = V_{k+1} H_k, V unit lower trapezoidal under the
  pivot order, |V| <= 1 under max-|.| pivoting.
* Sec. 1: the basis is the L factor of LU with partial pivoting of the Krylov
  matrix [b, Ab, ..., A^{k-1} b] (scipy's getrf as the library check).
* Sec. 3.2 with S = I: the sketched problem is the minimal-residual problem
  over K_k(A, b), i.e. GMRES (independent Arnoldi/MGS implementation).
* k = n, S = I: the dense least-squares / Tikhonov solutions (Eq. 2, Eq. 3).
* Eq. (eqthm) and the left inequality of Eq. (eqthm2): deterministic bounds.
* Sec. 3.2, Gaussian sketch: E[x_S] = x_LS and
  E||r_S||^2 = (1 + k/(l-k-1)) min ||r||^2 (Monte Carlo, 3-4 sigma bands).
* Breakdown (Algorithm 1, H(k+1,k) = 0 branch): exact solution in K_k.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from gen import problems as P
from oracle import gmres, operators as ops, scmrh, sketch as sk


def _rand_system(n, seed, shift=1.0, scale=0.3):
    rng = np.random.default_rng(seed)
    A = shift * np.eye(n) + scale * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    return A, b


def test_hessenberg_relation_and_trapezoid_random():
    A, b = _rand_system(40, 1)
    st = scmrh.run(lambda v: A @ v, b, sk.SparseSignSketch(5, 40, 32, 8), 15)
    k = st.k_done
    assert k == 15 and not st.breakdown
    V, H = st.V, st.H
    res = np.linalg.norm(A @ V[:, :k] - V @ H) / (np.linalg.norm(A, 2) * np.linalg.norm(V[:, :k], 2))
    assert res < 1e-13
    for i, p in enumerate(st.piv):
        assert V[p, i] == 1.0
        assert np.all(V[p, i + 1:] == 0.0)
    assert np.max(np.abs(V)) <= 1.0
    assert len(set(st.piv)) == len(st.piv)


def test_hessenberg_relation_deblur64():
    p = P.make("deblur64")
    A = ops.make_apply(p)
    st = scmrh.run(A, p.b[0], sk.SparseSignSketch(p.sketch_seed, p.n, p.m_s, p.zeta), p.k)
    k = st.k_done
    AV = np.stack([A(st.V[:, j]) for j in range(k)], axis=1)
    assert np.linalg.norm(AV - st.V @ st.H) / np.linalg.norm(AV) < 1e-13
    assert np.max(np.abs(st.V)) <= 1.0
    # the two forms of S A V_k agree in exact-ish arithmetic
    Zh = scmrh.projected_matrix(st, k, "hessenberg")
    Zd = scmrh.projected_matrix(st, k, "direct")
    assert np.linalg.norm(Zh - Zd) / np.linalg.norm(Zd) < 1e-12


def test_basis_is_lu_factor_of_krylov_matrix():
    n, k = 12, 6
    A, b = _rand_system(n, 2, shift=0.5, scale=1.0)
    K = np.stack([np.linalg.matrix_power(A, j) @ b for j in range(k)], axis=1)
    Pm, L, U = sla.lu(K)                       # K = Pm L U, L unit lower trapezoid
    lu_piv = [int(np.argmax(Pm[:, c])) for c in range(k)]
    st = scmrh.run(lambda v: A @ v, b, sk.IdentitySketch(n), k)
    assert st.piv[:k] == lu_piv
    assert np.allclose(st.V[:, :k], Pm @ L, atol=1e-10)


def test_identity_sketch_reproduces_gmres():
    n = 30
    A, b = _rand_system(n, 3)
    xs = gmres.gmres_iterates(A, b, 10)
    st = scmrh.run(lambda v: A @ v, b, sk.IdentitySketch(n), 10)
    for k, xg in enumerate(xs, start=1):
        x = scmrh.solve(st, k)
        assert np.linalg.norm(x - xg) / np.linalg.norm(xg) < 1e-10


def test_gmres_full_dimension_is_solve():
    n = 10
    A, b = _rand_system(n, 4)
    xs = gmres.gmres_iterates(A, b, n)
    assert np.allclose(xs[-1], np.linalg.solve(A, b), atol=1e-10)


@pytest.mark.parametrize("lam", [0.0, 0.3, 2.0])
def test_full_dimension_identity_sketch_is_dense_solution(lam):
    n = 14
    A, b = _rand_system(n, 5)
    st = scmrh.run(lambda v: A @ v, b, sk.IdentitySketch(n), n)
    assert st.k_done == n
    x = scmrh.solve(st, n, lam)
    want = np.linalg.solve(A.T @ A + lam ** 2 * np.eye(n), A.T @ b)
    assert np.allclose(x, want, rtol=0, atol=1e-10 * np.linalg.norm(want))


def test_penalty_on_y_matches_eq_tsp_form():
    """penalty 'y' solves min ||c - Z y||^2 + lam^2 ||y||^2 (Eq. TSP's penalty)."""
    n, k, lam = 20, 6, 0.7
    A, b = _rand_system(n, 6)
    st = scmrh.run(lambda v: A @ v, b, sk.IdentitySketch(n), k)
    y = scmrh.solve_y(st, k, lam, penalty="y")
    Z = A @ st.V[:, :k]
    want = np.linalg.solve(Z.T @ Z + lam ** 2 * np.eye(k), Z.T @ b)
    assert np.allclose(y, want, atol=1e-10)


def test_residual_inequalities():
    n, k = 60, 8
    A, b = _rand_system(n, 7, shift=1.0, scale=0.8)
    r = lambda x: np.linalg.norm(b - A @ x)
    st_I = scmrh.run(lambda v: A @ v, b, sk.IdentitySketch(n), k)
    x_ls = scmrh.solve(st_I, k)
    x_cm = scmrh.cmrh_solve(st_I, k)
    kappa = np.linalg.cond(st_I.V[:, :k + 1])
    assert r(x_ls) <= r(x_cm) * (1 + 1e-12)
    assert r(x_cm) <= kappa * r(x_ls) * (1 + 1e-12)
    for seed in range(10):
        st = scmrh.run(lambda v: A @ v, b, sk.SparseSignSketch(seed, n, 4 * k, 8), k)
        assert r(x_ls) <= r(scmrh.solve(st, k)) * (1 + 1e-12)


def test_gaussian_sketch_unbiased_and_expected_residual():
    n, k, ell, trials = 40, 4, 12, 3000
    A, b = _rand_system(n, 8, shift=1.0, scale=1.0)
    st_I = scmrh.run(lambda v: A @ v, b, sk.IdentitySketch(n), k)
    x_ls = scmrh.solve(st_I, k)
    r_ls2 = np.sum((b - A @ x_ls) ** 2)
    rng = np.random.default_rng(11)
    xs, ratios = [], []
    for _ in range(trials):
        S = rng.standard_normal((ell, n)) / np.sqrt(ell)
        st = scmrh.run(lambda v: A @ v, b, sk.DenseSketch(S), k)
        x = scmrh.solve(st, k)
        xs.append(x)
        ratios.append(np.sum((b - A @ x) ** 2) / r_ls2)
    xs = np.array(xs)
    se = xs.std(axis=0) / np.sqrt(trials)
    z = np.abs(xs.mean(axis=0) - x_ls) / se
    assert np.max(z) < 4.5                    # 40 components, Bonferroni-ish band
    want = 1 + k / (ell - k - 1)
    ratios = np.array(ratios)
    assert abs(ratios.mean() - want) < 4 * ratios.std() / np.sqrt(trials)


def test_breakdown_gives_exact_solution():
    d = np.array([2.0, 3.0, 5.0, 7.0, 11.0])
    A = np.diag(d)
    b = np.zeros(5)
    b[2] = 4.0
    st = scmrh.run(lambda v: A @ v, b, sk.IdentitySketch(5), 4)
    assert st.breakdown and st.k_done == 1
    assert st.H[1, 0] == 0.0
    assert np.allclose(scmrh.solve(st, 1), b / d)
    z = scmrh.run(lambda v: A @ v, np.zeros(5), sk.IdentitySketch(5), 3)
    assert z.k_done == 0 and z.breakdown


def test_all_rows_pivoted_breaks_down_at_n():
    n = 6
    A, b = _rand_system(n, 9)
    st = scmrh.run(lambda v: A @ v, b, sk.IdentitySketch(n), n + 3)
    assert st.k_done == n and st.breakdown
    assert np.allclose(scmrh.solve(st, n), np.linalg.solve(A, b), atol=1e-10)


def test_forced_pivots_replay():
    A, b = _rand_system(25, 10)
    S = sk.SparseSignSketch(3, 25, 24, 8)
    st = scmrh.run(lambda v: A @ v, b, S, 8)
    st2 = scmrh.run(lambda v: A @ v, b, S, 8, forced_pivots=st.piv)
    assert st2.piv == st.piv
    assert np.array_equal(st2.V, st.V) and np.array_equal(st2.H, st.H)
    # another admissible order still satisfies the Hessenberg relation
    alt = [st.piv[0]] + [p for p in range(25) if p != st.piv[0]][:8]
    st3 = scmrh.run(lambda v: A @ v, b, S, 8, forced_pivots=alt)
    k = st3.k_done
    assert np.linalg.norm(A @ st3.V[:, :k] - st3.V @ st3.H) < 1e-10 * np.linalg.norm(st3.H)


def test_pivot_ties_take_lowest_index():
    A = np.eye(4)
    b = np.array([1.0, -3.0, 3.0, 2.0])
    st = scmrh.run(lambda v: A @ v, b, sk.IdentitySketch(4), 1)
    assert st.piv[0] == 1 and st.beta == -3.0


@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_qmr_iterate_solves_its_normal_equations(lam):
    """Eq. (Hessenber_LS) / Eq. (TSP): y minimises ||beta e_1 - H y||^2 +
    lam^2 ||y||^2, i.e. (H^T H + lam^2 I) y = beta H^T e_1 (normal equations,
    solved independently), and for lam = 0 the residual of the CMRH iterate
    obeys the bounds of Eq. (eqthm) with M = L_{k+1}."""
    A, b = _rand_system(30, 8)
    st = scmrh.run(lambda v: A @ v, b, sk.IdentitySketch(30), 12)
    k = 10
    H = st.H[:k + 1, :k]
    y = scmrh.qmr_y(st.H, st.beta, k, lam)
    e1 = np.zeros(k + 1)
    e1[0] = st.beta
    y_ne = np.linalg.solve(H.T @ H + lam ** 2 * np.eye(k), H.T @ e1)
    assert np.linalg.norm(y - y_ne) <= 1e-10 * np.linalg.norm(y_ne)
    if lam == 0.0:
        x = scmrh.cmrh_solve(st, k)
        x_ls = scmrh.solve(st, k)                    # S = I: the minimal residual iterate
        r, r_ls = np.linalg.norm(A @ x - b), np.linalg.norm(A @ x_ls - b)
        kappa = np.linalg.cond(st.V[:, :k + 1])
        assert r_ls <= r * (1 + 1e-12) and r <= kappa * r_ls * (1 + 1e-12)
