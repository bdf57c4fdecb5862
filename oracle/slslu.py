"""sLSLU in float64: the generalized Hessenberg process with two sketches, then
the sketched projected (Tikhonov) least-squares solve.  Test infrastructure
only.

Paper, Sec. 3.1, Eq. (Hessenberg_r): for A (m x n),
    A L_k = D_{k+1} H_{k+1,k},    A^T D_{k+1} = L_{k+1} W_{k+1},
with D (m-space, range K_k(A A^T, b)) and L (n-space, range K_k(A^T A, A^T b))
unit lower triangular after their pivot permutations, H upper Hessenberg and
W upper triangular.  Sec. 3.2 / Algorithm 1 (sLSLU) and Sec. 3.3 /
Algorithm 2 (with Tikhonov):
    y_k = argmin ||S_2 (A L_k y - b)||^2 + lambda^2 ||S_1 L_k y||^2,
    x_k = L_k y_k,  x_0 = 0,
with S_2 (l x m) and S_1 (l x n), and S_2 A L_k = (S_2 D_{k+1}) H_{k+1,k}.

Readings of Algorithm 1 as printed (its loop has slips of notation): the
loop's first product is u = A l_k (it prints A^T applied to d_k); the vector
normalised from u is the new d_{k+1} (it reuses the name d_k); the second
product is q = A^T d_{k+1}; and the diagonal entry of W is the pivot entry
of q (it prints u).  Those readings are the ones that make both relations of
Eq. (Hessenberg_r) hold, which the tests check.

Steps, in the algorithm's order:
  init   r0 = b; t_1 = argmax |r0|; beta = r0(t_1); d_1 = r0 / beta
         v0 = A^T r0; g_1 = argmax |v0|; alpha = v0(g_1); l_1 = v0 / alpha
         W(1,1) = (A^T d_1)(g_1)
  loop   u = A l_k; z_k = S_2 u
         for j = 1..k: H(j,k) = u(t_j); u = u - H(j,k) d_j
         if k < m and u != 0: t_{k+1} = argmax over non-pivot rows of |u|
                              H(k+1,k) = u(t_{k+1}); d_{k+1} = u / H(k+1,k)
         else: H(k+1,k) = 0, stop
         q = A^T d_{k+1}
         for j = 1..k: W(j,k+1) = q(g_j); q = q - W(j,k+1) l_j
         if k < n and q != 0: g_{k+1} = argmax over non-pivot rows of |q|
                              W(k+1,k+1) = q(g_{k+1}); l_{k+1} = q / W(k+1,k+1)
         else: stop
Pivots are the largest magnitude with the lowest index on ties.

Storage precision (storage = "f32", "bf16", "f16"; default "f64"): each new
vector of D and of L is rounded to the storage type right after its
normalisation, and every later step reads the stored vector (the reading of
scmrh.py); all arithmetic stays float64.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import pivoting
from .storage import round_to
from .scmrh import _argmax_abs_excluding, _lstsq_qr, qmr_y


@dataclass
class GenHessenbergState:
    D: np.ndarray            # (m, k_done + 1)
    L: np.ndarray            # (n, k_done + 1); column k_done may be unset if the L side stopped
    H: np.ndarray            # (k_done + 1, k_done)
    W: np.ndarray            # (k_done + 1, k_done + 1) upper triangular
    pt: list                 # pivots of D (0-based rows of the m-space)
    pg: list                 # pivots of L (0-based rows of the n-space)
    SD: np.ndarray           # (l, k_done + 1) = S_2 D
    SL: np.ndarray           # (l, k_done + 1) = S_1 L
    Zd: np.ndarray           # (l, k_done) z_k = S_2 A l_k
    c: np.ndarray            # S_2 b
    beta: float
    alpha: float
    k_done: int              # completed steps: d_1..d_{k+1}, l_1..l_k at least
    l_done: int              # columns of L formed
    breakdown: bool
    gaps_t: list             # pivot-gap ratio (|u|_(1) - |u|_(2)) / |u|_(1) per pivot of D
    gaps_g: list             # the same for the pivots of L


def iterate(apply_A, apply_At, b, S1, S2, k_max: int, forced_t=None, forced_g=None, pivot_sample: int = 0,
            pivot_seeds=(0, 0), storage: str = "f64"):
    """Yields (k, state) after the initialisation (k = 0) and after each step.

    forced_t / forced_g: optional pivot sequences to use instead of the
    max-|.| choice (replays another run's order where two candidates are
    within rounding of each other).  pivot_sample > 0 chooses the pivots by
    sampled pivoting (pivoting.py), with sampling seeds pivot_seeds for D
    and L.  storage rounds each new basis vector to that type."""
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    m = b.size
    v0 = apply_At(b)
    n = v0.size
    ell = S2.m
    D = np.zeros((m, k_max + 1))
    L = np.zeros((n, k_max + 1))
    H = np.zeros((k_max + 1, k_max))
    W = np.zeros((k_max + 1, k_max + 1))
    SD = np.zeros((ell, k_max + 1))
    SL = np.zeros((S1.m, k_max + 1))
    Zd = np.zeros((ell, k_max))
    tpiv = np.zeros(m, dtype=bool)
    gpiv = np.zeros(n, dtype=bool)
    c = S2.apply(b)
    pt, pg = [], []
    gaps_t, gaps_g = [], []

    def state(k, beta, alpha, l_done, breakdown):
        return GenHessenbergState(D[:, :k + 1], L[:, :k + 1], H[:k + 1, :k], W[:k + 1, :k + 1], list(pt), list(pg),
                                  SD[:, :k + 1], SL[:, :k + 1], Zd[:, :k], c, beta, alpha, k, l_done, breakdown,
                                  list(gaps_t), list(gaps_g))

    def choose(vec, is_piv, forced, idx, gaps, side):
        i_max, _, gap = _argmax_abs_excluding(vec, is_piv)
        gaps.append(gap)
        if forced is not None and idx < len(forced):
            return int(forced[idx])
        if pivot_sample > 0:
            return pivoting.sampled_pivot(vec, is_piv, pivot_seeds[side], idx, pivot_sample)
        return i_max

    i = choose(b, tpiv, forced_t, 0, gaps_t, 0)
    beta = float(b[i])
    if beta == 0.0:
        yield 0, state(0, 0.0, 0.0, 0, True)
        return
    D[:, 0] = round_to(b / beta, storage)
    pt.append(i)
    tpiv[i] = True
    SD[:, 0] = S2.apply(D[:, 0])
    i2 = choose(v0, gpiv, forced_g, 0, gaps_g, 1)
    alpha = float(v0[i2])
    if alpha == 0.0:
        yield 0, state(0, beta, 0.0, 0, True)
        return
    L[:, 0] = round_to(v0 / alpha, storage)
    pg.append(i2)
    gpiv[i2] = True
    SL[:, 0] = S1.apply(L[:, 0])
    W[0, 0] = apply_At(D[:, 0])[i2]
    yield 0, state(0, beta, alpha, 1, False)

    for k in range(k_max):                         # 0-based: builds d_{k+2}, l_{k+2}
        u = apply_A(L[:, k])
        Zd[:, k] = S2.apply(u)
        for j in range(k + 1):
            H[j, k] = u[pt[j]]
            u = u - H[j, k] * D[:, j]
        assert not np.any(u[tpiv]), "elimination left a nonzero on a pivot row of D"
        if k + 1 >= m or not np.any(u):
            H[k + 1, k] = 0.0
            yield k + 1, state(k + 1, beta, alpha, k + 1, True)
            return
        p = choose(u, tpiv, forced_t, k + 1, gaps_t, 0)
        H[k + 1, k] = u[p]
        D[:, k + 1] = round_to(u / H[k + 1, k], storage)
        pt.append(p)
        tpiv[p] = True
        SD[:, k + 1] = S2.apply(D[:, k + 1])

        q = apply_At(D[:, k + 1])
        for j in range(k + 1):
            W[j, k + 1] = q[pg[j]]
            q = q - W[j, k + 1] * L[:, j]
        assert not np.any(q[gpiv]), "elimination left a nonzero on a pivot row of L"
        if k + 1 >= n or not np.any(q):
            yield k + 1, state(k + 1, beta, alpha, k + 1, True)
            return
        p2 = choose(q, gpiv, forced_g, k + 1, gaps_g, 1)
        W[k + 1, k + 1] = q[p2]
        L[:, k + 1] = round_to(q / W[k + 1, k + 1], storage)
        pg.append(p2)
        gpiv[p2] = True
        SL[:, k + 1] = S1.apply(L[:, k + 1])
        yield k + 1, state(k + 1, beta, alpha, k + 2, False)


def run(apply_A, apply_At, b, S1, S2, k_max: int, forced_t=None, forced_g=None, pivot_sample: int = 0,
        pivot_seeds=(0, 0), storage: str = "f64") -> GenHessenbergState:
    st = None
    for _, st in iterate(apply_A, apply_At, b, S1, S2, k_max, forced_t, forced_g, pivot_sample, pivot_seeds,
                         storage):
        pass
    return st


def projected_matrix(st: GenHessenbergState, k: int, zform: str = "hessenberg") -> np.ndarray:
    """Z = S_2 A L_k, as S_2 D_{k+1} H_{k+1,k} or from the sketched products."""
    if zform == "hessenberg":
        return st.SD[:, :k + 1] @ st.H[:k + 1, :k]
    if zform == "direct":
        return st.Zd[:, :k]
    raise ValueError(zform)


def solve_y(st: GenHessenbergState, k: int, lam: float = 0.0, zform: str = "hessenberg") -> np.ndarray:
    """y = argmin ||c - Z y||^2 + lam^2 ||S_1 L_k y||^2 (Algorithm 2)."""
    if k > st.k_done or k > st.l_done:
        raise ValueError("k exceeds the completed iterations")
    if k == 0:
        return np.zeros(0)
    Z = projected_matrix(st, k, zform)
    if lam == 0.0:
        return _lstsq_qr(Z, st.c)
    P = st.SL[:, :k]
    M = np.vstack([Z, lam * P])
    rhs = np.concatenate([st.c, np.zeros(P.shape[0])])
    return _lstsq_qr(M, rhs)


def solve(st: GenHessenbergState, k: int, lam: float = 0.0, zform: str = "hessenberg") -> np.ndarray:
    """x_k = L_k y_k (x_0 = 0)."""
    return st.L[:, :k] @ solve_y(st, k, lam, zform)


def lslu_solve(st: GenHessenbergState, k: int, lam: float = 0.0) -> np.ndarray:
    """LSLU quasi-minimal residual iterate (Eq. Hessenber_LS with M = D_{k+1}),
    with the Tikhonov term of Eq. (TSP) for lam > 0: x = L_k y."""
    return st.L[:, :k] @ qmr_y(st.H, st.beta, k, lam)
