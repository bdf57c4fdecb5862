"""sCMRH in float64: the pivoted Hessenberg process with a sketch, then the
sketched projected (Tikhonov) least-squares solve.  Test infrastructure only.

Paper, Sec. 3.1, Eq. (Hessenberg_s): A L_k = L_{k+1} H_{k+1,k} with L unit
lower triangular after the pivot permutation and range(L_k) = K_k(A, b).
Sec. 3.2, Eq. (sketched_LSLU): y_k = argmin_y ||S (A L_k y - b)||, x_k = L_k y_k
with x_0 = 0.  Algorithm 1 gives the loop (written there for the generalized
process; the square process applies A where Algorithm 1 applies A^T to the
left vector, and calls the new vector v_{j+1} where it reuses the name d_k).  Sec. 3.3 /
Algorithm 2 add the penalty lambda^2 ||S_1 L_k y||^2; for a square A one
sketch S serves as both S_1 and S_2.

The steps below follow Algorithm 1 in its order:
  init   r0 = b; i = argmax |r0| (lowest index on ties); beta = r0(i);
         v_1 = r0 / beta; pivot list p = [i]
  loop   u = A v_j;  z_j = S u
         for i = 1..j:  H(i, j) = u(p_i);  u = u - H(i, j) v_i
         if j < n and u != 0:  p_{j+1} = argmax over non-pivot rows of |u|
                                H(j+1, j) = u(p_{j+1});  v_{j+1} = u / H(j+1, j)
         else:                  H(j+1, j) = 0, stop (breakdown)
  solve  y = argmin ||c - Z y||^2 + lambda^2 ||S V_k y||^2,  c = S b,
         Z = S V_{k+1} H_k (or the sketched products z_j = S A v_j);
         x = V_k y
The sequential elimination leaves u(p_i) = 0 exactly (v_i(p_i) = 1 and
v_c(p_i) = 0 for c > i hold exactly in floating point), which run() asserts.

Storage precision (storage = "f32", "bf16", "f16"; default "f64"): each new
basis vector v_{j+1} = u / H(j+1, j) (and v_1 = b / beta) is rounded to the
storage type right after its normalisation, and every later step reads the
stored vector; all arithmetic stays float64.  Rounding keeps v(p_{j+1}) = 1
and the zeros on earlier pivot rows exact, so the elimination is unchanged.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from . import pivoting
from .storage import round_to


@dataclass
class HessenbergState:
    V: np.ndarray            # (n, k_done + 1) basis L_{k+1}; column k_done is zero on breakdown
    H: np.ndarray            # (k_done + 1, k_done) upper Hessenberg
    piv: list                # pivot rows p_1 .. p_{k_done + 1} (0-based)
    SV: np.ndarray           # (m, k_done + 1) = S V
    Zd: np.ndarray           # (m, k_done) columns z_j = S (A v_j)
    c: np.ndarray            # S b
    beta: float
    k_done: int
    breakdown: bool
    gaps: list = field(default_factory=list)   # pivot-gap ratio per chosen pivot


def _argmax_abs_excluding(u: np.ndarray, is_piv: np.ndarray):
    a = np.abs(u)
    a = np.where(is_piv, -1.0, a)
    i = int(np.argmax(a))                 # first occurrence: lowest index on ties
    top = a[i]
    a2 = a.copy()
    a2[i] = -1.0
    second = float(a2.max()) if a2.size > 1 else -1.0
    gap = (top - max(second, 0.0)) / top if top > 0 else 0.0
    return i, float(top), gap


def iterate(apply_A, b, sketch, k_max: int, forced_pivots=None, pivot_sample: int = 0, pivot_seed: int = 0,
            storage: str = "f64"):
    """Generator form of run(): yields (j, state) after the initialisation
    (j = 0) and after each Hessenberg step j = 1..k_done.  Each state holds
    views of the working arrays trimmed to the j completed steps.

    pivot_sample > 0 chooses each pivot by sampled pivoting (pivoting.py)
    with sampling seed pivot_seed.  storage rounds each new basis vector to
    that type (module docstring)."""
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    n = b.size
    m = sketch.m
    V = np.zeros((n, k_max + 1))
    H = np.zeros((k_max + 1, k_max))
    SV = np.zeros((m, k_max + 1))
    Zd = np.zeros((m, k_max))
    is_piv = np.zeros(n, dtype=bool)
    c = sketch.apply(b)
    gaps = []

    def state(k, beta, piv, breakdown):
        return HessenbergState(V[:, :k + 1], H[:k + 1, :k], list(piv), SV[:, :k + 1], Zd[:, :k], c,
                               beta, k, breakdown, list(gaps))

    # init: r0 = b - A x0 with x0 = 0
    if forced_pivots is not None:
        i = int(forced_pivots[0])
    else:
        i, _, g = _argmax_abs_excluding(b, is_piv)
        gaps.append(g)
        if pivot_sample > 0:
            i = pivoting.sampled_pivot(b, is_piv, pivot_seed, 0, pivot_sample)
    beta = float(b[i])
    if beta == 0.0:
        yield 0, state(0, 0.0, [], True)
        return
    V[:, 0] = round_to(b / beta, storage)
    piv = [i]
    is_piv[i] = True
    SV[:, 0] = sketch.apply(V[:, 0])
    yield 0, state(0, beta, piv, False)

    for j in range(k_max):
        u = apply_A(V[:, j])
        Zd[:, j] = sketch.apply(u)
        for ii in range(j + 1):                       # sequential elimination
            H[ii, j] = u[piv[ii]]
            u = u - H[ii, j] * V[:, ii]
        assert not np.any(u[is_piv]), "elimination left a nonzero on a pivot row"
        if j + 1 >= n or not np.any(u):
            H[j + 1, j] = 0.0
            yield j + 1, state(j + 1, beta, piv, True)
            return
        if forced_pivots is not None and j + 1 < len(forced_pivots):
            p = int(forced_pivots[j + 1])
        else:
            p, _, g = _argmax_abs_excluding(u, is_piv)
            gaps.append(g)
            if pivot_sample > 0:
                p = pivoting.sampled_pivot(u, is_piv, pivot_seed, j + 1, pivot_sample)
        H[j + 1, j] = u[p]
        V[:, j + 1] = round_to(u / H[j + 1, j], storage)
        piv.append(p)
        is_piv[p] = True
        SV[:, j + 1] = sketch.apply(V[:, j + 1])
        yield j + 1, state(j + 1, beta, piv, False)


def run(apply_A, b, sketch, k_max: int, forced_pivots=None, pivot_sample: int = 0,
        pivot_seed: int = 0, storage: str = "f64") -> HessenbergState:
    """k_max steps of the pivoted Hessenberg process with sketch S.

    forced_pivots: optional sequence of rows to use as p_1, p_2, ... instead
    of the max-|.| choice (replays another run's pivot order when two
    candidates are within rounding of each other).  storage: the type the
    basis is kept in (module docstring).
    """
    st = None
    for _, st in iterate(apply_A, b, sketch, k_max, forced_pivots, pivot_sample, pivot_seed, storage):
        pass
    return st


def _lstsq_qr(M: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """argmin ||rhs - M y|| by Householder QR (LAPACK geqrf)."""
    Q, R = np.linalg.qr(M, mode="reduced")
    return sla.solve_triangular(R, Q.T @ rhs, lower=False)


def projected_matrix(st: HessenbergState, k: int, zform: str = "hessenberg") -> np.ndarray:
    """Z = S A V_k, either as S V_{k+1} H_k or from the sketched products."""
    if zform == "hessenberg":
        return st.SV[:, :k + 1] @ st.H[:k + 1, :k]
    if zform == "direct":
        return st.Zd[:, :k]
    raise ValueError(zform)


def solve_y(st: HessenbergState, k: int, lam: float = 0.0, zform: str = "hessenberg",
            penalty: str = "sketched_x") -> np.ndarray:
    """y = argmin ||c - Z y||^2 + lam^2 ||P y||^2 with P = S V_k ('sketched_x')
    or P = I ('y', the form of Eq. TSP)."""
    if k > st.k_done:
        raise ValueError("k exceeds the completed iterations")
    if k == 0:
        return np.zeros(0)
    Z = projected_matrix(st, k, zform)
    if lam == 0.0:
        return _lstsq_qr(Z, st.c)
    P = st.SV[:, :k] if penalty == "sketched_x" else np.eye(k)
    M = np.vstack([Z, lam * P])
    rhs = np.concatenate([st.c, np.zeros(P.shape[0])])
    return _lstsq_qr(M, rhs)


def solve(st: HessenbergState, k: int, lam: float = 0.0, zform: str = "hessenberg",
          penalty: str = "sketched_x") -> np.ndarray:
    """x_k = V_k y_k (x_0 = 0)."""
    y = solve_y(st, k, lam, zform, penalty)
    return st.V[:, :k] @ y


def qmr_y(H: np.ndarray, beta: float, k: int, lam: float = 0.0) -> np.ndarray:
    """y = argmin ||beta e_1 - H_{k+1,k} y||^2 + lam^2 ||y||^2: the quasi-minimal
    residual problem of Eq. (Hessenber_LS) (M^+ (A x - b) = H y - beta e_1),
    with the Tikhonov term of Eq. (TSP) when lam > 0."""
    rhs = np.zeros(k + 1)
    rhs[0] = beta
    Hk = H[:k + 1, :k]
    if lam == 0.0:
        return _lstsq_qr(Hk, rhs)
    return _lstsq_qr(np.vstack([Hk, lam * np.eye(k)]), np.concatenate([rhs, np.zeros(k)]))


def cmrh_solve(st: HessenbergState, k: int, lam: float = 0.0) -> np.ndarray:
    """CMRH quasi-minimal residual iterate (Eq. Hessenber_LS with M = L_{k+1}),
    HCMRH for lam > 0 (Eq. TSP): x = V_k y."""
    return st.V[:, :k] @ qmr_y(st.H, st.beta, k, lam)
