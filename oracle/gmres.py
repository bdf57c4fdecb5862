"""GMRES by Arnoldi with modified Gram-Schmidt, x_0 = 0, in float64.

Test infrastructure only.  The paper compares sCMRH with GMRES (Sec. 4.1):
with S = I the sketched problem is the minimal-residual problem over
K_k(A, b), whose solution is the GMRES iterate; this independent
implementation is the pin for that special case.
"""
from __future__ import annotations

import numpy as np


def gmres_iterates(A: np.ndarray, b: np.ndarray, k_max: int):
    """Return [x_1, ..., x_k] for k = 1..k_max (stops early on breakdown)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    beta = np.linalg.norm(b)
    Q = np.zeros((n, k_max + 1))
    Hb = np.zeros((k_max + 1, k_max))
    Q[:, 0] = b / beta
    xs = []
    for j in range(k_max):
        w = A @ Q[:, j]
        for i in range(j + 1):
            Hb[i, j] = Q[:, i] @ w
            w = w - Hb[i, j] * Q[:, i]
        Hb[j + 1, j] = np.linalg.norm(w)
        rhs = np.zeros(j + 2)
        rhs[0] = beta
        y = np.linalg.lstsq(Hb[:j + 2, :j + 1], rhs, rcond=None)[0]
        xs.append(Q[:, :j + 1] @ y)
        if Hb[j + 1, j] <= 1e-14 * beta:
            break
        Q[:, j + 1] = w / Hb[j + 1, j]
    return xs
