"""Forward operators A of Eq. 1 for the oracle, accessed only through
products A v (Sec. 1: A is available through matrix-vector products).

conv2d_zero     w = P * v, zero boundary, odd kernel centred at its middle
                 (true convolution: w(y,x) = sum P[ky,kx] v(y-ky+cy, x-kx+cx)).
sep_motion       w = M * (G * v), each pass zero-boundary with the result
                 cropped to the image in between (G = g_col (x) g_row).
csr_apply        w = A v for a CSR matrix.

All sums are float64 shifted-array sums written straight from the
definitions; nothing is blocked or reordered.
"""
from __future__ import annotations

import numpy as np


def conv2d_zero(img: np.ndarray, K: np.ndarray) -> np.ndarray:
    img = np.asarray(img, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    H, W = img.shape
    ph, pw = K.shape
    if ph % 2 == 0 or pw % 2 == 0:
        raise ValueError("odd kernel sizes only")
    cy, cx = ph // 2, pw // 2
    vp = np.zeros((H + 2 * cy, W + 2 * cx))
    vp[cy:cy + H, cx:cx + W] = img
    out = np.zeros((H, W))
    for ky in range(ph):
        oy = 2 * cy - ky
        for kx in range(pw):
            k = K[ky, kx]
            if k != 0.0:
                ox = 2 * cx - kx
                out += k * vp[oy:oy + H, ox:ox + W]
    return out


def conv_rows(img: np.ndarray, g: np.ndarray) -> np.ndarray:
    """1-D zero-boundary convolution along x (axis 1)."""
    return conv2d_zero(img, np.asarray(g, dtype=np.float64)[None, :])


def conv_cols(img: np.ndarray, g: np.ndarray) -> np.ndarray:
    """1-D zero-boundary convolution along y (axis 0)."""
    return conv2d_zero(img, np.asarray(g, dtype=np.float64)[:, None])


def sep_motion(img, g_row, g_col, M):
    return conv2d_zero(conv_cols(conv_rows(img, g_row), g_col), M)


def csr_apply(rowptr, colind, vals, v):
    rowptr = np.asarray(rowptr, dtype=np.int64)
    m = rowptr.size - 1
    v = np.asarray(v, dtype=np.float64)
    prod = np.asarray(vals, dtype=np.float64) * v[np.asarray(colind, dtype=np.int64)]
    row_of = np.repeat(np.arange(m), np.diff(rowptr))
    return np.bincount(row_of, weights=prod, minlength=m)


def make_apply(problem):
    """A closure v -> A v (float64 vectors of length n) for a gen.Problem."""
    if problem.kind == "psf2d":
        H, W, K = problem.rows, problem.cols, problem.psf
        return lambda v: conv2d_zero(np.reshape(v, (H, W)), K).reshape(-1)
    if problem.kind == "psf_sep_motion":
        H, W = problem.rows, problem.cols
        gr, gc, M = problem.sep_row, problem.sep_col, problem.motion
        return lambda v: sep_motion(np.reshape(v, (H, W)), gr, gc, M).reshape(-1)
    if problem.kind == "csr":
        rp, ci, va = problem.rowptr, problem.colind, problem.vals
        return lambda v: csr_apply(rp, ci, va, v)
    raise ValueError(problem.kind)


def dense_matrix(apply_A, n: int) -> np.ndarray:
    """Columns A e_i (tiny n only)."""
    A = np.zeros((n, n))
    e = np.zeros(n)
    for i in range(n):
        e[i] = 1.0
        A[:, i] = apply_A(e)
        e[i] = 0.0
    return A
