"""Pins for the oracle's forward operators (A accessed through A v, Sec. 1)
and for the input generators: brute-force dense matrices written from the
definition, scipy's convolve2d / sparse products as independent library
routines, and closed-form chord lengths for the Siddon CT matrix."""
import math

import numpy as np
import pytest
from scipy.signal import convolve2d

from gen import problems as P
from oracle import operators as ops


def _dense_conv_matrix(H, W, K):
    """A[(y,x), (yy,xx)] = K[y - yy + cy, x - xx + cx] inside the kernel support."""
    ph, pw = K.shape
    cy, cx = ph // 2, pw // 2
    A = np.zeros((H * W, H * W))
    for y in range(H):
        for x in range(W):
            for yy in range(H):
                for xx in range(W):
                    ky, kx = y - yy + cy, x - xx + cx
                    if 0 <= ky < ph and 0 <= kx < pw:
                        A[y * W + x, yy * W + xx] = K[ky, kx]
    return A


def test_conv_matches_bruteforce_and_scipy():
    rng = np.random.default_rng(3)
    H, W = 7, 9
    K = rng.standard_normal((5, 3))       # deliberately not symmetric
    img = rng.standard_normal((H, W))
    got = ops.conv2d_zero(img, K)
    A = _dense_conv_matrix(H, W, K)
    assert np.allclose(got.reshape(-1), A @ img.reshape(-1), rtol=0, atol=1e-13)
    assert np.allclose(got, convolve2d(img, K, mode="same", boundary="fill"), atol=1e-13)


def test_sep_motion_equals_three_library_passes():
    rng = np.random.default_rng(4)
    img = rng.standard_normal((20, 23))
    g = P.gaussian_1d(7, 1.5)
    M = P.motion_kernel(5, 0.7)
    want = convolve2d(convolve2d(convolve2d(img, g[None, :], mode="same"), g[:, None],
                                 mode="same"), M, mode="same")
    assert np.allclose(ops.sep_motion(img, g, g, M), want, atol=1e-13)


def test_csr_apply_matches_scipy():
    rowptr, colind, vals = P.siddon_parallel(16, 16, 16)
    x = np.random.default_rng(5).standard_normal(256)
    assert np.allclose(ops.csr_apply(rowptr, colind, vals, x),
                       P.csr_matvec(rowptr, colind, vals, x), atol=1e-12)


def test_psfs_normalised_and_point_symmetric():
    for K in (P.gaussian_psf(15, 2.0), P.moffat_psf(31, 2.5, 4.0), P.motion_kernel(9, 1.1),
              np.outer(P.gaussian_1d(31, 3.0), P.gaussian_1d(31, 3.0))):
        assert abs(float(np.sum(K, dtype=np.float64)) - 1.0) < 1e-6
        assert np.allclose(K, K[::-1, ::-1], atol=1e-7)


def test_siddon_axis_aligned_rays_have_unit_chords():
    N = 32
    rowptr, colind, vals = P.siddon_parallel(N, 4, N)
    # angle 0: vertical rays through pixel-centre columns -> N entries of length 1
    for d in range(N):
        s, e = rowptr[d], rowptr[d + 1]
        assert e - s == N
        assert np.allclose(vals[s:e], 1.0)
        assert np.array_equal(np.sort(colind[s:e] % N), np.full(N, d))
    # angle pi/2 (a = 2 of 4): horizontal rays, each covering one image row
    for d in range(N):
        r = 2 * N + d
        s, e = rowptr[r], rowptr[r + 1]
        assert e - s == N and np.allclose(vals[s:e], 1.0)
        assert len(set((colind[s:e] // N).tolist())) == 1


def test_siddon_total_chord_equals_square_chord():
    """Sum of a row's weights = length of the ray's chord through the square
    (closed form from slab intersection)."""
    N, na, nd = 24, 7, 24
    rowptr, colind, vals = P.siddon_parallel(N, na, nd)
    h = N / 2
    for a in range(na):
        th = a * math.pi / na
        ct, st = math.cos(th), math.sin(th)
        for d in range(nd):
            s = d - (nd - 1) / 2
            px, py, ux, uy = s * ct, s * st, -st, ct
            lo, hi = -math.inf, math.inf
            for p0, u in ((px, ux), (py, uy)):
                if abs(u) < 1e-12:
                    if abs(p0) >= h:
                        lo, hi = 1.0, 0.0
                    continue
                t0, t1 = (-h - p0) / u, (h - p0) / u
                lo, hi = max(lo, min(t0, t1)), min(hi, max(t0, t1))
            chord = max(0.0, hi - lo)
            r = a * nd + d
            assert abs(vals[rowptr[r]:rowptr[r + 1]].astype(np.float64).sum() - chord) < 1e-4


def test_make_apply_kinds():
    p = P.make("deblur64")
    A = ops.make_apply(p)
    v = np.random.default_rng(6).standard_normal(p.n)
    w = A(v)
    assert w.shape == (p.n,)
    assert np.allclose(w.reshape(64, 64), convolve2d(v.reshape(64, 64), p.psf.astype(np.float64),
                                                     mode="same"), atol=1e-12)
