"""Seeded synthetic inverse problems b = A x_true + e (Eq. 1 of the paper).

This module only makes INPUTS: point-spread functions, phantoms, the CT
system matrix, noisy data.  It contains none of the solver's arithmetic, and
both the FP64 oracle and the CUDA library consume what it returns.

The forward blur used to make ``b`` is computed with an FFT product
(``scipy.signal.fftconvolve``), an algorithm that neither the oracle (direct
shifted sums) nor the CUDA kernels (tiled direct stencils) use; the CT data
are made with a ``scipy.sparse`` product.

The paper's datasets (the cameraman image, circuit.tiff, the FIPS cheese and
walnut scans; Sec. 4) are not available; the workloads below are synthetic
stand-ins with the shapes, PSF families, noise levels and phantom structure
named for each workload.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DATA_SEED_BASE = 2502021
SKETCH_SEED_OFFSET = 1000


# ----------------------------------------------------------------------------
# point-spread functions (all odd-sized, centred, normalised to sum 1, FP32)
# ----------------------------------------------------------------------------
def gaussian_1d(size: int, sigma: float) -> np.ndarray:
    c = size // 2
    t = np.arange(size, dtype=np.float64) - c
    g = np.exp(-0.5 * (t / sigma) ** 2)
    return (g / g.sum()).astype(np.float32)


def gaussian_psf(size: int, sigma: float) -> np.ndarray:
    c = size // 2
    t = np.arange(size, dtype=np.float64) - c
    r2 = t[:, None] ** 2 + t[None, :] ** 2
    p = np.exp(-0.5 * r2 / sigma ** 2)
    return (p / p.sum()).astype(np.float32)


def moffat_psf(size: int, beta: float, alpha: float) -> np.ndarray:
    c = size // 2
    t = np.arange(size, dtype=np.float64) - c
    r2 = t[:, None] ** 2 + t[None, :] ** 2
    p = (1.0 + r2 / alpha ** 2) ** (-beta)
    return (p / p.sum()).astype(np.float32)


def motion_kernel(length: int, theta: float) -> np.ndarray:
    """``length`` samples at t = -(length-1)/2 .. (length-1)/2 along the
    direction theta, bilinearly splatted onto a length x length grid centred
    at its middle, normalised to sum 1.  Samples come in +t/-t pairs, so the
    kernel is point-symmetric."""
    c = length // 2
    k = np.zeros((length, length), dtype=np.float64)
    for s in range(-c, c + 1):
        x = c + s * math.cos(theta)
        y = c + s * math.sin(theta)
        x0, y0 = math.floor(x), math.floor(y)
        fx, fy = x - x0, y - y0
        for dy, wy in ((0, 1.0 - fy), (1, fy)):
            for dx, wx in ((0, 1.0 - fx), (1, fx)):
                yy, xx = y0 + dy, x0 + dx
                if 0 <= yy < length and 0 <= xx < length:
                    k[yy, xx] += wy * wx
    # symmetrise exactly (rounding of cos/sin can break it by an ulp)
    k = 0.5 * (k + k[::-1, ::-1])
    return (k / k.sum()).astype(np.float32)


# ----------------------------------------------------------------------------
# phantoms
# ----------------------------------------------------------------------------
def blobs_phantom(h: int, w: int, nblobs: int, rng: np.random.Generator) -> np.ndarray:
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    x = np.zeros((h, w))
    for _ in range(nblobs):
        cy, cx = rng.uniform(0, h), rng.uniform(0, w)
        amp = rng.uniform(0.2, 1.0)
        wid = rng.uniform(2.0, 6.0)
        x += amp * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * wid ** 2))
    return x


def ellipse_phantom(h: int, w: int, nell: int, rng: np.random.Generator) -> np.ndarray:
    """Piecewise-constant sum of ``nell`` seeded ellipses; sizes scale with the image."""
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    yy = (yy + 0.5) / h
    xx = (xx + 0.5) / w
    x = np.zeros((h, w))
    for _ in range(nell):
        cy, cx = rng.uniform(0.15, 0.85), rng.uniform(0.15, 0.85)
        a, b = rng.uniform(0.03, 0.22), rng.uniform(0.03, 0.22)
        th = rng.uniform(0, math.pi)
        val = rng.uniform(0.1, 1.0)
        ct, st = math.cos(th), math.sin(th)
        u = (xx - cx) * ct + (yy - cy) * st
        v = -(xx - cx) * st + (yy - cy) * ct
        x[(u / a) ** 2 + (v / b) ** 2 <= 1.0] += val
    return x


def head_phantom(n: int, rng: np.random.Generator, nsmall: int = 8) -> np.ndarray:
    """Shepp-Logan-like head: an outer ellipse, a darker interior, and
    ``nsmall`` seeded small ellipses of low contrast."""
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    yy = 2.0 * (yy + 0.5) / n - 1.0
    xx = 2.0 * (xx + 0.5) / n - 1.0
    x = np.zeros((n, n))

    def add(cx, cy, a, b, th, val):
        ct, st = math.cos(th), math.sin(th)
        u = (xx - cx) * ct + (yy - cy) * st
        v = -(xx - cx) * st + (yy - cy) * ct
        x[(u / a) ** 2 + (v / b) ** 2 <= 1.0] += val

    add(0.0, 0.0, 0.69, 0.92, 0.0, 1.0)
    add(0.0, -0.02, 0.62, 0.85, 0.0, -0.8)
    for _ in range(nsmall):
        add(rng.uniform(-0.4, 0.4), rng.uniform(-0.5, 0.5), rng.uniform(0.04, 0.25),
            rng.uniform(0.04, 0.3), rng.uniform(0, math.pi), rng.uniform(-0.2, 0.3))
    return x


# ----------------------------------------------------------------------------
# forward models used only to make b
# ----------------------------------------------------------------------------
def blur_fft(img: np.ndarray, kernel: np.ndarray) -> np.ndarray:
    """Zero-boundary 'same' convolution by FFT (used only to synthesise b)."""
    from scipy.signal import fftconvolve
    return fftconvolve(img.astype(np.float64), kernel.astype(np.float64), mode="same")


def siddon_parallel(nimg: int, nangles: int, ndet: int, det_spacing: float = 1.0):
    """Parallel-beam system matrix by Siddon's ray tracing (chord lengths).

    Image: nimg x nimg unit pixels centred at the origin, row 0 at the top,
    column index r*nimg + c.  Ray (a, d): angle theta_a = a*pi/nangles, offset
    s_d = (d - (ndet-1)/2)*det_spacing; points s*(cos, sin) + t*(-sin, cos).
    Row index a*ndet + d.  Returns (rowptr int64, colind int32, vals float32).
    """
    half = nimg / 2.0
    grid = np.arange(nimg + 1, dtype=np.float64) - half
    rows_cols, rows_vals, counts = [], [], []
    for a in range(nangles):
        th = a * math.pi / nangles
        ct, st = math.cos(th), math.sin(th)
        s = (np.arange(ndet, dtype=np.float64) - (ndet - 1) / 2.0) * det_spacing
        px, py = s * ct, s * st            # point on ray at t = 0
        ux, uy = -st, ct                   # unit direction
        ts = []
        if abs(ux) > 1e-12:
            ts.append((grid[None, :] - px[:, None]) / ux)
        if abs(uy) > 1e-12:
            ts.append((grid[None, :] - py[:, None]) / uy)
        T = np.concatenate(ts, axis=1)
        # clip to the part of the ray inside the square
        with np.errstate(divide="ignore", invalid="ignore"):
            if abs(ux) > 1e-12:
                tx0, tx1 = (-half - px) / ux, (half - px) / ux
                txmin, txmax = np.minimum(tx0, tx1), np.maximum(tx0, tx1)
            else:
                inside = np.abs(px) < half
                txmin = np.where(inside, -np.inf, np.inf)
                txmax = np.where(inside, np.inf, -np.inf)
            if abs(uy) > 1e-12:
                ty0, ty1 = (-half - py) / uy, (half - py) / uy
                tymin, tymax = np.minimum(ty0, ty1), np.maximum(ty0, ty1)
            else:
                inside = np.abs(py) < half
                tymin = np.where(inside, -np.inf, np.inf)
                tymax = np.where(inside, np.inf, -np.inf)
        tlo = np.maximum(txmin, tymin)
        thi = np.minimum(txmax, tymax)
        # rays that miss the square have an empty (or infinite) interval: they
        # get empty rows, and only the others reach the arithmetic below
        hit = np.isfinite(tlo) & np.isfinite(thi) & (tlo < thi)
        Th = np.sort(np.clip(T[hit], tlo[hit, None], thi[hit, None]), axis=1)
        t0, t1 = Th[:, :-1], Th[:, 1:]
        L = t1 - t0
        tm = 0.5 * (t0 + t1)
        xm = px[hit, None] + tm * ux
        ym = py[hit, None] + tm * uy
        c = np.floor(xm + half).astype(np.int64)
        r = (nimg - 1) - np.floor(ym + half).astype(np.int64)
        ok = (L > 1e-9) & (c >= 0) & (c < nimg) & (r >= 0) & (r < nimg)
        hit_row = np.cumsum(hit) - 1
        for d in range(ndet):
            if not hit[d]:
                rows_cols.append(np.zeros(0, np.int32))
                rows_vals.append(np.zeros(0, np.float32))
                counts.append(0)
                continue
            h = hit_row[d]
            m = ok[h]
            col = (r[h][m] * nimg + c[h][m])
            val = L[h][m]
            # merge duplicate pixels (a crossing can split one pixel's chord)
            if col.size:
                order = np.argsort(col, kind="stable")
                col, val = col[order], val[order]
                uq, start = np.unique(col, return_index=True)
                val = np.add.reduceat(val, start)
                col = uq
            rows_cols.append(col.astype(np.int32))
            rows_vals.append(val.astype(np.float32))
            counts.append(col.size)
    rowptr = np.zeros(len(counts) + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(counts)
    colind = np.concatenate(rows_cols) if rows_cols else np.zeros(0, np.int32)
    vals = np.concatenate(rows_vals) if rows_vals else np.zeros(0, np.float32)
    return rowptr, colind, vals


def csr_matvec(rowptr, colind, vals, x):
    from scipy.sparse import csr_matrix
    m = rowptr.size - 1
    A = csr_matrix((vals.astype(np.float64), colind, rowptr), shape=(m, x.size))
    return A @ x.astype(np.float64)


def add_noise(clean: np.ndarray, level: float, rng: np.random.Generator) -> np.ndarray:
    """e = level * ||A x|| * g / ||g||, g ~ N(0, I)."""
    g = rng.standard_normal(clean.shape)
    return clean + level * np.linalg.norm(clean) * g / np.linalg.norm(g)


# ----------------------------------------------------------------------------
# workload descriptions
# ----------------------------------------------------------------------------
@dataclass
class Problem:
    """One workload: operator description + data, in plain numpy arrays.

    kind: 'psf2d' (psf), 'psf_sep_motion' (sep_row, sep_col, motion) or 'csr'.
    b:    (nrhs, n) float32, rows are independent right-hand sides.
    """
    name: str
    kind: str
    rows: int
    cols: int
    b: np.ndarray
    x_true: np.ndarray
    k: int
    m_s: int
    zeta: int
    sketch_seed: int
    lambdas: list = field(default_factory=lambda: [0.0])
    psf: np.ndarray | None = None
    sep_row: np.ndarray | None = None
    sep_col: np.ndarray | None = None
    motion: np.ndarray | None = None
    rowptr: np.ndarray | None = None
    colind: np.ndarray | None = None
    vals: np.ndarray | None = None

    @property
    def n(self) -> int:
        return self.rows * self.cols if self.kind != "csr" else int(self.rowptr.size - 1)

    @property
    def nrhs(self) -> int:
        return int(self.b.shape[0])


def deblur_gauss64(seed: int = DATA_SEED_BASE + 0) -> Problem:
    """64x64 deblurring, 15x15 Gaussian PSF sigma=2, 8 blobs, 1% noise, k=50, m_s=200."""
    rng = np.random.default_rng(seed)
    psf = gaussian_psf(15, 2.0)
    x = blobs_phantom(64, 64, 8, rng)
    clean = blur_fft(x, psf)
    b = add_noise(clean, 0.01, rng).astype(np.float32)
    return Problem("deblur64_gauss15", "psf2d", 64, 64, b.reshape(1, -1), x.reshape(-1),
                   k=50, m_s=200, zeta=8, sketch_seed=seed + SKETCH_SEED_OFFSET,
                   lambdas=[0.0, 1e-3], psf=psf)


def deblur_sep_motion256(seed: int = DATA_SEED_BASE + 1, side: int = 256) -> Problem:
    """256x256 deblurring: separable 31-tap Gaussian (sigma=3) then a seeded
    9-px linear motion blur, zero boundary, 2% noise, 20 ellipses, k=100,
    m_s=400, 8 log-spaced lambdas 1e-4..1e-1."""
    rng = np.random.default_rng(seed)
    g = gaussian_1d(31, 3.0)
    theta = rng.uniform(0, math.pi)
    mk = motion_kernel(9, theta)
    x = ellipse_phantom(side, side, 20, rng)
    clean = blur_fft(blur_fft(x, np.outer(g, g)), mk)
    b = add_noise(clean, 0.02, rng).astype(np.float32)
    lams = list(np.logspace(-4, -1, 8))
    return Problem(f"deblur{side}_sep31_motion9", "psf_sep_motion", side, side, b.reshape(1, -1),
                   x.reshape(-1), k=100, m_s=400, zeta=8, sketch_seed=seed + SKETCH_SEED_OFFSET,
                   lambdas=lams, sep_row=g, sep_col=g, motion=mk)


def deblur_moffat(side: int = 2048, seed: int = DATA_SEED_BASE + 2, k: int = 200,
                  m_s: int = 800) -> Problem:
    """side x side deblurring, 31x31 Moffat PSF (beta=2.5, alpha=4), ellipse
    phantom at scale, 1% noise, k=200, m_s=800."""
    rng = np.random.default_rng(seed)
    psf = moffat_psf(31, 2.5, 4.0)
    x = ellipse_phantom(side, side, 20, rng)
    clean = blur_fft(x, psf)
    b = add_noise(clean, 0.01, rng).astype(np.float32)
    return Problem(f"deblur{side}_moffat31", "psf2d", side, side, b.reshape(1, -1), x.reshape(-1),
                   k=k, m_s=m_s, zeta=8, sketch_seed=seed + SKETCH_SEED_OFFSET, psf=psf)


_CSR_CACHE: dict = {}


def ct_parallel(side: int = 256, nrhs: int = 32, seed: int = DATA_SEED_BASE + 3, k: int = 150,
                m_s: int = 600, noise: float = 0.005) -> Problem:
    """Square parallel-beam CT: side x side image, side angles x side
    detectors (m = n), Siddon chord-length CSR, head phantoms, 0.5% noise,
    ``nrhs`` independent right-hand sides (phantom and noise seeded per RHS)."""
    key = (side, side, side)
    if key not in _CSR_CACHE:
        _CSR_CACHE[key] = siddon_parallel(side, side, side)
    rowptr, colind, vals = _CSR_CACHE[key]
    bs, xs = [], []
    for r in range(nrhs):
        rng = np.random.default_rng(seed * 1000 + r)
        x = head_phantom(side, rng).reshape(-1)
        clean = csr_matvec(rowptr, colind, vals, x)
        bs.append(add_noise(clean, noise, rng).astype(np.float32))
        xs.append(x)
    return Problem(f"ct{side}_parallel_siddon", "csr", side, side, np.stack(bs), np.stack(xs),
                   k=k, m_s=m_s, zeta=8, sketch_seed=seed + SKETCH_SEED_OFFSET,
                   rowptr=rowptr, colind=colind, vals=vals)


def make(name: str, **kw) -> Problem:
    table = {
        "deblur64": deblur_gauss64,
        "deblur256": deblur_sep_motion256,
        "deblur2048": deblur_moffat,
        "ct256": ct_parallel,
    }
    return table[name](**kw)
