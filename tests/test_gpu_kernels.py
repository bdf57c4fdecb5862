"""Kernel-level parity through the C ABI: the sparse-sign sketch and the
forward operators against the FP64 oracle on the same seeded inputs, at
sizes that span several tiles and ragged edges."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from _gpu_common import ensure_lib  # noqa: E402
from gen import problems as P  # noqa: E402
from oracle import operators as ops, sketch as sk  # noqa: E402


@pytest.fixture(scope="module")
def torch():
    import torch as t
    ensure_lib()
    return t


@pytest.mark.parametrize("n,m_s,zeta", [(1, 8, 8), (4096, 200, 8), (100003, 400, 8), (65536, 124, 3),
                                        (300001, 600, 16), (4194304, 800, 8)])
def test_sketch_apply_matches_oracle(torch, n, m_s, zeta):
    from paper_2502_02721_gb300 import binding as bd
    rng = np.random.default_rng(n + m_s)
    x = (rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    y = torch.zeros(m_s, dtype=torch.float64, device="cuda")
    seed = 0x1234ABCD + n
    bd.sketch_apply(xd, m_s, zeta, seed, y)
    torch.cuda.synchronize()
    S = sk.SparseSignSketch(seed, n, m_s, zeta)
    want = S.apply(x.astype(np.float64))
    got = y.cpu().numpy()
    # each term is rounded once to a multiple of 2^-F (F = 61 - ceil(log2(n+1))
    # - e_max, |x| < 2^e_max); the rounding errors are symmetric, so a row
    # with c terms is off by a few sqrt(c) 2^-(F+1) / sqrt(zeta)
    e_max = int(np.frexp(np.float64(np.abs(x).max()))[1])
    lg = int(np.ceil(np.log2(n + 1)))
    F = 61 - lg - e_max
    rows, _ = sk.sparse_sign_structure(seed, np.arange(n), m_s, zeta)
    cmax = np.bincount(rows.ravel(), minlength=m_s).max()
    tol = 10.0 * np.sqrt(cmax) * 2.0 ** (-F - 1) / np.sqrt(zeta)
    assert np.max(np.abs(got - want)) <= tol, (np.max(np.abs(got - want)), tol)


def test_sketch_apply_zero_vector(torch):
    from paper_2502_02721_gb300 import binding as bd
    x = torch.zeros(1000, dtype=torch.float32, device="cuda")
    y = torch.full((64,), 7.0, dtype=torch.float64, device="cuda")
    bd.sketch_apply(x, 64, 8, 5, y)
    assert torch.count_nonzero(y).item() == 0


def _apply_gpu(torch, opdesc, v, nrhs=1):
    from paper_2502_02721_gb300 import binding as bd
    keep = []
    op = bd.operator_from_problem(opdesc, keep) if hasattr(opdesc, "kind") else opdesc
    h = bd.Operator(op, keep)
    vd = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).cuda()
    wd = torch.zeros_like(vd)
    h.apply(vd, wd, nrhs)
    torch.cuda.synchronize()
    out = wd.cpu().numpy()
    h.close()
    return out


class _Desc:
    def __init__(self, **kw):
        self.__dict__.update(dict(psf=None, sep_row=None, sep_col=None, motion=None,
                                  rowptr=None, colind=None, vals=None))
        self.__dict__.update(kw)


@pytest.mark.parametrize("H,W,K", [(64, 64, "gauss15"), (300, 257, "moffat31"), (129, 70, "rand5x7"),
                                   (33, 900, "gauss7"), (70, 65, "rand41x41")])
def test_psf_conv_matches_oracle(torch, H, W, K):
    rng = np.random.default_rng(H * W)
    psf = {"gauss15": P.gaussian_psf(15, 2.0), "moffat31": P.moffat_psf(31, 2.5, 4.0),
           "gauss7": P.gaussian_psf(7, 1.0),
           "rand5x7": rng.standard_normal((5, 7)).astype(np.float32),
           "rand41x41": rng.standard_normal((41, 41)).astype(np.float32)}[K]
    v = rng.standard_normal(H * W).astype(np.float32)
    got = _apply_gpu(torch, _Desc(kind="psf2d", rows=H, cols=W, psf=psf), v)
    want = ops.conv2d_zero(v.reshape(H, W), psf).reshape(-1)
    scale = np.abs(psf).sum() * np.abs(v).max()
    assert np.max(np.abs(got - want)) <= 2e-6 * scale


# The BF16 product w = P * v for a BF16 vector v.  On the tensor cores each
# PSF tap F is carried as hi + lo, two BF16 numbers: hi is F rounded to 8
# significant bits and lo the remainder rounded to 8 more, so
# |F - hi - lo| <= 2^-17 |F|.  Each output sums, in FP32, at most 2*32
# products inside one MMA and then 2*KW partial sums in the epilogue: even with
# truncating adds that is <= (64 + 62) 2^-23 of the sum of |terms|.  Hence
# |w - w_exact| <= (2^-17 + 126 2^-23) (|F| * |v|) elementwise.  The FP32 FMA
# path (kept for other sizes, and selectable) is bounded by KW^2 2^-24 (|F|*|v|).
TC_REL = 2.0 ** -17 + 126 * 2.0 ** -23


def _psf(name, rng):
    return {"gauss15": P.gaussian_psf(15, 2.0), "moffat31": P.moffat_psf(31, 2.5, 4.0),
            "gauss11": P.gaussian_psf(11, 1.5),
            "rand31": rng.standard_normal((31, 31)).astype(np.float32),
            "rand9x13": rng.standard_normal((9, 13)).astype(np.float32)}[name]


def _oracle_windows(v, psf, wins, size):
    """Exact FP64 products on size x size windows at (Y, X): the oracle runs on
    the window plus a halo of the PSF radius cut from the zero-padded image."""
    H, W = v.shape
    cy, cx = psf.shape[0] // 2, psf.shape[1] // 2
    vp = np.zeros((H + 2 * cy + size, W + 2 * cx + size))
    vp[cy:cy + H, cx:cx + W] = v
    out = []
    for (Y, X) in wins:
        crop = vp[Y:Y + size + 2 * cy, X:X + size + 2 * cx]
        full = ops.conv2d_zero(crop, psf)
        out.append(full[cy:cy + size, cx:cx + size][:H - Y, :W - X])
    return out


@pytest.mark.parametrize("H,W,K", [(64, 64, "gauss15"), (200, 136, "moffat31"), (257, 264, "rand31"),
                                   (33, 1032, "gauss11"), (96, 104, "rand9x13"), (300, 130, "moffat31"),
                                   (2048, 2048, "moffat31")])
def test_psf_conv_bf16_matches_oracle(torch, H, W, K):
    """Tensor-core product (PSF padding to 15x15 or 31x31, W % 8 == 0) and the
    FP32 FMA product against the FP64 oracle on the same BF16 vector; W = 130
    is not a multiple of 8 and takes the FMA kernel on both calls."""
    from paper_2502_02721_gb300 import binding as bd
    rng = np.random.default_rng(H * 7 + W)
    psf = _psf(K, rng)
    vb = torch.from_numpy(rng.standard_normal(H * W).astype(np.float32)).cuda().to(torch.bfloat16)
    v = vb.float().cpu().numpy().astype(np.float64).reshape(H, W)
    keep = []
    op = bd.Operator(bd.make_operator("psf2d", H, W, psf=psf, keep=keep), keep)
    got = {}
    for fma in (False, True):
        wd = torch.full((H * W,), float("nan"), dtype=torch.float32, device="cuda")
        op.apply_bf16(vb, wd, use_fma=fma)
        torch.cuda.synchronize()
        got[fma] = wd.cpu().numpy().astype(np.float64).reshape(H, W)
    op.close()
    kw = max(psf.shape)
    if H * W <= 300 * 300:
        want = ops.conv2d_zero(v, psf)
        mag = ops.conv2d_zero(np.abs(v), np.abs(psf))
        cmp = [(got[False], want, mag), (got[True], want, mag)]
    else:
        # full size: the corners, the image edges and random interior windows
        S = 64
        wins = [(0, 0), (0, W - S), (H - S, 0), (H - S, W - S), (H // 2, 0), (0, W // 2)]
        wins += [(int(rng.integers(0, H - S)), int(rng.integers(0, W - S))) for _ in range(10)]
        want = _oracle_windows(v, psf, wins, S)
        mag = _oracle_windows(np.abs(v), np.abs(psf), wins, S)
        cmp = []
        for fma in (False, True):
            g = np.concatenate([got[fma][Y:Y + S, X:X + S].ravel() for (Y, X) in wins])
            cmp.append((g, np.concatenate([a.ravel() for a in want]), np.concatenate([a.ravel() for a in mag])))
    for (g, wnt, mg), rel_bound in zip(cmp, (TC_REL, kw * kw * 2.0 ** -24)):
        assert np.all(np.isfinite(g))
        err = np.abs(g - wnt)
        assert np.all(err <= rel_bound * mg + 1e-30), (np.max(err / (mg + 1e-30)), rel_bound)


@pytest.mark.parametrize("H,W", [(256, 256), (100, 130), (37, 300)])
def test_sep_motion_matches_oracle(torch, H, W):
    rng = np.random.default_rng(H + W)
    g = P.gaussian_1d(31, 3.0)
    M = P.motion_kernel(9, rng.uniform(0, np.pi))
    v = rng.standard_normal(H * W).astype(np.float32)
    got = _apply_gpu(torch, _Desc(kind="psf_sep_motion", rows=H, cols=W, sep_row=g, sep_col=g, motion=M), v)
    want = ops.sep_motion(v.reshape(H, W), g, g, M).reshape(-1)
    assert np.max(np.abs(got - want)) <= 2e-6 * np.abs(v).max()


@pytest.mark.parametrize("nrhs", [1, 4, 32])
def test_csr_matches_oracle(torch, nrhs):
    rowptr, colind, vals = P.siddon_parallel(48, 48, 48)
    n = 48 * 48
    rng = np.random.default_rng(nrhs)
    v = rng.standard_normal((nrhs, n)).astype(np.float32)
    # rows x cols of a CSR problem description is the image (48 x 48); the
    # operator is n x n with n = 48 * 48
    got = _apply_gpu(torch, _Desc(kind="csr", rows=48, cols=48, rowptr=rowptr, colind=colind, vals=vals),
                     v.reshape(-1), nrhs).reshape(nrhs, n)
    for r in range(nrhs):
        want = ops.csr_apply(rowptr, colind, vals, v[r])
        assert np.max(np.abs(got[r] - want)) <= 1e-5 * np.abs(want).max()
