"""The allocation-free sketch entry point (ipf_sketch_apply_noalloc) against
the allocating one (ipf_sketch_apply) and the oracle, through the C ABI.

Both entry points run the same kernels with exact 64-bit integer sums, so
their results must be bit-identical; a partial clear of the shared scratch
(which keeps the previous call's contents) would leave stale residues that
this equality catches.  The two cases run back to back with different sizes,
largest first, so the second call starts from a scratch array the first one
filled.  The result is also compared with the oracle's sparse-sign S x
within the rounding bound of the fixed-point sums.  This file is collected
last so a run that stops at its failure has run everything else.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _tol(x, n, m_s, zeta, seed):
    # rounding bound of the exact fixed-point sums: each of the at most cmax
    # contributions to a row is rounded once to the quantum 2^-F (half a
    # quantum each, taken as a random walk with a factor 10 of margin)
    from oracle import sketch as sk
    e_max = int(np.frexp(np.float64(np.abs(x).max()))[1])
    F = 61 - int(np.ceil(np.log2(n + 1))) - e_max
    rows, _ = sk.sparse_sign_structure(seed, np.arange(n), m_s, zeta)
    cmax = np.bincount(rows.ravel(), minlength=m_s).max()
    return 10.0 * np.sqrt(cmax) * 2.0 ** (-F - 1) / np.sqrt(zeta)


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    from _gpu_common import ensure_lib
    from oracle import sketch as sk
    from paper_2502_02721_gb300 import binding as bd
    ensure_lib()
    cases = [(300001, 800, 8, 0xABCDEF), (4097, 120, 3, 77)]
    for n, m_s, zeta, seed in cases:
        rng = np.random.default_rng(n)
        x = (rng.standard_normal(n) * np.exp(rng.uniform(-2, 2, n))).astype(np.float32)
        xd = torch.from_numpy(x).cuda()
        y_ref = torch.zeros(m_s, dtype=torch.float64, device="cuda")
        y_new = torch.full((m_s,), np.nan, dtype=torch.float64, device="cuda")
        bd.sketch_apply(xd, m_s, zeta, seed, y_ref)
        bd.sketch_apply_noalloc(xd, m_s, zeta, seed, y_new)
        torch.cuda.synchronize()
        a, b = y_ref.cpu().numpy(), y_new.cpu().numpy()
        assert np.all(np.isfinite(b))
        assert np.array_equal(a, b), (n, m_s, int(np.count_nonzero(a != b)))
        want = sk.SparseSignSketch(seed, n, m_s, zeta).apply(x.astype(np.float64))
        assert np.max(np.abs(b - want)) <= _tol(x, n, m_s, zeta, seed)


def test_noalloc_rejects_too_many_rows():
    import torch
    from _gpu_common import ensure_lib
    from paper_2502_02721_gb300 import binding as bd
    ensure_lib()
    x = torch.ones(64, dtype=torch.float32, device="cuda")
    y = torch.zeros(4097, dtype=torch.float64, device="cuda")
    with pytest.raises(bd.IpfError) as ei:
        bd.sketch_apply_noalloc(x, 4097, 8, 1, y)
    assert ei.value.code == bd.IPF_ERR_UNSUPPORTED
