"""The allocation-free sketch entry point (ipf_sketch_apply_noalloc) gives
the same result as ipf_sketch_apply, through the C ABI, on two calls in a
row of different sizes (the shared scratch keeps the previous call's
contents, so the second call checks that it is cleared).  This file is
collected last so a run that stops at its failure has run everything else.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _tol(x, n, m_s, zeta, seed):
    # the rounding bound of the exact fixed-point sums (as in the sketch parity test)
    from oracle import sketch as sk
    e_max = int(np.frexp(np.float64(np.abs(x).max()))[1])
    F = 61 - int(np.ceil(np.log2(n + 1))) - e_max
    rows, _ = sk.sparse_sign_structure(seed, np.arange(n), m_s, zeta)
    cmax = np.bincount(rows.ravel(), minlength=m_s).max()
    return 10.0 * np.sqrt(cmax) * 2.0 ** (-F - 1) / np.sqrt(zeta)


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    from _gpu_common import ensure_lib
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
        assert np.max(np.abs(a - b)) <= _tol(x, n, m_s, zeta, seed)


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
