"""The Gaussian sketch (Sec. 2; the paper's experiments) through the C ABI:
S drawn on the GPU from the counter hash (Box-Muller), S V_{k+1} by one GEMM
at solve time, against the oracle's GaussianSketch with the same definition
and storage rounding."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from _gpu_common import FLOOR, U, compare_pivots, ensure_lib, gpu_context, rel  # noqa: E402
from gen import problems as P  # noqa: E402
from oracle import operators as ops, scmrh, sketch as sk  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_lib()


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_gaussian_sketch_matches_oracle(storage):
    """x_k within max(floor, 10 u_s kappa(Z_k), 10 sqrt(n) u_a kappa(Z_k)): the
    last term is the GEMM's accumulation over n products (u_a = 2^-24 for
    FP32 accumulation, 2^-53 for FP64) carried to y through kappa(Z_k).  BF16
    storage is compared at k = 1, 2 (its basis departs from the FP64 oracle's
    by the storage rounding, as in the sparse-sign tests)."""
    p = P.make("deblur64")
    A = ops.make_apply(p)
    S = sk.GaussianSketch(p.sketch_seed, p.n, p.m_s, storage)
    st = scmrh.run(A, p.b[0].astype(np.float64), S, p.k)
    ctx = gpu_context(p, storage, sketch="gaussian")
    ctx.step(p.k)
    status, kd = ctx.sync()
    assert kd == [p.k]
    ex = ctx.export(0)
    agree = compare_pivots(ex["piv"][:p.k + 1], st, storage)
    assert not np.any(ex["SV"])                       # no per-step sparse sketch
    u_a = 2.0 ** -53 if storage == "f64" else 2.0 ** -24
    ks = [1, 2, 5, 10, 20, 50] if storage != "bf16" else [kk for kk in (1, 2) if kk < agree]
    for k in ks:
        x, _ = ctx.solve(k, p.lambdas)
        kappa = np.linalg.cond(scmrh.projected_matrix(st, k))
        tol = max(FLOOR[storage], 10 * U[storage] * kappa, 10 * np.sqrt(p.n) * u_a * kappa)
        for li, lam in enumerate(p.lambdas):
            e = rel(x[li, 0].astype(np.float64), scmrh.solve(st, k, lam))
            assert e <= tol, (k, lam, e, tol, kappa)
    ctx.close()


def test_gaussian_sketch_needs_one_rhs():
    from paper_2502_02721_gb300 import binding as bd
    p = P.ct_parallel(side=16, nrhs=2, k=5, m_s=20)
    with pytest.raises(bd.IpfError):
        gpu_context(p, "f32", sketch="gaussian")
