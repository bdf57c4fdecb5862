"""The quasi-minimal residual iterate (Eq. Hessenber_LS; CMRH and LSLU, with
the Tikhonov term of Eq. TSP) through ipf_solve_qmr against the oracle on
the same basis."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from _gpu_common import FLOOR, U, ensure_lib, gpu_context, oracle_run, rel  # noqa: E402
from gen import problems as P  # noqa: E402
from oracle import scmrh  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_lib()


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_cmrh_iterate_matches_oracle(storage):
    """Pivots of deblur64 agree exactly in FP64 and FP32 (checked by the
    parity suite), so the QMR iterate of each k follows from the same H and
    V: within max(floor, 10 u_s kappa(H_{k+1,k}))."""
    p = P.make("deblur64")
    st = oracle_run(p)
    ctx = gpu_context(p, storage)
    ctx.step(p.k)
    status, kd = ctx.sync()
    assert kd == [p.k]
    for k in (1, 5, 10, 20, 50):
        x, info = ctx.solve(k, [0.0, 1e-3, 1e-1], qmr=True)
        kappa = np.linalg.cond(st.H[:k + 1, :k])
        tol = max(FLOOR[storage], 10.0 * U[storage] * kappa)
        for li, lam in enumerate((0.0, 1e-3, 1e-1)):
            e = rel(x[li, 0].astype(np.float64), scmrh.cmrh_solve(st, k, lam))
            assert e <= tol, (k, lam, e, tol)
        # the sketched and the quasi-minimal residual iterates differ in general
        xs, _ = ctx.solve(k, [0.0])
        if k >= 5:
            assert rel(xs[0, 0].astype(np.float64), x[0, 0].astype(np.float64)) > 1e-6
    ctx.close()


def test_qmr_needs_room_in_the_workspace():
    from paper_2502_02721_gb300 import binding as bd
    p = P.make("deblur64")
    ctx = gpu_context(p, "f32", k=20, m_s=16)
    ctx.step(20)
    with pytest.raises(bd.IpfError):
        ctx.solve(20, [0.0], qmr=True)
    ctx.close()
