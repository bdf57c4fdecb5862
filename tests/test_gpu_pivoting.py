"""Sampled pivoting (Sec. 3.2, Sec. 4) through the C ABI against the oracle
drawing the same samples: pivots identical (FP64) or identical up to a near
tie among the sampled entries (FP32), and x_k per iterate up to the full k
(the oracle replaying the GPU's pivots)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from _gpu_common import TIE, compare_solution, ensure_lib, gpu_context, tolerance, verify_scmrh  # noqa: E402
from gen import problems as P  # noqa: E402
from oracle import operators as ops, scmrh, sketch as sk  # noqa: E402

PIVOT_SEED_XOR = 0xA5A5A5A5A5A5A5A5       # include/ipf.h, config.pivot_sample


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_lib()


@pytest.mark.parametrize("storage,sample", [("f64", 5), ("f64", 25), ("f32", 25)])
def test_sampled_pivoting_scmrh(storage, sample):
    p = P.make("deblur64")
    A = ops.make_apply(p)
    S = sk.SparseSignSketch(p.sketch_seed, p.n, p.m_s, p.zeta)
    b = p.b[0].astype(np.float64)
    st = scmrh.run(A, b, S, p.k, pivot_sample=sample, pivot_seed=p.sketch_seed ^ PIVOT_SEED_XOR)
    full = scmrh.run(A, b, S, p.k)
    assert st.piv != full.piv                       # the samples change the pivot order
    ctx = gpu_context(p, storage, pivot_sample=sample)
    ctx.step(p.k)
    status, kd = ctx.sync()
    assert kd == [p.k]
    piv = [int(v) for v in ctx.export(0)["piv"][:p.k + 1]]
    j = next((i for i in range(p.k + 1) if piv[i] != st.piv[i]), p.k + 1)
    if storage == "f64":
        assert j == p.k + 1, j
    elif j <= p.k:
        # a near tie between the two sampled entries in the oracle's vector at
        # that choice (v_j = u / u(p_j), so the ratio test is the one on u)
        vec = b if j == 0 else scmrh.run(A, b, S, j, forced_pivots=st.piv[:j + 1]).V[:, j]
        a, bb = abs(vec[piv[j]]), abs(vec[st.piv[j]])
        assert abs(a - bb) <= TIE[storage] * max(a, bb), (j, a, bb)
    # iterates up to the full k: the oracle replays the GPU's sampled pivots
    verify_scmrh(ctx, p, storage, [1, 2, 5, 10, 20, 30, 50], p.lambdas, check_pivots=False,
                 name=f"deblur64_{storage}_sampled{sample}")
    ctx.close()


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_sampled_pivot_growth_keeps_sketch_exact(storage):
    """Basis growth under sampled pivoting: a right-hand side with one entry
    1e4 and the rest in [1e-3, 1e-2], with one-entry samples, gives pivots far
    below the largest entry and |v_j| of about 1e6 (full pivoting keeps
    |v| <= 1).  The sketch sums must stay exact for such columns: S v_j from
    the library equals S applied to the stored v_j up to the fixed-point
    quantum, n * 2^-34 relative to max |v_j| (overflowing integer counters
    would be off by about max |v_j|); the pivots are the oracle's and, in
    FP64, so are the sketches and the iterates."""
    p = P.make("deblur64")
    rng = np.random.default_rng(8)
    b = rng.uniform(1e-3, 1e-2, p.n).astype(np.float32)
    b[1234] = 1e4
    k = 5
    A = ops.make_apply(p)
    S = sk.SparseSignSketch(p.sketch_seed, p.n, p.m_s, p.zeta)
    st = scmrh.run(A, b.astype(np.float64), S, k, pivot_sample=1, pivot_seed=p.sketch_seed ^ PIVOT_SEED_XOR)
    assert np.abs(st.V).max() > 1e5
    ctx = gpu_context(p, storage, k=k, b=b.reshape(1, -1), pivot_sample=1)
    ctx.step(k)
    status, kd = ctx.sync()
    assert kd == [k]
    ex = ctx.export(0)
    assert [int(v) for v in ex["piv"][:k + 1]] == list(st.piv)
    Sd = S.matrix()
    for j in range(k + 1):
        vj = st.V[:, j] if storage == "f64" else ctx.basis(j).astype(np.float64)
        ref = Sd @ vj
        tol = p.n * 2.0 ** -34 * np.abs(vj).max()
        assert np.abs(ex["SV"][:, j] - ref).max() <= tol, (j, np.abs(vj).max())
    if storage == "f64":
        compare_solution(ctx, st, storage, [1, 2, 3, 4, 5], [0.0])
    ctx.close()


def test_inverse_growth_switches_to_forward_substitution():
    """The pivot-block solve in inverse form keeps a row of L_p^{-1} per
    step; a row larger than 2^20 in magnitude switches the solve to forward
    substitution for the rest of the run.  Sampled pivoting with one-entry
    samples and a right-hand side with one entry 1e6 gives |v_j| up to 4e9
    and, in the oracle's L_p, rows of the inverse of 0.45, 0.81, 1.2e2 and
    then 1.5e7 at step 4, so the switch happens inside this 8-step run.  In
    FP64 the pivots are the oracle's and x_k follows it, both with the
    default solve (inverse form, then the switch) and with forward
    substitution throughout (pivot_fwd = 1), and the two runs agree to FP64
    rounding."""
    p = P.make("deblur64")
    rng = np.random.default_rng(8)
    b = rng.uniform(1e-3, 1e-2, p.n).astype(np.float32)
    b[1234] = 1e6
    k = 8
    A = ops.make_apply(p)
    S = sk.SparseSignSketch(p.sketch_seed, p.n, p.m_s, p.zeta)
    st = scmrh.run(A, b.astype(np.float64), S, k, pivot_sample=1, pivot_seed=p.sketch_seed ^ PIVOT_SEED_XOR)
    L = st.V[st.piv[:k + 1], :k + 1]
    Minv = np.linalg.inv(L)
    rows = [np.abs(Minv[j, :j]).max() for j in range(1, k + 1)]
    assert max(rows[:3]) < 2.0 ** 20 < rows[3], rows           # the switch comes at step 4
    xs = []
    for fwd in (0, 1):
        ctx = gpu_context(p, "f64", k=k, b=b.reshape(1, -1), pivot_sample=1, pivot_fwd=fwd)
        ctx.step(k)
        status, kd = ctx.sync()
        assert kd == [k]
        assert [int(v) for v in ctx.export(0)["piv"][:k + 1]] == list(st.piv)
        compare_solution(ctx, st, "f64", list(range(1, k + 1)), [0.0], name=f"growth_switch_fwd{fwd}")
        x, _ = ctx.solve(k, [0.0])
        xs.append(x[0, 0].astype(np.float64))
        ctx.close()
    tol = tolerance("f64", np.linalg.cond(scmrh.projected_matrix(st, k, "hessenberg")))
    assert np.linalg.norm(xs[0] - xs[1]) <= tol * np.linalg.norm(xs[1])
