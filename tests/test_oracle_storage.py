"""Pins for the oracle's storage-precision mode (each new basis vector
rounded to FP32, BF16 or FP16 right after its normalisation; every later
step reads the stored vector), checked against facts that hold for any
correct implementation of that reading:

* storage "f64" changes nothing, bit for bit;
* round_to gives the nearest value of the storage type (ties to even),
  checked against a brute-force search over the type's neighbours;
* the stored basis stays exactly unit lower trapezoidal under the pivots,
  with |v| <= 1, and every entry is a value of the storage type;
* Eq. (Hessenberg_s) holds for the stored basis up to the rounding of the
  newest vector: column j of A V_k - V_{k+1} H_k is H(j+1, j) times the
  rounding error of v_{j+1}, so its max-norm is at most |H(j+1, j)| u_s and
  is not zero (the rounding really happens);
* at k = n with S = I the stored basis still spans R^n, so x_n = A^{-1} b;
* the deviation of x_k from the FP64 oracle grows with the unit roundoff of
  the storage type (FP32 << FP16 << BF16, in about the ratio of the units);
* the generalized process (sLSLU): both stored bases exact unit lower
  trapezoidal and both relations of Eq. (Hessenberg_r) to the rounding of
  their newest vectors.
"""
import numpy as np
import pytest

from gen import problems as P
from oracle import operators as ops, scmrh, slslu, sketch as sk
from oracle.storage import UNIT, round_to


def _rand_system(n, seed, shift=1.0, scale=0.3):
    rng = np.random.default_rng(seed)
    A = shift * np.eye(n) + scale * rng.standard_normal((n, n)) / np.sqrt(n)
    return A, rng.standard_normal(n)


def _representable(v, storage):
    return np.array_equal(round_to(v, storage), v)


def test_f64_storage_is_the_unrounded_process():
    p = P.make("deblur64")
    A = ops.make_apply(p)
    S = sk.SparseSignSketch(p.sketch_seed, p.n, p.m_s, p.zeta)
    a = scmrh.run(A, p.b[0], S, 20)
    b = scmrh.run(A, p.b[0], S, 20, storage="f64")
    assert a.piv == b.piv
    for f in ("V", "H", "SV", "Zd", "c"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


@pytest.mark.parametrize("storage,mant", [("bf16", 7), ("f16", 10), ("f32", 23)])
def test_round_to_is_nearest_value_of_the_type(storage, mant):
    """Brute force: the two values of the type around x (x's binade with
    `mant` fraction bits) are found by flooring the scaled fraction; the
    result must be the nearer one, the even one on a tie."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal(4000) * np.exp(rng.uniform(-6, 6, 4000))
    # exact ties and values just around them
    ties = (1.0 + (2 * np.arange(1, 60) + 1) * 2.0 ** -(mant + 1)) * 2.0 ** rng.integers(-5, 5, 59)
    x = np.concatenate([x, ties, -ties, np.nextafter(ties, 0), np.nextafter(ties, 2 * ties)])
    if storage == "f16":
        x = x[np.abs(x) < 6.0e4]
        x = x[np.abs(x) > 2.0 ** -14]            # normal range of FP16
    r = round_to(x, storage)
    for xi, ri in zip(x, r):
        e = int(np.frexp(abs(xi))[1]) - 1            # xi in [2^e, 2^(e+1))
        q = 2.0 ** (e - mant)                      # spacing of the type in xi's binade
        lo = np.floor(abs(xi) / q) * q
        hi = lo + q
        d_lo, d_hi = abs(xi) - lo, hi - abs(xi)
        if d_lo < d_hi:
            want = lo
        elif d_hi < d_lo:
            want = hi
        else:
            want = lo if (int(round(lo / q)) % 2 == 0) else hi
        want = np.copysign(want, xi)
        if storage == "bf16" and want != ri:
            # a value within float32 rounding of a bf16 tie may round the other
            # way after the float32 step; that is the only difference allowed
            x32 = float(np.float32(xi))
            assert abs(abs(x32) - (lo + q / 2)) <= 2.0 ** (e - 23), (xi, ri, want)
            continue
        assert ri == want, (storage, xi, ri, want)


@pytest.mark.parametrize("storage", ["bf16", "f16", "f32"])
def test_stored_basis_is_exact_unit_lower_trapezoid(storage):
    p = P.make("deblur64")
    A = ops.make_apply(p)
    st = scmrh.run(A, p.b[0], sk.SparseSignSketch(p.sketch_seed, p.n, p.m_s, p.zeta), p.k, storage=storage)
    assert st.k_done == p.k
    V = st.V
    assert _representable(V, storage)
    for i, pi in enumerate(st.piv):
        assert V[pi, i] == 1.0 and np.all(V[pi, i + 1:] == 0.0)
    assert np.abs(V).max() <= 1.0
    assert len(set(st.piv)) == len(st.piv)


@pytest.mark.parametrize("storage", ["bf16", "f16", "f32"])
def test_stored_basis_hessenberg_relation_per_column(storage):
    p = P.make("deblur64")
    A = ops.make_apply(p)
    st = scmrh.run(A, p.b[0], sk.SparseSignSketch(p.sketch_seed, p.n, p.m_s, p.zeta), 30, storage=storage)
    u = UNIT[storage]
    worst_ratio = 0.0
    for j in range(st.k_done):
        Av = A(st.V[:, j])
        r = Av - st.V[:, :j + 2] @ st.H[:j + 2, j]
        bound = abs(st.H[j + 1, j]) * u
        fp64 = 64 * 2.0 ** -53 * (np.abs(Av).max() + np.abs(st.H[:j + 2, j]).sum())
        assert np.abs(r).max() <= bound + fp64, (j, np.abs(r).max(), bound)
        worst_ratio = max(worst_ratio, np.abs(r).max() / bound)
    # the rounding is applied: some column carries a sizeable part of its bound
    assert worst_ratio > 0.25


def test_stored_basis_reaches_the_dense_solution_at_k_equal_n():
    """At k = n the stored basis is a permuted unit lower triangle, so it
    spans R^n and the problem over it (Z = S A V_k, the sketched products of
    Algorithm 1) is solved by x = A^{-1} b.  S V_{k+1} H_k equals S A V_k
    only up to the rounding of the stored vectors (|H(j+1, j)| u_s per
    column), so that form is off by about u_s."""
    n = 12
    A, b = _rand_system(n, 8)
    st = scmrh.run(lambda v: A @ v, b, sk.IdentitySketch(n), n, storage="bf16")
    # every row is a pivot after n steps: the process stops there (no candidates)
    assert st.k_done == n and st.breakdown
    x = scmrh.solve(st, n, zform="direct")
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-9 * np.linalg.norm(x)
    xh = scmrh.solve(st, n, zform="hessenberg")
    d = np.linalg.norm(xh - x) / np.linalg.norm(x)
    assert 1e-5 < d < 10 * np.linalg.cond(A) * UNIT["bf16"]


def test_deviation_from_fp64_grows_with_the_storage_unit():
    p = P.make("deblur64")
    A = ops.make_apply(p)
    S = sk.SparseSignSketch(p.sketch_seed, p.n, p.m_s, p.zeta)
    ref = scmrh.run(A, p.b[0], S, 10)
    dev = {}
    for storage in ("f32", "f16", "bf16"):
        st = scmrh.run(A, p.b[0], S, 10, forced_pivots=ref.piv, storage=storage)
        xs, xr = scmrh.solve(st, 10, 1e-3), scmrh.solve(ref, 10, 1e-3)
        dev[storage] = np.linalg.norm(xs - xr) / np.linalg.norm(xr)
    assert dev["f32"] > 0.0
    r1 = dev["bf16"] / dev["f16"]              # units differ by 2^3
    r2 = dev["f16"] / dev["f32"]               # units differ by 2^13
    assert 2.0 <= r1 <= 32.0, dev
    assert 500.0 <= r2 <= 1e5, dev


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_generalized_process_stored_bases(storage):
    p = P.make("deblur64")
    psf = p.psf.astype(np.float64)
    A = lambda v: ops.conv2d_zero(v.reshape(p.rows, p.cols), psf).reshape(-1)
    At = lambda v: ops.conv2d_zero(v.reshape(p.rows, p.cols), psf[::-1, ::-1]).reshape(-1)
    S1 = sk.SparseSignSketch(p.sketch_seed ^ 0x5DEECE66DA3B1F27, p.n, p.m_s, p.zeta)
    S2 = sk.SparseSignSketch(p.sketch_seed, p.n, p.m_s, p.zeta)
    k = 20
    st = slslu.run(A, At, p.b[0].astype(np.float64), S1, S2, k, storage=storage)
    assert st.k_done == k
    u = UNIT[storage]
    for M, piv in ((st.D, st.pt), (st.L, st.pg)):
        assert _representable(M, storage)
        for i, pi in enumerate(piv):
            assert M[pi, i] == 1.0 and np.all(M[pi, i + 1:] == 0.0)
        assert np.abs(M).max() <= 1.0
    for j in range(k):
        Al = A(st.L[:, j])
        r = Al - st.D[:, :j + 2] @ st.H[:j + 2, j]
        assert np.abs(r).max() <= abs(st.H[j + 1, j]) * u + 64 * 2.0 ** -53 * np.abs(Al).max() * (j + 2)
        Ad = At(st.D[:, j + 1])
        q = Ad - st.L[:, :j + 2] @ st.W[:j + 2, j + 1]
        assert np.abs(q).max() <= abs(st.W[j + 1, j + 1]) * u + 64 * 2.0 ** -53 * np.abs(Ad).max() * (j + 2)
