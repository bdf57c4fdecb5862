"""End-to-end parity of the CUDA path (ipf_create / ipf_step / ipf_solve
through the C ABI) with the FP64 oracle on the same seeded inputs: pivots
identical up to near ties, the sketch of the first basis vector, and x_k per
iterate up to the full k for plain and Tikhonov problems, in every storage
precision (against the oracle keeping its basis in the same storage type and
replaying the GPU's pivots, and against the FP64 oracle at the stated
tolerance wherever that storage type can reach it); plus breakdown,
batching and ragged sizes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from _gpu_common import (U, compare_pivots, ensure_lib, gpu_context, oracle_run, rel,  # noqa: E402
                         verify_scmrh)
from gen import problems as P  # noqa: E402
from oracle import operators as ops, scmrh, sketch as sk  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_lib()


@pytest.fixture(scope="module")
def deblur64():
    p = P.make("deblur64")
    return p, oracle_run(p)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_deblur64_parity(deblur64, storage):
    p, st = deblur64
    ctx = gpu_context(p, storage)
    ctx.step(p.k)
    status, kd = ctx.sync()
    assert kd == [p.k]
    ex = ctx.export(0)
    agree = compare_pivots(ex["piv"][:p.k + 1], st, storage)
    assert agree == p.k + 1, "pivots diverged (near tie)"
    assert abs(ex["beta"] - st.beta) <= 1e-6 * abs(st.beta)
    # sketch of v_1 = b / beta and c = S b
    assert rel(ex["SV"][:, 0], st.SV[:, 0]) < (1e-12 if storage == "f64" else 1e-6)
    assert rel(ex["c"], st.c) < (1e-12 if storage == "f64" else 1e-6)
    if storage == "f32":
        # z_j = S A v_j (the sketched product of Algorithm 1).  z_0 involves one FP32 product;
        # later columns inherit the drift of individual basis vectors, which
        # is larger than that of x_k (errors inside the Krylov subspace leave
        # x_k unchanged), hence the looser bound
        assert rel(ex["SZ"][:, 0], st.Zd[:, 0]) < 1e-6
        for j in range(1, 5):
            assert rel(ex["SZ"][:, j], st.Zd[:, j]) < 1e-4
    # Hessenberg columns: the first tightly, the next ones with the basis drift
    assert rel(ex["H"][:2, 0], st.H[:2, 0]) < (1e-12 if storage == "f64" else 1e-6)
    for j in range(1, 5):
        assert rel(ex["H"][:j + 2, j], st.H[:j + 2, j]) < (1e-10 if storage == "f64" else 1e-4)
    verify_scmrh(ctx, p, storage, [1, 2, 5, 10, 20, 30, 40, 50], p.lambdas, name=f"deblur64_{storage}",
                 require_all_pivots=True)
    ctx.close()


@pytest.mark.parametrize("storage,conv_fma", [("bf16", 0), ("bf16", 1), ("f16", 0)])
def test_deblur64_low_precision(deblur64, storage, conv_fma):
    """BF16 runs the 15x15 product on the tensor cores (conv_fma 0) and on
    the FP32 FMA path (conv_fma 1); both must meet the same bounds."""
    p, st = deblur64
    ctx = gpu_context(p, storage, conv_fma=conv_fma)
    ctx.step(p.k)
    status, kd = ctx.sync()
    ex = ctx.export(0)
    assert kd == [p.k]
    # exact structure of the stored basis (unit lower trapezoid, |v| <= 1)
    k = kd[0]
    V = np.stack([ctx.basis(j) for j in range(k + 1)], axis=1).astype(np.float64)
    piv = ex["piv"][:k + 1]
    for i, pi in enumerate(piv):
        assert V[pi, i] == 1.0 and np.all(V[pi, i + 1:] == 0.0)
    assert np.abs(V).max() <= 1.0
    # Hessenberg relation of the stored basis: column j is off by the rounding
    # of v_{j+1} to storage (|H(j+1,j)| u_s) plus FP32 accumulation
    A = ops.make_apply(p)
    H = ex["H"][:k + 1, :k]
    for j in range(k):
        r = A(V[:, j]) - V[:, :j + 2] @ H[:j + 2, j]
        bound = abs(H[j + 1, j]) * U[storage] + 1e-5 * (np.abs(A(V[:, j])).max() + np.abs(H[:j + 2, j]).sum())
        assert np.abs(r).max() <= bound, (j, np.abs(r).max(), bound)
    # iterates at every k up to the full k against the oracle with the same
    # storage, replaying the GPU's pivots; 1e-3 against FP64 where reachable
    verify_scmrh(ctx, p, storage, [1, 5, 10, 20, 30, 50], p.lambdas, conv_fma=conv_fma,
                 name=f"deblur64_{storage}" + ("_fma" if conv_fma else ""))
    ctx.close()


@pytest.mark.parametrize("storage,overlap", [("f32", 0), ("f32", 1), ("f32", 2), ("bf16", 0), ("bf16", 2)])
def test_step_modes_match_oracle(deblur64, storage, overlap):
    """The one-stream step and the two-stream steps (operator beside V_j h, or
    beside the pivot-row products and the FP64 pivot-block solve) against the
    oracle, with graph replay and eager launches giving the same bits."""
    p, st = deblur64
    xs = []
    for graphs in (1, 0):
        ctx = gpu_context(p, storage, graphs=graphs, overlap=overlap)
        ctx.step(p.k)
        status, kd = ctx.sync()
        assert kd == [p.k]
        verify_scmrh(ctx, p, storage, [1, 5, 20, 50], p.lambdas, require_all_pivots=storage == "f32",
                     name=f"deblur64_{storage}_overlap{overlap}_graphs{graphs}")
        xs.append(ctx.solve(p.k, [0.0])[0])
        ctx.close()
    assert np.array_equal(xs[0], xs[1])


def test_zforms_agree_f32(deblur64):
    from paper_2502_02721_gb300 import binding as bd
    p, st = deblur64
    xs = []
    for zf in (bd.IPF_Z_DIRECT, bd.IPF_Z_HESSENBERG):
        ctx = gpu_context(p, "f32", zform=zf)
        ctx.step(20)
        x, _ = ctx.solve(20, [0.0])
        xs.append(x[0, 0].astype(np.float64))
        ctx.close()
    assert rel(xs[0], xs[1]) < 1e-6


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_direct_zform_low_precision(deblur64, storage):
    """The DIRECT form (z_j = S A v_j of the stored basis) with BF16/FP16
    storage against the oracle's sketched products of its stored basis, up
    to the full k."""
    from paper_2502_02721_gb300 import binding as bd
    p, _ = deblur64
    ctx = gpu_context(p, storage, zform=bd.IPF_Z_DIRECT)
    ctx.step(p.k)
    verify_scmrh(ctx, p, storage, [1, 5, 10, 20, 30, 50], p.lambdas, zform="direct",
                 name=f"deblur64_{storage}_direct")
    ctx.close()


def test_penalty_on_y(deblur64):
    from paper_2502_02721_gb300 import binding as bd
    p, st = deblur64
    ctx = gpu_context(p, "f64", penalty=bd.IPF_PEN_Y)
    ctx.step(30)
    lam = [0.05, 0.5]
    x, _ = ctx.solve(30, lam)
    for li, l in enumerate(lam):
        assert rel(x[li, 0], scmrh.solve(st, 30, l, penalty="y")) < 2e-7     # x is float32
    ctx.close()


@pytest.fixture(scope="module")
def deblur256():
    return P.make("deblur256")


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_deblur256_sep_motion_lambda_sweep(deblur256, storage):
    """The separable + motion operator, all 8 lambdas for FP32, a plain and a
    regularised one for BF16 / FP16, up to k = 100."""
    p = deblur256
    ctx = gpu_context(p, storage)
    ctx.step(p.k)
    status, kd = ctx.sync()
    assert kd == [p.k]
    lams = p.lambdas if storage == "f32" else [0.0, p.lambdas[5]]
    verify_scmrh(ctx, p, storage, [5, 25, 50, 100], lams, require_all_pivots=storage == "f32",
                 name=f"deblur256_{storage}")
    ctx.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_graph_and_eager_paths_give_identical_bits(deblur64, storage):
    """Steps launched eagerly, from the one-step graph and from the
    eight-step graph (step(7): one eager step and six one-step replays;
    step(13) and step(20): eight-step replays and one-step remainders) give
    the same bits."""
    p, _ = deblur64
    outs = []
    for graphs in (0, 1):
        ctx = gpu_context(p, storage, k=40, graphs=graphs)
        ctx.step(7)
        ctx.step(13)
        ctx.step(20)
        x, _ = ctx.solve(40, [0.0, 1e-3])
        outs.append((x.copy(), ctx.export(0)))
        ctx.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1]["SV"], outs[1][1]["SV"])
    assert np.array_equal(outs[0][1]["piv"], outs[1][1]["piv"])


@pytest.mark.parametrize("storage,overlap", [("bf16", 2), ("bf16", 0), ("f32", 2)])
def test_interleaved_solves_and_exports_keep_sketch_exact(deblur64, storage, overlap):
    """With one float right-hand side the sketch of each new column is taken
    by the next step's update, and the newest column's before a solve or an
    export (each column exactly once).  Solving and exporting between steps,
    twice in a row, must leave S V, the pivots and x_k bit-identical to an
    uninterrupted run: a column sketched twice or never would show in S V."""
    p, _ = deblur64
    ref = gpu_context(p, storage, k=30, overlap=overlap)
    ref.step(30)
    x_ref, _ = ref.solve(30, [0.0, 1e-3])
    ex_ref = ref.export(0)
    x_ref12, _ = ref.solve(12, [0.0])
    ref.close()
    ctx = gpu_context(p, storage, k=30, overlap=overlap)
    ctx.step(5)
    ctx.solve(5, [0.0])
    ctx.export(0)
    ctx.export(0)
    ctx.step(7)
    x12, _ = ctx.solve(12, [0.0])
    ctx.solve(12, [0.0])
    ctx.step(1)
    ctx.export(0)
    ctx.step(17)
    x, _ = ctx.solve(30, [0.0, 1e-3])
    ex = ctx.export(0)
    ctx.close()
    assert np.array_equal(ex["piv"], ex_ref["piv"])
    assert np.array_equal(ex["SV"], ex_ref["SV"])
    assert np.array_equal(x, x_ref)
    assert np.array_equal(x12, x_ref12)


@pytest.mark.parametrize("storage,pivot_fwd", [("f64", 0), ("f32", 0), ("bf16", 0), ("f64", 1), ("bf16", 1)])
def test_large_k_pivot_block(storage, pivot_fwd):
    """k = 300, m_s = 1200: the pivot-block solve in inverse form (rows of
    L_p^{-1} over ten blocks of 32 columns, h as a product with 300
    independent rows) and by forward substitution (pivot_fwd = 1: L_p read
    from L2, four row groups per warp, up to 512 rows); pivots and x_k
    against the oracle up to the full k."""
    p = P.make("deblur64")
    k, m_s = 300, 1200
    ctx = gpu_context(p, storage, k=k, m_s=m_s, pivot_fwd=pivot_fwd)
    ctx.step(k)
    status, kd = ctx.sync()
    assert kd == [k]
    # past j ~ 70 this smooth operator's residual is at rounding level and the
    # pivot order chaotic even in FP64, so the pivots are checked against the
    # oracle's own divergence under perturbations of the same size (in every
    # storage type), and x_k by replaying the GPU's pivots
    verify_scmrh(ctx, p, storage, [50, 150, 225, 300], [0.0, 1e-3], k=k, m_s=m_s,
                 name=f"large_k300_{storage}_fwd{pivot_fwd}")
    ctx.close()


def test_ragged_psf_image():
    rng = np.random.default_rng(7)
    H, W = 100, 130
    psf = P.gaussian_psf(9, 1.5)
    x = P.ellipse_phantom(H, W, 6, rng)
    b = P.add_noise(P.blur_fft(x, psf), 0.01, rng).astype(np.float32)
    p = P.Problem("ragged", "psf2d", H, W, b.reshape(1, -1), x.reshape(-1), k=25, m_s=100, zeta=8,
                  sketch_seed=99, psf=psf)
    ctx = gpu_context(p, "f32")
    ctx.step(p.k)
    verify_scmrh(ctx, p, "f32", [3, 10, 25], [0.0, 1e-2], require_all_pivots=True, name="ragged100x130_f32")
    ctx.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_ct_batched_rhs(storage):
    p = P.ct_parallel(side=48, nrhs=4, k=30, m_s=120)
    ctx = gpu_context(p, storage)
    ctx.step(p.k)
    status, kd = ctx.sync()
    assert kd == [p.k] * 4
    for r in range(4):
        verify_scmrh(ctx, p, storage, [1, 5, 15, 30], [0.0, 1.0], r=r, kd=kd[r],
                     require_all_pivots=storage == "f32", name=f"ct48_batch4_{storage}_rhs{r}")
    ctx.close()


def test_batch_equals_single():
    """A RHS solved inside a batch gives the same bits as solved alone."""
    p = P.ct_parallel(side=32, nrhs=8, k=12, m_s=48)
    ctx = gpu_context(p, "f32")
    ctx.step(p.k)
    xb, _ = ctx.solve(p.k, [0.0, 0.5])
    ctx.close()
    for r in (0, 5):
        single = gpu_context(p, "f32", nrhs=1, b=p.b[r:r + 1])
        single.step(p.k)
        xs, _ = single.solve(p.k, [0.0, 0.5])
        single.close()
        assert np.array_equal(xb[:, r], xs[:, 0])


def test_breakdown_on_invariant_subspace():
    n = 64
    d = np.linspace(1.0, 2.0, n).astype(np.float32)
    rowptr = np.arange(n + 1, dtype=np.int64)
    colind = np.arange(n, dtype=np.int32)
    b = np.zeros((2, n), np.float32)
    b[0, 5] = 3.0                 # eigenvector: breakdown after one step
    b[1, :] = 0.0                 # zero RHS: nothing to do
    p = P.Problem("diag", "csr", 8, 8, b, np.zeros((2, n)), k=4, m_s=16, zeta=8, sketch_seed=3,
                  rowptr=rowptr, colind=colind, vals=d)
    from paper_2502_02721_gb300 import binding as bd
    ctx = gpu_context(p, "f32", nrhs=2)
    ctx.step(4)
    status, kd = ctx.sync()
    assert status == bd.IPF_BREAKDOWN and kd == [1, 0]
    x, info = ctx.solve(4, [0.0])
    assert info[0][:2] == (1, 1) and info[1][:2] == (0, 0)
    want = np.zeros(n)
    want[5] = 3.0 / d[5]
    assert rel(x[0, 0], want) < 1e-6
    assert not np.any(x[0, 1])
    ctx.close()


def test_state_errors():
    from paper_2502_02721_gb300 import binding as bd
    p = P.make("deblur64")
    ctx = gpu_context(p, "f32", k=5)
    with pytest.raises(bd.IpfError) as ei:
        ctx.solve(3, [0.0])
    assert ei.value.code == bd.IPF_ERR_STATE
    assert ctx.step(10) == 5                       # clipped to k_max
    x, info = ctx.solve(5, [0.0])
    assert info[0][0] == 5
    ctx.close()
