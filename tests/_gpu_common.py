"""Shared helpers for the GPU parity tests: run the CUDA path through the
C ABI, run the FP64 oracle on the same seeded inputs, compare, and record
the errors reached.

The comparison of iterates (verify_scmrh) has two parts.

Parity.  The oracle runs the same method with the basis kept in the same
storage type (oracle/storage.py) and replays the GPU's pivot sequence;
what is left between the two is the GPU's FP32 accumulation (FP64 for F64
storage) in the products and the elimination.  The bound is taken from the
oracle's own response to that: the replay is run again with every product
perturbed elementwise by a relative N(0, delta^2) error, delta = sqrt(K)
u_acc for K-term sums (plus the 2^-17 PSF split of the tensor-core product),
and the GPU must stay within max(floor, 10 x that response).

The stated tolerance.  1e-4 (FP32) and 1e-3 (BF16, FP16) relative to the
FP64 oracle are asserted wherever they are reachable in that storage type,
by two criteria taken from the arithmetic, both required: the first-order
least-squares bound kappa(Z_k) u_s is within the stated tolerance, and the
oracle's storage-rounded run, with every product perturbed by the RMS
rounding error of a K-term sum in the accumulation type (delta =
sqrt(K / 12) u_acc: K roundings, each uniform within half a unit), stays
within a third of it.  Where either fails (BF16 from k = 1 on, FP16 beyond
the first steps, FP32 where kappa(Z_k) amplifies its rounding past 1e-4),
the record says so; the parity check still holds there.

Every comparison is appended to RECORD (test, storage, k, lambda, the
errors and bounds); conftest.py prints the worst cases at the end of the
run and writes all of them to parity_errors.json in the folder named by
IPF_PARITY_RECORD_DIR when that is set.
"""
import os

import numpy as np

from gen import problems as P
from oracle import operators as ops, scmrh, sketch as sk

U = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}
# accumulation unit of each storage mode's arithmetic
U_ACC = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -24, "f16": 2.0 ** -24}
# the stated tolerances against the FP64 oracle; x is returned in float32, so
# even F64 storage cannot beat ~1e-7
STATED = {"f64": 2e-7, "f32": 1e-4, "bf16": 1e-3, "f16": 1e-3}
FLOOR = STATED
# floor of the parity bound: the float32 rounding of x itself
PAR_FLOOR = 2e-7
TIE = {"f64": 1e-12, "f32": 1e-6, "bf16": 3 * 2.0 ** -8, "f16": 3 * 2.0 ** -11}
PSF_SPLIT = 2.0 ** -17           # |F - hi - lo| / |F| of the tensor-core PSF operand

RECORD = []


def ensure_lib():
    import torch
    from paper_2502_02721_gb300 import binding, build
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    if not os.path.exists(build.lib_path()):
        build.build()
    return binding.load()


def gpu_context(p, storage, k=None, m_s=None, zform=None, penalty=None, graphs=1, nrhs=None, b=None, **extra):
    from paper_2502_02721_gb300 import binding as bd
    keep = []
    op = bd.operator_from_problem(p, keep)
    kw = dict(k_max=k or p.k, m_s=m_s or p.m_s, zeta=p.zeta, seed=p.sketch_seed, storage=storage,
              nrhs=nrhs or p.nrhs, use_graphs=graphs)
    if zform is not None:
        kw["zform"] = zform
    if penalty is not None:
        kw["penalty"] = penalty
    kw.update(extra)
    cfg = bd.default_config(**kw)
    return bd.Context(op, p.b if b is None else b, cfg, keep)


def oracle_run(p, r=0, k=None, m_s=None, forced=None, storage="f64", apply=None, sketch=None):
    A = apply or ops.make_apply(p)
    S = sketch or sk.SparseSignSketch(p.sketch_seed, p.n, m_s or p.m_s, p.zeta)
    return scmrh.run(A, p.b[r].astype(np.float64), S, k or p.k, forced_pivots=forced, storage=storage)


def tolerance(storage, kappa):
    """max(floor, 10 u_s kappa(Z_k)): the first-order least-squares bound
    for a basis perturbed at the storage rounding (used where the iterate
    is compared with the unrounded FP64 oracle, e.g. the sLSLU tests)."""
    return max(FLOOR[storage], 10.0 * U[storage] * kappa)


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def first_divergence(a, b, k):
    return next((j for j in range(min(len(a), len(b), k + 1)) if int(a[j]) != int(b[j])),
                min(len(a), len(b), k + 1))


def compare_pivots(gpu_piv, st, storage):
    """Pivots identical up to near ties.  Returns the number of leading
    pivots that agree (all of them unless a near tie was resolved the other
    way, which is then checked to be a near tie)."""
    n = min(len(gpu_piv), len(st.piv))
    for j in range(n):
        if int(gpu_piv[j]) != int(st.piv[j]):
            assert st.gaps[j] < TIE[storage], (j, gpu_piv[j], st.piv[j], st.gaps[j])
            return j
    return n


def perturbed(apply_A, delta, seed):
    """apply_A with every output entry perturbed by a relative N(0, delta^2) error."""
    rng = np.random.default_rng(seed)
    return lambda v: (lambda w: w * (1.0 + delta * rng.standard_normal(w.size)))(apply_A(v))


def product_terms(p):
    """K: the number of nonzero terms of one output entry of A v."""
    if p.kind == "csr":
        return int(np.max(np.diff(p.rowptr)))
    if p.kind == "psf2d":
        return int(np.count_nonzero(p.psf))
    return int(np.count_nonzero(p.sep_row) + np.count_nonzero(p.sep_col) + np.count_nonzero(p.motion))


def uses_tensor_cores(p, storage, conv_fma=0):
    kw = max(p.psf.shape) if p.kind == "psf2d" else 0
    return storage == "bf16" and not conv_fma and p.kind == "psf2d" and 7 < kw <= 31 and p.cols % 8 == 0


_REF64 = {}


def _ref64(p, r, k, apply, sketch=None, m_s=None):
    key = (p.name, p.rows, p.cols, p.sketch_seed, r, k, m_s or p.m_s, id(sketch))
    if key not in _REF64:
        _REF64[key] = oracle_run(p, r=r, k=k, apply=apply, sketch=sketch, m_s=m_s)
    return _REF64[key]


def verify_scmrh(ctx, p, storage, ks, lambdas, r=0, k=None, conv_fma=0, zform="hessenberg", name="", kd=None,
                 require_all_pivots=False, check_pivots=True, penalty="sketched_x", sketch=None, sketch64=None,
                 m_s=None, contraction_terms=0):
    """Pivots and iterates of the GPU context against the oracle (module
    docstring).  check_pivots=False leaves the pivot check to the caller
    (e.g. sampled pivoting, whose choices the caller checks); the iterates
    are compared by replaying the GPU's pivots either way.  sketch /
    sketch64: the oracle's sketch in the storage type and in FP64 (default:
    the sparse-sign sketch of the problem, m_s rows).  contraction_terms > 0
    (the Gaussian sketch, S V_{k+1} formed at solve time by a sum of that
    many products per entry) adds 10 sqrt(terms) u_acc kappa(Z_k) to the
    parity bound: that sum's rounding carried to y.  Returns the records of
    this call."""
    kk = k or p.k
    A = ops.make_apply(p)
    ex = ctx.export(r)
    if kd is None:
        kd = ctx.sync()[1][r]
    gpiv = [int(v) for v in ex["piv"][:kd + 1]]
    assert min(gpiv) >= 0
    ref64 = _ref64(p, r, kk, A, sketch64 or sketch, m_s)
    run = lambda **kw: oracle_run(p, r=r, k=kk, m_s=m_s, sketch=sketch, **kw)
    own = ref64 if storage == "f64" and sketch64 is None else run(storage=storage, apply=A)
    delta = np.sqrt(product_terms(p)) * U_ACC[storage] + (PSF_SPLIT if uses_tensor_cores(p, storage, conv_fma) else 0.0)
    # pivots: identical to the storage-rounded oracle's own choices until at
    # least the step where that oracle, perturbed at the GPU's accumulation
    # level, first departs from itself (earliest of three seeds, less 3)
    j_gpu = first_divergence(gpiv, own.piv, kd)
    if require_all_pivots:
        assert compare_pivots(gpiv, own, storage) == kd + 1, "pivots diverged (near tie)"
    if check_pivots and j_gpu <= kd:
        j_or = kd + 1
        for seed in (1, 2, 3):
            sp = run(storage=storage, apply=perturbed(A, delta, seed))
            j_or = min(j_or, first_divergence(sp.piv, own.piv, kd))
        assert j_gpu >= j_or - 3, (j_gpu, j_or)
    rep = run(forced=gpiv, storage=storage, apply=A)
    rep_p = run(forced=gpiv, storage=storage, apply=perturbed(A, delta, 12345))
    # the RMS rounding of a K-term sum of the products
    delta_typ = np.sqrt(product_terms(p) / 12.0) * U_ACC[storage] + \
        (PSF_SPLIT if uses_tensor_cores(p, storage, conv_fma) else 0.0)
    rep_m = run(forced=gpiv, storage=storage, apply=perturbed(A, delta_typ, 54321))
    out = []
    for k1 in ks:
        if k1 > kd:
            continue
        x, info = ctx.solve(k1, lambdas)
        for li, lam in enumerate(lambdas):
            xg = x[li, r].astype(np.float64)
            xr = scmrh.solve(rep, k1, lam, zform, penalty)
            resp = rel(scmrh.solve(rep_p, k1, lam, zform, penalty), xr)
            tol_par = max(PAR_FLOOR, 10.0 * resp)
            kappa = np.linalg.cond(scmrh.projected_matrix(rep, k1, zform))
            if contraction_terms:
                tol_par = max(tol_par, 10.0 * np.sqrt(contraction_terms) * U_ACC[storage] * kappa)
            e_par = rel(xg, xr)
            x64 = scmrh.solve(ref64, k1, lam, "hessenberg", penalty)
            e64 = rel(xg, x64)
            d_s = rel(xr, x64)
            r_typ = rel(scmrh.solve(rep_m, k1, lam, zform, penalty), xr)
            stated = STATED[storage]
            reach = kappa * U[storage] <= stated and d_s + 3.0 * r_typ <= stated
            rec = {"test": name, "storage": storage, "k": k1, "lam": lam, "e_par": e_par, "tol_par": tol_par,
                   "e64": e64, "stated": stated, "storage_only": d_s, "rms_rounding": r_typ, "kappa": kappa,
                   "stated_reachable": bool(reach), "pivots_agree": j_gpu}
            RECORD.append(rec)
            out.append(rec)
            assert e_par <= tol_par, rec
            if reach:
                assert e64 <= stated, rec
    return out


def compare_solution(ctx, st, storage, ks, lambdas, r=0, zform="hessenberg", name=""):
    """x_k from the GPU against the FP64 oracle state st for each k and
    lambda, within the stated tolerance widened to the first-order
    perturbation bound (kept for callers that compare with an unrounded
    oracle directly); records what was reached."""
    worst = []
    for k in ks:
        x, info = ctx.solve(k, lambdas)
        Z = scmrh.projected_matrix(st, k, zform)
        kappa = np.linalg.cond(Z)
        tol = tolerance(storage, kappa)
        for li, lam in enumerate(lambdas):
            x_or = scmrh.solve(st, k, lam)
            e = rel(x[li, r].astype(np.float64), x_or)
            RECORD.append({"test": name, "storage": storage, "k": k, "lam": lam, "e64": e, "tol": tol,
                           "stated": STATED[storage]})
            worst.append((k, lam, e, tol))
            assert e <= tol, (k, lam, e, tol, kappa)
    return worst
