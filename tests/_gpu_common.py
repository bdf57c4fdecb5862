"""Shared helpers for the GPU parity tests: run the CUDA path through the
C ABI, run the FP64 oracle on the same seeded inputs, compare."""
import os

import numpy as np

from gen import problems as P
from oracle import operators as ops, scmrh, sketch as sk

U = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}
# x is returned in float32 by the ABI, so even F64 storage cannot beat ~1e-7
FLOOR = {"f64": 2e-7, "f32": 1e-4, "bf16": 1e-3, "f16": 1e-3}
TIE = {"f64": 1e-12, "f32": 1e-6, "bf16": 3 * 2.0 ** -8, "f16": 3 * 2.0 ** -11}


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


def oracle_run(p, r=0, k=None, m_s=None, forced=None):
    A = ops.make_apply(p)
    S = sk.SparseSignSketch(p.sketch_seed, p.n, m_s or p.m_s, p.zeta)
    return scmrh.run(A, p.b[r].astype(np.float64), S, k or p.k, forced_pivots=forced)


def tolerance(storage, kappa):
    """max(floor, 10 u_s kappa(Z_k)): the stated floor, widened to the
    first-order least-squares perturbation bound where kappa makes the floor
    unreachable in the storage precision."""
    return max(FLOOR[storage], 10.0 * U[storage] * kappa)


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


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


def compare_solution(ctx, st, storage, ks, lambdas, r=0, zform="hessenberg"):
    """x_k from the GPU against the oracle for each k and lambda."""
    worst = []
    for k in ks:
        x, info = ctx.solve(k, lambdas)
        Z = scmrh.projected_matrix(st, k, zform)
        kappa = np.linalg.cond(Z)
        tol = tolerance(storage, kappa)
        for li, lam in enumerate(lambdas):
            x_or = scmrh.solve(st, k, lam)
            e = rel(x[li, r].astype(np.float64), x_or)
            worst.append((k, lam, e, tol))
            assert e <= tol, (k, lam, e, tol, kappa)
    return worst
