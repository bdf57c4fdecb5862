"""Serving (ipf_server_*): requests of different operators and sizes are
admitted while others run, overlap on the GPU, and each result equals the
same solve run alone through ipf_create/ipf_step/ipf_solve (the kernels of
one context do not depend on what else runs, so the bits agree).

With the batched step (the default), the requests it can drive share one
launch per phase per step: each result must be bit-identical served alone
and served in a mix of requests of other sizes, operators and k; on the FMA
column convolution and the CSR product it must also equal the solve alone
through a context; on the tensor-core convolution too, when the tuner's
choice is pinned to the band height the context uses."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from _gpu_common import ensure_lib  # noqa: E402
from gen import problems as P  # noqa: E402


def _requests():
    rng = np.random.default_rng(11)
    reqs = []
    for t in range(10):
        side = int(rng.choice([48, 64, 96]))
        sigma = float(rng.uniform(1.0, 2.5))
        psf = P.gaussian_psf(2 * int(np.ceil(3 * sigma)) + 1, sigma)
        x = P.ellipse_phantom(side, side, 6, rng)
        b = P.add_noise(P.blur_fft(x, psf), 0.01, rng).astype(np.float32)
        k = int(rng.integers(5, 25))
        reqs.append(dict(kind="psf2d", rows=side, cols=side, psf=psf, b=b.reshape(1, -1), k=k, m_s=4 * k,
                         lam=float(10 ** rng.uniform(-4, -1)), storage=["f32", "bf16"][t % 2], seed=1000 + t))
    ct = P.ct_parallel(side=32, nrhs=1, k=20, m_s=80)
    for t in range(4):
        k = int(rng.integers(8, 20))
        reqs.append(dict(kind="csr", rows=32, cols=32, rowptr=ct.rowptr, colind=ct.colind, vals=ct.vals,
                         b=ct.b, k=k, m_s=4 * k, lam=0.0, storage="bf16", seed=2000 + t))
    return reqs


def _op(bd, r, keep):
    if r["kind"] == "psf2d":
        return bd.make_operator("psf2d", r["rows"], r["cols"], psf=r["psf"], keep=keep)
    n = r["rows"] * r["cols"]
    return bd.make_operator("csr", n, n, rowptr=r["rowptr"], colind=r["colind"], vals=r["vals"], keep=keep)


def _serve(bd, reqs, keep, per_request=False, max_inflight=6, steps_per_slice=4, extra=None):
    """Submit all requests at once; returns the results by request index and
    the server's batch statistics."""
    srv = bd.Server(hbm_budget_bytes=2 << 30, max_inflight=max_inflight, steps_per_slice=steps_per_slice,
                    per_request=per_request)
    tickets = []
    for r in reqs:
        cfg = bd.default_config(k_max=r["k"], m_s=r["m_s"], zeta=8, seed=r["seed"], storage=r["storage"],
                                **(extra or {}))
        tickets.append(srv.submit(_op(bd, r, keep), r["b"], cfg, r["k"], r["lam"]))
    results = {}
    t0 = time.time()
    while len(results) < len(tickets) and time.time() - t0 < 120:
        for t in tickets:
            if t not in results:
                out = srv.poll(t)
                if out is not None:
                    results[t] = out
        time.sleep(0.002)
    stats = srv.batch_stats()
    srv.close()
    assert len(results) == len(tickets)
    return [results[t] for t in tickets], stats


def _alone(bd, r, keep, overlap=0, **extra):
    cfg = bd.default_config(k_max=r["k"], m_s=r["m_s"], zeta=8, seed=r["seed"], storage=r["storage"],
                            overlap=overlap, **extra)
    ctx = bd.Context(_op(bd, r, keep), r["b"], cfg, keep)
    ctx.step(r["k"])
    xa, _ = ctx.solve(r["k"], [r["lam"]])
    ctx.close()
    return xa[0]


def test_served_results_equal_solves_alone():
    ensure_lib()
    from paper_2502_02721_gb300 import binding as bd
    reqs = _requests()
    keep = []
    res, stats = _serve(bd, reqs, keep, per_request=True)
    assert stats[0] == 0                               # no request took the batched step
    results = {i: r for i, r in enumerate(res)}
    tickets = list(range(len(reqs)))
    # several requests were on the GPU at the same time
    spans = [(results[t][2][1], results[t][2][2]) for t in tickets]
    overlapping = sum(1 for i, a in enumerate(spans) for b in spans[i + 1:] if a[0] < b[1] and b[0] < a[1])
    assert overlapping > 0
    for r, t in zip(reqs, tickets):
        status, k_used, _, x = results[t]
        assert status == bd.IPF_OK and k_used == r["k"]
        # the server steps every request on one stream (overlap 0), so the
        # solve alone uses the same step
        assert np.array_equal(x, _alone(bd, r, keep)), (r["kind"], r["storage"])


def test_batched_results_alone_and_in_the_mix():
    """The batched step: every request served alone (one at a time) and in
    the mix (all at once, six in flight, so requests of different sizes,
    operators, k and step counts share launches) gives the same bits; the
    mix ran in batch slots, partly from captured graphs."""
    ensure_lib()
    from paper_2502_02721_gb300 import binding as bd
    reqs = _requests()
    keep = []
    mix, stats = _serve(bd, reqs, keep)
    assert stats[0] == len(reqs)                       # every request took a batch slot
    assert stats[1] + stats[2] > 0
    for i, r in enumerate(reqs):
        (one,), _ = _serve(bd, [r], keep, max_inflight=1)
        assert mix[i][0] == bd.IPF_OK and one[0] == bd.IPF_OK and mix[i][1] == r["k"]
        assert np.array_equal(mix[i][3], one[3]), (i, r["kind"], r["storage"])


def test_batched_fma_and_csr_equal_the_context():
    """FMA column convolution (BF16 with conv_fma, and FP32) and CSR: the
    batched step computes each element as the one-context kernels of step
    mode 2 do (products at the pivot rows beside the operator), so the served
    x equals such a context's x bit for bit."""
    ensure_lib()
    from paper_2502_02721_gb300 import binding as bd
    reqs = _requests()
    keep = []
    res, stats = _serve(bd, reqs, keep, extra={"conv_fma": 1})
    assert stats[0] == len(reqs)
    for r, out in zip(reqs, res):
        assert out[0] == bd.IPF_OK
        assert np.array_equal(out[3], _alone(bd, r, keep, overlap=2, conv_fma=1)), (r["kind"], r["storage"])


def test_batched_csr_requests_sharing_a_matrix():
    """CSR requests on one operator (one set of device arrays) share each
    pass over its nonzeros in the batched step (groups of up to sixteen);
    each request's sums keep the one-request order, so every x equals the
    context's x bit for bit, whatever the group it ran in."""
    import torch
    ensure_lib()
    from paper_2502_02721_gb300 import binding as bd
    ct = P.ct_parallel(side=32, nrhs=1, k=20, m_s=80)
    keep = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (ct.rowptr, ct.colind, ct.vals)]
    n = 32 * 32
    # device arrays: referenced by every request, not copied
    op = bd.make_operator("csr", n, n, rowptr=keep[0], colind=keep[1], vals=keep[2], keep=keep)
    rng = np.random.default_rng(5)
    reqs = []
    for t in range(20):                       # one full group of sixteen and one of four
        k = int(rng.integers(6, 20))
        b = (ct.b * (1.0 + 0.1 * rng.standard_normal(ct.b.shape))).astype(np.float32)
        reqs.append(dict(b=b, k=k, m_s=4 * k, lam=float(10 ** rng.uniform(-4, -2)),
                         storage=["bf16", "f32"][t % 3 == 2], seed=4000 + t))
    srv = bd.Server(hbm_budget_bytes=2 << 30, max_inflight=20, steps_per_slice=4)
    tickets = [srv.submit(op, r["b"], bd.default_config(k_max=r["k"], m_s=r["m_s"], zeta=8, seed=r["seed"],
                                                        storage=r["storage"]), r["k"], r["lam"]) for r in reqs]
    results = {}
    t0 = time.time()
    while len(results) < len(tickets) and time.time() - t0 < 120:
        for t in tickets:
            if t not in results:
                out = srv.poll(t)
                if out is not None:
                    results[t] = out
        time.sleep(0.002)
    stats = srv.batch_stats()
    srv.close()
    assert len(results) == len(tickets) and stats[0] == len(reqs)
    for r, t in zip(reqs, tickets):
        out = results[t]
        assert out[0] == bd.IPF_OK and out[1] == r["k"]
        cfg = bd.default_config(k_max=r["k"], m_s=r["m_s"], zeta=8, seed=r["seed"], storage=r["storage"], overlap=2)
        ctx = bd.Context(op, r["b"], cfg, keep)
        ctx.step(r["k"])
        xa, _ = ctx.solve(r["k"], [r["lam"]])
        ctx.close()
        assert np.array_equal(out[3], xa[0]), (r["storage"], r["k"])


def test_batched_tensor_cores_equal_the_context(tmp_path, monkeypatch):
    """BF16 PSF requests on the tensor-core convolution, with the tuner's
    choice pinned (IPF_TUNE_CACHE) to the band height a context uses on a
    64 x 64 image (32 output rows per CTA): the served x equals the x of a
    context in step mode 2 bit for bit."""
    ensure_lib()
    from paper_2502_02721_gb300 import binding as bd
    cache = tmp_path / "tune.json"
    cache.write_text('{"version": 1, "entries": [\n'
                     '  {"key": "conv/bf16/kw15/64x64", "variant": 1, "param": 32, "us": 1.0},\n'
                     '  {"key": "conv/bf16/kw31/64x64", "variant": 1, "param": 32, "us": 1.0}\n]}\n')
    monkeypatch.setenv("IPF_TUNE_CACHE", str(cache))
    rng = np.random.default_rng(23)
    reqs = []
    for t, sigma in enumerate((1.5, 2.0, 3.0, 3.5)):
        psf = P.gaussian_psf(2 * int(np.ceil(3 * sigma)) + 1, sigma)
        x = P.ellipse_phantom(64, 64, 6, rng)
        b = P.add_noise(P.blur_fft(x, psf), 0.01, rng).astype(np.float32)
        k = 12 + 3 * t
        reqs.append(dict(kind="psf2d", rows=64, cols=64, psf=psf, b=b.reshape(1, -1), k=k, m_s=4 * k, lam=1e-3,
                         storage="bf16", seed=3000 + t))
    keep = []
    res, stats = _serve(bd, reqs, keep)
    assert stats[0] == len(reqs)
    for r, out in zip(reqs, res):
        assert out[0] == bd.IPF_OK
        assert np.array_equal(out[3], _alone(bd, r, keep, overlap=2)), r["psf"].shape


def test_server_rejects_what_can_never_fit():
    ensure_lib()
    from paper_2502_02721_gb300 import binding as bd
    srv = bd.Server(hbm_budget_bytes=8 << 20, max_inflight=2)
    psf = P.gaussian_psf(7, 1.0)
    keep = []
    op = bd.make_operator("psf2d", 512, 512, psf=psf, keep=keep)
    cfg = bd.default_config(k_max=100, m_s=400, storage="f32")
    with pytest.raises(bd.IpfError) as ei:
        srv.submit(op, np.ones(512 * 512, np.float32), cfg, 100)
    assert ei.value.code == bd.IPF_ERR_REJECTED
    srv.close()


def test_requests_wait_for_memory_to_free():
    """An HBM budget that holds two requests at a time: six are submitted at
    once with eight slots free, so four wait for memory (not for a slot);
    the server never holds more than two, the budget is never exceeded, and
    every result equals the same request served alone."""
    import ctypes as C
    ensure_lib()
    from paper_2502_02721_gb300 import binding as bd
    lib = bd.load()
    rng = np.random.default_rng(31)
    side, k = 96, 20
    keep = []
    psf = P.gaussian_psf(9, 1.5)
    reqs = []
    for t in range(6):
        x = P.ellipse_phantom(side, side, 6, rng)
        b = P.add_noise(P.blur_fft(x, psf), 0.01, rng).astype(np.float32)
        reqs.append(dict(kind="psf2d", rows=side, cols=side, psf=psf, b=b.reshape(1, -1), k=k, m_s=4 * k,
                         lam=1e-3, storage="bf16", seed=5000 + t))
    cfg0 = bd.default_config(k_max=k, m_s=4 * k, zeta=8, seed=1, storage="bf16")
    op0 = _op(bd, reqs[0], keep)
    need = lib.ipf_footprint(C.byref(op0), C.byref(cfg0)) + 4 * side * side + (64 << 10)
    budget = int(2.5 * need)
    srv = bd.Server(hbm_budget_bytes=budget, max_inflight=8, steps_per_slice=2)
    tickets = []
    for r in reqs:
        cfg = bd.default_config(k_max=r["k"], m_s=r["m_s"], zeta=8, seed=r["seed"], storage=r["storage"])
        tickets.append(srv.submit(_op(bd, r, keep), r["b"], cfg, r["k"], r["lam"]))
    results, most, queued_seen = {}, 0, 0
    t0 = time.time()
    while len(results) < len(tickets) and time.time() - t0 < 120:
        active, queued, used = srv.stats()
        most = max(most, active)
        queued_seen = max(queued_seen, queued)
        assert used <= budget
        for t in tickets:
            if t not in results:
                out = srv.poll(t)
                if out is not None:
                    results[t] = out
        time.sleep(0.001)
    srv.close()
    assert len(results) == len(tickets)
    assert most <= 2 and queued_seen >= 1
    spans = sorted((results[t][2][1], results[t][2][2]) for t in tickets)
    for i, (a0, _) in enumerate(spans):
        assert sum(1 for b0, b1 in spans if b0 <= a0 < b1) <= 2, i       # never three admitted at once
    for r, t in zip(reqs, tickets):
        assert results[t][0] == bd.IPF_OK and results[t][1] == r["k"]
        (one,), _ = _serve(bd, [r], keep, max_inflight=1)
        assert np.array_equal(results[t][3], one[3])
