#!/usr/bin/env python
"""Throughput of the sCMRH hot path on GB300 (one JSON line on rank 0).

One step = one whole solve through the C ABI: initialisation (pivot of b,
v_1, sketches), k Hessenberg steps (operator, pivot-block solve, update +
argmax + the sketch of the newest column, normalise) and the sketched
projected solve with x = V_k y.  The timed region runs the library default
(Hessenberg steps replayed from CUDA graphs, eight steps per launch); per-kernel
times and the roofline come
from a second, profiled pass of the same workload (CUDA events around every
launch on the library's streams).

Default workload: 2048 x 2048 deblurring with a 31 x 31 Moffat PSF
(beta 2.5, alpha 4), ellipse phantom, 1% noise, k = 200, m_s = 800, zeta 8,
basis stored in BF16 with FP32 accumulation (FP64 pivot-block and projected
solves).  The FP32-storage form of the same workload is timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica (the method
does not shard across GPUs here); value = all ranks' iterations / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "iters/s & solves/s, BF16 vs FP32 GPU at rel-err<=1e-3 vs FP64; p50/p99 latency"
WORKLOAD = ("deblur 2048x2048, Moffat 31x31 PSF (beta 2.5, alpha 4), ellipse phantom, 1% noise; "
            "k=200, m_s=800, zeta=8; basis BF16 storage, FP32 accumulate; x = V_k y per solve")
K_ITERS = 200

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# kernels named in the roofline, averaged over the steps of this workload,
# from ncu on single launches of the 1024 x 1024 case (--small bf16) scaled
# to 2048 x 2048 by the units processed: the update at steps j = 19 and 49
# (54.71 and 120.32 MB) fits T(j) = 1.043 (j+1) 2n + 10.47 n bytes, which at
# n = 2048^2 averages 923.1 MB over j = 0..199; the convolution read 2.25 MB
# for 2n = 2.10 MB of v_j, 8.98 MB at 2048^2.  Cleared whenever a kernel
# changes.
TRAFFIC: dict = {"update": 923.1e6, "conv": 8.98e6}

# the accuracy gate: FP64 oracle iterates of the 1024 x 1024 Moffat case
# (k = 64, m_s = 256) and of the first steps of the 2048 x 2048 workload,
# against which the GPU's BF16, FP16 and FP32 forms are measured
GATE_SIDE, GATE_K, GATE_MS = 1024, 64, 256
GATE_KS = (1, 8, 64)
GATE_LAMS = (0.0, 1e-2)
GATE2048_K = 5


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _bf16_peak():
    """Dense BF16 tensor peak for a kernel timed inside a long step: the
    sustained measured figure, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]), "measured bf16_tflops_sustained"
    except Exception:
        return 1700.0, "fallback (sustained)"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _gpu_id(torch, dev):
    try:
        props = torch.cuda.get_device_properties(dev)
        bus = getattr(props, "pci_bus_id", None)
        dom = getattr(props, "pci_domain_id", 0)
        devid = getattr(props, "pci_device_id", 0)
        if bus is not None:
            return f"{dom:08X}:{bus:02X}:{devid:02X}.0"
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        return vis.split(",")[dev]
    return str(dev)


# ---------------------------------------------------------------------------
# the FP64 oracle on a bounded sample (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
ORACLE_SAMPLE = ("oracle (numpy float64) on the full 2048x2048 problem: Hessenberg steps 1..{s} after the "
                 "initialisation (each: one 31x31 convolution, the sequential elimination, the max pivot, two "
                 "sketches); {r} replicas at once, one per host core, one thread each; its step cost grows with j "
                 "(the elimination is O(j n)), so this rate is an upper bound on its rate over j = 1..200")


def oracle_gate_child(side: int, k: int, m_s: int, ks, lams, out_path: str):
    """The FP64 oracle on the side x side Moffat workload for k steps (one
    thread), x_k for each k in ks and lambda in lams, and the step times."""
    from gen import problems as P
    from oracle import operators as ops, scmrh, sketch as sk
    p = P.make("deblur2048") if side == 2048 else P.deblur_moffat(side=side, k=k, m_s=m_s)
    A = ops.make_apply(p)
    S = sk.SparseSignSketch(p.sketch_seed, p.n, p.m_s, p.zeta)
    t0 = time.perf_counter()
    times, xs = [], {}
    for j, st in scmrh.iterate(A, p.b[0], S, k):
        times.append(time.perf_counter() - t0)
        if j in ks:
            for li, lam in enumerate(lams):
                xs[f"x{j}_{li}"] = scmrh.solve(st, j, lam)
    np.savez(out_path, times=np.array(times), **xs)


def start_child(fn: str, args: tuple):
    """Start bench.<fn>(*args, out) in a fresh interpreter (one BLAS thread);
    returns (process, output path)."""
    import tempfile
    out = os.path.join(tempfile.mkdtemp(prefix="ipf_oracle_"), "o.npz")
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = f"import sys; sys.path.insert(0, {ROOT!r}); import bench; bench.{fn}(*{args!r}, {out!r})"
    return subprocess.Popen([sys.executable, "-c", code], env=env), out


def finish_child(h) -> dict:
    proc, out = h
    if proc.wait() != 0:
        raise RuntimeError(f"oracle child failed ({proc.returncode})")
    d = np.load(out)
    times = d["times"]
    x = {}
    for key in d.files:
        if key.startswith("x"):
            kk, li = key[1:].split("_")
            x[(int(kk), int(li))] = d[key]
    return {"init_s": float(times[0]), "step_s": [float(times[i] - times[i - 1]) for i in range(1, len(times))],
            "x": x}


def oracle_replicas(steps: int, cores: int) -> dict:
    """`cores` independent replicas of the oracle (init + `steps` steps of the
    2048 x 2048 workload, one thread each) at once on the host: the
    oracle's aggregate rate on all cores."""
    hs = [start_child("oracle_gate_child", (2048, steps, 800, (), ())) for _ in range(cores)]
    res = [finish_child(h) for h in hs]
    rate = sum(len(r["step_s"]) / sum(r["step_s"]) for r in res)
    return {"iters_per_s": rate, "replicas": cores, "steps_each": steps,
            "step_s_median": float(np.median([t for r in res for t in r["step_s"]]))}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def max_over_ranks(torch, dist, t_ms: float, device: str) -> float:
    """The slowest rank's time (all ranks get it); t_ms itself on one process."""
    if dist is None:
        return float(t_ms)
    tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def replica_throughput(world: int, steps: int, k: int, t_max_ms: float) -> float:
    """Whole-job Hessenberg iterations/s: every rank solves `steps` times with
    k iterations each (independent replicas), over the slowest rank's time."""
    return world * steps * k / (t_max_ms * 1e-3)


def run_ours(args, rank, world, torch, dist):
    from gen import problems as P
    from paper_2502_02721_gb300 import binding as bd, build as bl
    if not os.path.exists(bl.lib_path()):
        bl.build()
    bd.load()
    lead = rank == 0 and world == 1 and not args.no_cpu_baseline
    # the FP64 oracle legs of the accuracy gate run on host cores beside the
    # GPU work (fresh interpreters, one thread each)
    gate_h = None
    if lead:
        gate_h = (start_child("oracle_gate_child", (GATE_SIDE, GATE_K, GATE_MS, GATE_KS, GATE_LAMS)),
                  start_child("oracle_gate_child", (2048, GATE2048_K, 800, tuple(range(1, GATE2048_K + 1)),
                                                    GATE_LAMS)))
    dev = torch.cuda.current_device()
    p = P.make("deblur2048")
    n = p.n
    k = K_ITERS
    stream = torch.cuda.current_stream()
    keep = []
    op = bd.operator_from_problem(p, keep)
    b_dev = torch.from_numpy(p.b.copy()).to(f"cuda:{dev}")

    def make_ctx(storage, profile):
        cfg = bd.default_config(k_max=k, m_s=p.m_s, zeta=p.zeta, seed=p.sketch_seed, storage=storage,
                                profile=profile, use_graphs=0 if profile else 1, stream=stream.cuda_stream,
                                overlap=args.overlap)
        return bd.Context(op, b_dev, cfg, keep)

    def timed_solves(ctx, x_out, steps, warmup, lam=(0.0,)):
        for _ in range(warmup):
            ctx.reset(b_dev)
            ctx.step(k)
            ctx.solve(k, lam, out=x_out, wait=False)
        torch.cuda.synchronize()
        ctx.profile_read()                       # drop warm-up kernel times
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        evs[0].record(stream)
        for s_ in range(steps):
            ctx.reset(b_dev)
            ctx.step(k)
            ctx.solve(k, lam, out=x_out, wait=False)
            evs[s_ + 1].record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        per = [evs[s_].elapsed_time(evs[s_ + 1]) for s_ in range(steps)]
        total = evs[0].elapsed_time(evs[-1])
        prof = ctx.profile_read()
        st, kd = ctx.sync()
        return total, per, prof, kd

    # --- BF16 (headline) --------------------------------------------------
    clocks = ClockSampler(_gpu_id(torch, dev))
    ctx16 = make_ctx("bf16", 0)
    x16 = torch.zeros((1, 1, n), dtype=torch.float32, device=f"cuda:{dev}")
    clocks.start()
    t16, per16, prof16, kd16 = timed_solves(ctx16, x16, args.steps, args.warmup)
    clk = clocks.stop()
    t_max = max_over_ranks(torch, dist, t16, f"cuda:{dev}")

    # --- per-kernel times: the same workload in profile mode (events around
    # every launch, eager), a separate pass after the timed region --------
    ctx16p = make_ctx("bf16", 1)
    x16p = torch.zeros((1, 1, n), dtype=torch.float32, device=f"cuda:{dev}")
    steps_p = max(1, min(args.steps, 3))
    tp, _, prof16, _ = timed_solves(ctx16p, x16p, steps_p, 1)
    ctx16p.close()
    del x16p

    # --- FP32 and FP16 storage, same workload -------------------------------
    ctx32 = make_ctx("f32", 0)
    x32 = torch.zeros((1, 1, n), dtype=torch.float32, device=f"cuda:{dev}")
    steps32 = max(1, min(args.steps, 5))
    t32, per32, prof32, kd32 = timed_solves(ctx32, x32, steps32, 1)
    ctxh = make_ctx("f16", 0)
    xh = torch.zeros((1, 1, n), dtype=torch.float32, device=f"cuda:{dev}")
    th, perh, _, kdh = timed_solves(ctxh, xh, steps32, 1)

    nrm = lambda a: float(np.linalg.norm(a))
    acc = {}
    xb = x16[0, 0].double().cpu().numpy()
    xf = x32[0, 0].double().cpu().numpy()
    acc["k200_relerr_bf16_vs_fp32"] = nrm(xb - xf) / nrm(xf)
    acc["k200_err_vs_xtrue"] = {"bf16": nrm(xb - p.x_true) / nrm(p.x_true), "fp32": nrm(xf - p.x_true) / nrm(p.x_true)}

    # --- accuracy gate, GPU side: the first steps of this workload, and the
    # 1024 x 1024 case up to k = 64, in every storage form ------------------
    gate_gpu = {}
    for name, ctx in (("bf16", ctx16), ("fp32", ctx32), ("fp16", ctxh)):
        ctx.reset(b_dev)
        ctx.step(GATE2048_K)
        for kk in range(1, GATE2048_K + 1):
            xs_, _ = ctx.solve(kk, list(GATE_LAMS))
            for li in range(len(GATE_LAMS)):
                gate_gpu[("2048", name, kk, li)] = xs_[li, 0].astype(np.float64)
    p1k = P.deblur_moffat(side=GATE_SIDE, k=GATE_K, m_s=GATE_MS)
    keep1k = []
    op1k = bd.operator_from_problem(p1k, keep1k)
    for name, stg in (("bf16", "bf16"), ("fp32", "f32"), ("fp16", "f16")):
        cfg = bd.default_config(k_max=GATE_K, m_s=GATE_MS, zeta=8, seed=p1k.sketch_seed, storage=stg,
                                stream=stream.cuda_stream)
        ctx = bd.Context(op1k, p1k.b, cfg, keep1k)
        ctx.step(GATE_K)
        for kk in GATE_KS:
            xs_, _ = ctx.solve(kk, list(GATE_LAMS))
            for li in range(len(GATE_LAMS)):
                gate_gpu[(str(GATE_SIDE), name, kk, li)] = xs_[li, 0].astype(np.float64)
        ctx.close()

    # --- end to end: pinned host b in, host x out, through the C ABI ------
    b_host = torch.from_numpy(p.b.copy()).pin_memory()
    x_host = torch.zeros((1, 1, n), dtype=torch.float32).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))
    ctx16.reset(b_host)
    ctx16.step(k)
    ctx16.solve(k, [0.0], out=x_host)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx16.reset(b_host)
        ctx16.step(k)
        ctx16.solve(k, [0.0], out=x_host)
    torch.cuda.synchronize()
    t_e2e_ms = max_over_ranks(torch, dist, 1e3 * (time.perf_counter() - t0), f"cuda:{dev}")
    ctx16.profile_read()

    # --- roofline of the dominant kernel ------------------------------------
    ms, cnt, byts = prof16
    names = ["operator", "pivot_solve", "update_or_Vh", "normalize", "init", "solve_qr", "solve_x",
             "pivot_rows", "combine", "gauss_gemm", "sample_pivot", "sketch_deferred"]
    busy = sum(ms)
    kern = {names[i]: {"ms_total": ms[i], "launches": int(cnt[i]),
                       "share": ms[i] / max(busy, 1e-9),
                       "GBps_incl_overhead": (byts[i] / (ms[i] * 1e-3) / 1e9) if ms[i] > 0 and byts[i] > 0 else None}
            for i in range(len(names)) if cnt[i] > 0}
    peak, peak_kind = _peaks()
    # the method's bytes of one update launch: step j reads V_j, (j+1) n s_V
    # bytes, averaged over j = 0..k-1 of the profiled solves
    alg_upd = 2.0 * n * (k + 1) / 2.0
    over_upd = 8.0 * n + n / 8.0 + 8.0 * n
    t_upd = ms[2] / max(cnt[2], 1) * 1e-3
    ach = alg_upd / t_upd / 1e9 if ms[2] > 0 else None
    roof = {"kernel": "k_update_f<bf16,1> (w -= V_j h, the max-|w| pivot, S v_j of the newest column)",
            "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": (ach / peak) if ach else None, "traffic": TRAFFIC.get("update"),
            "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_launch": alg_upd,
            "algorithmic_bytes": "per launch at step j: (j+1)*n*2, the read of V_j (BF16), averaged over "
                                 "j = 0..199",
            "overhead_bytes_per_launch": over_upd,
            "overhead_bytes": "8n (read and write of the FP32 work vector w) + n/8 (pivot bitmap) + 8n (sketch "
                              "table: the kernel also sketches the newest column v_j); implementation choices, "
                              "not counted in frac",
            "us_per_launch": t_upd * 1e6}
    # the convolution runs on the tensor cores (BF16 operands, FP32
    # accumulation); useful work is the convolution itself, 2 x 31 x 31 flops
    # per pixel, against the dense BF16 tensor peak
    conv_flops = 2.0 * 961 * n * cnt[0]
    conv_tf = conv_flops / (ms[0] * 1e-3) / 1e12 if ms[0] > 0 else None
    tpeak, tpeak_src = _bf16_peak()
    roof_conv = {"kernel": "k_conv2d_tc<32> (w = P * v_j, tcgen05)", "bound": "tensor", "achieved": conv_tf,
                 "peak": tpeak, "unit": "TFLOP/s", "frac": (conv_tf / tpeak) if conv_tf else None,
                 "traffic": TRAFFIC.get("conv"), "peak_source": tpeak_src,
                 "us_per_launch": ms[0] / max(cnt[0], 1) * 1e3,
                 "algorithmic_flops": "2 x 31 x 31 x n per launch (n = 2048^2); the MMAs execute 2 x 2 x 80 x 256 "
                                      "per 8 image rows x 128 columns (K and N padding, two PSF parts)"}
    dominant = max(range(len(ms)), key=lambda i: ms[i])
    launches_p = int(cnt[0] + cnt[1] + cnt[2] + cnt[3] + 4 * cnt[4] + 2 * cnt[5] + 2 * cnt[6] + cnt[7] + cnt[8]
                     + cnt[9] + cnt[10] + cnt[11])
    launches = launches_p * args.steps // steps_p          # the profiled pass ran steps_p solves

    value = replica_throughput(world, args.steps, k, t_max)
    config = static_config(args, world)
    out = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config,
        "solves_per_s": world * args.steps / (t_max * 1e-3),
        "latency_ms": {"p50": float(np.percentile(per16, 50)), "p99": float(np.percentile(per16, 99))},
        "fp32": {"iters_per_s": steps32 * k / (t32 * 1e-3), "solves_per_s": steps32 / (t32 * 1e-3),
                 "ms_per_solve": t32 / steps32},
        "fp16": {"iters_per_s": steps32 * k / (th * 1e-3), "solves_per_s": steps32 / (th * 1e-3),
                 "ms_per_solve": th / steps32},
        "bf16_speedup_over_fp32": (args.steps / t16) / (steps32 / t32),
        "accuracy": acc,
        "roofline": roof if dominant in (2, 3, 6) else roof_conv,
        "roofline_other": roof_conv if dominant in (2, 3, 6) else roof,
        "kernels": kern,
        "profiled_pass": {"solves": steps_p, "ms_per_solve": tp / steps_p,
                          "how": "CUDA events around each launch on the library's streams, eager launches"},
        "gpu_launches": launches * world,
        "e2e": {"value": replica_throughput(world, e2e_steps, k, t_e2e_ms), "unit": "iters/s",
                "h2d_bytes_per_step": int(4 * n),
                "d2h_bytes_per_step": int(4 * n)},
        "clocks": {k2: clk[k2] for k2 in ("sm_mhz", "sm_max_mhz", "reasons")},
        "k_done": kd16,
    }
    ctx16.close()
    ctx32.close()
    ctxh.close()
    gate_o = None
    if rank == 0 and not args.no_extra:
        out["deblur64"] = run_deblur64(torch, stream)
        out["deblur256"] = run_deblur256(torch, stream)
        out["ct256_batch32"] = run_ct_batch(torch, stream)
        out["gaussian_sketch"] = run_gaussian(torch, stream, args.overlap)
        # the oracle children of the accuracy gate finish first: the serving
        # loop's scheduler thread must not share the host cores with them
        if gate_h is not None:
            gate_o = (finish_child(gate_h[0]), finish_child(gate_h[1]))
        sv = run_serving(args, duration=5.0)
        out["serving"] = {k2: v for k2, v in sv.items() if k2 not in ("metric", "unit", "value")}

    # --- accuracy gate against the FP64 oracle, and the CPU baseline --------
    if gate_h is not None:
        o1k, o2k = gate_o if gate_o is not None else (finish_child(gate_h[0]), finish_child(gate_h[1]))
        gate = accuracy_gate(gate_gpu, o1k, o2k, p1k)
        config.update(gate)
        acc["gate"] = gate
        cores = os.cpu_count() or 1
        rep = oracle_replicas(2, cores)
        one = len(o2k["step_s"]) / sum(o2k["step_s"])
        out["cpu_baseline"] = {
            "value": rep["iters_per_s"], "unit": "iters/s", "cores": cores, "kind": "oracle",
            "sample": ORACLE_SAMPLE.format(s=2, r=cores),
            "one_thread": {"value": one, "unit": "iters/s", "cores": 1,
                           "sample": "the same oracle alone, steps 1..%d of the 2048x2048 workload, one thread "
                                     "(init %.1f s; step times %s s)" % (
                                         len(o2k["step_s"]), o2k["init_s"],
                                         ", ".join("%.1f" % t for t in o2k["step_s"]))},
            "replica_step_s_median": rep["step_s_median"]}
    return out


def static_config(args, world: int) -> dict:
    """The workload description both arms print (the accuracy gate's
    results are added to ours)."""
    return {"workload": WORKLOAD, "n": 2048 * 2048, "k": K_ITERS, "m_s": 800, "zeta": 8, "storage": "bf16",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "inputs larger than L2: the BF16 basis is 1.69 GB (L2 129 MB)",
            "launch": "CUDA graphs of eight Hessenberg steps (the library default); kernel times and the roofline "
                      "from a second, profiled pass",
            "overlap": args.overlap}


def accuracy_gate(gpu: dict, o1k: dict, o2k: dict, p1k) -> dict:
    """Relative error of the GPU's iterates (BF16, FP16 and FP32 storage)
    against the FP64 oracle's, per k and lambda, for the config; and whether
    each form meets its stated tolerance (FP32 1e-4, BF16 / FP16 1e-3)."""
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    g = {}
    stated = {"fp32": 1e-4, "bf16": 1e-3, "fp16": 1e-3}
    met = {nm: [] for nm in stated}
    for (side, nm, kk, li), x in sorted(gpu.items()):
        o = o1k if side == str(GATE_SIDE) else o2k
        ref = o["x"][(kk, li)]
        e = rel(x, ref)
        lam = GATE_LAMS[li]
        key = f"acc_{nm}_{side}_k{kk}" + ("" if lam == 0.0 else f"_lam{lam:g}")
        if side == str(GATE_SIDE) or kk in (1, GATE2048_K):
            g[key] = e
        if e <= stated[nm]:
            met[nm].append(f"{side}k{kk}" + ("" if lam == 0.0 else "r"))
    # error against x_true of BF16 and FP32 at the 1024^2 case (regularised)
    xt = p1k.x_true
    for kk in GATE_KS:
        eb = rel(gpu[(str(GATE_SIDE), "bf16", kk, 1)], xt)
        ef = rel(gpu[(str(GATE_SIDE), "fp32", kk, 1)], xt)
        g[f"acc_xtrue_bf16_minus_fp32_k{kk}_lam{GATE_LAMS[1]:g}"] = eb - ef
    g["acc_meets_stated"] = "; ".join(f"{nm}<={stated[nm]:g}: " + (",".join(v) if v else "none")
                                      for nm, v in met.items())
    return g


def _time_ctx(torch, stream, ctx, b_dev, k, lams, steps, warmup):
    """ms per solve (reset + k steps + the solve for every lambda, x on the
    device), CUDA events on the library's caller stream."""
    x = torch.zeros((len(lams), 1, b_dev.shape[-1]), dtype=torch.float32, device=b_dev.device)
    for _ in range(warmup):
        ctx.reset(b_dev)
        ctx.step(k)
        ctx.solve(k, lams, out=x, wait=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.reset(b_dev)
        ctx.step(k)
        ctx.solve(k, lams, out=x, wait=False)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, x


def run_deblur64(torch, stream, steps: int = 50) -> dict:
    """The plain method on 64 x 64 deblurring (15 x 15 Gaussian PSF, k = 50,
    m_s = 200, lambda in {0, 1e-3}), FP64 and FP32 storage: one step = one
    solve with both lambdas."""
    from gen import problems as P
    from paper_2502_02721_gb300 import binding as bd
    p = P.make("deblur64")
    keep = []
    op = bd.operator_from_problem(p, keep)
    b_dev = torch.from_numpy(p.b.copy()).cuda()
    out = {"workload": "deblur 64x64, Gaussian 15x15 sigma 2, k=50, m_s=200, lambda {0, 1e-3}; latency-bound "
                       "(V 1.6 MB in FP64)"}
    for stg in ("f64", "f32"):
        cfg = bd.default_config(k_max=p.k, m_s=p.m_s, zeta=p.zeta, seed=p.sketch_seed, storage=stg,
                                stream=stream.cuda_stream)
        ctx = bd.Context(op, b_dev, cfg, keep)
        ms, _ = _time_ctx(torch, stream, ctx, b_dev, p.k, list(p.lambdas), steps, 3)
        out[stg] = {"ms_per_solve": ms, "solves_per_s": 1e3 / ms, "iters_per_s": p.k * 1e3 / ms}
        ctx.close()
    return out


def run_deblur256(torch, stream, steps: int = 10) -> dict:
    """256 x 256 deblurring with the separable 31-tap Gaussian then the
    9-px motion blur, k = 100, m_s = 400, the 8-lambda sweep, FP32 storage:
    one step = one solve with all 8 lambdas."""
    from gen import problems as P
    from paper_2502_02721_gb300 import binding as bd
    p = P.make("deblur256")
    keep = []
    op = bd.operator_from_problem(p, keep)
    b_dev = torch.from_numpy(p.b.copy()).cuda()
    cfg = bd.default_config(k_max=p.k, m_s=p.m_s, zeta=p.zeta, seed=p.sketch_seed, storage="f32",
                            stream=stream.cuda_stream)
    ctx = bd.Context(op, b_dev, cfg, keep)
    ms, _ = _time_ctx(torch, stream, ctx, b_dev, p.k, list(p.lambdas), steps, 2)
    ctx.close()
    return {"workload": "deblur 256x256, separable 31-tap Gaussian sigma 3 + 9-px motion, k=100, m_s=400, "
                        "8 lambdas 1e-4..1e-1; FP32 basis (V 26.5 MB, L2-resident)",
            "f32": {"ms_per_solve": ms, "solves_per_s": 1e3 / ms, "iters_per_s": p.k * 1e3 / ms}}


# ---------------------------------------------------------------------------
# reference arm: the oracle as it stands, on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    from gen import problems as P
    from oracle import operators as ops, scmrh, sketch as sk
    p = P.make("deblur2048")
    A = ops.make_apply(p)
    S = sk.SparseSignSketch(p.sketch_seed, p.n, p.m_s, p.zeta)
    total = args.warmup + args.steps
    it = scmrh.iterate(A, p.b[0], S, total)
    next(it)                                   # initialisation (not a step)
    times = []
    for s in range(total):
        t0 = time.perf_counter()
        next(it)
        times.append(time.perf_counter() - t0)
    timed = times[args.warmup:]
    t = sum(timed)
    value = args.steps / t
    sample = (f"each step = one Hessenberg step of the float64 oracle on the full 2048x2048 problem "
              f"(steps {args.warmup + 1}..{total} of one run after {args.warmup} warm-up steps), one thread")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": static_config(args, 1),
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_ct_batch(torch, stream, steps: int = 3) -> dict:
    """CT 256x256 parallel beam (256 angles x 256 detectors, CSR Siddon
    weights), 32 right-hand sides in one context, k = 150, m_s = 600: one
    step = all 32 solves (150 Hessenberg iterations each + x = V_k y), with
    the Hessenberg process on A (sCMRH) and with the generalized process on
    A and A^T (sLSLU, two products per iteration)."""
    from gen import problems as P
    from paper_2502_02721_gb300 import binding as bd
    p = P.make("ct256")
    dev = torch.cuda.current_device()
    keep = []
    op = bd.operator_from_problem(p, keep)
    b_dev = torch.from_numpy(p.b.copy()).to(f"cuda:{dev}")
    out = {"workload": "CT 256x256, 256 angles x 256 detectors, CSR FP32 (%d nonzeros), 32 RHS batched, "
                       "k=150, m_s=600" % int(p.rowptr[-1])}
    variants = (("scmrh", "f32", 0), ("scmrh", "bf16", 0), ("slslu", "f32", 0), ("slslu", "bf16", 0),
                ("slslu", "bf16", 25))
    for method, storage, sample in variants:
        cfg = bd.default_config(k_max=p.k, m_s=p.m_s, zeta=p.zeta, seed=p.sketch_seed, storage=storage,
                                nrhs=p.nrhs, use_graphs=1, stream=stream.cuda_stream, method=method,
                                pivot_sample=sample)
        ctx = bd.Context(op, b_dev, cfg, keep)
        xo = torch.zeros((1, p.nrhs, p.n), dtype=torch.float32, device=f"cuda:{dev}")
        ctx.reset(b_dev)
        ctx.step(p.k)
        ctx.solve(p.k, [0.0], out=xo, wait=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.reset(b_dev)
            ctx.step(p.k)
            ctx.solve(p.k, [0.0], out=xo, wait=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        def med_err(x):
            return float(np.median([np.linalg.norm(x[r] - p.x_true[r]) / np.linalg.norm(p.x_true[r])
                                    for r in range(p.nrhs)]))
        err = med_err(xo[0].double().cpu().numpy())
        # the iterates semi-converge on noisy data: also the best k of a few
        errs = {}
        for kk in (10, 20, 40, 80):
            xk, _ = ctx.solve(kk, [0.0])
            errs[kk] = med_err(xk[0].astype(np.float64))
        key = storage if method == "scmrh" else f"slslu_{storage}" + (f"_sampled{sample}" if sample else "")
        out[key] = {"ms_per_batch": ms, "solves_per_s": p.nrhs / (ms * 1e-3),
                    "iters_per_s": p.nrhs * p.k / (ms * 1e-3), "median_err_vs_xtrue": err,
                    "median_err_vs_xtrue_by_k": {str(kk): v for kk, v in errs.items()}}
        ctx.close()
    return out


def run_gaussian(torch, stream, overlap: int, steps: int = 3) -> dict:
    """The headline deblurring workload (2048^2, k = 200, m_s = 800, BF16
    basis) with the Gaussian embedding in place of the sparse sign sketch:
    S (800 x 2048^2, BF16, 6.7 GB) is drawn once when the context is created,
    the steps do no sketching, and each solve forms [S V_{k+1} | S b] by one
    tensor-core contraction (k_gauss_mma)."""
    from gen import problems as P
    from paper_2502_02721_gb300 import binding as bd
    p = P.make("deblur2048")
    dev = torch.cuda.current_device()
    keep = []
    op = bd.operator_from_problem(p, keep)
    b_dev = torch.from_numpy(p.b.copy()).to(f"cuda:{dev}")
    out = {"workload": "deblur 2048x2048, 31x31 Moffat PSF, k=200, m_s=800, BF16 basis, one RHS"}
    xs = {}
    for sketch in ("gaussian", "sparse_sign"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cfg = bd.default_config(k_max=p.k, m_s=p.m_s, zeta=p.zeta, seed=p.sketch_seed, storage="bf16",
                                profile=1, use_graphs=0, stream=stream.cuda_stream, overlap=overlap, sketch=sketch)
        ctx = bd.Context(op, b_dev, cfg, keep)
        torch.cuda.synchronize()
        create_s = time.perf_counter() - t0
        xo = torch.zeros((1, 1, p.n), dtype=torch.float32, device=f"cuda:{dev}")
        ctx.reset(b_dev)
        ctx.step(p.k)
        ctx.solve(p.k, [0.0], out=xo, wait=False)
        torch.cuda.synchronize()
        ctx.profile_read()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.reset(b_dev)
            ctx.step(p.k)
            ctx.solve(p.k, [0.0], out=xo, wait=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        pm, pc, pb = ctx.profile_read()
        x = xo[0, 0].double().cpu().numpy()
        xs[sketch] = x
        r = {"ms_per_solve": ms, "iters_per_s": p.k / (ms * 1e-3), "create_s": create_s,
             "err_vs_xtrue_k200": float(np.linalg.norm(x - p.x_true) / np.linalg.norm(p.x_true)),
             "normalize_ms_per_solve": pm[3] / steps, "sketch_deferred_ms_per_solve": pm[11] / steps,
             "init_ms_per_solve": pm[4] / steps}
        if sketch == "gaussian" and pc[9] > 0:
            gbs = pb[9] / (pm[9] * 1e-3) / 1e9
            peak, kind = _peaks()
            fl = 2.0 * p.m_s * p.n * (p.k + 1) * pc[9] / (pm[9] * 1e-3) / 1e12
            r["gemm"] = {"kernel": "k_gauss_mma<bf16> + k_gauss_reduce ([S V_{k+1} | S b], tcgen05, FP32 sums per "
                                   "slice, FP64 across slices)", "bound": "hbm",
                         "ms": pm[9] / pc[9], "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "peak_source": f"{kind} hbm_gbs", "tensor_tflops_useful": fl,
                         "algorithmic_bytes": "m_s*n*2 (S) + n*(k+1)*2 (V_{k+1}) per solve"}
        out[sketch] = r
        ctx.close()
    a, g = xs["sparse_sign"], xs["gaussian"]
    out["relerr_gaussian_vs_sparse_sign_k200"] = float(np.linalg.norm(g - a) / np.linalg.norm(a))
    return out


def run_serving(args, duration=None):
    """Serving workload: Poisson arrivals (200 req/s) of mixed solves, 70%
    deblurring (side U{128,256,512,1024}, Gaussian sigma U(1,4)), 30% CT
    (128^2 or 256^2 parallel beam), k U{30..150}, m_s = 4k, lambda
    log-U(1e-4, 1e-1), BF16 basis, at most 64 in flight."""
    import torch
    from gen import problems as P
    from paper_2502_02721_gb300 import binding as bd, build as bl
    if not os.path.exists(bl.lib_path()):
        bl.build()
    rng = np.random.default_rng(2502021 + 4)
    keep = []
    # pools of distinct inputs, made before the timed window
    deblur = []
    for side in (128, 256, 512, 1024):
        for _ in range(3):
            sigma = float(rng.uniform(1.0, 4.0))
            psf = P.gaussian_psf(2 * int(np.ceil(3 * sigma)) + 1, sigma)
            x = P.ellipse_phantom(side, side, 20, rng)
            b = P.add_noise(P.blur_fft(x, psf), 0.01, rng).astype(np.float32)
            deblur.append((side, psf, b.reshape(1, -1)))
    ct = []
    for side in (128, 256):
        pr = P.ct_parallel(side=side, nrhs=3)
        dev = [torch.from_numpy(a).cuda() for a in (pr.rowptr, pr.colind, pr.vals)]
        keep += dev
        n = side * side
        op = bd.make_operator("csr", n, n, rowptr=dev[0], colind=dev[1], vals=dev[2], keep=keep)
        for r in range(pr.nrhs):
            ct.append((op, pr.b[r:r + 1]))

    def serve_cfg(kind):
        kw = {}
        if args.serve_overlap is not None:
            kw["overlap"] = args.serve_overlap
        if args.serve_conv_fma is not None:
            kw["conv_fma"] = args.serve_conv_fma
        return kw

    def draw(n_req):
        plan = []
        for _ in range(n_req):
            k = int(rng.integers(30, 151))
            lam = float(10 ** rng.uniform(-4, -1))
            if rng.uniform() < 0.7:
                side, psf, b = deblur[int(rng.integers(len(deblur)))]
                op = bd.make_operator("psf2d", side, side, psf=psf, keep=keep)
                kind = f"deblur{side}"
            else:
                op, b = ct[int(rng.integers(len(ct)))]
                kind = "ct"
            cfg = bd.default_config(k_max=k, m_s=4 * k, zeta=8, seed=int(rng.integers(1 << 30)), storage="bf16",
                                    **serve_cfg(kind))
            plan.append((op, b, cfg, k, lam, kind))
        return plan

    def serve(arrivals, plan):
        srv = bd.Server(hbm_budget_bytes=64 << 30, max_inflight=64, steps_per_slice=args.serve_slice,
                        per_request=args.serve_per_request)
        tickets = []
        t0 = time.perf_counter()
        for a, (op, b, cfg, k, lam, kind) in zip(arrivals, plan):
            delay = t0 + a - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append((srv.submit(op, b, cfg, k, lam), kind))
        results = {}
        limit = float(arrivals[-1]) + 120.0
        while len(results) < len(tickets) and time.perf_counter() - t0 < limit:
            for t, kind in tickets:
                if t not in results:
                    out = srv.poll(t, want_x=False)
                    if out is not None:
                        results[t] = (out, kind)
            time.sleep(0.001)
        bstats = srv.batch_stats()
        srv.close()
        lat = np.array([r[0][2][2] - r[0][2][0] for r in results.values()])
        wait = np.array([r[0][2][1] - r[0][2][0] for r in results.values()])      # submit -> admitted
        ok = sum(1 for r in results.values() if r[0][0] in (0, 1))
        t_first = min(r[0][2][0] for r in results.values())
        span = float(max(r[0][2][2] for r in results.values()) - t_first)
        by = {}
        for (out, kind) in results.values():
            by.setdefault(kind, []).append(out[2][2] - out[2][0])
        return {"submitted": len(tickets), "completed_ok": ok, "solves_per_s": ok / span if span > 0 else 0.0,
                "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3),
                               "p99": float(np.percentile(lat, 99) * 1e3), "mean": float(lat.mean() * 1e3)},
                "latency_ms_by_kind_p50": {k2: float(np.percentile(v, 50) * 1e3) for k2, v in sorted(by.items())},
                "latency_ms_by_kind_p99": {k2: float(np.percentile(v, 99) * 1e3) for k2, v in sorted(by.items())},
                "queue_ms": {"p50": float(np.percentile(wait, 50) * 1e3), "p99": float(np.percentile(wait, 99) * 1e3)},
                "span_s": span,
                "batched_step": {"requests_batched": bstats[0], "graph_turns": bstats[1], "eager_turns": bstats[2],
                                 "graph_captures": bstats[3]}}

    rate = 200.0
    duration = float(args.serve_seconds if duration is None else duration)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * duration * 1.5) + 10))
    arrivals = arrivals[arrivals < duration]
    poisson = serve(arrivals, draw(len(arrivals)))
    # the same mix submitted all at once: what the loop sustains when saturated
    n_burst = 400
    burst = serve(np.zeros(n_burst), draw(n_burst))
    return {"metric": METRIC, "value": poisson["solves_per_s"], "unit": "solves/s",
            "workload": "serving: Poisson 200 req/s, 70% deblur (side U{128,256,512,1024}, Gaussian sigma U(1,4)), "
                        "30% CT 128^2/256^2; k U{30..150}, m_s=4k, lambda log-U(1e-4,1e-1); BF16; <=64 in flight",
            "offered_req_per_s": rate, "duration_s": duration, **{k2: v for k2, v in poisson.items()},
            "saturated": {"burst_requests": n_burst, **burst}}


def run_small(storage: str):
    """One solve of a small case (1024x1024 Moffat, k=64, m_s=256; the basis
    plus work vector exceed L2) with eager launches: the ncu target.
    storage "gauss": the same with a BF16 basis and the Gaussian sketch (S is
    256 x 1024^2 BF16, 0.5 GB), whose solve runs the tensor-core
    contraction [S V_{k+1} | S b]; "gauss800": the Gaussian sketch with the
    shape of the 2048^2 workload's contraction (m_s = 800, k = 200: four row
    groups of S, 201 basis columns) on the 1024^2 image (S 1.7 GB);
    "gauss2k256": the 2048^2 image with k = 200 and m_s = 256 (one row group,
    S 2.1 GB, V_{k+1} 1.7 GB), the full-size basis in a capture of a few GB."""
    import torch
    from gen import problems as P
    from paper_2502_02721_gb300 import binding as bd, build as bl
    if not os.path.exists(bl.lib_path()):
        bl.build()
    torch.cuda.set_device(0)
    kk, ms = (200, 800) if storage == "gauss800" else (200, 256) if storage == "gauss2k256" else (64, 256)
    side = 2048 if storage == "gauss2k256" else 1024
    p = P.deblur_moffat(side=side, k=kk, m_s=ms)
    keep = []
    op = bd.operator_from_problem(p, keep)
    gauss = storage.startswith("gauss")
    extra = {"sketch": "gaussian"} if gauss else {}
    cfg = bd.default_config(k_max=kk, m_s=ms, zeta=8, seed=p.sketch_seed,
                            storage="bf16" if gauss else storage, use_graphs=0, **extra)
    ctx = bd.Context(op, p.b, cfg, keep)
    ctx.step(kk)
    x, info = ctx.solve(kk, [0.0, 1e-3])
    print(json.dumps({"small_case": f"deblur{side} moffat31 k={kk} m_s={ms}", "storage": storage, "info": info,
                      "x_norm": float(np.linalg.norm(x[0, 0]))}))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--overlap", type=int, default=2, choices=[0, 1, 2],
                    help="second stream per step: 0 none, 1 operator beside V_j h, "
                         "2 (library default) operator beside the pivot-block solve")
    ap.add_argument("--workload", default="deblur2048", choices=["deblur2048", "serving"])
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-overlap", type=int, default=None, choices=[0, 1, 2])
    ap.add_argument("--serve-conv-fma", type=int, default=None, choices=[0, 1])
    ap.add_argument("--serve-slice", type=int, default=8, help="Hessenberg steps per serving turn")
    ap.add_argument("--serve-per-request", action="store_true",
                    help="serve without the batched step (each request on its own streams)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the CT 32-RHS batch and the 5 s serving run on the default line")
    ap.add_argument("--small", default=None, choices=["f32", "bf16", "f16", "f64", "gauss", "gauss800", "gauss2k256"],
                    help="run one small solve (profiling target) and exit")
    args = ap.parse_args()
    if args.small:
        run_small(args.small)
        return
    if args.workload == "serving" and args.impl == "ours":
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(run_serving(args)), flush=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
        if rank != 0:
            return
        print(json.dumps(run_reference(args)), flush=True)
        return
    import torch
    dist = None
    if world > 1:
        import torch.distributed as tdist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)
    out = run_ours(args, rank, world, torch, dist)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
