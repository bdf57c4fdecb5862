import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Errors reached by the GPU parity tests: the worst case per test
    against the storage-matched oracle (e_par / bound) and against the FP64
    oracle (e64 / stated, or why the stated bound is out of reach); the full
    record goes to parity_errors.json in the folder named by the environment
    variable IPF_PARITY_RECORD_DIR, when it is set and exists."""
    try:
        import _gpu_common as gc
    except Exception:
        return
    rec = gc.RECORD
    if not rec:
        return
    import json
    out = os.environ.get("IPF_PARITY_RECORD_DIR", "")
    if out and os.path.isdir(out):
        with open(os.path.join(out, "parity_errors.json"), "w") as f:
            json.dump(rec, f)
    by = {}
    for r in rec:
        by.setdefault((r["test"], r["storage"]), []).append(r)
    tr = terminalreporter
    tr.write_sep("-", "parity: worst e_par/bound, worst e64 (k at which the stated bound is out of reach)")
    for (name, stg), rs in sorted(by.items()):
        par = [r for r in rs if "e_par" in r]
        if par:
            w = max(par, key=lambda r: r["e_par"] / r["tol_par"])
            gate = [r for r in par if r["stated_reachable"]]
            wg = max(gate, key=lambda r: r["e64"]) if gate else None
            out_k = sorted({r["k"] for r in par if not r["stated_reachable"]})
            tr.write_line(f"{name}: par {w['e_par']:.1e}/{w['tol_par']:.1e}@k{w['k']}; "
                          + (f"e64 {wg['e64']:.1e}<={wg['stated']:.0e}" if wg else "e64 -")
                          + (f"; stated out of reach k={out_k[0]}..{out_k[-1]}" if out_k else ""))
        else:
            w = max(rs, key=lambda r: r["e64"] / r["tol"])
            tr.write_line(f"{name}: e64 {w['e64']:.1e}/{w['tol']:.1e}@k{w['k']}")
    par = [r for r in rec if "e_par" in r]
    reach = [r for r in par if r["stated_reachable"]]
    tr.write_line(f"parity summary: {len(par)} storage-matched comparisons (worst e_par/bound "
                  f"{max((r['e_par'] / r['tol_par'] for r in par), default=0):.2f}); stated bound vs FP64 "
                  f"asserted at {len(reach)}, out of reach at {len(par) - len(reach)} "
                  f"({sorted({r['storage'] for r in par if not r['stated_reachable']})})")
