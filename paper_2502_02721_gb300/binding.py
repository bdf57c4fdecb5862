"""ctypes binding over libipf.so (include/ipf.h).  Argument marshalling only:
every step of the method runs in the library's CUDA kernels.  There is no
CPU fallback; if the library is missing the import fails loudly.

torch provides device memory and streams: device arrays are passed as
``tensor.data_ptr()`` and streams as ``torch.cuda.current_stream().cuda_stream``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

IPF_OK, IPF_BREAKDOWN, IPF_PENDING = 0, 1, 2
IPF_ERR_ARG, IPF_ERR_OOM, IPF_ERR_CUDA, IPF_ERR_NONFINITE = -1, -2, -3, -4
IPF_ERR_TIMEOUT, IPF_ERR_STATE, IPF_ERR_UNSUPPORTED, IPF_ERR_REJECTED = -5, -6, -7, -8

IPF_OP_PSF2D, IPF_OP_PSF2D_SEP_MOTION, IPF_OP_CSR = 1, 2, 3
IPF_MEM_HOST, IPF_MEM_DEVICE = 0, 1
IPF_STORE_F64, IPF_STORE_F32, IPF_STORE_BF16, IPF_STORE_F16 = 0, 1, 2, 3
IPF_PEN_SKETCHED_X, IPF_PEN_Y = 0, 1
IPF_Z_DIRECT, IPF_Z_HESSENBERG, IPF_Z_AUTO = 0, 1, 2

STORAGE = {"f64": IPF_STORE_F64, "f32": IPF_STORE_F32, "bf16": IPF_STORE_BF16, "f16": IPF_STORE_F16}

_fp = C.POINTER(C.c_float)
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class ipf_operator(C.Structure):
    _fields_ = [("kind", C.c_int), ("rows", C.c_int), ("cols", C.c_int),
                ("psf", C.c_void_p), ("ph", C.c_int), ("pw", C.c_int),
                ("sep_row", C.c_void_p), ("sep_col", C.c_void_p), ("slen", C.c_int),
                ("motion", C.c_void_p), ("mlen", C.c_int),
                ("rowptr", C.c_void_p), ("colind", C.c_void_p), ("vals", C.c_void_p), ("nnz", C.c_longlong),
                ("mem", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


METHOD = {"scmrh": 0, "slslu": 1}
SKETCH = {"sparse_sign": 0, "gaussian": 1}


class ipf_config(C.Structure):
    _fields_ = [("k_max", C.c_int), ("m_s", C.c_int), ("zeta", C.c_int), ("seed", C.c_ulonglong),
                ("storage", C.c_int), ("penalty", C.c_int), ("zform", C.c_int), ("nrhs", C.c_int),
                ("use_graphs", C.c_int), ("profile", C.c_int), ("overlap", C.c_int), ("method", C.c_int), ("sketch", C.c_int),
                ("pivot_sample", C.c_int),
                ("conv_fma", C.c_int), ("pivot_fwd", C.c_int),
                ("stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p)]


class ipf_server_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("pinned_bytes", C.c_size_t), ("max_inflight", C.c_int),
                ("steps_per_slice", C.c_int), ("per_request", C.c_int)]


class ipf_request(C.Structure):
    _fields_ = [("op", ipf_operator), ("b", C.c_void_p), ("cfg", ipf_config), ("k", C.c_int),
                ("lambda_", C.c_double)]


class ipf_result(C.Structure):
    _fields_ = [("status", C.c_int), ("k_used", C.c_int), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double)]


class ipf_solve_info(C.Structure):
    _fields_ = [("k_used", C.c_int), ("k_done", C.c_int), ("status", C.c_int), ("pad", C.c_int)]


# name -> (restype, argtypes), one entry per declaration in include/ipf.h
SIGNATURES = {
    "ipf_config_default": (None, [C.POINTER(ipf_config)]),
    "ipf_footprint": (C.c_size_t, [C.POINTER(ipf_operator), C.POINTER(ipf_config)]),
    "ipf_create": (C.c_int, [C.POINTER(ipf_operator), C.c_void_p, C.c_int, C.POINTER(ipf_config),
                             C.POINTER(C.c_void_p)]),
    "ipf_reset": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "ipf_step": (C.c_int, [C.c_void_p, C.c_int, _ip]),
    "ipf_profile_read": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_longlong), _dp]),
    "ipf_sync": (C.c_int, [C.c_void_p, _ip]),
    "ipf_solve": (C.c_int, [C.c_void_p, C.c_int, _dp, C.c_int, C.c_void_p, C.c_int,
                            C.POINTER(ipf_solve_info)]),
    "ipf_export": (C.c_int, [C.c_void_p, C.c_int, _ip, _dp, _dp, _dp, _dp, _dp]),
    "ipf_export_basis": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _fp]),
    "ipf_destroy": (None, [C.c_void_p]),
    "ipf_status_str": (C.c_char_p, [C.c_int]),
    "ipf_last_error": (C.c_char_p, [C.c_void_p]),
    "ipf_op_create": (C.c_int, [C.POINTER(ipf_operator), C.POINTER(C.c_void_p)]),
    "ipf_op_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "ipf_solve_qmr": (C.c_int, [C.c_void_p, C.c_int, _dp, C.c_int, C.c_void_p, C.c_int,
                                C.POINTER(ipf_solve_info)]),
    "ipf_export_dual": (C.c_int, [C.c_void_p, C.c_int, _ip, _dp, _dp, _dp]),
    "ipf_export_basis_l": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _fp]),
    "ipf_op_apply_bf16": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "ipf_op_destroy": (None, [C.c_void_p]),
    "ipf_sketch_apply": (C.c_int, [C.c_void_p, C.c_longlong, C.c_int, C.c_int, C.c_ulonglong, C.c_void_p,
                                   C.c_void_p]),
    "ipf_sketch_apply_noalloc": (C.c_int, [C.c_void_p, C.c_longlong, C.c_int, C.c_int, C.c_ulonglong,
                                           C.c_void_p, C.c_void_p]),
    "ipf_sketch_gaussian": (C.c_int, [C.c_int, C.c_ulonglong, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p]),
    "ipf_server_create": (C.c_int, [C.POINTER(ipf_server_config), C.POINTER(C.c_void_p)]),
    "ipf_submit": (C.c_int, [C.c_void_p, C.POINTER(ipf_request), C.POINTER(C.c_ulonglong)]),
    "ipf_poll": (C.c_int, [C.c_void_p, C.c_ulonglong, C.POINTER(ipf_result), C.c_void_p]),
    "ipf_server_stats": (C.c_int, [C.c_void_p, _ip, _ip, C.POINTER(C.c_size_t)]),
    "ipf_server_batch_stats": (C.c_int, [C.c_void_p, _ip, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                         C.POINTER(C.c_longlong)]),
    "ipf_server_destroy": (None, [C.c_void_p]),
}

_LIB = None


def load(path: str | None = None):
    """Load libipf.so (built by build.py); raises if it is absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.lib_path()
    if not os.path.exists(path):
        raise ImportError(f"libipf.so not built at {path}; run paper_2502_02721_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class IpfError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"{status_str(code)}{': ' + msg if msg else ''}")


def _check_size(a, want: int, name: str):
    """Refuse buffers whose element count does not match the operator: the C
    ABI takes raw pointers and cannot check them itself."""
    got = int(a.size) if isinstance(a, np.ndarray) else int(a.numel())
    if got != int(want):
        raise ValueError(f"{name} has {got} elements, expected {want}")


def _check_device(a, name: str, elem_bytes: int):
    """Refuse a tensor that is not in device memory or has the wrong element
    size for a call that writes it from a kernel."""
    if not getattr(a, "is_cuda", False):
        raise ValueError(f"{name} must be a CUDA tensor")
    if int(a.element_size()) != elem_bytes:
        raise ValueError(f"{name} has {a.element_size()}-byte elements, expected {elem_bytes}")


def status_str(code: int) -> str:
    return load().ipf_status_str(int(code)).decode()


def _ptr(a):
    """Host numpy array or torch tensor -> (address, mem flag)."""
    if a is None:
        return None, IPF_MEM_HOST
    if isinstance(a, np.ndarray):
        return a.ctypes.data, IPF_MEM_HOST
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), (IPF_MEM_DEVICE if a.is_cuda else IPF_MEM_HOST)
    raise TypeError(type(a))


def make_operator(kind: str, rows: int, cols: int, *, psf=None, sep_row=None, sep_col=None, motion=None,
                  rowptr=None, colind=None, vals=None, keep: list | None = None) -> ipf_operator:
    """Fill an ipf_operator from numpy arrays (host) or torch CUDA tensors.
    Arrays must be contiguous float32 (rowptr int64, colind int32); the
    caller keeps them alive (``keep`` collects the converted copies)."""
    keep = keep if keep is not None else []
    op = ipf_operator()
    op.rows, op.cols = int(rows), int(cols)
    mems = set()

    def put(a, dtype):
        if a is None:
            return None
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=dtype)
        keep.append(a)
        p, m = _ptr(a)
        mems.add(m)
        return p

    if kind == "psf2d":
        op.kind = IPF_OP_PSF2D
        op.psf = put(psf, np.float32)
        op.ph, op.pw = int(psf.shape[0]), int(psf.shape[1])
    elif kind == "psf_sep_motion":
        op.kind = IPF_OP_PSF2D_SEP_MOTION
        op.sep_row = put(sep_row, np.float32)
        op.sep_col = put(sep_col, np.float32)
        op.slen = int(sep_row.shape[0])
        op.motion = put(motion, np.float32)
        op.mlen = int(motion.shape[0])
    elif kind == "csr":
        op.kind = IPF_OP_CSR
        op.rowptr = put(rowptr, np.int64)
        op.colind = put(colind, np.int32)
        op.vals = put(vals, np.float32)
        op.nnz = int(vals.shape[0])
    else:
        raise ValueError(kind)
    if len(mems) > 1:
        raise ValueError("operator arrays must all be host or all be device")
    op.mem = mems.pop() if mems else IPF_MEM_HOST
    return op


def operator_from_problem(p, keep: list | None = None) -> ipf_operator:
    """ipf_operator for a gen.problems.Problem (host arrays).  For CSR the
    problem's rows x cols is the image; the operator is m x n = rays x pixels."""
    rows, cols = p.rows, p.cols
    if p.kind == "csr":
        rows, cols = int(np.asarray(p.rowptr).size - 1), int(p.rows * p.cols)
    return make_operator(p.kind, rows, cols, psf=p.psf, sep_row=p.sep_row, sep_col=p.sep_col,
                         motion=p.motion, rowptr=p.rowptr, colind=p.colind, vals=p.vals, keep=keep)


def default_config(**kw) -> ipf_config:
    cfg = ipf_config()
    load().ipf_config_default(C.byref(cfg))
    for k, v in kw.items():
        if k == "storage" and isinstance(v, str):
            v = STORAGE[v]
        if k == "method" and isinstance(v, str):
            v = METHOD[v]
        if k == "sketch" and isinstance(v, str):
            v = SKETCH[v]
        setattr(cfg, k, v)
    return cfg


class Context:
    """One ipf_ctx: nrhs right-hand sides sharing an operator."""

    def __init__(self, op: ipf_operator, b, cfg: ipf_config, keep=None):
        self._lib = load()
        self._keep = list(keep or [])
        if isinstance(b, np.ndarray):
            b = np.ascontiguousarray(b, dtype=np.float32)
        self.cfg = cfg
        self.nrhs = cfg.nrhs
        # x has n entries per RHS; b has m (= n except for a rectangular CSR
        # operator under the generalized process)
        self.n = op.cols if op.kind == IPF_OP_CSR else op.rows * op.cols
        self.m = op.rows if (op.kind == IPF_OP_CSR and cfg.method == METHOD["slslu"]) else self.n
        _check_size(b, self.nrhs * self.m, "b")
        self._keep.append(b)
        ptr, mem = _ptr(b)
        h = C.c_void_p()
        st = self._lib.ipf_create(C.byref(op), ptr, mem, C.byref(cfg), C.byref(h))
        if st != IPF_OK:
            raise IpfError(st, "ipf_create")
        self.h = h

    def _check(self, st, what):
        if st < 0:
            raise IpfError(st, f"{what}: {self._lib.ipf_last_error(self.h).decode()}")
        return st

    def reset(self, b):
        """New right-hand side(s) on the same context (no allocation)."""
        if isinstance(b, np.ndarray):
            b = np.ascontiguousarray(b, dtype=np.float32)
            self._keep.append(b)
        _check_size(b, self.nrhs * self.m, "b")
        ptr, mem = _ptr(b)
        self._check(self._lib.ipf_reset(self.h, ptr, mem), "ipf_reset")

    def profile_read(self):
        """(ms[12], launches[12], bytes[12]) per kernel kind since the last read."""
        ms = (C.c_double * 12)()
        n = (C.c_longlong * 12)()
        by = (C.c_double * 12)()
        self._check(self._lib.ipf_profile_read(self.h, ms, n, by), "ipf_profile_read")
        return list(ms), list(n), list(by)

    def step(self, nsteps: int) -> int:
        k = C.c_int(0)
        self._check(self._lib.ipf_step(self.h, int(nsteps), C.byref(k)), "ipf_step")
        return k.value

    def sync(self):
        kd = (C.c_int * self.nrhs)()
        st = self._check(self._lib.ipf_sync(self.h, kd), "ipf_sync")
        return st, list(kd)

    def solve(self, k: int, lambdas=(0.0,), out=None, wait: bool = True, qmr: bool = False):
        """x for every lambda: numpy (nl, nrhs, n) float32, or into ``out``
        (a CUDA tensor or pinned host tensor of that shape, written in place).
        wait=False with a CUDA ``out`` returns without synchronising.
        qmr=True gives the quasi-minimal residual iterate (ipf_solve_qmr)."""
        lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64).reshape(-1))
        nl = lam.size
        info = (ipf_solve_info * self.nrhs)() if wait or out is None or not getattr(out, "is_cuda", False) else None
        if out is None:
            x = np.zeros((nl, self.nrhs, self.n), dtype=np.float32)
            ptr, mem = x.ctypes.data, IPF_MEM_HOST
        else:
            x = out
            _check_size(out, nl * self.nrhs * self.n, "out")
            ptr, mem = _ptr(out)
        fn = self._lib.ipf_solve_qmr if qmr else self._lib.ipf_solve
        st = fn(self.h, int(k), lam.ctypes.data_as(_dp), nl, ptr, mem, info)
        self._check(st, "ipf_solve_qmr" if qmr else "ipf_solve")
        return x, ([(i.k_used, i.k_done, i.status) for i in info] if info is not None else None)

    def export(self, r: int = 0):
        K1 = self.cfg.k_max + 1
        piv = np.zeros(K1, dtype=np.int32)
        H = np.zeros(K1 * self.cfg.k_max, dtype=np.float64)
        SV = np.zeros(K1 * self.cfg.m_s, dtype=np.float64)
        SZ = np.zeros(self.cfg.k_max * self.cfg.m_s, dtype=np.float64)
        c = np.zeros(self.cfg.m_s, dtype=np.float64)
        beta = np.zeros(1, dtype=np.float64)
        st = self._lib.ipf_export(self.h, r, piv.ctypes.data_as(_ip), H.ctypes.data_as(_dp),
                                  SV.ctypes.data_as(_dp), SZ.ctypes.data_as(_dp), c.ctypes.data_as(_dp),
                                  beta.ctypes.data_as(_dp))
        self._check(st, "ipf_export")
        return {"piv": piv, "H": H.reshape(self.cfg.k_max, K1).T, "SV": SV.reshape(K1, self.cfg.m_s).T,
                "SZ": SZ.reshape(self.cfg.k_max, self.cfg.m_s).T, "c": c, "beta": float(beta[0])}

    def basis(self, j: int, r: int = 0) -> np.ndarray:
        """Column j of the basis (D for the generalized process)."""
        v = np.zeros(self.m, dtype=np.float32)
        self._check(self._lib.ipf_export_basis(self.h, r, j, v.ctypes.data_as(_fp)), "ipf_export_basis")
        return v

    def export_dual(self, r: int = 0):
        """Generalized process: pivots of L, the W table, S_1 L and W(1,1)."""
        K1 = self.cfg.k_max + 1
        piv = np.zeros(K1, dtype=np.int32)
        W = np.zeros(K1 * self.cfg.k_max, dtype=np.float64)
        SL = np.zeros(K1 * self.cfg.m_s, dtype=np.float64)
        w11 = np.zeros(1, dtype=np.float64)
        st = self._lib.ipf_export_dual(self.h, r, piv.ctypes.data_as(_ip), W.ctypes.data_as(_dp),
                                       SL.ctypes.data_as(_dp), w11.ctypes.data_as(_dp))
        self._check(st, "ipf_export_dual")
        return {"piv": piv, "W": W.reshape(self.cfg.k_max, K1).T, "SL": SL.reshape(K1, self.cfg.m_s).T,
                "w11": float(w11[0])}

    def basis_l(self, j: int, r: int = 0) -> np.ndarray:
        """Column j of the L basis of the generalized process (n floats)."""
        v = np.zeros(self.n, dtype=np.float32)
        self._check(self._lib.ipf_export_basis_l(self.h, r, j, v.ctypes.data_as(_fp)), "ipf_export_basis_l")
        return v

    def close(self):
        if getattr(self, "h", None):
            self._lib.ipf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    """ipf_op handle: standalone w = A v on device float32 tensors."""

    def __init__(self, op: ipf_operator, keep=None):
        self._lib = load()
        self._keep = keep
        self.m = op.rows if op.kind == IPF_OP_CSR else op.rows * op.cols
        self.n = op.cols if op.kind == IPF_OP_CSR else op.rows * op.cols
        h = C.c_void_p()
        st = self._lib.ipf_op_create(C.byref(op), C.byref(h))
        if st != IPF_OK:
            raise IpfError(st, "ipf_op_create")
        self.h = h

    def apply(self, v, w, nrhs: int = 1, stream=None):
        """w (float32, nrhs x m) = A v (float32, nrhs x n), device tensors."""
        _check_size(v, nrhs * self.n, "v")
        _check_size(w, nrhs * self.m, "w")
        _check_device(v, "v", 4)
        _check_device(w, "w", 4)
        st = self._lib.ipf_op_apply(self.h, v.data_ptr(), w.data_ptr(), int(nrhs), stream)
        if st != IPF_OK:
            raise IpfError(st, "ipf_op_apply")

    def apply_bf16(self, v, w, use_fma: bool = False, stream=None):
        """w (float32, m) = A v for v a bfloat16 device tensor of n values."""
        if str(v.dtype) != "torch.bfloat16" or str(w.dtype) != "torch.float32":
            raise TypeError("apply_bf16 takes a bfloat16 v and a float32 w")
        _check_size(v, self.n, "v")
        _check_size(w, self.m, "w")
        _check_device(v, "v", 2)
        _check_device(w, "w", 4)
        st = self._lib.ipf_op_apply_bf16(self.h, v.data_ptr(), w.data_ptr(), 1 if use_fma else 0, stream)
        if st != IPF_OK:
            raise IpfError(st, "ipf_op_apply_bf16")

    def close(self):
        if getattr(self, "h", None):
            self._lib.ipf_op_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """ipf_server: continuous serving of many solves on one GPU."""

    def __init__(self, hbm_budget_bytes: int = 0, max_inflight: int = 64, steps_per_slice: int = 8,
                 pinned_bytes: int = 0, per_request: bool = False):
        self._lib = load()
        cfg = ipf_server_config(hbm_budget_bytes=int(hbm_budget_bytes), pinned_bytes=int(pinned_bytes),
                                max_inflight=int(max_inflight), steps_per_slice=int(steps_per_slice),
                                per_request=1 if per_request else 0)
        h = C.c_void_p()
        st = self._lib.ipf_server_create(C.byref(cfg), C.byref(h))
        if st != IPF_OK:
            raise IpfError(st, "ipf_server_create")
        self.h = h
        self._n = {}

    def submit(self, op: ipf_operator, b: np.ndarray, cfg: ipf_config, k: int, lam: float = 0.0) -> int:
        b = np.ascontiguousarray(b, dtype=np.float32)
        n = op.cols if op.kind == IPF_OP_CSR else op.rows * op.cols
        _check_size(b, n * cfg.nrhs, "b")
        rq = ipf_request(op=op, b=b.ctypes.data, cfg=cfg, k=int(k), lambda_=float(lam))
        t = C.c_ulonglong(0)
        st = self._lib.ipf_submit(self.h, C.byref(rq), C.byref(t))
        if st != IPF_OK:
            raise IpfError(st, "ipf_submit")
        self._n[t.value] = (n, cfg.nrhs)
        return t.value

    def poll(self, ticket: int, want_x: bool = True):
        """None while pending, else (status, k_used, (t_submit, t_admit, t_done), x or None)."""
        n, nrhs = self._n[ticket]
        res = ipf_result()
        x = np.zeros((nrhs, n), dtype=np.float32) if want_x else None
        st = self._lib.ipf_poll(self.h, int(ticket), C.byref(res), x.ctypes.data if want_x else None)
        if st == IPF_PENDING:
            return None
        del self._n[ticket]
        return res.status, res.k_used, (res.t_submit, res.t_admit, res.t_done), x

    def stats(self):
        a, q = C.c_int(0), C.c_int(0)
        m = C.c_size_t(0)
        self._lib.ipf_server_stats(self.h, C.byref(a), C.byref(q), C.byref(m))
        return a.value, q.value, m.value

    def batch_stats(self):
        """(requests that took a batch slot, graph turns, eager turns, graph captures)."""
        b = C.c_int(0)
        g, e, c = C.c_longlong(0), C.c_longlong(0), C.c_longlong(0)
        self._lib.ipf_server_batch_stats(self.h, C.byref(b), C.byref(g), C.byref(e), C.byref(c))
        return b.value, g.value, e.value, c.value

    def close(self):
        if getattr(self, "h", None):
            self._lib.ipf_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sketch_apply(x, m_s: int, zeta: int, seed: int, y, stream=None):
    """y (device float64, m_s) = S x (device float32, n)."""
    _check_size(y, m_s, "y")
    _check_device(x, "x", 4)
    _check_device(y, "y", 8)
    st = load().ipf_sketch_apply(x.data_ptr(), int(x.numel()), int(m_s), int(zeta), int(seed), y.data_ptr(), stream)
    if st != IPF_OK:
        raise IpfError(st, "ipf_sketch_apply")


def sketch_gaussian(storage: str, seed: int, n: int, m_s: int, S, stream=None):
    """ipf_sketch_gaussian: the Gaussian sketch (m_s x n, row-major) into
    the device tensor S of the storage type (m_s * n elements)."""
    _check_size(S, int(m_s) * int(n), "S")
    _check_device(S, "S", {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[storage])
    st = load().ipf_sketch_gaussian(STORAGE[storage], int(seed), int(n), int(m_s), S.data_ptr(), stream)
    if st != IPF_OK:
        raise IpfError(st, "ipf_sketch_gaussian")


def sketch_apply_noalloc(x, m_s: int, zeta: int, seed: int, y, stream=None):
    """ipf_sketch_apply_noalloc: y = S x with the library's fixed scratch
    (no device allocation; m_s <= 4096; calls must not overlap on the GPU)."""
    _check_size(y, m_s, "y")
    _check_device(x, "x", 4)
    _check_device(y, "y", 8)
    st = load().ipf_sketch_apply_noalloc(x.data_ptr(), int(x.numel()), int(m_s), int(zeta), int(seed),
                                         y.data_ptr(), stream)
    if st != IPF_OK:
        raise IpfError(st, "ipf_sketch_apply_noalloc")
