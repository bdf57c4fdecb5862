"""The C-ABI library loads on a CPU-only machine and exports every function
declared in include/ipf.h (no compute calls: they need a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\*?\s*(ipf_[a-z_0-9]+)\s*\(", text, re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2502_02721_gb300 import binding, build
    if not os.path.exists(build.lib_path()):
        build.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ipf_create", "ipf_step", "ipf_solve", "ipf_destroy", "ipf_status_str"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2502_02721_gb300 import binding
    assert set(_declared()) <= set(binding.SIGNATURES)


def test_status_strings_and_config_defaults(lib):
    from paper_2502_02721_gb300 import binding as b
    assert b.status_str(b.IPF_ERR_TIMEOUT) == "IPF_ERR_TIMEOUT"
    cfg = b.default_config()
    assert (cfg.k_max, cfg.m_s, cfg.zeta, cfg.nrhs) == (50, 200, 8, 1)


def test_argument_errors_need_no_gpu(lib):
    """Validation happens before any CUDA call."""
    import ctypes as C
    import numpy as np
    from paper_2502_02721_gb300 import binding as b
    keep = []
    op = b.make_operator("psf2d", 8, 8, psf=np.ones((4, 3), np.float32), keep=keep)   # even size
    cfg = b.default_config()
    h = C.c_void_p()
    bb = np.ones(64, np.float32)
    assert lib.ipf_create(C.byref(op), bb.ctypes.data, 0, C.byref(cfg), C.byref(h)) == b.IPF_ERR_ARG
    op = b.make_operator("psf2d", 8, 8, psf=np.ones((3, 3), np.float32), keep=keep)
    cfg = b.default_config(nrhs=3)
    assert lib.ipf_create(C.byref(op), bb.ctypes.data, 0, C.byref(cfg), C.byref(h)) == b.IPF_ERR_ARG
    cfg = b.default_config(nrhs=2)
    assert lib.ipf_create(C.byref(op), bb.ctypes.data, 0, C.byref(cfg), C.byref(h)) == b.IPF_ERR_UNSUPPORTED
    cfg = b.default_config(m_s=4, zeta=8)
    assert lib.ipf_create(C.byref(op), bb.ctypes.data, 0, C.byref(cfg), C.byref(h)) == b.IPF_ERR_ARG
    # k_max: at most 480 (512 pivot rows in registers), 247 with the Gaussian
    # sketch (its contraction's B tile holds 256 rows)
    cfg = b.default_config(k_max=481, m_s=2000)
    assert lib.ipf_create(C.byref(op), bb.ctypes.data, 0, C.byref(cfg), C.byref(h)) == b.IPF_ERR_UNSUPPORTED
    cfg = b.default_config(k_max=248, m_s=1000, sketch="gaussian")
    assert lib.ipf_create(C.byref(op), bb.ctypes.data, 0, C.byref(cfg), C.byref(h)) == b.IPF_ERR_UNSUPPORTED
    # m_s: the normaliser's two sets of shared sketch counters fit 227 KB
    cfg = b.default_config(m_s=7233)
    assert lib.ipf_create(C.byref(op), bb.ctypes.data, 0, C.byref(cfg), C.byref(h)) == b.IPF_ERR_UNSUPPORTED
    # pivot-block solve: 0 inverse form (default), 1 forward substitution
    cfg = b.default_config(pivot_fwd=2)
    assert lib.ipf_create(C.byref(op), bb.ctypes.data, 0, C.byref(cfg), C.byref(h)) == b.IPF_ERR_ARG
    assert lib.ipf_step(None, 1, None) == b.IPF_ERR_ARG
    assert lib.ipf_footprint(C.byref(op), C.byref(b.default_config())) > 64 * 51 * 4


def test_default_config_maps_string_options(lib):
    """Library defaults (ipf_config_default, host only) and the binding's
    names for the enums of include/ipf.h."""
    from paper_2502_02721_gb300 import binding as bd
    d = bd.default_config()
    assert d.overlap == 2 and d.pivot_sample == 0 and d.sketch == 0 and d.method == 0 and d.pivot_fwd == 0
    cfg = bd.default_config(storage="bf16", method="slslu", sketch="gaussian", pivot_sample=25)
    assert cfg.storage == bd.STORAGE["bf16"]
    assert cfg.method == bd.METHOD["slslu"] == 1
    assert cfg.sketch == bd.SKETCH["gaussian"] == 1
    assert cfg.pivot_sample == 25


def test_footprint_counts_the_gaussian_sketch(lib):
    """ipf_footprint (host arithmetic): a Gaussian sketch adds the stored S,
    m_s x n elements of the basis storage type."""
    import ctypes as C
    from gen import problems as P
    from paper_2502_02721_gb300 import binding as bd
    p = P.make("deblur64")
    keep = []
    op = bd.operator_from_problem(p, keep)
    base = bd.default_config(k_max=p.k, m_s=p.m_s, storage="bf16")
    gauss = bd.default_config(k_max=p.k, m_s=p.m_s, storage="bf16", sketch="gaussian")
    f0 = lib.ipf_footprint(C.byref(op), C.byref(base))
    f1 = lib.ipf_footprint(C.byref(op), C.byref(gauss))
    assert f1 - f0 >= p.m_s * p.n * 2


def test_binding_refuses_host_buffers_for_device_calls(lib):
    """Calls whose kernels write a buffer check, before reaching the
    library, that it is a device tensor of the right size and element size."""
    import torch
    from paper_2502_02721_gb300 import binding as bd
    S = torch.empty(8 * 100, dtype=torch.bfloat16)            # host memory
    with pytest.raises(ValueError):
        bd.sketch_gaussian("bf16", 1, 100, 8, S)
    with pytest.raises(ValueError):
        bd.sketch_gaussian("bf16", 1, 100, 8, torch.empty(10, dtype=torch.bfloat16))
    x, y = torch.empty(100), torch.empty(8, dtype=torch.float64)
    with pytest.raises(ValueError):
        bd.sketch_apply(x, 8, 8, 1, y)


def test_operator_apply_refuses_host_buffers(lib):
    """Operator.apply / apply_bf16 check their tensors before the library call
    (the handle is built without ipf_op_create, which needs a GPU)."""
    import torch
    from paper_2502_02721_gb300 import binding as bd
    op = bd.Operator.__new__(bd.Operator)
    op._lib, op.m, op.n, op.h = lib, 16, 16, None
    with pytest.raises(ValueError):
        op.apply(torch.empty(16), torch.empty(16))
    with pytest.raises(ValueError):
        op.apply_bf16(torch.empty(16, dtype=torch.bfloat16), torch.empty(16))
    with pytest.raises(ValueError):
        op.apply(torch.empty(15), torch.empty(16))
