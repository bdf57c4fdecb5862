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
    assert lib.ipf_step(None, 1, None) == b.IPF_ERR_ARG
    assert lib.ipf_footprint(C.byref(op), C.byref(b.default_config())) > 64 * 51 * 4
