"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/qmcur.h (host-only calls exercised; no kernels launched)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qmcur.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qmcur_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2402_19147_gb300 import build as B
    srcs = [os.path.join(B.CSRC, f) for f in os.listdir(B.CSRC)] + [HEADER]
    if not os.path.exists(B.LIB) or os.path.getmtime(B.LIB) < max(map(os.path.getmtime, srcs)):
        try:
            B.build()
        except RuntimeError as e:
            if "nvcc not found" in str(e):
                pytest.skip("no nvcc on this host")
            raise
    return B.LIB


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("qmcur_probs", "qmcur_sample", "qmcur_pinv_core", "qmcur_reconstruct",
                     "qmcur_residual"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(libpath):
    from paper_2402_19147_gb300 import qmcur as Q
    assert set(declared_functions()) <= set(Q.SIGNATURES)


def test_host_only_calls(libpath):
    from paper_2402_19147_gb300 import qmcur as Q
    L = Q.lib()
    assert L.qmcur_status_str(0) == b"QMCUR_OK"
    assert L.qmcur_status_str(6) == b"QMCUR_ERR_NO_CONVERGENCE"
    for prec in range(6):
        assert Q.workspace_size(2048, 2048, 200, 200, prec) > 0
    assert Q.workspace_size(0, 10, 1, 1, 1) == 0
    # the CTA budget is host state of the calling thread
    assert L.qmcur_set_max_ctas(-1) == 1            # INVALID_ARG
    assert L.qmcur_set_max_ctas(76) == 0 and L.qmcur_set_max_ctas(0) == 0


def test_decompose_many_checks_its_lists():
    # host-side validation before any device work
    from paper_2402_19147_gb300 import qmcur as Q
    with pytest.raises(ValueError):
        Q.decompose_many([object()], [], [0])
    Q.decompose_many([], [], [])           # nothing to do
