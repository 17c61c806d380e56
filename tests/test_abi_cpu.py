"""The C-ABI library builds, loads and exports every symbol include/mdp.h
declares; without a GPU every compute call fails loudly (no CPU fallback)."""
import ctypes as C
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "mdp.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2109_00857_gb300 import build_native, mdp
    build_native.build()
    return mdp.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(mdp_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ("mdp_build", "mdp_solve", "mdp_export_csr", "mdp_model_free", "mdp_serve_create",
              "mdp_serve_submit", "mdp_serve_poll", "mdp_batch_create", "mdp_sample_coeffs"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2109_00857_gb300 import mdp
    names = declared_functions()
    assert names, "no declarations parsed"
    for n in names:
        assert hasattr(lib, n), f"{n} not exported"
        assert n in mdp.SIGNATURES, f"{n} missing from the Python binding"
    assert set(mdp.SIGNATURES) == set(names)


def test_version_string(lib):
    assert b"sm_103a" in lib.mdp_version()


def test_no_cpu_fallback_without_a_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2109_00857_gb300 import mdp
    sig = (C.c_double * 2)(0.2, 0.1)
    code = lib.mdp_sample_coeffs(2, 4, 2, C.cast(sig, C.c_void_p), 1, 0, 0, None, None)
    assert code == -6      # MDP_ERR_CUDA
    assert b"no usable CUDA device" in lib.mdp_last_error()
    h = C.c_void_p()
    code = lib.mdp_build(None, None, None, 10, 7, None, 1, None, None, C.byref(h))
    assert code == -6 and not h.value


def test_build_is_quick_and_in_tree():
    from paper_2109_00857_gb300 import build_native
    assert build_native.LIB.startswith(os.path.join(ROOT, "paper_2109_00857_gb300"))
    assert "-fmad=false" in build_native.UNITS["check_fp64.cu"]
    assert build_native.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
