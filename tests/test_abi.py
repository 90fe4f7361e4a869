"""The C ABI library builds for sm_103a, loads, and exports every function
that include/iwpp.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(iwpp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1209_3314_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("iwpp_ctx_create", "iwpp_ctx_destroy", "iwpp_recon", "iwpp_edt",
                     "iwpp_recon_batched", "iwpp_edt_batched", "iwpp_recon_async", "iwpp_edt_async",
                     "iwpp_sync", "iwpp_stats", "iwpp_submit", "iwpp_poll", "iwpp_wait"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1209_3314_gb300.binding import SIGNATURES

    assert set(SIGNATURES) == set(declared_functions())


def test_version_without_gpu(lib):
    assert lib.iwpp_version() >= 100


def test_context_creation_fails_cleanly_without_gpu(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.iwpp_ctx_create(ctypes.byref(h), 0, ctypes.c_size_t(0))
    assert rc != 0 and not h.value
