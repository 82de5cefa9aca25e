"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point that include/exactsum.h declares; host-side argument
checks fail cleanly without a GPU.  No kernel runs here."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import pytest

import paper_1605_05436_gb300 as es
from paper_1605_05436_gb300 import buildlib as esbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:exactsum_status|const char\*|int|void)\s+(exactsum_\w+)\s*\(",
                            text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    return esbuild.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("exactsum_create", "exactsum_destroy", "exactsum_sum", "exactsum_last_error",
                     "exactsum_sum_host", "exactsum_acc_add", "exactsum_acc_round"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib_path]).decode()
    exported = set(re.findall(r"\bT (exactsum_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_mirrors_the_header(lib_path):
    names = declared_functions()
    for n in names:
        assert hasattr(es, n), f"binding lacks {n}"


def test_host_checks_without_gpu(lib_path):
    """With no usable GPU, create() reports an error instead of crashing, and
    calls on a NULL handle are rejected with EINVAL."""
    lib = es.library()
    h = ctypes.c_void_p()
    st = lib.exactsum_create(ctypes.byref(h), 0, 0)
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except ImportError:
        has_gpu = False
    if not has_gpu:
        assert st in (es.ECUDA, es.EINVAL, es.EUNSUPPORTED)
        assert h.value is None
        assert lib.exactsum_last_error(None)
    else:
        assert st in (es.OK, es.EUNSUPPORTED)
        if st == es.OK:
            lib.exactsum_destroy(h)
    assert lib.exactsum_sum(None, None, 0, 0, 0, 0, None, None) == es.EINVAL
    assert b"null handle" in lib.exactsum_last_error(None)
    assert lib.exactsum_create(None, 0, 0) == es.EINVAL


def test_product_path_has_no_oracle_dependency():
    """The library package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_1605_05436_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "exactsum_oracle" not in text and "liboracle" not in text, f
