"""The C ABI from plain C: tests/abi_example.c is compiled as C99 against
include/exactsum.h with warnings as errors, linked against the library and
the CUDA runtime, and run -- without a GPU (creation must fail cleanly) and,
marked gpu, on a GB300 (the sums must be exact)."""
from __future__ import annotations

import os
import subprocess

import pytest

from paper_1605_05436_gb300 import buildlib as esbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = "/usr/local/cuda"


@pytest.fixture(scope="module")
def example(tmp_path_factory):
    lib = esbuild.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path_factory.mktemp("cabi") / "abi_example")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), "-isystem", os.path.join(CUDA, "include"),
           os.path.join(ROOT, "tests", "abi_example.c"), "-o", exe,
           "-L", libdir, "-lexactsum", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           "-Wl,-rpath," + libdir, "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except ImportError:
        return False


def test_header_is_c99_and_the_call_fails_cleanly_without_gpu(example):
    if _has_gpu():
        pytest.skip("a GPU is present (the gpu-marked test covers it)")
    p = subprocess.run([example, "nogpu"], capture_output=True, text=True, timeout=60)
    assert p.returncode == 0, p.stdout + p.stderr
    assert p.stdout.startswith("OK no GPU")


@pytest.mark.gpu
def test_c_program_sums_exactly(example):
    if not _has_gpu():
        pytest.skip("no CUDA device")
    p = subprocess.run([example, "gpu"], capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stdout + p.stderr
    assert p.stdout.startswith("OK 500500 500500 1")
