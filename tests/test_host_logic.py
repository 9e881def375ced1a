"""Host-side decisions of the serving engine, checked without a GPU.

The engine moves a caller's buffer with one direct copy (a copy engine, beside
the kernels) when it can, and through its page-locked staging buffer
otherwise.  Device memory of any device is copied directly (cudaMemcpyDefault
crosses devices); page-locked host memory is read directly, but written
directly only when CUDA allocated it: memory registered with cudaHostRegister
may be read-only for the device.  Pageable and managed memory are staged.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2311_00482_gb300", "csrc")


def cuda_include():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            return os.path.join(cand, "include")
    return None


def test_kernel_path_decisions(tmp_path):
    inc = cuda_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "ptr_decision_check")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I" + CSRC, "-I" + inc,
                    os.path.join(ROOT, "tests", "ptr_decision_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {name: int(k) for name, k in (line.split() for line in out.splitlines())}
    expect_direct = {"device_read": 1, "device_write": 1, "host_alloc_read": 1,
                     "host_alloc_write": 1, "host_registered_read": 1,
                     "host_registered_write": 0, "managed_read": 0, "managed_write": 0,
                     "unregistered_read": 0, "unregistered_write": 0}
    assert got == expect_direct
