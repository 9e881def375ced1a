"""Host-side decisions of the serving engine, checked without a GPU.

The engine copies records in and images out with a kernel where it can use
the buffer's address on its own device, and with cudaMemcpyAsync otherwise.
Device memory of another GPU (no peer mapping) and page-locked host memory
that was registered rather than allocated by CUDA (it may be read-only for
the device) must take the copy-call path when the kernel would write them.
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
    got = {name: (int(k), int(ok)) for name, k, ok in (line.split() for line in out.splitlines())}
    expect_kernel = {"device_same": 1, "device_same_write": 1, "device_foreign": 0,
                     "device_foreign_write": 0, "host_alloc_read": 1, "host_alloc_write": 1,
                     "host_registered_read": 1, "host_registered_write": 0,
                     "host_other_current": 0, "managed": 0, "unregistered": 0}
    for name, k in expect_kernel.items():
        assert got[name][0] == k, name
        assert got[name][1] == 1, name + ": wrong address"
