"""The library's decision on where an array argument lives (host code, no GPU).

An array on another GPU than the current one must be refused before any
launch: the library launches on the current GPU and enables no peer access, so
a kernel reading it would fault.  crhyb::place_of turns the attributes the
driver reports into 1 (current GPU or managed memory), 0 (host) or -1
(another GPU); this test compiles it with the host compiler against the
library's internal header and checks every case, including the ordinals of a
second GPU, which this test needs no second GPU to exercise.
"""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"

SRC = r"""
#include <cstdio>
#include "internal.h"
int main() {
    using crhyb::place_of;
    int bad = 0;
    auto expect = [&](int got, int want, const char* what) {
        if (got != want) { std::printf("%s: got %d want %d\n", what, got, want); ++bad; }
    };
    expect(place_of(cudaMemoryTypeDevice, 0, 0), 1, "device of the current GPU");
    expect(place_of(cudaMemoryTypeDevice, 3, 3), 1, "device 3 with GPU 3 current");
    expect(place_of(cudaMemoryTypeDevice, 1, 0), -1, "device of GPU 1 with GPU 0 current");
    expect(place_of(cudaMemoryTypeDevice, 0, 5), -1, "device of GPU 0 with GPU 5 current");
    expect(place_of(cudaMemoryTypeManaged, 2, 0), 1, "managed memory");
    expect(place_of(cudaMemoryTypeHost, 0, 0), 0, "pinned host memory");
    expect(place_of(cudaMemoryTypeUnregistered, 0, 0), 0, "pageable host memory");
    std::printf("%s\n", bad ? "FAIL" : "OK");
    return bad;
}
"""


def test_arrays_of_another_gpu_are_refused(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("no host C++ compiler or CUDA headers")
    src = tmp_path / "place.cpp"
    exe = tmp_path / "place"
    src.write_text(SRC)
    csrc = os.path.join(ROOT, "paper_2101_03777_gb300", "csrc")
    subprocess.run([cxx, "-std=c++17", "-I", csrc, "-I", CUDA_INC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout
