"""Builds synth/lib/libsynthgen.so, the device implementation of the seeded input generator
(synth/csrc/gen.cu), in-tree with nvcc for sm_103a. It is separate from the embedded-ERI library:
it draws input numbers and holds none of the method's arithmetic."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "gen.cu")
LIB = os.path.join(HERE, "lib", "libsynthgen.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp"
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-fvisibility=hidden", "-shared", SRC, "-o", tmp, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for gen.cu:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB
