"""The C ABI's host code under AddressSanitizer and UndefinedBehaviorSanitizer:
a variant of libmd_b300 with sanitized host code is built into a temporary
directory (the device code is the same), and tests/abi_sanitize_main.c drives
the argument checks and error paths of every entry point through it.  Runs on
a machine without a GPU, where a valid md_create also exercises the cleanup
of a context whose device setup fails."""
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
# one flag per sanitizer: nvcc splits -Xcompiler values at commas
SAN = ["-fsanitize=address", "-fsanitize=undefined", "-fsanitize=float-cast-overflow",
       "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"]


def _gpu_present():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


def test_abi_error_paths_under_asan_ubsan(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    sys.path.insert(0, os.path.join(ROOT, "paper_2109_09056_b300"))
    try:
        import build as B
    finally:
        sys.path.pop(0)
    try:
        B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    tmp = str(tmp_path)
    extra = []
    for f in SAN + ["-g"]:
        extra += ["-Xcompiler", f]
    lib = os.path.join(tmp, "libmd_b300_asan.so")
    B.build(force=True, extra=extra, lib=lib, objdir=os.path.join(tmp, "obj"))
    exe = os.path.join(tmp, "abi_sanitize")
    cmd = ["gcc", "-std=c11", "-g", *SAN, "-Wall", "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "abi_sanitize_main.c"), lib, f"-Wl,-rpath,{tmp}", "-o", exe, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    args = [] if _gpu_present() else ["create"]
    env = dict(os.environ, ASAN_OPTIONS="protect_shadow_gap=0:detect_leaks=1",
               UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe, *args], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == "ok"
