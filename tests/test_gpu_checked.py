"""Checked build on a B300: the library compiled with -DMD_CHECKED (index checks
at the gathers and scatters of the sort, the list build, the force kernels,
the adjoint and the SPME real-space pass; a failing check is recorded and the
access redirected or skipped, so the kernels never touch memory out of
range) runs small workloads of every kind (tests/checked_run.py) in a
subprocess, and no check may fire.  The checked library is built in-tree
beside the default one; the default build's kernels carry no checks."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PKG = os.path.join(ROOT, "paper_2109_09056_b300")


def test_checked_build_runs_clean():
    sys.path.insert(0, PKG)
    try:
        import build as B
    finally:
        sys.path.pop(0)
    lib = os.path.join(PKG, "_build_checked", "libmd_b300_checked.so")
    B.build(extra=["-DMD_CHECKED"], lib=lib, objdir=os.path.join(PKG, "_build_checked", "obj"))
    env = dict(os.environ, MD_B300_LIB=lib,
               PYTHONPATH=os.pathsep.join([ROOT, HERE, os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert r.stdout.strip().splitlines()[-1] == "ok"
