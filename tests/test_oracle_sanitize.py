"""The C oracle under AddressSanitizer and UndefinedBehaviorSanitizer (host
only): tests/oracle_sanitize_main.c drives every exported oracle function on
small seeded systems and edge cases (2- and 3-cell boxes, atoms outside the
box, truncated rows, one atom, empty cells), checks the oracle's internal
consistency, and aborts on the first sanitizer finding.  The oracle is built
without OpenMP here, so the run is serial and deterministic."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _sanitizer_works(tmp):
    src = os.path.join(tmp, "probe.c")
    with open(src, "w") as fh:
        fh.write("int main(void) { return 0; }\n")
    r = subprocess.run(["gcc", "-fsanitize=address,undefined", src, "-o",
                        os.path.join(tmp, "probe")], capture_output=True, text=True)
    return r.returncode == 0


def test_oracle_under_asan_ubsan(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    tmp = str(tmp_path)
    if not _sanitizer_works(tmp):
        pytest.skip("gcc has no ASan/UBSan runtime here")
    exe = os.path.join(tmp, "oracle_sanitize")
    cmd = ["gcc", "-std=c11", "-O1", "-g", "-fno-omit-frame-pointer", "-ffp-contract=off",
           "-fsanitize=address,undefined,float-cast-overflow", "-fno-sanitize-recover=all", "-Wall",
           "-Wno-unknown-pragmas",
           os.path.join(HERE, "oracle_sanitize_main.c"), os.path.join(ROOT, "oracle", "oracle_md.c"),
           "-o", exe, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == "ok"
