"""The Ewald / SPME oracle pins catch plausible mistakes: each mutant plants
one (a dropped or wrong factor, a wrong sign, a swapped axis, a wrong stencil
direction) in a copy of oracle/ewald.py and runs tests/test_oracle_ewald.py
against it in a subprocess; at least one pin must fail.  CPU only; the
mutants live in a temporary directory."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ewald.py")

MUTANTS = {
    "moduli_dropped": ("    return B * C\n", "    return C\n"),
    "influence_exponent": ("np.exp(-math.pi ** 2 * msq / alpha ** 2) / (math.pi * V * msq)",
                           "np.exp(-math.pi * msq / alpha ** 2) / (math.pi * V * msq)"),
    "spme_energy_factor": ("E = 0.5 * float(np.sum(theta", "E = float(np.sum(theta"),
    "stencil_direction": ("(k0.astype(np.int64)[:, :, None] - np.arange(n))",
                          "(k0.astype(np.int64)[:, :, None] + np.arange(n))"),
    "spline_deriv_sign": ("return bspline(n - 1, x) - bspline(n - 1, np.asarray(x, dtype=np.float64) - 1.0)",
                          "return bspline(n - 1, np.asarray(x, dtype=np.float64) - 1.0) - bspline(n - 1, x)"),
    "spme_axis_scale_swap": ("[gx * (K[0] / L[0]), gy * (K[1] / L[1]), gz * (K[2] / L[2])]",
                             "[gx * (K[1] / L[1]), gy * (K[0] / L[0]), gz * (K[2] / L[2])]"),
    "recip_force_factor": ("F += (2.0 / V) * q[:, None]", "F += (1.0 / V) * q[:, None]"),
    "recip_energy_factor": ("/ (2.0 * math.pi * V)", "/ (math.pi * V)"),
    "real_gaussian_term": ("(er / r + 2.0 * alpha / math.sqrt(math.pi)",
                           "(er / r + alpha / math.sqrt(math.pi)"),
    "real_min_image": ("np.where(d > 0.5 * L, d - L,", "np.where(d > 0.5 * L, d + L,"),
    "self_factor": ("return -alpha / math.sqrt(math.pi) * float(np.dot(q, q))",
                    "return -alpha / math.pi * float(np.dot(q, q))"),
    "background_sign": ("return -math.pi * Qt * Qt", "return math.pi * Qt * Qt"),
    "spline_recursion": ("return (x * bspline(n - 1, x) + (n - x) * bspline(n - 1, x - 1.0)) / (n - 1)",
                         "return (x * bspline(n - 1, x) + (n - x) * bspline(n - 1, x - 1.0)) / n"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_ewald_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = tmp_path / "ewald_mut.py"
    path.write_text(src.replace(old, new))
    env = dict(os.environ, ORACLE_EWALD=str(path))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_ewald.py"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
