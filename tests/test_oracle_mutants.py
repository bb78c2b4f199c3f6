"""The oracle pins catch plausible mistakes: each mutant below plants one
(dropped term, wrong sign or factor, wrong index order, broken stability,
swapped integrator order, wrong adjoint factor) in a copy of oracle_md.c,
compiles it, and runs the oracle pin tests against it in a subprocess; at
least one pin must fail.  CPU only; the mutants live in a temporary
directory and never replace the real oracle."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle_md.c")
PINS = ["tests/test_oracle_pair.py", "tests/test_oracle_lists.py", "tests/test_oracle_md.py",
        "tests/test_oracle_adjoint.py"]

MUTANTS = {
    "pair_sign": ("*phi = 24.0 * eps * r2inv * (2.0 * s12 - s6);",
                  "*phi = 24.0 * eps * r2inv * (2.0 * s12 + s6);"),
    "pair_factor": ("*phi = 24.0 * eps * r2inv * (2.0 * s12 - s6);",
                    "*phi = 48.0 * eps * r2inv * (2.0 * s12 - s6);"),
    "energy_half": ("double e = 4.0 * eps * (s12 - s6);", "double e = 2.0 * eps * (s12 - s6);"),
    "cutoff_inclusive": ("if (!(u < rc2)) continue;\n            int32_t ab = type[i] * ntypes + type[j];\n            double phi, U;\n            lj_pair(u, eps[ab], sigma[ab], rc, shift, &phi, &U);\n            for (int a = 0; a < 3; ++a) fi[a] += phi * d[a];\n            ei += 0.5 * U;\n        }\n        for (int a = 0; a < 3; ++a) f[3 * i + a] = fi[a];\n        ea[i] = ei;\n    }\n    double tot = 0.0;\n    for (int64_t i = 0; i < n; ++i) tot += ea[i];\n    if (pe) *pe = tot;\n    if (!e_atom) free(ea);\n}\n\n/* Forces and energies by brute",
                         "if (!(u <= rc2)) continue;\n            int32_t ab = type[i] * ntypes + type[j];\n            double phi, U;\n            lj_pair(u, eps[ab], sigma[ab], rc, shift, &phi, &U);\n            for (int a = 0; a < 3; ++a) fi[a] += phi * d[a];\n            ei += 0.5 * U;\n        }\n        for (int a = 0; a < 3; ++a) f[3 * i + a] = fi[a];\n        ea[i] = ei;\n    }\n    double tot = 0.0;\n    for (int64_t i = 0; i < n; ++i) tot += ea[i];\n    if (pe) *pe = tot;\n    if (!e_atom) free(ea);\n}\n\n/* Forces and energies by brute"),
    "min_image_sign": ("        if (t > h) t = t - L[a];\n        else if (t < -h) t = t + L[a];\n        d[a] = t;\n    }\n    double sx",
                       "        if (t > h) t = t + L[a];\n        else if (t < -h) t = t + L[a];\n        d[a] = t;\n    }\n    double sx"),
    "no_stencil_dedupe": ("if (seen) continue;", "(void)seen;"),
    "unstable_sort": ("for (int64_t i = 0; i < n; ++i) perm[start[cell[i]]++] = (int32_t)i;",
                      "for (int64_t i = n - 1; i >= 0; --i) perm[start[cell[i]]++] = (int32_t)i;"),
    "cell_order": ("cell[i] = (c[2] * nc[1] + c[1]) * nc[0] + c[0];",
                   "cell[i] = (c[0] * nc[1] + c[1]) * nc[2] + c[2];"),
    "wrap_upper": ("if (w >= L) { w = w - L; k += 1; }", "(void)0;"),
    "drift_before_kick": ("v[3 * i + a] = v[3 * i + a] + hm * f[3 * i + a];\n                    x[3 * i + a] = x[3 * i + a] + dt * v[3 * i + a];",
                          "x[3 * i + a] = x[3 * i + a] + dt * v[3 * i + a];\n                    v[3 * i + a] = v[3 * i + a] + hm * f[3 * i + a];"),
    "adjoint_psi": ("double psi = 2.0 * dphidu;", "double psi = dphidu;"),
    "adjoint_dsigma": ("double dphids = (24.0 * e / u) * (24.0 * s12 - 6.0 * s6) / s;",
                       "double dphids = (24.0 * e / u) * (12.0 * s12 - 6.0 * s6) / s;"),
    "adjoint_energy_half": ("row[0] += dGi * dphide + 0.5 * gE * dUde;", "row[0] += dGi * dphide + gE * dUde;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(old, new, 1)
    c_path = tmp_path / "oracle_mut.c"
    so_path = tmp_path / "liboracle_mut.so"
    c_path.write_text(mutated)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-std=c11", "-shared", "-fPIC",
                    "-o", str(so_path), str(c_path), "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB=str(so_path))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu", *PINS], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
