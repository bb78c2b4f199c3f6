"""Degenerate inputs of the method against the FP64 oracle (GPU, both
precisions): a single atom (no neighbors), a dimer, a sparse gas with empty
cells and empty rows, and a dense cluster whose cells hold more than 32 atoms
and whose stencils hold more than one shared-memory window of candidates (the
build's multi-pass paths).  Bars as in the parity tests: permutation and
neighbor sets bit-exact, forces within 1e-10 (FP64) / 1e-5 (mixed)."""
import numpy as np
import pytest

import md_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import RS, gpu_sets_by_original_id, make, oracle_sets_by_original_id, rel_l2  # noqa: E402


def system(x, L):
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    v = mi.maxwell_velocities(n, 1.0, np.random.default_rng(n)) if n > 1 else np.zeros((n, 3))
    return mi.LJSystem(x=x, v=np.ascontiguousarray(v), types=np.zeros(n, dtype=np.int32),
                       box=np.full(3, float(L)))


def single():
    return system([[3.1, 4.2, 5.3]], 10.0)


def dimer():
    # r = 1.3: away from the minimum at 2^(1/6), where the pair force itself
    # cancels to ~0 and FP32 pair arithmetic keeps only an absolute accuracy
    return system([[5.0, 5.0, 5.0], [6.25, 5.3, 4.8]], 10.0)


def gas():
    rng = np.random.default_rng(7)
    return system(rng.uniform(0, 20.0, size=(33, 3)), 20.0)


def cluster():
    """About 3,000 atoms: a dense FCC blob (rho 1.6, nearest neighbors 0.95
    sigma apart, ~1000 atoms) inside a dilute FCC background (rho 0.5):
    up to 62 atoms in a cell, ~1200 candidates in a blob stencil, rows of ~150
    entries (the automatic pad overflows and grows)."""
    a = mi.fcc_lattice_constant(1.6)
    blob = mi.fcc_sites(7, 7, 7, a)[:1000] + 4.0
    lo, hi = 3.0, 4.0 + 7 * a + 1.0
    nb = 9
    L = (4 * nb ** 3 / 0.5) ** (1 / 3)
    bg = mi.fcc_sites(nb, nb, nb, L / nb) + 0.25
    outside = np.any((bg < lo) | (bg > hi), axis=1)
    return system(np.vstack([blob, bg[outside]]), L)


CASES = {"single": single, "dimer": dimer, "gas_33": gas, "cluster": cluster}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_degenerate_inputs(case, precision):
    s = CASES[case]()
    sysm = make(s, precision)
    perm_o, _, _ = oracle.bin_sort(s.x, s.box, RS)
    assert np.array_equal(sysm.permutation(), perm_o)
    assert gpu_sets_by_original_id(sysm) == oracle_sets_by_original_id(s.x, s.box)
    f_o, _, pe_o = oracle.lj_forces(oracle.wrap(s.x, s.box)[0], s.types, s.box)
    pe = sysm.compute_forces()
    f = sysm.state()["f"]
    if np.linalg.norm(f_o) == 0.0:
        assert np.all(f == 0.0) and pe == 0.0
    else:
        assert rel_l2(f, f_o) <= (1e-10 if precision == "fp64" else 1e-5)
    # a few steps run and stay finite
    th = sysm.step(10)
    assert np.isfinite(th["etot"])
    sysm.close()
