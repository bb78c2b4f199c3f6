"""Parity at the benchmark's full size (the 4M-atom LJ melt, 100^3 FCC cells)
in the launch configuration bench.py times (library-default lanes per atom and
CTA size, rebuild every 20, CUDA-graph periods).  After 27 steps (one rebuild
at step 20, then drift) the GPU state is snapshot and:

* the re-sort's permutation equals the oracle's counting sort of the snapshot
  (all 4M atoms, bit-exact);
* the neighbor rows of sampled atoms equal the oracle's brute-force rows over
  all 4M atoms (bit-exact sets), sampled atoms including the first and last
  slots and the atoms with the longest and shortest rows;
* the forces of sampled atoms match the oracle's brute-force forces (relative
  L2 over the sample: 1e-5 mixed, 1e-10 FP64).
"""
import numpy as np
import pytest

import md_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import RS, make, rel_l2  # noqa: E402
from paper_2109_09056_b300 import api as A  # noqa: E402

NSAMPLE = 192


@pytest.fixture(scope="module")
def workload():
    return mi.workload("lj_fcc100_4m")


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_fullsize_sort_list_forces_sampled(workload, precision):
    s = workload
    sysm = make(s, precision)
    sysm.step(27)
    st = sysm.state(forces=False)
    x_int = st["x"][st["ids"]]                    # positions in the GPU's internal order
    sysm.bin_sort()
    perm_o, xs_o, _ = oracle.bin_sort(x_int, s.box, RS)
    assert np.array_equal(sysm.permutation(), perm_o)
    sysm.build_neighbors()

    dev = torch.device("cuda")
    nn_d, rows_d = A.md_get_neighbors(sysm.ctx, device=dev)
    nn = nn_d.cpu().numpy()
    rng = np.random.default_rng(2026)
    idx = np.unique(np.concatenate([
        rng.choice(s.n, NSAMPLE, replace=False),
        [0, s.n - 1, int(np.argmax(nn)), int(np.argmin(nn))]]))
    rows = rows_d[torch.as_tensor(idx, device=dev)].cpu().numpy()
    sets_o = oracle.neighbors_sample(xs_o, s.box, RS, idx)
    for k, i in enumerate(idx):
        assert nn[i] == len(sets_o[k]), i
        assert frozenset(rows[k, : nn[i]].tolist()) == sets_o[k], i

    sysm.compute_forces()
    st = sysm.state()
    ids = st["ids"]                               # original id of each internal slot
    sample_ids = ids[idx]
    xw = oracle.wrap(st["x"], s.box)[0]
    f_o, _ = oracle.lj_forces_sample(xw, s.types, s.box, sample_ids)
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert rel_l2(st["f"][sample_ids], f_o) <= tol
    sysm.close()
