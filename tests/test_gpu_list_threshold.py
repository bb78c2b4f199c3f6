"""Neighbor decisions at the list radius (Section "Neighbor List Creation":
a pair is listed iff its nearest-image FP64 distance is below rs = rc + skin).

The build decides most candidates in FP32 and re-tests those whose FP32 r^2
lies within 3e-5 rs^2 of rs^2 with the exact FP64 rule.  These boxes hold
pairs placed at distances rs (1 + delta) for delta from -5e-5 to +5e-5, down
to +-1e-12 and 0 (so that many canonical FP64 r^2 fall inside the band and
some within a few ulps of rs^2), at random positions inside their cells and
across the periodic faces, in boxes of 2, 3 and 5 cells per axis.  Bar: the
GPU neighbor sets equal the FP64 oracle's, bit-exact, in both precisions and
with half lists (whose rows, symmetrised, equal the oracle's full list).
"""
import numpy as np
import pytest

import md_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import RS, gpu_sets_by_original_id, make, oracle_sets_by_original_id  # noqa: E402

DELTAS = [-5e-5, -2.9e-5, -1e-5, -1e-6, -1e-9, -1e-12, 0.0, 1e-12, 1e-9, 1e-6, 1e-5, 2.9e-5, 5e-5]


def threshold_box(L, npairs, seed):
    """npairs pairs at distance RS (1 + delta), no two atoms closer than 0.8."""
    rng = np.random.default_rng(seed)
    pts = np.zeros((0, 3))

    def clear(p):
        if len(pts) == 0:
            return True
        d = pts - p
        d -= L * np.round(d / L)
        return np.min(np.sum(d * d, axis=1)) > 0.64

    tries = 0
    while len(pts) < 2 * npairs and tries < 200000:
        tries += 1
        a = rng.uniform(0.0, L, 3)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        b = np.mod(a + RS * (1.0 + DELTAS[rng.integers(len(DELTAS))]) * u, L)
        if clear(a) and clear(b):
            pts = np.vstack([pts, a, b])
    n = len(pts)
    v = mi.maxwell_velocities(n, 1.0, rng)
    return mi.LJSystem(x=np.ascontiguousarray(pts), v=np.ascontiguousarray(v),
                       types=np.zeros(n, dtype=np.int32), box=np.full(3, float(L)))


def band_pairs(s):
    """Pairs whose canonical FP64 r^2 lies within 3e-5 rs^2 of rs^2."""
    xw = oracle.wrap(s.x, s.box)[0]
    d = xw[None, :, :] - xw[:, None, :]
    d -= s.box * np.round(d / s.box)
    r2 = np.sum(d * d, axis=2)
    iu = np.triu_indices(s.n, 1)
    return int(np.sum(np.abs(r2[iu] - RS * RS) <= 3e-5 * RS * RS))


BOXES = {"nc2": (6.0, 30, 1), "nc3": (9.0, 120, 2), "nc5": (14.5, 300, 3)}


@pytest.mark.parametrize("name", list(BOXES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_list_decisions_at_rs_match_the_oracle(name, precision):
    L, npairs, seed = BOXES[name]
    s = threshold_box(L, npairs, seed)
    assert band_pairs(s) >= npairs // 3       # the band is exercised
    sysm = make(s, precision)
    assert gpu_sets_by_original_id(sysm) == oracle_sets_by_original_id(s.x, s.box)
    sysm.close()


@pytest.mark.parametrize("name", list(BOXES))
def test_half_list_decisions_at_rs_match_the_oracle(name):
    L, npairs, seed = BOXES[name]
    s = threshold_box(L, npairs, seed)
    sysm = make(s, "mixed", half_list=True)
    half = gpu_sets_by_original_id(sysm)
    full = {i: set() for i in range(s.n)}
    for i, js in half.items():
        for j in js:
            assert i not in half[j]               # each pair once
            full[i].add(j)
            full[j].add(i)
    assert {i: frozenset(v) for i, v in full.items()} == oracle_sets_by_original_id(s.x, s.box)
    sysm.close()
