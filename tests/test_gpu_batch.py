"""Batched ensemble: many independent periodic boxes of uneven size in one
context (every kernel runs over all boxes in one launch; the force kernel is
the persistent one; the rebuild period replays as a CUDA graph).

Bars: a batched run is bitwise identical to running each box in its own
context (the per-atom work and its order do not depend on the other boxes);
per-box forces match the FP64 oracle (relative L2 1e-5 mixed, 1e-10 FP64);
per-box thermo matches the oracle; boxes with only 2 cells per axis included.
"""
import numpy as np
import pytest

import md_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import rel_l2  # noqa: E402
from paper_2109_09056_b300 import MDSystem  # noqa: E402


def small_ensemble():
    boxes = mi.ensemble(nbox=12, seed=5, n_lo=256, n_hi=3000)
    # 250 atoms (6 vacancies) at rho 0.9: L = 6.52, 2 cells per axis
    boxes[0] = mi.vacancy_box(250, 0.9, 1.2, np.random.default_rng(1))
    return boxes


def batch_system(boxes, precision, **kw):
    x = np.concatenate([b.x for b in boxes])
    v = np.concatenate([b.v for b in boxes])
    t = np.concatenate([b.types for b in boxes])
    return MDSystem(x, v, t, None, precision=precision, n_per_box=[b.n for b in boxes],
                    boxes=[b.box for b in boxes], stream=torch.cuda.Stream(), **kw)


def offsets(boxes):
    return np.concatenate([[0], np.cumsum([b.n for b in boxes])])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_forces_match_oracle_per_box(precision):
    boxes = small_ensemble()
    sysm = batch_system(boxes, precision)
    sysm.compute_forces()
    f = sysm.state()["f"]
    off = offsets(boxes)
    tol = 1e-5 if precision == "mixed" else 1e-10
    th = sysm.batch_thermo()
    for k, b in enumerate(boxes):
        xw = oracle.wrap(b.x, b.box)[0]
        f_o, _, pe_o = oracle.lj_forces(xw, b.types, b.box)
        if np.linalg.norm(f_o) > 1e-6:
            assert rel_l2(f[off[k]:off[k + 1]], f_o) <= tol, k
        else:  # a perfect crystal: forces vanish
            assert np.abs(f[off[k]:off[k + 1]]).max() < 1e-4, k
        assert th[k]["pe"] == pytest.approx(pe_o, rel=tol)
        ke_o, t_o, _ = oracle.thermo(b.v, b.types)
        assert th[k]["ke"] == pytest.approx(ke_o, rel=1e-12)


def test_batch_run_equals_separate_runs_bitwise():
    boxes = small_ensemble()
    sysm = batch_system(boxes, "mixed")
    sysm.step(45)
    st = sysm.state()
    th = sysm.batch_thermo()
    off = offsets(boxes)
    for k, b in enumerate(boxes):
        one = MDSystem(b.x, b.v, b.types, b.box, precision="mixed", stream=torch.cuda.Stream())
        t1 = one.step(45)
        s1 = one.state()
        for key in ("x", "v", "f"):
            assert np.array_equal(st[key][off[k]:off[k + 1]], s1[key]), (k, key)
        assert th[k]["etot"] == t1["etot"]
        one.close()


def test_batch_fp64_trajectory_matches_oracle():
    boxes = small_ensemble()[:4]
    sysm = batch_system(boxes, "fp64")
    sysm.step(40)
    st = sysm.state()
    off = offsets(boxes)
    for k, b in enumerate(boxes):
        r = oracle.md_run(b.x, b.v, b.types, b.box, 40)
        x_o = r.by_id(r.x + r.img * b.box)
        x_g = st["x"][off[k]:off[k + 1]] + st["img"][off[k]:off[k + 1]] * b.box
        assert np.abs(x_g - x_o).max() < 1e-9, k
