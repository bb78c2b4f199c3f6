"""Particle-layout variants of the mixed force kernel's neighbor gathers
(md_params.shadow_vl): the float4 shadow per atom (default) against AoSoA
copies of vector length 8 and 32 (blocks of x[V], y[V], z[V], type[V]).  The
kernel reads the same FP32 values either way, so forces, energies and whole
trajectories must be bitwise identical to the default layout, and match the
oracle to the mixed bar; invalid combinations are refused.
"""
import numpy as np
import pytest

import md_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import make, rel_l2  # noqa: E402
from paper_2109_09056_b300 import MDError  # noqa: E402


@pytest.mark.parametrize("vl", [8, 32])
def test_aosoa_gathers_give_the_same_forces_and_trajectory(vl):
    s = mi.lj_melt(10, seed=12, jitter=0.1)
    ref = make(s, "mixed")
    var = make(s, "mixed", shadow_vl=vl)
    assert var.compute_forces() == ref.compute_forces()
    fv, fr = var.state()["f"], ref.state()["f"]
    assert np.array_equal(fv, fr)
    f_o, _, _ = oracle.lj_forces(oracle.wrap(s.x, s.box)[0], s.types, s.box)
    assert rel_l2(fv, f_o) <= 1e-5
    tv, tr = var.step(45), ref.step(45)
    sv, sr = var.state(), ref.state()
    for k in ("x", "v", "f"):
        assert np.array_equal(sv[k], sr[k]), k
    assert tv["etot"] == tr["etot"]
    var.close()
    ref.close()


def test_aosoa_two_types():
    s = mi.workload("lj_2type_fcc20_32000")
    ref = make(s, "mixed")
    var = make(s, "mixed", shadow_vl=32)
    ref.compute_forces()
    var.compute_forces()
    assert np.array_equal(var.state()["f"], ref.state()["f"])
    var.close()
    ref.close()


def test_aosoa_refusals():
    s = mi.lj_melt(6, seed=3)
    for kw in (dict(precision="fp64", shadow_vl=8), dict(shadow_vl=16),
               dict(shadow_vl=8, lanes_per_atom=2), dict(shadow_vl=8, half_list=True)):
        prec = kw.pop("precision", "mixed")
        with pytest.raises(MDError):
            make(s, prec, **kw)
