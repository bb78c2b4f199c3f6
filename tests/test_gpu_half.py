"""Half Verlet lists (md_params.half_list, Newton's third law): each unordered
pair is listed once, by the atom whose cell is behind the partner's in the
stencil order (or, in one cell, by the earlier atom), and its reaction is added
to the partner's accumulator (FP32 atomics in a mixed context, FP64 in an FP64
one).  4 lanes per atom.

Bars: the half rows hold every pair once, and together with their reversals
they are exactly the FP64 oracle's full list (integer sets, bit-exact); forces
within relative L2 1e-5 (mixed) / 1e-10 (FP64) of the oracle and potential
energy to 1e-5 / 1e-10 for single boxes (2, 3 and 5 cells per axis, and a
compressed box whose home cells straddle the build's staging windows); in a
batch, forces to 1e-5 and energies against the full-list run; a 45-step run
stays within 1e-6 (mixed) / 1e-10 (FP64) of the full-list run; the adjoint,
which needs full lists, refuses a half-list context (the SPME solver takes
half lists: tests/test_gpu_spme*.py).
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
from paper_2109_09056_b300 import MDError, MDSystem  # noqa: E402


def boxes():
    rng = np.random.default_rng(4)
    return {"fcc10_nc5": mi.lj_melt(10, seed=21, jitter=0.2),
            "fcc6_nc3": mi.lj_melt(6, seed=3, jitter=0.1),
            "vac250_nc2": mi.vacancy_box(250, 0.9, 1.2, rng),
            # compressed lattice, 3 cells per axis, up to 62 atoms per cell: a
            # home cell's atoms come in two 32-candidate chunks, and for several
            # home batches the staging window fills between them, so the chunk
            # before the batch's own atoms lies in an earlier window
            "dense_fcc7_nc3": mi.lj_melt(7, rho=1.2, seed=1, jitter=0.1)}


NAMES = ["fcc10_nc5", "fcc6_nc3", "vac250_nc2", "dense_fcc7_nc3"]


def half_pairs_by_id(sysm):
    """Unordered pairs (original ids) of the half rows, and the row count."""
    st = sysm.state(forces=False)
    ids = np.asarray(st["ids"])
    nn, rows = sysm.neighbors()
    pairs = []
    for k in range(len(nn)):
        i = int(ids[k])
        for j in ids[rows[k, : nn[k]]]:
            pairs.append((min(i, int(j)), max(i, int(j))))
    return pairs, int(nn.sum())


@pytest.mark.parametrize("name", NAMES)
def test_half_rows_hold_each_pair_once_and_symmetrize_to_the_oracle(name):
    s = boxes()[name]
    sysm = make(s, "mixed", half_list=True)
    pairs, total = half_pairs_by_id(sysm)
    assert len(set(pairs)) == total == len(pairs)           # no pair twice
    xw = oracle.wrap(s.x, s.box)[0]
    nn_o, nbr_o = oracle.neighbors(xw, s.box, RS)
    full = set()
    for i in range(s.n):
        for j in nbr_o[i, : nn_o[i]]:
            full.add((min(i, int(j)), max(i, int(j))))
    assert set(pairs) == full
    sysm.close()


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_half_list_forces_and_energy_match_the_oracle(name, precision):
    s = boxes()[name]
    tol = 1e-5 if precision == "mixed" else 1e-10
    sysm = make(s, precision, half_list=True)
    pe = sysm.compute_forces()
    f = sysm.state()["f"]
    f_o, _, pe_o = oracle.lj_forces(oracle.wrap(s.x, s.box)[0], s.types, s.box)
    assert rel_l2(f, f_o) <= tol
    assert pe == pytest.approx(pe_o, rel=tol)
    sysm.close()


def test_half_list_fp64_after_steps_and_rebuilds_matches_the_full_list_run():
    """FP64: 45 steps (rebuilds at 20 and 40) with half lists against full
    lists, positions and total energy to 1e-10, forces on the final positions
    against the oracle to 1e-10."""
    s = mi.lj_melt(10, seed=10)
    half = make(s, "fp64", half_list=True)
    full = make(s, "fp64")
    th_h = half.step(45)
    th_f = full.step(45)
    sh, sf = half.state(), full.state()
    f_o, _, _ = oracle.lj_forces(oracle.wrap(sh["x"], s.box)[0], s.types, s.box)
    assert rel_l2(sh["f"], f_o) <= 1e-10
    xh = sh["x"] + sh["img"] * s.box
    xf = sf["x"] + sf["img"] * s.box
    assert rel_l2(xh, xf) <= 1e-10
    assert th_h["etot"] == pytest.approx(th_f["etot"], rel=1e-10)
    half.close()
    full.close()


def test_half_list_after_steps_and_rebuilds_matches_the_oracle():
    """45 steps (rebuilds at 20 and 40): forces on the final positions and the
    trajectory against the full-list mixed run."""
    s = mi.lj_melt(10, seed=10)
    half = make(s, "mixed", half_list=True)
    full = make(s, "mixed")
    th_h = half.step(45)
    th_f = full.step(45)
    sh, sf = half.state(), full.state()
    f_o, _, _ = oracle.lj_forces(oracle.wrap(sh["x"], s.box)[0], s.types, s.box)
    assert rel_l2(sh["f"], f_o) <= 1e-5
    xh = sh["x"] + sh["img"] * s.box
    xf = sf["x"] + sf["img"] * s.box
    assert rel_l2(xh, xf) <= 1e-6
    assert th_h["etot"] == pytest.approx(th_f["etot"], rel=1e-5)
    half.close()
    full.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_half_list_batch_per_box(precision):
    """Per box: forces against the oracle (1e-5 mixed, 1e-10 FP64); potential
    energy against the full-list run of the same batch, to 1e-6 (mixed) /
    1e-12 (FP64) of the summed per-atom energy magnitudes (in the mixed path
    both share the FP32 pair arithmetic, whose energy error shows most in box
    7, a compressed lattice of 286 atoms on 500 sites where pair energies of
    both signs sum to a small total); FP64 energies also against the oracle's
    (1e-10)."""
    ens = mi.ensemble(nbox=8, seed=5, n_lo=256, n_hi=3000)
    x = np.concatenate([b.x for b in ens])
    v = np.concatenate([b.v for b in ens])
    t = np.concatenate([b.types for b in ens])
    th, f = {}, None
    for half in (True, False):
        sysm = MDSystem(x, v, t, None, precision=precision, n_per_box=[b.n for b in ens],
                        boxes=[b.box for b in ens], half_list=half, lanes_per_atom=4,
                        stream=torch.cuda.Stream())
        sysm.compute_forces()
        if half:
            f = sysm.state()["f"]
        th[half] = sysm.batch_thermo()
        sysm.close()
    ftol, etol = (1e-5, 1e-6) if precision == "mixed" else (1e-10, 1e-12)
    off = np.concatenate([[0], np.cumsum([b.n for b in ens])])
    for k, b in enumerate(ens):
        f_o, e_o, pe_o = oracle.lj_forces(oracle.wrap(b.x, b.box)[0], b.types, b.box)
        assert rel_l2(f[off[k]:off[k + 1]], f_o) <= ftol, k
        assert abs(th[True][k]["pe"] - th[False][k]["pe"]) <= etol * np.abs(e_o).sum(), k
        if precision == "fp64":
            assert th[True][k]["pe"] == pytest.approx(pe_o, rel=1e-10), k


def test_half_list_refusals():
    s = mi.lj_melt(6, seed=3)
    with pytest.raises(MDError):
        make(s, "fp64", half_list=True, lanes_per_atom=8)
    with pytest.raises(MDError):
        make(s, "mixed", half_list=True, lanes_per_atom=8)
    sysm = make(s, "mixed", half_list=True)
    with pytest.raises(MDError):
        sysm.force_backward(np.zeros((s.n, 3)))
    sysm.close()
