"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Bars: cell permutations and neighbor sets bit-exact; forces relative L2
<= 1e-10 (FP64 path) and <= 1e-5 (mixed path) on the same positions; the
FP64 trajectory within 1e-9 of the oracle's over 100 steps.
"""
import numpy as np
import pytest

import md_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import RS, gpu_sets_by_original_id, make, oracle_sets_by_original_id, rel_l2  # noqa: E402


def ragged_box(n=1000, rho=0.8442, seed=5):
    rng = np.random.default_rng(seed)
    return mi.vacancy_box(n, rho, 1.44, rng)


CASES = {
    "fcc10_4000": lambda: mi.lj_melt(10, seed=1),
    "fcc10_jitter": lambda: mi.lj_melt(10, seed=2, jitter=0.1),
    "ragged_1000": lambda: ragged_box(1000),
    "nc3_864": lambda: mi.lj_melt(6, seed=3, jitter=0.15),
    "nc2_256": lambda: ragged_box(256, rho=0.7, seed=6),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_create_sort_list_forces(case, precision):
    s = CASES[case]()
    sysm = make(s, precision)
    # permutation of the first sort, relative to the input order
    perm_o, xs_o, _ = oracle.bin_sort(s.x, s.box, RS)
    assert np.array_equal(sysm.permutation(), perm_o)
    # neighbor sets by original id
    assert gpu_sets_by_original_id(sysm) == oracle_sets_by_original_id(s.x, s.box)
    # forces and energy on the same positions
    f_o, _, pe_o = oracle.lj_forces(oracle.wrap(s.x, s.box)[0], s.types, s.box)
    pe = sysm.compute_forces()
    f = sysm.state()["f"]
    tol = 1e-10 if precision == "fp64" else 1e-5
    if np.linalg.norm(f_o) > 1e-8:
        assert rel_l2(f, f_o) <= tol
    else:  # perfect lattice: forces vanish
        assert np.abs(f).max() < (1e-10 if precision == "fp64" else 1e-4)
    assert abs(pe - pe_o) <= (1e-11 if precision == "fp64" else 1e-6) * abs(pe_o)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_lanes_per_atom_variants(precision, lanes):
    s = mi.lj_melt(8, seed=7, jitter=0.1)
    sysm = make(s, precision, lanes_per_atom=lanes)
    f_o, _, pe_o = oracle.lj_forces(oracle.wrap(s.x, s.box)[0], s.types, s.box)
    pe = sysm.compute_forces()
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert rel_l2(sysm.state()["f"], f_o) <= tol
    assert gpu_sets_by_original_id(sysm) == oracle_sets_by_original_id(s.x, s.box)


@pytest.mark.parametrize("lanes,block", [(1, 768), (2, 768), (4, 384), (8, 64)])
def test_cta_sizes_and_wide_rows(lanes, block):
    """Explicit CTA sizes, including ones whose per-warp list buffers do not all
    fit in shared memory at 768 threads (the kernel then runs fewer warps per
    CTA): same forces as the oracle and the same trajectory as the default."""
    s = mi.lj_melt(12, seed=13, jitter=0.1)         # 6912 atoms
    a = make(s, "mixed", lanes_per_atom=lanes, block_threads=block)
    f_o, _, _ = oracle.lj_forces(oracle.wrap(s.x, s.box)[0], s.types, s.box)
    a.compute_forces()
    assert rel_l2(a.state()["f"], f_o) <= 1e-5
    b = make(s, "mixed", lanes_per_atom=lanes)
    a.step(30)
    b.step(30)
    assert np.array_equal(a.state()["x"], b.state()["x"])   # the CTA size changes no arithmetic


def test_two_types_forces_both_precisions():
    s = mi.two_type_melt(8, seed=8)
    f_o, _, pe_o = oracle.lj_forces(oracle.wrap(s.x, s.box)[0], s.types, s.box, eps=s.eps,
                                    sigma=s.sigma)
    for precision, tol in (("fp64", 1e-10), ("mixed", 1e-5)):
        sysm = make(s, precision)
        pe = sysm.compute_forces()
        assert rel_l2(sysm.state()["f"], f_o) <= tol
        assert abs(pe - pe_o) <= tol * abs(pe_o)


def test_shifted_energy():
    s = mi.lj_melt(8, seed=9, jitter=0.1)
    _, _, pe_o = oracle.lj_forces(oracle.wrap(s.x, s.box)[0], s.types, s.box, shift=True)
    sysm = make(s, "fp64", shift_energy=True)
    assert sysm.compute_forces() == pytest.approx(pe_o, rel=1e-12)


def test_build_after_steps_resorts_first():
    """md_build_neighbors on a drifted state re-sorts before building: the
    permutation and the lists equal the oracle's sort and list of the snapshot."""
    s = mi.lj_melt(10, seed=12)
    sysm = make(s, "mixed")
    sysm.step(27)                        # rebuilt at 20; drifted since
    st = sysm.state(forces=False)
    x_int = st["x"][st["ids"]]
    sysm.build_neighbors()               # no explicit bin_sort
    perm_o, xs_o, _ = oracle.bin_sort(x_int, s.box, RS)
    assert np.array_equal(sysm.permutation(), perm_o)
    nn, rows = sysm.neighbors()
    nn_o, rows_o = oracle.neighbors(xs_o, s.box, RS)
    assert np.array_equal(nn, nn_o)
    for k in range(len(nn)):
        assert set(rows[k, : nn[k]].tolist()) == set(rows_o[k, : nn_o[k]].tolist())


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_resort_and_list_after_steps_on_gpu_snapshot(precision):
    """Per-stage parity on the GPU's own state: run, snapshot, then the GPU's
    re-sort and list must equal the oracle's on that snapshot."""
    s = mi.lj_melt(10, seed=10)
    sysm = make(s, precision)
    sysm.step(33)                        # rebuilt at 20; drifted since
    st = sysm.state(forces=False)
    x_int = st["x"][st["ids"]]           # positions in the GPU's internal order
    sysm.bin_sort()
    perm_o, xs_o, _ = oracle.bin_sort(x_int, s.box, RS)
    assert np.array_equal(sysm.permutation(), perm_o)
    sysm.build_neighbors()
    nn, rows = sysm.neighbors()
    nn_o, rows_o = oracle.neighbors(xs_o, s.box, RS)
    assert np.array_equal(nn, nn_o)
    for k in range(len(nn)):
        assert set(rows[k, : nn[k]].tolist()) == set(rows_o[k, : nn_o[k]].tolist())
    # forces on the snapshot positions (original order)
    pe = sysm.compute_forces()
    f_o, _, pe_o = oracle.lj_forces(oracle.wrap(st["x"], s.box)[0], s.types, s.box)
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert rel_l2(sysm.state()["f"], f_o) <= tol


def test_fp64_trajectory_matches_oracle_100_steps():
    s = mi.lj_melt(10, seed=1)
    sysm = make(s, "fp64", thermo_every=10)
    th = sysm.step(100)
    st = sysm.state()
    r = oracle.md_run(s.x, s.v, s.types, s.box, 100)
    x_o = r.by_id(r.x + r.img * s.box)
    x_g = st["x"] + st["img"] * s.box
    assert np.abs(x_g - x_o).max() < 1e-9
    assert np.abs(st["v"] - r.by_id(r.v)).max() < 1e-8
    assert th["etot"] == pytest.approx(r.thermo[-1, 2], rel=1e-10)
    log = sysm.thermo_log()
    assert log.shape[0] == 11
    assert np.allclose(log[:, 3], r.thermo[::10, 2], rtol=1e-10)


def test_mixed_trajectory_close_and_energy_drift():
    s = mi.lj_melt(10, seed=1)
    th64 = make(s, "fp64", thermo_every=10)
    thmx = make(s, "mixed", thermo_every=10)
    a = th64.step(100)
    b = thmx.step(100)
    r = oracle.md_run(s.x, s.v, s.types, s.box, 100)
    # chaotic divergence is slow over 0.5 time units: positions stay close
    xa = thmx.state()["x"] + thmx.state()["img"] * s.box
    x_o = r.by_id(r.x + r.img * s.box)
    assert np.abs(xa - x_o).max() < 1e-3
    la, lb = th64.thermo_log(), thmx.thermo_log()
    assert np.abs((lb[:, 3] - la[:, 3]) / s.n).max() < 1e-5
    assert b["etot"] / s.n == pytest.approx(a["etot"] / s.n, abs=1e-5)


def test_determinism_and_graph_equivalence():
    s = mi.lj_melt(10, seed=11)
    runs = []
    for graphs in (True, True, False):
        sysm = make(s, "mixed", use_graphs=graphs)
        sysm.step(45)
        st = sysm.state()
        runs.append((st["x"], st["v"], st["f"]))
    for k in range(3):
        assert np.array_equal(runs[0][k], runs[1][k])     # run to run, bitwise
        assert np.array_equal(runs[0][k], runs[2][k])     # graph replay == direct launches


def test_overflow_recovery_matches_roomy_pad():
    # From a perfect lattice every row holds 78 entries; an explicit pad grows
    # only to what a build needs (80), so rows growing as the crystal melts
    # overflow inside md_step and exercise the freeze / grow / resume path.
    s = mi.lj_melt(8, seed=12)
    big = make(s, "mixed", neigh_pad=160)
    small = make(s, "mixed", neigh_pad=8)
    assert small.thermo()["pad"] == 80
    big.step(50)
    small.step(50)
    a, b = big.state(), small.state()
    for k in ("x", "v", "f"):
        assert np.array_equal(a[k], b[k])
    assert small.thermo()["pad"] >= small.thermo()["nn_max"]


def test_error_paths_return_status():
    from paper_2109_09056_b300 import MDError, MDSystem
    s = mi.lj_melt(10, seed=1)
    with pytest.raises(MDError) as e:
        MDSystem(s.x, s.v, s.types, [5.5, 20.0, 20.0])
    assert "BOX_TOO_SMALL" in str(e.value)
    bad_t = s.types.copy()
    bad_t[3] = 4
    with pytest.raises(MDError) as e:
        MDSystem(s.x, s.v, bad_t, s.box)
    assert "MD_ERR_ARG" in str(e.value)
    x = s.x.copy()
    x[7, 1] = np.nan
    with pytest.raises(MDError) as e:
        MDSystem(x, s.v, s.types, s.box)
    assert "NONFINITE" in str(e.value)
    with pytest.raises(MDError):
        MDSystem(s.x, s.v, s.types, s.box, lanes_per_atom=3)


def test_dangerous_build_flag_when_checked():
    from paper_2109_09056_b300 import MDError
    s = mi.lj_melt(10, seed=1)
    sysm = make(s, "mixed", check_displacement=True)
    with pytest.raises(MDError) as e:
        sysm.step(100)                      # T*=1.44, rebuild every 20 > skin/2 motion
    assert "DANGEROUS" in str(e.value)
    assert sysm.thermo()["dangerous_builds"] >= 1


def test_device_and_host_pointers_agree():
    s = mi.lj_melt(8, seed=14, jitter=0.1)
    a = make(s, "fp64")
    xd = torch.from_numpy(s.x).cuda()
    vd = torch.from_numpy(s.v).cuda()
    td = torch.from_numpy(s.types).cuda()
    from paper_2109_09056_b300 import MDSystem
    b = MDSystem(xd, vd, td, s.box, precision="fp64", stream=torch.cuda.Stream())
    a.step(25)
    b.step(25)
    sa = a.state()
    sb = b.state(device="cuda")
    for k in ("x", "v", "f"):
        assert np.array_equal(sa[k], sb[k].cpu().numpy())


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_set_state_from_host_pinned_and_device(precision):
    """md_set_state with host velocities copies them beside the re-sort and
    puts them in place by atom id: numpy (pageable), pinned and device inputs
    give the same state, which continues like the run it came from."""
    s = mi.lj_melt(8, seed=15, jitter=0.1)
    a = make(s, precision)
    a.step(10)
    st = a.state()
    runs = []
    for kind in ("numpy", "pinned", "device"):
        b = make(s, precision)
        if kind == "numpy":
            b.set_state(st["x"], st["v"])
        elif kind == "pinned":
            b.set_state(torch.from_numpy(st["x"]).pin_memory(), torch.from_numpy(st["v"]).pin_memory())
        else:
            b.set_state(torch.from_numpy(st["x"]).cuda(), torch.from_numpy(st["v"]).cuda())
        sb = b.state()
        assert np.array_equal(sb["v"], st["v"])
        assert np.abs(periodic_diff(sb["x"], st["x"], s.box)).max() < 1e-12
        tol = 1e-10 if precision == "fp64" else 1e-5
        assert rel_l2(sb["f"], st["f"]) <= tol
        b.step(10)
        runs.append(b.state())
    for r in runs[1:]:
        for k in ("x", "v", "f"):
            assert np.array_equal(r[k], runs[0][k])
    # velocities alone, positions kept
    c = make(s, precision)
    v2 = -st["v"]
    c.set_state(None, v2)
    sc = c.state()
    assert np.array_equal(sc["v"], v2)
    assert np.abs(periodic_diff(sc["x"], s.x, s.box)).max() < 1e-12


def periodic_diff(a, b, L):
    """a - b folded into [-L/2, L/2) (positions may sit in different images)."""
    d = np.asarray(a) - np.asarray(b)
    return d - L * np.round(d / L)
