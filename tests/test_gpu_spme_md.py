"""Coulomb + LJ dynamics (md_spme_step) against a velocity-Verlet loop over
the oracles' forces (C LJ oracle + numpy Ewald/SPME oracle), through the C
ABI, on a B300; and energy conservation of the combined dynamics.

Trajectory: 864 atoms (6^3 FCC melt cells, jitter 0.1), neutral random +-1
charges, alpha 1.25, rc 2.5, 24^3 grid, order 4, dt 0.005, 30 steps with a
re-sort and list rebuild every 4 steps.  The oracle takes every pair by brute
force at every step; the GPU takes them from its Verlet list, which holds every
pair within rc only while no atom has moved more than skin/2 since the build,
so the cadence is kept short enough for that to hold throughout (the Coulomb
forces accelerate atoms beyond what a 20-step cadence allows at this
temperature).  Positions (modulo the box) and velocities must match the
oracle's to 1e-9 (FP64) / 1e-5 (mixed) relative, and the final energies to the
same bars.
"""
import dataclasses

import numpy as np
import pytest

import md_inputs as mi
import oracle
from oracle import ewald as ew

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import make, rel_l2  # noqa: E402
from paper_2109_09056_b300 import SPME  # noqa: E402

ALPHA, RC, K, ORDER = 1.25, 2.5, (24, 24, 24), 4


def small_charged():
    s = mi.lj_melt(6, seed=3, jitter=0.1)
    s.rebuild_every = 4
    q = mi.neutral_charges(s.n, np.random.default_rng(17))
    return s, q


def oracle_forces(x, q, s, shift=False):
    xw = oracle.wrap(x, s.box)[0]
    f_lj, _, pe = oracle.lj_forces(xw, s.types, s.box, eps=s.eps, sigma=s.sigma, shift=shift)
    ek, fk = ew.spme_reciprocal(xw, q, s.box, ALPHA, K, ORDER)
    er, fr = ew.ewald_real(xw, q, s.box, ALPHA, RC)
    ec = ek + er + ew.ewald_self(q, ALPHA) + ew.ewald_background(q, s.box, ALPHA)
    return f_lj + fk + fr, pe, ec


def oracle_verlet(s, q, nsteps, shift=False):
    """Velocity Verlet (m = 1): v += dt/2 F; x += dt v; F = F(x); v += dt/2 F."""
    x, v = s.x.copy(), s.v.copy()
    f, pe, ec = oracle_forces(x, q, s, shift)
    for _ in range(nsteps):
        v = v + 0.5 * s.dt * f
        x = x + s.dt * v
        f, pe, ec = oracle_forces(x, q, s, shift)
        v = v + 0.5 * s.dt * f
    return x, v, pe, ec, 0.5 * float((v * v).sum())


def periodic_diff(a, b, box):
    d = a - b
    return d - box * np.round(d / box)


@pytest.fixture(scope="module")
def reference():
    s, q = small_charged()
    return s, q, oracle_verlet(s, q, 30)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_step_trajectory_matches_oracle(reference, precision):
    s, q, (x_o, v_o, pe_o, ec_o, ke_o) = reference
    tol = 1e-9 if precision == "fp64" else 1e-5
    sysm = make(s, precision)
    sp = SPME(sysm, q, alpha=ALPHA, rc=RC, K=K, order=ORDER)
    e = sp.step(30)
    st = sysm.state(forces=False)
    dx = periodic_diff(st["x"], x_o, s.box)
    assert np.linalg.norm(dx) <= tol * np.linalg.norm(x_o)
    assert rel_l2(st["v"], v_o) <= tol
    assert abs(e["pe_lj"] - pe_o) <= tol * abs(pe_o)
    assert abs(e["coulomb"] - ec_o) <= tol * abs(ec_o)
    assert abs(e["ke"] - ke_o) <= tol * abs(ke_o)
    assert e["total"] == pytest.approx(e["pe_lj"] + e["coulomb"] + e["ke"], rel=1e-14)
    # zero steps: the energies of the current state, state unchanged
    e0 = sp.step(0)
    assert e0["ke"] == pytest.approx(e["ke"], rel=1e-12)
    st0 = sysm.state(forces=False)
    assert np.array_equal(st0["x"], st["x"])
    sp.close()
    sysm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_step_chunks_equal_one_run(precision):
    """Two calls of 15 steps give the state of one call of 30 (the forces of
    the starting state are recomputed at each call)."""
    s, q = small_charged()
    a = make(s, precision)
    b = make(s, precision)
    sa = SPME(a, q, alpha=ALPHA, rc=RC, K=K, order=ORDER)
    sb = SPME(b, q, alpha=ALPHA, rc=RC, K=K, order=ORDER)
    ea = sa.step(30)
    sb.step(15)
    eb = sb.step(15)
    xa, xb = a.state(forces=False)["x"], b.state(forces=False)["x"]
    tol = 1e-11 if precision == "fp64" else 1e-6
    assert np.linalg.norm(periodic_diff(xa, xb, s.box)) <= tol * np.linalg.norm(xa)
    assert eb["total"] == pytest.approx(ea["total"], rel=tol)
    for o in (sa, sb):
        o.close()
    a.close()
    b.close()


def test_spme_step_energy_conservation():
    """NVE with the shifted LJ potential (energy continuous at rc) and SPME
    Coulomb on the 4,000-atom charged melt over 2 time units, both
    precisions: no dangerous build (list rebuilt every 0.02 time units), the
    total energy's largest deviation falls with dt^2 (ratio 2.5-6 for dt
    halved) and stays below 1e-4 per atom at dt = 0.002, and the two
    precisions' energy traces agree to a tenth of that deviation (their
    trajectories drift apart chaotically, so the bar is set by the energy's
    own integration fluctuation, not by a fixed number)."""
    cs = mi.charged_workload("coulomb_fcc10_4000")
    s = cs.lj
    dev = {}
    for prec in ("fp64", "mixed"):
        for dt, every in ((0.004, 5), (0.002, 10)):
            m = make(dataclasses.replace(s, dt=dt, rebuild_every=every), prec,
                     shift_energy=True, check_displacement=True)
            sp = SPME(m, cs.q, alpha=cs.alpha, rc=cs.rc, K=cs.K, order=cs.order)
            chunk = int(round(0.1 / dt))
            E = [sp.step(0)["total"]] + [sp.step(chunk)["total"] for _ in range(20)]
            assert m.thermo()["dangerous_builds"] == 0
            dev[prec, dt] = np.abs(np.array(E) - E[0]).max() / s.n
            dev[prec, dt, "E"] = np.array(E) / s.n
            sp.close()
            m.close()
    for prec in ("fp64", "mixed"):
        ratio = dev[prec, 0.004] / dev[prec, 0.002]
        assert 2.5 <= ratio <= 6.0, (prec, ratio)
        assert dev[prec, 0.002] <= 1e-4
    assert (np.abs(dev["fp64", 0.002, "E"] - dev["mixed", 0.002, "E"]).max()
            <= 0.1 * dev["fp64", 0.002])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_step_two_types_shifted(precision):
    """The fused LJ + Coulomb pass with two atom types (per-pair eps, sigma in
    [0.8, 1.2]) and the shifted LJ potential: 12 steps against the oracle loop."""
    rng = np.random.default_rng(41)
    s = mi.lj_melt(6, seed=5, jitter=0.1)
    s.types = np.zeros(s.n, dtype=np.int32)
    s.types[rng.permutation(s.n)[: s.n // 2]] = 1
    s.eps, s.sigma = mi.random_pair_params(2, rng)
    s.mass = np.ones(2)
    s.rebuild_every = 4
    q = mi.neutral_charges(s.n, rng)
    x_o, v_o, pe_o, ec_o, ke_o = oracle_verlet(s, q, 12, shift=True)
    tol = 1e-9 if precision == "fp64" else 1e-5
    sysm = make(s, precision, shift_energy=True)
    sp = SPME(sysm, q, alpha=ALPHA, rc=RC, K=K, order=ORDER)
    e = sp.step(12)
    st = sysm.state(forces=False)
    assert np.linalg.norm(periodic_diff(st["x"], x_o, s.box)) <= tol * np.linalg.norm(x_o)
    assert rel_l2(st["v"], v_o) <= tol
    assert abs(e["pe_lj"] - pe_o) <= tol * abs(pe_o)
    assert abs(e["coulomb"] - ec_o) <= tol * abs(ec_o)
    sp.close()
    sysm.close()


def test_spme_step_reuses_forces_only_while_valid():
    """Between md_spme_step calls the total forces are reused when nothing
    touched the context: ten single steps give the trajectory of one call of
    ten (FP64, 1e-11); md_set_params between two calls is seen (the oracle loop
    switches eps at the same point), and so are another solver's step and
    md_spme_set_charges."""
    s, q = small_charged()
    a = make(s, "fp64")
    b = make(s, "fp64")
    sa = SPME(a, q, alpha=ALPHA, rc=RC, K=K, order=ORDER)
    sb = SPME(b, q, alpha=ALPHA, rc=RC, K=K, order=ORDER)
    for _ in range(10):
        sa.step(1)
    sb.step(10)
    xa, xb = a.state(forces=False)["x"], b.state(forces=False)["x"]
    assert np.linalg.norm(periodic_diff(xa, xb, s.box)) <= 1e-11 * np.linalg.norm(xa)
    # parameters changed between calls: the next call must use the new forces
    eps2 = np.full((1, 1), 0.8)
    a.set_params(eps=eps2, sigma=np.ones((1, 1)))
    sa.step(8)
    s2 = dataclasses.replace(s, eps=eps2)
    x1, v1, _, _, _ = oracle_verlet(s, q, 10)
    x_o, v_o, _, _, _ = oracle_verlet(dataclasses.replace(s2, x=x1, v=v1), q, 8)
    st = a.state(forces=False)
    assert np.linalg.norm(periodic_diff(st["x"], x_o, s.box)) <= 1e-9 * np.linalg.norm(x_o)
    assert rel_l2(st["v"], v_o) <= 1e-9
    # another solver (other charges) stepping the same context in between
    sc = SPME(b, -q, alpha=ALPHA, rc=RC, K=K, order=ORDER)
    sc.step(0)
    eb = sb.step(0)
    e_fresh = SPME(b, q, alpha=ALPHA, rc=RC, K=K, order=ORDER).step(0)
    assert eb["coulomb"] == pytest.approx(e_fresh["coulomb"], rel=1e-12)
    for o in (sa, sb, sc):
        o.close()
    a.close()
    b.close()
    # new charges between two calls: the opening half-kick must use the forces
    # of the new charges (the oracle loop switches q at the same point), and the
    # energy of a zero-step call must be that of a fresh solver with them
    c = make(s, "fp64")
    sd = SPME(c, q, alpha=ALPHA, rc=RC, K=K, order=ORDER)
    sd.step(3)
    q2 = np.roll(q, 1) * 0.5
    sd.set_charges(q2)
    e0 = sd.step(0)
    e_new = SPME(c, q2, alpha=ALPHA, rc=RC, K=K, order=ORDER).step(0)
    assert e0["coulomb"] == pytest.approx(e_new["coulomb"], rel=1e-12)
    sd.step(5)
    x3, v3, _, _, _ = oracle_verlet(s, q, 3)
    x_o, v_o, _, _, _ = oracle_verlet(dataclasses.replace(s, x=x3, v=v3), q2, 5)
    st = c.state(forces=False)
    assert np.linalg.norm(periodic_diff(st["x"], x_o, s.box)) <= 1e-9 * np.linalg.norm(x_o)
    assert rel_l2(st["v"], v_o) <= 1e-9
    sd.close()
    c.close()


@pytest.fixture(scope="module")
def reference8():
    s, q = small_charged()
    return s, q, oracle_verlet(s, q, 8)


@pytest.mark.parametrize("lanes", [1, 2, 8])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_step_lanes_per_atom(reference8, precision, lanes):
    """The fused LJ + Coulomb pass on every list layout (1, 2, 8 lanes per atom
    besides the default 4): 8 steps against the oracle loop."""
    s, q, (x_o, v_o, pe_o, ec_o, ke_o) = reference8
    tol = 1e-9 if precision == "fp64" else 1e-5
    sysm = make(s, precision, lanes_per_atom=lanes)
    sp = SPME(sysm, q, alpha=ALPHA, rc=RC, K=K, order=ORDER)
    e = sp.step(8)
    st = sysm.state(forces=False)
    assert np.linalg.norm(periodic_diff(st["x"], x_o, s.box)) <= tol * np.linalg.norm(x_o)
    assert rel_l2(st["v"], v_o) <= tol
    assert abs(e["pe_lj"] - pe_o) <= tol * abs(pe_o)
    assert abs(e["coulomb"] - ec_o) <= tol * abs(ec_o)
    sp.close()
    sysm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_step_half_lists(reference8, precision):
    """The fused LJ + Coulomb pass on half Verlet lists (reactions added to the
    partner): 8 steps against the oracle loop."""
    s, q, (x_o, v_o, pe_o, ec_o, ke_o) = reference8
    tol = 1e-9 if precision == "fp64" else 1e-5
    sysm = make(s, precision, half_list=True)
    sp = SPME(sysm, q, alpha=ALPHA, rc=RC, K=K, order=ORDER)
    e = sp.step(8)
    st = sysm.state(forces=False)
    assert np.linalg.norm(periodic_diff(st["x"], x_o, s.box)) <= tol * np.linalg.norm(x_o)
    assert rel_l2(st["v"], v_o) <= tol
    assert abs(e["pe_lj"] - pe_o) <= tol * abs(pe_o)
    assert abs(e["coulomb"] - ec_o) <= tol * abs(ec_o)
    sp.close()
    sysm.close()
