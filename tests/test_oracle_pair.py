"""Pins of the oracle's Lennard-Jones pair term and force/energy sums against
closed-form facts of the 12-6 potential and against invariants (CPU only).

The paper names the LJ short-range kernel (Section "CabanaMD") without a
formula; these pins fix the textbook 12-6 form independently of the oracle's
own expression: the minimum sits at 2^(1/6) sigma with depth -eps, U(sigma)=0,
F = -dU/dr, the eps/sigma scaling law, and Newton's third law.
"""
import json
import math
import os

import numpy as np
import pytest

import md_inputs as mi

BIG = np.array([30.0, 30.0, 30.0])


def dimer(orc, r, eps=1.0, sig=1.0, shift=False, rc=2.5):
    x = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
    f, ea, pe = orc.lj_forces(x, [0, 0], BIG, eps=[[eps]], sigma=[[sig]], rc=rc, shift=shift,
                              brute=True)
    return f, pe


def test_minimum_location_and_depth(orc):
    for eps, sig in [(1.0, 1.0), (1.1, 0.9), (0.8, 1.2)]:
        rmin = 2.0 ** (1.0 / 6.0) * sig
        f, pe = dimer(orc, rmin, eps, sig)
        assert abs(f[0, 0]) < 1e-12 * eps / sig
        assert pe == pytest.approx(-eps, rel=1e-14)
        # it is a minimum: energy rises on both sides
        assert dimer(orc, rmin * 0.999, eps, sig)[1] > pe
        assert dimer(orc, rmin * 1.001, eps, sig)[1] > pe


def test_zero_at_sigma_and_repulsive_inside(orc):
    for sig in (1.0, 0.9, 1.2):
        f, pe = dimer(orc, sig, 1.0, sig)
        assert abs(pe) < 1e-13   # 4*eps*(s12 - s6) with s6 = 1 up to rounding
        # inside the minimum the force pushes atom 0 away from atom 1 (-x)
        assert f[0, 0] < 0 and f[1, 0] > 0


def test_force_is_minus_energy_gradient(orc):
    h = 1e-6
    for r in np.linspace(0.95, 2.45, 16):
        f, _ = dimer(orc, r)
        ep = dimer(orc, r + h)[1]
        em = dimer(orc, r - h)[1]
        dUdr = (ep - em) / (2 * h)
        # atom 1 sits at +r: F_1x = -dU/dr
        assert f[1, 0] == pytest.approx(-dUdr, rel=1e-6, abs=1e-9)


def test_eps_sigma_scaling_law(orc):
    """U(r; eps, sig) = eps * U(r/sig; 1, 1) with the cutoff scaled by sig."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        eps, sig = rng.uniform(0.5, 2.0, 2)
        r = rng.uniform(0.95, 2.4)
        f1, pe1 = dimer(orc, r, 1.0, 1.0)
        f2, pe2 = dimer(orc, r * sig, eps, sig, rc=2.5 * sig)
        assert pe2 == pytest.approx(eps * pe1, rel=1e-13)
        assert f2[1, 0] == pytest.approx(eps / sig * f1[1, 0], rel=1e-12)


def test_cutoff_strict_and_shift(orc):
    f, pe = dimer(orc, 2.5)                    # r^2 == rc^2 exactly: no interaction
    assert pe == 0.0 and np.all(f == 0.0)
    # the same through the neighbor-list path (the pair is inside rc + skin)
    x = np.array([[10.0, 10.0, 10.0], [12.5, 10.0, 10.0]])
    fl, _, pel = orc.lj_forces(x, [0, 0], BIG)
    assert pel == 0.0 and np.all(fl == 0.0)
    x[1, 0] = 12.5 - 1e-9
    assert orc.lj_forces(x, [0, 0], BIG)[2] < 0
    f, pe = dimer(orc, 2.5 - 1e-9)
    assert pe < 0 and f[1, 0] < 0               # attractive just inside
    _, pes = dimer(orc, 2.5 - 1e-9, shift=True)  # shifted: continuous at rc
    assert abs(pes) < 1e-9
    # shift changes energies only
    f1, pe1 = dimer(orc, 1.3)
    f2, pe2 = dimer(orc, 1.3, shift=True)
    assert np.array_equal(f1, f2) and pe2 > pe1


def test_fcc_lattice_sum_and_zero_forces(orc):
    """Perfect FCC crystal: every force vanishes by symmetry, and PE/N equals
    the coordination-shell sum 1/2 sum_k n_k U(r_k) over shells inside rc."""
    shells = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fcc_shells.json")))["shells"]
    s = mi.lj_melt(6, seed=1)           # 864 atoms, L = 10.08
    a = mi.fcc_lattice_constant(mi.RHO_MELT)
    f, ea, pe = orc.lj_forces(s.x, s.types, s.box)
    assert np.abs(f).max() < 1e-12
    # the pair energy at each shell radius, from a dimer evaluation
    expect = 0.0
    expect_shift = 0.0
    for m, count in shells:
        r = math.sqrt(m) * a
        if r * r < 2.5 ** 2:
            expect += 0.5 * count * dimer(orc, r)[1]
            expect_shift += 0.5 * count * dimer(orc, r, shift=True)[1]
    assert pe / s.n == pytest.approx(expect, rel=1e-13)
    assert np.allclose(ea, expect, rtol=1e-13)
    _, _, pes = orc.lj_forces(s.x, s.types, s.box, shift=True)
    assert pes / s.n == pytest.approx(expect_shift, rel=1e-13)
    assert expect == pytest.approx(-6.773368053252958, rel=1e-12)


def test_newton_third_law_and_list_vs_brute(orc):
    s = mi.lj_melt(5, seed=4, jitter=0.08)
    f, ea, pe = orc.lj_forces(s.x, s.types, s.box)
    fb, eb, peb = orc.lj_forces(s.x, s.types, s.box, brute=True)
    assert np.abs(f.sum(axis=0)).max() <= 1e-12 * np.abs(f).sum()
    assert np.allclose(f, fb, rtol=0, atol=1e-12 * np.abs(f).max())
    assert pe == pytest.approx(peb, rel=1e-13)


def test_total_force_is_minus_gradient_of_pe(orc):
    s = mi.lj_melt(5, seed=5, jitter=0.1)
    f, _, _ = orc.lj_forces(s.x, s.types, s.box, brute=True)
    rng = np.random.default_rng(0)
    h = 1e-6
    checked = 0
    for i in rng.choice(s.n, 12, replace=False):
        # skip atoms with a pair within 10h of the cutoff (the FD would cross it)
        d = s.x - s.x[i]
        d -= s.box * np.round(d / s.box)
        r = np.sqrt((d * d).sum(1))
        if np.any(np.abs(r - 2.5) < 10 * h):
            continue
        for a in range(3):
            xp = s.x.copy(); xp[i, a] += h
            xm = s.x.copy(); xm[i, a] -= h
            # only pairs that contain i depend on x_i, and they sum to 2 e_i
            ep = 2.0 * orc.lj_forces(xp, s.types, s.box, brute=True)[1][i]
            em = 2.0 * orc.lj_forces(xm, s.types, s.box, brute=True)[1][i]
            assert f[i, a] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6, abs=1e-7)
            # and the same through the total energy, at the rounding level of PE
            Ep = orc.lj_forces(xp, s.types, s.box, brute=True)[2]
            Em = orc.lj_forces(xm, s.types, s.box, brute=True)[2]
            assert f[i, a] == pytest.approx(-(Ep - Em) / (2 * h), abs=1e-5)
        checked += 1
    assert checked >= 8


def test_type_relabeling_invariance(orc):
    s = mi.two_type_melt(5, seed=9)
    f, ea, pe = orc.lj_forces(s.x, s.types, s.box, eps=s.eps, sigma=s.sigma)
    perm = [1, 0]
    f2, ea2, pe2 = orc.lj_forces(s.x, 1 - s.types, s.box, eps=s.eps[np.ix_(perm, perm)],
                                 sigma=s.sigma[np.ix_(perm, perm)])
    assert np.array_equal(f, f2) and pe == pe2
