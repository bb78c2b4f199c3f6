"""Pins of the Ewald / SPME oracle (oracle/ewald.py) against what mathematics
fixes independently of its own formulas:

* the B-spline recursion against the exact truncated-power form of the
  cardinal B-spline, evaluated in rational arithmetic;
* partition of unity of the splines and of their derivatives; symmetry;
* the Euler exponential spline moduli |b(m)|^2 for orders 4 and 6 against
  closed forms derived by hand from the spline values at the integers;
* the rock-salt Madelung constant 1.7475645946331822 (total Ewald energy);
* independence of the total energy and forces from the splitting parameter
  (neutral box, and a charged box through the background term);
* forces equal to minus the gradient of the energy (central differences), for
  the direct sum and for SPME;
* SPME converging to the direct Ewald reciprocal sum as the grid and order
  grow; exact invariance of the SPME energy under a shift by one grid spacing;
* the vectorised real-space sum against a plain double loop on a tiny box.
"""
import importlib.util
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import md_inputs as mi

# ORACLE_EWALD: a deliberately broken copy of oracle/ewald.py (the mutation
# test checks that these pins catch each planted mistake)
if os.environ.get("ORACLE_EWALD"):
    _spec = importlib.util.spec_from_file_location("ewald_mutant", os.environ["ORACLE_EWALD"])
    ew = importlib.util.module_from_spec(_spec)
    _spec.loader.exec_module(ew)
else:
    from oracle import ewald as ew

MADELUNG_NACL = 1.7475645946331822


def exact_bspline(n, x: Fraction) -> Fraction:
    """M_n(x) = 1/(n-1)! sum_{k=0}^{n} (-1)^k C(n,k) max(x-k, 0)^(n-1)."""
    s = Fraction(0)
    for k in range(n + 1):
        if x > k:
            s += (-1) ** k * math.comb(n, k) * (x - k) ** (n - 1)
    return s / math.factorial(n - 1)


@pytest.mark.parametrize("n", [3, 4, 6, 8])
def test_bspline_recursion_matches_exact_form(n):
    xs = [Fraction(j, 8) for j in range(-4, 8 * n + 5)]
    got = ew.bspline(n, np.array([float(x) for x in xs]))
    want = np.array([float(exact_bspline(n, x)) for x in xs])
    assert np.max(np.abs(got - want)) <= 2e-16 * n


@pytest.mark.parametrize("n", [4, 6, 8])
def test_bspline_partition_symmetry_derivative(n):
    t = np.random.default_rng(n).uniform(0.0, 1.0, 64)
    a = np.arange(n)
    W = ew.bspline(n, t[:, None] + a)
    D = ew.bspline_deriv(n, t[:, None] + a)
    assert np.allclose(W.sum(axis=1), 1.0, rtol=0, atol=1e-15)
    assert np.allclose(D.sum(axis=1), 0.0, rtol=0, atol=1e-14)
    x = t * n
    assert np.allclose(ew.bspline(n, x), ew.bspline(n, n - x), rtol=0, atol=1e-15)
    h = 1e-6
    fd = (ew.bspline(n, x + h) - ew.bspline(n, x - h)) / (2 * h)
    assert np.allclose(ew.bspline_deriv(n, x), fd, rtol=0, atol=1e-8)
    assert np.all(ew.bspline(n, np.array([-0.5, 0.0, float(n), n + 0.5])) == 0.0)


def test_bspline_order4_at_integers():
    assert np.allclose(ew.bspline(4, np.array([1.0, 2.0, 3.0])), [1 / 6, 2 / 3, 1 / 6],
                       rtol=0, atol=1e-16)


@pytest.mark.parametrize("K", [16, 25, 40])
def test_moduli_closed_forms(K):
    w = 2 * np.pi * np.arange(K) / K
    # n = 4: sum_k M_4(k+1) e^{iwk} = e^{iw} (2/3 + cos(w)/3)
    assert np.allclose(ew.bspline_moduli(4, K), 9.0 / (2.0 + np.cos(w)) ** 2, rtol=1e-14)
    # n = 6: M_6(1..5) = (1, 26, 66, 26, 1)/120, so the sum is
    # e^{2iw} (66 + 52 cos w + 2 cos 2w) / 120
    want6 = (120.0 / (66.0 + 52.0 * np.cos(w) + 2.0 * np.cos(2 * w))) ** 2
    assert np.allclose(ew.bspline_moduli(6, K), want6, rtol=1e-13)
    for n in (4, 6, 8):
        assert abs(ew.bspline_moduli(n, K)[0] - 1.0) <= 1e-15


def test_moduli_odd_order_even_grid_rejected():
    with pytest.raises(ValueError):
        ew.bspline_moduli(3, 16)


def test_madelung_rocksalt():
    x, q, box = mi.rocksalt(6)                  # 216 ions, nearest-neighbor distance 1
    E, F = ew.ewald_total(x, q, box, alpha=1.7, rc=2.95, kmax=20)
    assert abs(E / (len(q) / 2) + MADELUNG_NACL) <= 1e-10
    assert np.abs(F).max() <= 1e-12              # every ion is a centre of symmetry


def _random_box(n, seed, charged=False):
    rng = np.random.default_rng(seed)
    L = np.array([10.0, 11.0, 9.5])
    x = rng.uniform(0.0, 1.0, (n, 3)) * L
    q = mi.neutral_charges(n, rng)
    if charged:
        q = q + 0.3
    return x, q, L


@pytest.mark.parametrize("charged", [False, True])
def test_total_independent_of_alpha(charged):
    x, q, L = _random_box(120, 5, charged)
    E1, F1 = ew.ewald_total(x, q, L, 1.15, 4.7, kmax=24)
    E2, F2 = ew.ewald_total(x, q, L, 1.35, 4.7, kmax=28)
    assert abs(E1 - E2) <= 1e-10 * abs(E1)
    assert np.linalg.norm(F1 - F2) <= 1e-9 * np.linalg.norm(F1)
    if charged:
        # without the background term the totals differ: the pin sees it
        assert abs(ew.ewald_background(q, L, 1.15) - ew.ewald_background(q, L, 1.35)) > 1e-3


def _fd_check(energy, x, F, coords, h=1e-5, tol=1e-7):
    scale = np.abs(F).max()
    for i, d in coords:
        xp = x.copy(); xp[i, d] += h
        xm = x.copy(); xm[i, d] -= h
        g = (energy(xp) - energy(xm)) / (2 * h)
        assert abs(-g - F[i, d]) <= tol * scale, (i, d, -g, F[i, d])


def test_direct_forces_are_minus_gradient():
    x, q, L = _random_box(40, 9)
    E, F = ew.ewald_total(x, q, L, 1.2, 4.7, kmax=20)
    coords = [(i, d) for i in (0, 7, 19, 33) for d in range(3)]
    _fd_check(lambda y: ew.ewald_total(y, q, L, 1.2, 4.7, kmax=20)[0], x, F, coords)


@pytest.mark.parametrize("n", [4, 6])
def test_spme_forces_are_minus_gradient(n):
    x, q, L = _random_box(60, 11)
    K = (20, 24, 18)
    E, F = ew.spme_reciprocal(x, q, L, 1.1, K, n)
    coords = [(i, d) for i in (1, 12, 40) for d in range(3)]
    _fd_check(lambda y: ew.spme_reciprocal(y, q, L, 1.1, K, n)[0], x, F, coords, tol=1e-7)


def test_spme_converges_to_direct_sum():
    x, q, L = _random_box(120, 1)
    Ed, Fd = ew.ewald_reciprocal(x, q, L, 1.1, 24)
    errs = []
    for K, n in ((16, 4), (32, 4), (32, 6), (32, 8), (64, 8)):
        Es, Fs = ew.spme_reciprocal(x, q, L, 1.1, (K, K + 2, K - 2), n)
        errs.append((abs(Es - Ed) / abs(Ed), np.linalg.norm(Fs - Fd) / np.linalg.norm(Fd)))
    for k in range(len(errs) - 1):
        assert errs[k + 1][0] < errs[k][0] and errs[k + 1][1] < errs[k][1]
    assert errs[-1][0] <= 1e-8 and errs[-1][1] <= 1e-7
    assert errs[0][1] >= 1e-3                       # the coarse grid is visibly worse


def test_spme_invariant_under_one_grid_shift():
    x, q, L = _random_box(50, 3)
    K = (20, 24, 18)
    E0, F0 = ew.spme_reciprocal(x, q, L, 1.1, K, 6)
    shift = np.array([L[0] / K[0], 0.0, 2 * L[2] / K[2]])
    E1, F1 = ew.spme_reciprocal(x + shift, q, L, 1.1, K, 6)
    assert abs(E1 - E0) <= 1e-13 * abs(E0)
    assert np.linalg.norm(F1 - F0) <= 1e-12 * np.linalg.norm(F0)
    # a shift by a non-grid amount changes the SPME energy (it is not exact)
    E2, _ = ew.spme_reciprocal(x + 0.37 * shift, q, L, 1.1, K, 6)
    assert abs(E2 - E0) > 1e-9 * abs(E0)


def test_real_space_against_double_loop():
    rng = np.random.default_rng(4)
    L = np.array([6.0, 6.5, 7.0])
    x = rng.uniform(-3.0, 9.0, (30, 3))            # some atoms outside the box
    q = rng.normal(size=30)
    alpha, rc = 0.9, 2.9
    E, F = ew.ewald_real(x, q, L, alpha, rc)
    Ee, Fe = 0.0, np.zeros((30, 3))
    for i in range(30):
        for j in range(i + 1, 30):
            d = [0.0, 0.0, 0.0]
            for a in range(3):
                di = (x[j, a] % L[a]) - (x[i, a] % L[a])
                d[a] = di - L[a] * round(di / L[a])
            r = math.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
            if r < rc:
                Ee += q[i] * q[j] * math.erfc(alpha * r) / r
                g = q[i] * q[j] * (math.erfc(alpha * r) / r
                                   + 2 * alpha / math.sqrt(math.pi) * math.exp(-(alpha * r) ** 2)) / r ** 2
                for a in range(3):
                    Fe[i, a] -= g * d[a]
                    Fe[j, a] += g * d[a]
    assert abs(E - Ee) <= 1e-13 * abs(Ee)
    assert np.allclose(F, Fe, rtol=0, atol=1e-13 * np.abs(Fe).max())
    assert np.allclose(ew.ewald_real_sample(x, q, L, alpha, rc, [3, 17]), F[[3, 17]],
                       rtol=0, atol=1e-14 * np.abs(Fe).max())


def test_self_energy_of_point_charges():
    # E_self is the alpha-dependent interaction of each charge with its own
    # screening Gaussian: -alpha/sqrt(pi) q^2; E_bg vanishes for a neutral box
    assert ew.ewald_self([2.0, -1.0], 0.5) == pytest.approx(-0.5 / math.sqrt(math.pi) * 5.0, rel=1e-15)
    assert ew.ewald_background([1.0, -1.0], [3.0, 3.0, 3.0], 1.0) == 0.0
