"""Pins of the oracle's force-matching adjoint (CPU only).

Loss L = sum_i |F_i - F_target,i|^2 + c * PE with targets from the same
configuration at pair parameters shifted by +5%.  The analytic gradient with
respect to every (eps, sigma) of the symmetric two-type table and to sampled
coordinates must agree with central finite differences (h = 1e-6) to 1e-6
relative; dL/dx with G = 0, gE = 1 must equal -F.
"""
import numpy as np
import pytest

import md_inputs as mi

H = 1e-6


@pytest.fixture(scope="module")
def fm(orc):
    s = mi.two_type_melt(5, seed=21)        # 500 atoms, L = 8.4
    ft, _, _ = orc.lj_forces(s.x, s.types, s.box, eps=1.05 * s.eps, sigma=1.05 * s.sigma)
    return s, ft


def loss(orc, s, ft, x, eps, sig, c, shift):
    f, _, pe = orc.lj_forces(x, s.types, s.box, eps=eps, sigma=sig, shift=shift)
    return float(((f - ft) ** 2).sum() + c * pe)


@pytest.mark.parametrize("shift", [False, True])
def test_param_gradient_matches_finite_differences(orc, fm, shift):
    s, ft = fm
    c = 0.37
    f, _, _ = orc.lj_forces(s.x, s.types, s.box, eps=s.eps, sigma=s.sigma, shift=shift)
    G = 2.0 * (f - ft)
    _, de, ds = orc.lj_adjoint(s.x, s.types, s.box, G, c, eps=s.eps, sigma=s.sigma, shift=shift)
    assert np.allclose(de, de.T) and np.allclose(ds, ds.T)
    for table, grad in (("eps", de), ("sig", ds)):
        for a, b in [(0, 0), (0, 1), (1, 1)]:
            vals = []
            for sgn in (+1, -1):
                e, sg = s.eps.copy(), s.sigma.copy()
                t = e if table == "eps" else sg
                t[a, b] += sgn * H
                if a != b:
                    t[b, a] += sgn * H
                vals.append(loss(orc, s, ft, s.x, e, sg, c, shift))
            fd = (vals[0] - vals[1]) / (2 * H)
            assert grad[a, b] == pytest.approx(fd, rel=1e-6), (table, a, b)


def test_position_gradient_matches_finite_differences(orc, fm):
    s, ft = fm
    c = 0.37
    f, _, _ = orc.lj_forces(s.x, s.types, s.box, eps=s.eps, sigma=s.sigma)
    G = 2.0 * (f - ft)
    dx, _, _ = orc.lj_adjoint(s.x, s.types, s.box, G, c, eps=s.eps, sigma=s.sigma)
    rng = np.random.default_rng(5)
    checked = 0
    for flat in rng.choice(s.n * 3, 96, replace=False):
        i, a = divmod(int(flat), 3)
        d = s.x - s.x[i]
        d -= s.box * np.round(d / s.box)
        r = np.sqrt((d * d).sum(1))
        if np.any(np.abs(r[np.arange(s.n) != i] - 2.5) < 10 * H):
            continue                       # a pair within 10h of rc: FD would cross it
        xp = s.x.copy(); xp[i, a] += H
        xm = s.x.copy(); xm[i, a] -= H
        fd = (loss(orc, s, ft, xp, s.eps, s.sigma, c, False)
              - loss(orc, s, ft, xm, s.eps, s.sigma, c, False)) / (2 * H)
        assert dx[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(dx).mean())
        checked += 1
        if checked == 64:
            break
    assert checked == 64


def test_energy_gradient_is_minus_force_and_brute_equals_list(orc, fm):
    s, _ = fm
    f, _, _ = orc.lj_forces(s.x, s.types, s.box, eps=s.eps, sigma=s.sigma)
    dx, de, ds = orc.lj_adjoint(s.x, s.types, s.box, np.zeros_like(f), 1.0, eps=s.eps,
                                sigma=s.sigma)
    assert np.allclose(dx, -f, rtol=1e-13, atol=1e-13 * np.abs(f).max())
    G = np.random.default_rng(1).standard_normal(f.shape)
    a = orc.lj_adjoint(s.x, s.types, s.box, G, 0.5, eps=s.eps, sigma=s.sigma)
    b = orc.lj_adjoint(s.x, s.types, s.box, G, 0.5, eps=s.eps, sigma=s.sigma, brute=True)
    for u, w in zip(a, b):
        assert np.allclose(u, w, rtol=1e-12, atol=1e-12 * np.abs(u).max())
