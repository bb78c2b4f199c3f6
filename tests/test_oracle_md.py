"""Pins of the oracle's velocity-Verlet NVE run (CPU only).

The paper's timestep propagates particles with the computed forces and then
re-sorts them (Introduction, anatomy of a timestep).  Pins: a free particle
moves on a straight line exactly; a bound LJ dimer follows the exact ODE
solution with a global error of order dt^2; the scheme is time reversible
through re-sorts and list rebuilds; momentum is conserved; with the shifted
potential the energy fluctuation shrinks ~4x when dt halves.
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

import md_inputs as mi

BOX = np.array([30.0, 30.0, 30.0])


def test_free_particles_move_straight(orc):
    x = np.array([[5.0, 5.0, 5.0], [20.0, 20.0, 20.0]])
    v = np.array([[0.3, -0.2, 0.1], [-0.1, 0.25, 0.05]])
    r = orc.md_run(x, v, [0, 0], BOX, 50, dt=0.01, rebuild_every=7)
    xs, vs = r.by_id(r.x), r.by_id(r.v)
    assert np.array_equal(vs, v)
    assert np.allclose(xs, x + 50 * 0.01 * v, rtol=0, atol=1e-12)


def _dimer_final_r(orc, dt, t_end):
    x = np.array([[10.0, 10.0, 10.0], [11.3, 10.0, 10.0]])
    v = np.array([[0.3, 0.0, 0.0], [-0.3, 0.0, 0.0]])
    nsteps = int(round(t_end / dt))
    r = orc.md_run(x, v, [0, 0], BOX, nsteps, dt=dt, rebuild_every=10)
    xs = r.by_id(r.x)
    return xs[1, 0] - xs[0, 0]


def test_dimer_matches_ode_with_second_order_error(orc):
    t_end = 2.0
    # relative coordinate of two unit masses: r'' = 2 F(r), F = -dU/dr of 12-6 LJ
    def rhs(t, y):
        r, u = y
        return [u, 2.0 * (48.0 * r ** -13 - 24.0 * r ** -7)]
    sol = solve_ivp(rhs, (0, t_end), [1.3, -0.6], method="DOP853", rtol=1e-13, atol=1e-14)
    r_exact = sol.y[0, -1]
    errs = [abs(_dimer_final_r(orc, dt, t_end) - r_exact) for dt in (0.004, 0.002, 0.001)]
    assert errs[0] < 1e-3
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.2 < e1 / e2 < 4.8          # global error ~ dt^2


def test_time_reversibility_through_resorts(orc):
    # Rebuild every 5 steps: atoms then move far less than skin/2 between
    # builds, so no pair within rc is ever missing from a list and both
    # directions see the same forces.  (With rebuild every 20 at T*=1.44 some
    # atoms move more than skin/2 between builds, lists built at different
    # instants miss different pairs, and reversibility only holds to ~1e-4.)
    s = mi.lj_melt(6, seed=12, jitter=0.05)
    f1 = orc.md_run(s.x, s.v, s.types, s.box, 40, rebuild_every=5)
    back = orc.md_run(f1.x, -f1.v, f1.types, s.box, 40, rebuild_every=5, step0=40, ids=f1.ids,
                      img=f1.img)
    x_back = back.by_id(back.x + back.img * s.box)
    v_back = back.by_id(back.v)
    assert np.allclose(x_back, s.x, rtol=0, atol=1e-9)
    assert np.allclose(-v_back, s.v, rtol=0, atol=1e-9)


def test_momentum_conserved_and_ids_permutation(orc):
    s = mi.lj_melt(6, seed=13)
    r = orc.md_run(s.x, s.v, s.types, s.box, 60)
    _, _, p = orc.thermo(r.v, r.types)
    assert np.abs(p).max() < 1e-10
    assert np.array_equal(np.sort(r.ids), np.arange(s.n))


def test_energy_fluctuation_scales_with_dt_squared(orc):
    s = mi.lj_melt(6, seed=14)
    t_end = 0.5
    fl = []
    for dt in (0.004, 0.002):
        r = orc.md_run(s.x, s.v, s.types, s.box, int(round(t_end / dt)), dt=dt,
                       shift=True)
        e = r.thermo[:, 2] / s.n
        fl.append(np.abs(e - e[0]).max())
    assert fl[0] < 5e-3
    assert 2.5 < fl[0] / fl[1] < 6.0


def test_run_records_displacement_and_resets_at_rebuild(orc):
    s = mi.lj_melt(6, seed=15)
    r = orc.md_run(s.x, s.v, s.types, s.box, 25)
    d = r.thermo[:, 3]
    assert d[0] == 0.0 and d[20] == 0.0 and d[19] > 0 and d[25] > 0
