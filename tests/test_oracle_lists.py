"""Pins of the oracle's wrap, cell binning, stable cell-order sort and Verlet
neighbor list (CPU only).

Sorting by geometric binning is the paper's "Particle Sorting" step and the
Verlet list built by binning is its "Neighbor List Creation" step; the pins
are: wrap/bin invariants, equality with a library stable sort, equality of the
cell-list search with an O(n^2) brute force (including boxes with only 2 or 3
cells per axis, where the 27-cell stencil folds onto itself), list symmetry,
and the exact FCC coordination counts (78 within 2.8, 54 within 2.5).
"""
import json
import os

import numpy as np
import pytest

import md_inputs as mi


def test_cell_grid_of_named_workloads(orc):
    rs = 2.8
    for ncell, nc in [(10, 5), (32, 19), (100, 59), (20, 11)]:
        L = ncell * mi.fcc_lattice_constant(mi.RHO_MELT)
        assert list(orc.cell_grid([L, L, L], rs)) == [nc] * 3
    with pytest.raises(ValueError):
        orc.cell_grid([5.6, 10.0, 10.0], rs)         # L == 2 rs is rejected
    assert list(orc.cell_grid([5.6000001, 10.0, 10.0], rs)) == [2, 3, 3]


def test_wrap_properties(orc):
    L = np.array([7.15, 10.08, 16.79596191382507])
    rng = np.random.default_rng(1)
    x = rng.uniform(-3, 4, size=(5000, 3)) * L
    x[:10] = rng.uniform(0, 1, size=(10, 3)) * L       # already inside: unchanged
    x[10] = L                                          # exactly L -> 0
    x[11] = -1e-300                                    # tiny negative
    x[12] = L * (1 - 2.0 ** -53)                        # just below L
    x[13] = L * 1.5                                    # in [L, 2L): x - L is exact
    w, img = orc.wrap(x, L)
    assert np.all(w >= 0) and np.all(w < L)
    assert np.array_equal(w[:10], x[:10])
    assert np.all(w[10] == 0.0)
    assert np.array_equal(w[13], x[13] - L)
    back = w + img * L
    assert np.allclose(back, x, rtol=0, atol=4e-16 * np.abs(x).max() * 4)


def test_cell_index_contains_atom(orc):
    L = np.array([16.79596191382507] * 3)
    nc = orc.cell_grid(L, 2.8)
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, size=(20000, 3)) * L
    cell = orc.cell_index(x, L, nc)
    h = L / nc
    c = np.stack([cell % nc[0], (cell // nc[0]) % nc[1], cell // (nc[0] * nc[1])], axis=1)
    assert np.all(c >= 0) and np.all(c < nc)
    assert np.all(x >= c * h - 1e-12) and np.all(x <= (c + 1) * h + 1e-12)


def test_cell_linear_order(orc):
    """c = (cz * nc_y + cy) * nc_x + cx, x fastest, on a box with distinct nc per axis."""
    L = np.array([12.0, 15.0, 18.0])
    nc = orc.cell_grid(L, 2.8)
    assert list(nc) == [4, 5, 6]
    h = L / nc
    rng = np.random.default_rng(4)
    for _ in range(50):
        c = rng.integers(0, nc)
        x = (c + rng.uniform(0.1, 0.9, 3)) * h
        cell = orc.cell_index(x[None, :], L, nc)[0]
        assert cell == (c[2] * nc[1] + c[1]) * nc[0] + c[0]


def test_stable_sort_equals_library_sort(orc):
    rng = np.random.default_rng(3)
    for ncell, n in [(5, 1000), (125, 4000), (6859, 50000), (1, 7)]:
        cell = rng.integers(0, ncell, n).astype(np.int32)
        perm = orc.stable_sort_by_cell(cell, ncell)
        assert np.array_equal(perm, np.argsort(cell, kind="stable"))
        assert perm.tolist() == sorted(range(n), key=lambda i: cell[i])
    assert orc.stable_sort_by_cell(np.zeros(0, np.int32), 4).size == 0


def test_bin_sort_orders_by_cell_then_prior_index(orc):
    s = mi.lj_melt(8, seed=6, jitter=0.3)
    x = s.x.copy()
    x[::7] += s.box * 1.3                              # some atoms outside the box
    perm, xs, cells = orc.bin_sort(x, s.box, 2.8)
    assert np.array_equal(np.sort(perm), np.arange(s.n))
    assert np.all(np.diff(cells) >= 0)
    same = np.diff(cells) == 0
    assert np.all(np.diff(perm)[same] > 0)


def _sets(orc, x, L, rs, brute):
    nn, nbr = orc.neighbors(x, L, rs, brute=brute)
    return nn, orc.neighbor_sets(nn, nbr)


@pytest.mark.parametrize("case", ["nc2", "nc3", "nc5_jitter", "gas", "nc2x3x4"])
def test_cell_list_equals_brute_force(orc, case):
    rng = np.random.default_rng(11)
    if case == "nc2":                    # 256 atoms at rho 0.7: L = 7.15, 2 cells per axis
        n = 256
        L = np.full(3, (n / 0.7) ** (1 / 3))
        x = rng.uniform(0, 1, size=(n, 3)) * L
    elif case == "nc3":                  # 6^3 FCC: 864 atoms, L = 10.08, 3 cells per axis
        s = mi.lj_melt(6, seed=2, jitter=0.2)
        x, L = s.x, s.box
    elif case == "nc5_jitter":
        s = mi.lj_melt(10, seed=3, jitter=0.05)
        x, L = s.x, s.box
    elif case == "gas":
        n = 3000
        L = np.full(3, 15.0)
        x = rng.uniform(-1, 2, size=(n, 3)) * L         # unwrapped coordinates too
        x = orc.wrap(x, L)[0]
    else:
        n = 1500
        L = np.array([5.7, 9.0, 12.0])
        x = rng.uniform(0, 1, size=(n, 3)) * L
    nn_c, sets_c = _sets(orc, x, L, 2.8, brute=False)
    nn_b, sets_b = _sets(orc, x, L, 2.8, brute=True)
    assert np.array_equal(nn_c, nn_b)
    assert sets_c == sets_b
    # full list: symmetric, no self
    for i, si in enumerate(sets_c):
        assert i not in si
        for j in si:
            assert i in sets_c[j]


def test_fcc_coordination_counts(orc):
    shells = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fcc_shells.json")))["shells"]
    a = mi.fcc_lattice_constant(mi.RHO_MELT)
    expect_rs = sum(c for m, c in shells if m * a * a < 2.8 ** 2)
    expect_rc = sum(c for m, c in shells if m * a * a < 2.5 ** 2)
    assert (expect_rs, expect_rc) == (78, 54)
    s = mi.lj_melt(10, seed=1)
    nn, nbr = orc.neighbors(s.x, s.box, 2.8)
    assert np.all(nn == 78)
    nn, nbr = orc.neighbors(s.x, s.box, 2.5)
    assert np.all(nn == 54)


def test_sampled_rows_and_forces_equal_full_versions(orc):
    s = mi.lj_melt(6, seed=16, jitter=0.1)
    xw, _ = orc.wrap(s.x, s.box)
    idx = np.array([0, 5, 17, 300, 863])
    nn, nbr = orc.neighbors(xw, s.box, 2.8)
    full = orc.neighbor_sets(nn, nbr)
    assert orc.neighbors_sample(xw, s.box, 2.8, idx) == [full[i] for i in idx]
    f, ea, _ = orc.lj_forces(xw, s.types, s.box, brute=True)
    fs, es = orc.lj_forces_sample(xw, s.types, s.box, idx)
    assert np.array_equal(fs, f[idx]) and np.array_equal(es, ea[idx])
