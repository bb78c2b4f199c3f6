"""FP64 CPU oracle for the short-range Lennard-Jones MD timestep.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; the product package never imports
it.  It wraps ``oracle_md.c`` (plain C, FP64, no FMA contraction) through
ctypes.  It shares no code with the CUDA library.

Each wrapper takes and returns numpy arrays: positions, velocities and forces
as (n, 3) float64 (AoS), types as (n,) int32.  See ``oracle_md.c`` for the
definition each function follows and the paper passage it cites.

Parity status: every function is pinned by closed forms, invariants, brute
force or finite differences (tests/test_oracle_*.py); none is pinned to a
number printed in the paper, which prints none for this path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_md.c")
_LIB = os.path.join(_HERE, "liboracle_md.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_BOX = 1
ERR_ALLOC = 2
ERR_ARG = 3


def build(force: bool = False) -> str:
    """Compile oracle_md.c into liboracle_md.so next to it (gcc, -O2,
    -ffp-contract=off, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-std=c11",
               "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB: an alternative build of oracle_md.c (the mutation
            # test loads deliberately broken copies to check the pins catch them)
            alt = os.environ.get("ORACLE_LIB")
            if not alt:
                build()
            lib = C.CDLL(alt or _LIB)
            P = C.c_void_p
            i64, i32, dbl = C.c_int64, C.c_int32, C.c_double
            sig = {
                "oracle_num_threads": ([], C.c_int),
                "oracle_set_num_threads": ([C.c_int], None),
                "oracle_cell_grid": ([P, dbl, P], C.c_int),
                "oracle_wrap": ([i64, P, P, P], None),
                "oracle_cell_index": ([i64, P, P, P, P], None),
                "oracle_stable_sort_by_cell": ([i64, P, i64, P], C.c_int),
                "oracle_neighbors_cells": ([i64, P, P, P, dbl, i32, P, P], C.c_int),
                "oracle_neighbors_brute": ([i64, P, P, dbl, i32, P, P], C.c_int),
                "oracle_lj_forces": ([i64, P, P, P, i32, P, P, dbl, C.c_int, P, P, i32, P, P, P], None),
                "oracle_lj_forces_brute": ([i64, P, P, P, i32, P, P, dbl, C.c_int, P, P, P], None),
                "oracle_thermo": ([i64, P, P, P, P], None),
                "oracle_md_run": ([i64, P, P, P, P, P, P, P, i32, P, P, P, dbl, dbl, dbl, i32,
                                   C.c_int, i64, i32, i32, P], C.c_int),
                "oracle_lj_adjoint": ([i64, P, P, P, i32, P, P, dbl, C.c_int, P, P, i32, P, dbl,
                                       P, P, P], None),
                "oracle_lj_forces_sample": ([i64, P, P, P, i32, P, P, dbl, C.c_int, i64, P, P, P],
                                            None),
                "oracle_neighbors_sample": ([i64, P, P, dbl, i64, P, i32, P, P], C.c_int),
            }
            for name, (args, res) in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(t: int) -> None:
    _load().oracle_set_num_threads(int(t))


def cell_grid(box, rs: float) -> np.ndarray:
    """nc[d] = floor(L[d]/rs); raises ValueError when some L[d] <= 2 rs."""
    L = _f64(box, (3,))
    nc = np.zeros(3, dtype=np.int32)
    if _load().oracle_cell_grid(_p(L), float(rs), _p(nc)) != OK:
        raise ValueError("box edge must exceed 2*(rc+skin)")
    return nc


def wrap(x, box, img=None):
    """Wrapped copy of x (n,3) and the updated image counts (n,3) int32."""
    x = _f64(x).copy()
    n = x.shape[0]
    im = np.zeros((n, 3), dtype=np.int32) if img is None else _i32(img).copy()
    _load().oracle_wrap(n, _p(x), _p(im), _p(_f64(box, (3,))))
    return x, im


def cell_index(x, box, nc) -> np.ndarray:
    x = _f64(x)
    cell = np.zeros(x.shape[0], dtype=np.int32)
    _load().oracle_cell_index(x.shape[0], _p(x), _p(_f64(box, (3,))), _p(_i32(nc)), _p(cell))
    return cell


def stable_sort_by_cell(cell, ncell: int) -> np.ndarray:
    cell = _i32(cell)
    perm = np.zeros(cell.shape[0], dtype=np.int32)
    rc = _load().oracle_stable_sort_by_cell(cell.shape[0], _p(cell), int(ncell), _p(perm))
    if rc != OK:
        raise MemoryError("oracle sort failed")
    return perm


def bin_sort(x, box, rs: float):
    """The resort step on a state given in its current order: wrap, bin and
    stably sort by cell.  Returns (perm[new]=old, wrapped x in new order,
    cell id of each atom in new order)."""
    L = _f64(box, (3,))
    nc = cell_grid(L, rs)
    xw, _ = wrap(x, L)
    cell = cell_index(xw, L, nc)
    perm = stable_sort_by_cell(cell, int(np.prod(nc.astype(np.int64))))
    return perm, xw[perm], cell[perm]


def neighbors(x, box, rs: float, maxnb: int = 256, brute: bool = False):
    """Full neighbor list (pairs with canonical r^2 < rs^2).  Returns
    (nn (n,), rows (n, maxnb) int32 with row i valid up to nn[i])."""
    x = _f64(x)
    n = x.shape[0]
    L = _f64(box, (3,))
    while True:
        nn = np.zeros(n, dtype=np.int32)
        nbr = np.full((n, maxnb), -1, dtype=np.int32)
        if brute:
            rc = _load().oracle_neighbors_brute(n, _p(x), _p(L), float(rs), int(maxnb), _p(nn), _p(nbr))
        else:
            nc = cell_grid(L, rs)
            rc = _load().oracle_neighbors_cells(n, _p(x), _p(L), _p(nc), float(rs), int(maxnb),
                                                _p(nn), _p(nbr))
        if rc < 0:
            maxnb = -rc
            continue
        if rc != OK:
            raise RuntimeError(f"oracle neighbor build failed ({rc})")
        return nn, nbr


def neighbor_sets(nn, nbr):
    """List of frozensets, one per row."""
    return [frozenset(nbr[i, : nn[i]].tolist()) for i in range(len(nn))]


def _params(ntypes, eps, sigma):
    eps = _f64(eps).reshape(ntypes * ntypes)
    sigma = _f64(sigma).reshape(ntypes * ntypes)
    return eps, sigma


def lj_forces(x, types, box, eps=((1.0,),), sigma=((1.0,),), rc: float = 2.5, shift: bool = False,
              skin: float = 0.3, nn=None, nbr=None, brute: bool = False):
    """Forces (n,3), per-atom energies (n,), total PE (float).  Uses the
    given full list (nn, nbr) if provided, else builds one with rs = rc+skin,
    or sums over all pairs when brute=True."""
    x = _f64(x)
    n = x.shape[0]
    L = _f64(box, (3,))
    types = _i32(types)
    eps_a = np.atleast_2d(np.asarray(eps, dtype=np.float64))
    nt = eps_a.shape[0]
    e, s = _params(nt, eps_a, sigma)
    f = np.zeros((n, 3))
    ea = np.zeros(n)
    pe = C.c_double(0.0)
    if brute:
        _load().oracle_lj_forces_brute(n, _p(x), _p(types), _p(L), nt, _p(e), _p(s), float(rc),
                                       int(shift), _p(f), _p(ea), C.byref(pe))
    else:
        if nn is None:
            nn, nbr = neighbors(x, L, rc + skin)
        nn = _i32(nn)
        nbr = _i32(nbr)
        _load().oracle_lj_forces(n, _p(x), _p(types), _p(L), nt, _p(e), _p(s), float(rc), int(shift),
                                 _p(nn), _p(nbr), nbr.shape[1], _p(f), _p(ea), C.byref(pe))
    return f, ea, float(pe.value)


def thermo(v, types, mass=(1.0,)):
    """(KE, T, P[3]) with T = 2KE/(3n-3)."""
    v = _f64(v)
    out = np.zeros(5)
    _load().oracle_thermo(v.shape[0], _p(v), _p(_i32(types)), _p(_f64(mass)), _p(out))
    return out[0], out[1], out[2:5].copy()


class RunResult:
    """State after an oracle NVE run, in the oracle's internal (cell) order."""

    def __init__(self, x, v, f, types, ids, img, thermo):
        self.x, self.v, self.f, self.types, self.ids, self.img = x, v, f, types, ids, img
        self.thermo = thermo          # (nsteps+1, 4): PE, KE, Etot, max displacement

    def by_id(self, a):
        out = np.empty_like(a)
        out[self.ids] = a
        return out


def md_run(x, v, types, box, nsteps: int, eps=((1.0,),), sigma=((1.0,),), mass=(1.0,),
           rc: float = 2.5, skin: float = 0.3, dt: float = 0.005, rebuild_every: int = 20,
           shift: bool = False, step0: int = 0, ids=None, img=None, maxnb: int = 160) -> RunResult:
    """Velocity-Verlet NVE run of ``nsteps`` steps from (x, v) at counter step0."""
    x = _f64(x).copy()
    v = _f64(v).copy()
    n = x.shape[0]
    types = _i32(types).copy()
    ids = np.arange(n, dtype=np.int32) if ids is None else _i32(ids).copy()
    img = np.zeros((n, 3), dtype=np.int32) if img is None else _i32(img).copy()
    f = np.zeros((n, 3))
    L = _f64(box, (3,))
    eps_a = np.atleast_2d(np.asarray(eps, dtype=np.float64))
    nt = eps_a.shape[0]
    e, s = _params(nt, eps_a, sigma)
    mass = _f64(mass)
    th = np.zeros((nsteps + 1, 4))
    while True:
        xx, vv, tt, ii, mm = x.copy(), v.copy(), types.copy(), ids.copy(), img.copy()
        rc_ = _load().oracle_md_run(n, _p(xx), _p(vv), _p(f), _p(tt), _p(ii), _p(mm), _p(L), nt,
                                    _p(e), _p(s), _p(mass), float(rc), float(skin), float(dt),
                                    int(rebuild_every), int(shift), int(step0), int(nsteps),
                                    int(maxnb), _p(th))
        if rc_ < 0:
            maxnb = -rc_ + 16
            continue
        if rc_ != OK:
            raise RuntimeError(f"oracle md_run failed ({rc_})")
        return RunResult(xx, vv, f, tt, ii, mm, th)


def lj_adjoint(x, types, box, G, gE: float, eps=((1.0,),), sigma=((1.0,),), rc: float = 2.5,
               shift: bool = False, skin: float = 0.3, brute: bool = False):
    """(dL/dx (n,3), dL/deps (nt,nt), dL/dsigma (nt,nt)) for upstream
    gradients G = dL/dF (n,3) and gE = dL/dE."""
    x = _f64(x)
    n = x.shape[0]
    L = _f64(box, (3,))
    types = _i32(types)
    eps_a = np.atleast_2d(np.asarray(eps, dtype=np.float64))
    nt = eps_a.shape[0]
    e, s = _params(nt, eps_a, sigma)
    G = _f64(G, (n, 3))
    dx = np.zeros((n, 3))
    de = np.zeros(nt * nt)
    ds = np.zeros(nt * nt)
    if brute:
        _load().oracle_lj_adjoint(n, _p(x), _p(types), _p(L), nt, _p(e), _p(s), float(rc), int(shift),
                                  None, None, 0, _p(G), float(gE), _p(dx), _p(de), _p(ds))
    else:
        nn, nbr = neighbors(x, L, rc + skin)
        _load().oracle_lj_adjoint(n, _p(x), _p(types), _p(L), nt, _p(e), _p(s), float(rc), int(shift),
                                  _p(nn), _p(nbr), nbr.shape[1], _p(G), float(gE), _p(dx), _p(de),
                                  _p(ds))
    return dx, de.reshape(nt, nt), ds.reshape(nt, nt)


def lj_forces_sample(x, types, box, idx, eps=((1.0,),), sigma=((1.0,),), rc: float = 2.5,
                     shift: bool = False):
    """Forces (m,3) and per-atom energies (m,) of atoms idx, by brute force
    over all atoms (for systems too large to list in full)."""
    x = _f64(x)
    L = _f64(box, (3,))
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    eps_a = np.atleast_2d(np.asarray(eps, dtype=np.float64))
    nt = eps_a.shape[0]
    e, s = _params(nt, eps_a, sigma)
    f = np.zeros((idx.size, 3))
    ea = np.zeros(idx.size)
    _load().oracle_lj_forces_sample(x.shape[0], _p(x), _p(_i32(types)), _p(L), nt, _p(e), _p(s),
                                    float(rc), int(shift), idx.size, _p(idx), _p(f), _p(ea))
    return f, ea


def neighbors_sample(x, box, rs: float, idx, maxnb: int = 256):
    """Neighbor rows (canonical r^2 < rs^2) of atoms idx by brute force:
    list of frozensets of atom indices."""
    x = _f64(x)
    L = _f64(box, (3,))
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    while True:
        nn = np.zeros(idx.size, dtype=np.int32)
        nbr = np.zeros((idx.size, maxnb), dtype=np.int32)
        rc_ = _load().oracle_neighbors_sample(x.shape[0], _p(x), _p(L), float(rs), idx.size,
                                              _p(idx), int(maxnb), _p(nn), _p(nbr))
        if rc_ < 0:
            maxnb = -rc_
            continue
        return [frozenset(nbr[s, : nn[s]].tolist()) for s in range(idx.size)]
