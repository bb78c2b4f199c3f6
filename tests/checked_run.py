"""Workloads run through a checked build of the library (every index check of
the hot path's gathers and scatters compiled in): started by
tests/test_gpu_checked.py in a subprocess whose MD_B300_LIB names that build.
Each call raises if a check failed (the library then reports MD_ERR_CUDA with
the site and index), so reaching the end means no check fired.  Prints one
line per workload and "ok" at the end."""
import numpy as np
import torch

import md_inputs as mi
from paper_2109_09056_b300 import SPME, MDSystem, _native


def single(prec, lanes, types2=False):
    s = mi.lj_melt(6, seed=3, jitter=0.1)
    kw = {}
    if types2:
        rng = np.random.default_rng(41)
        s.types = (np.arange(s.n) % 2).astype(np.int32)
        s.eps, s.sigma = mi.random_pair_params(2, rng)
        s.mass = np.ones(2)
        kw = dict(ntypes=2, eps=s.eps, sigma=s.sigma, mass=s.mass)
    m = MDSystem(s.x, s.v, s.types, s.box, precision=prec, lanes_per_atom=lanes,
                 rebuild_every=4, stream=torch.cuda.Stream(), **kw)
    m.step(13)
    m.neighbors()
    m.permutation()
    st = m.state()
    m.set_state(st["x"], st["v"])
    m.step(5)
    if prec == "fp64":
        m.force_backward(np.ones((s.n, 3)), 0.5)
    return s, m


def main():
    assert "checked" in _native.LIB_PATH_USED, _native.LIB_PATH_USED
    for prec in ("mixed", "fp64"):
        for lanes in (1, 2, 4, 8):
            s, m = single(prec, lanes)
            m.close()
            print("single", prec, lanes, flush=True)
        # two types: the type tables, the adjoint's parameter sums and the
        # fused LJ + Coulomb pass's type gathers of sentinel entries
        s, m = single(prec, 4, types2=True)
        q = mi.neutral_charges(s.n, np.random.default_rng(17))
        sp = SPME(m, q, alpha=1.25, rc=2.5, K=(24, 24, 24), order=4)
        sp.compute()
        sp.step(9)
        sp.close()
        m.close()
        print("spme", prec, flush=True)
        boxes = mi.ensemble(nbox=6, seed=5, n_lo=256, n_hi=2000)
        x = np.concatenate([b.x for b in boxes])
        v = np.concatenate([b.v for b in boxes])
        t = np.concatenate([b.types for b in boxes])
        bm = MDSystem(x, v, t, None, precision=prec, n_per_box=[b.n for b in boxes],
                      boxes=[b.box for b in boxes], rebuild_every=5,
                      stream=torch.cuda.Stream())
        bm.step(12)
        bm.batch_thermo()
        bm.close()
        print("batch", prec, flush=True)
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
