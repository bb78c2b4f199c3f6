"""Helpers shared by the GPU parity tests (imported only when a GPU test runs)."""
import numpy as np
import torch

import oracle
from paper_2109_09056_b300 import MDSystem

RS = 2.8


def stream():
    return torch.cuda.Stream()


def make(sysd, precision="mixed", **kw):
    """MDSystem from an md_inputs.LJSystem."""
    kw.setdefault("stream", torch.cuda.Stream())
    return MDSystem(sysd.x, sysd.v, sysd.types, sysd.box, ntypes=sysd.ntypes, eps=sysd.eps,
                    sigma=sysd.sigma, mass=sysd.mass, rc=sysd.rc, skin=sysd.skin, dt=sysd.dt,
                    rebuild_every=sysd.rebuild_every, precision=precision, **kw)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_sets_by_original_id(sysm):
    """Neighbor sets keyed by original atom id, from the GPU list."""
    st = sysm.state(forces=False)
    ids = st["ids"]
    nn, rows = sysm.neighbors()
    out = {}
    for k in range(len(nn)):
        out[int(ids[k])] = frozenset(ids[rows[k, : nn[k]]].tolist())
    return out


def oracle_sets_by_original_id(x_orig, box):
    xw, _ = oracle.wrap(x_orig, box)
    nn, nbr = oracle.neighbors(xw, box, RS)
    return {i: frozenset(nbr[i, : nn[i]].tolist()) for i in range(len(nn))}
