"""The batched-ensemble workload at its full configured scale: the 512
independent boxes of mi.ensemble(512, seed 11) (atom counts log-uniform in
[256, 32768], 3,246,941 atoms in all, densities U[0.7, 0.9], temperatures
U[0.8, 1.6]), mixed precision, in the launch configuration the autotuner picks
for it on B300 (4 lanes per atom, 768-thread CTAs, rebuild every 10 steps, list
pad 103), one context, graph-replayed rebuild periods.

After 20 steps (list builds at steps 10 and 20), on 16 sampled boxes (the
smallest, the largest, the densest, the hottest and 12 drawn at random):
  * each atom's neighbor set, from md_get_neighbors mapped back to original ids
    through the box offsets, equals the FP64 oracle's list on the same
    positions (bit-exact: integer sets);
  * the box's forces match the FP64 oracle to relative L2 1e-5 (the mixed bar);
  * the box's potential energy (md_batch_thermo) matches the oracle's to 1e-5.
"""
import numpy as np
import pytest

import md_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import RS, rel_l2  # noqa: E402
from paper_2109_09056_b300 import MDSystem  # noqa: E402

TUNED = dict(lanes_per_atom=4, block_threads=768, rebuild_every=10, neigh_pad=103)


def sample_boxes(ens, k=16, seed=3):
    n = np.array([b.n for b in ens])
    rho = np.array([b.n / np.prod(b.box) for b in ens])
    picks = [int(n.argmin()), int(n.argmax()), int(rho.argmax())]
    ke = np.array([0.5 * np.sum(b.v ** 2) / b.n for b in ens])
    picks.append(int(ke.argmax()))
    rng = np.random.default_rng(seed)
    rest = [b for b in rng.permutation(len(ens)) if b not in picks]
    picks += [int(b) for b in rest[: k - len(set(picks))]]
    return sorted(set(picks))


def test_ensemble_512_tuned_launch_lists_forces_energies():
    ens = mi.ensemble(nbox=512, seed=11)
    counts = [b.n for b in ens]
    off = np.concatenate([[0], np.cumsum(counts)])
    assert off[-1] == 3246941
    sysm = MDSystem(np.concatenate([b.x for b in ens]), np.concatenate([b.v for b in ens]),
                    np.concatenate([b.types for b in ens]), None, precision="mixed",
                    n_per_box=counts, boxes=[b.box for b in ens], rc=ens[0].rc,
                    skin=ens[0].skin, dt=ens[0].dt, stream=torch.cuda.Stream(), **TUNED)
    sysm.step(20)
    th = sysm.batch_thermo()
    st = sysm.state()
    x, f = st["x"], st["f"]
    ids = np.asarray(st["ids"])
    nn_d, rows_d = sysm.neighbors(device="cuda")
    picks = sample_boxes(ens)
    assert len(picks) == 16
    for k in picks:
        b = ens[k]
        lo, hi = int(off[k]), int(off[k + 1])
        xw = oracle.wrap(x[lo:hi], b.box)[0]
        # neighbor sets keyed by box-local original id
        nn = nn_d[lo:hi].cpu().numpy()
        rows = rows_d[lo:hi].cpu().numpy()
        gpu = {}
        for u in range(hi - lo):
            gpu[int(ids[lo + u]) - lo] = frozenset((ids[rows[u, : nn[u]]] - lo).tolist())
        nn_o, nbr_o = oracle.neighbors(xw, b.box, RS)
        assert len(gpu) == b.n, k
        for i in range(b.n):
            assert gpu[i] == frozenset(nbr_o[i, : nn_o[i]].tolist()), (k, i)
        # forces and energy on the same positions
        f_o, _, pe_o = oracle.lj_forces(xw, b.types, b.box, nn=nn_o, nbr=nbr_o)
        assert rel_l2(f[lo:hi], f_o) <= 1e-5, k
        assert th[k]["pe"] == pytest.approx(pe_o, rel=1e-5), k
    sysm.close()
