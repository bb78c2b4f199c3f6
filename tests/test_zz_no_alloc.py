"""md_bin_sort_noalloc: the binning + stable cell-order permutation for callers
that may not allocate device memory (code running under an allocator that
owns the device's memory, or a loop that must not pay the device-wide
synchronisation cudaMalloc/cudaFree can cause).  Its intermediates live in a
fixed array inside the library, shared by every call.

Checked through the C ABI against the FP64 oracle's binning permutation
(oracle.bin_sort) and against the existing path (md_create bins and re-sorts
its input; md_get_permutation returns that permutation): integer results, so
all three must be identical, on consecutive calls of different sizes (the
second call must not see the first call's leftovers), and on a box with one
dense cell (the per-cell ordering is quadratic in the cell's population).
This file is collected last on purpose.
"""
import numpy as np
import pytest

import md_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2109_09056_b300 import MDError, MDSystem, md_bin_sort_noalloc  # noqa: E402


def existing_path_perm(s):
    sysm = MDSystem(s.x, s.v, s.types, s.box, stream=torch.cuda.Stream())
    perm = np.array(sysm.permutation())
    sysm.close()
    return perm


def noalloc_perm(box, x_np, rs, stream):
    x = torch.from_numpy(np.ascontiguousarray(x_np)).cuda()
    perm = torch.full((x.shape[0],), -1, dtype=torch.int32, device="cuda")
    md_bin_sort_noalloc(box, x, rs, perm, stream=stream)
    stream.synchronize()
    return perm.cpu().numpy()


def test_noalloc_permutation_equals_oracle_and_md_create_on_consecutive_calls():
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(31)
    cases = [mi.lj_melt(10, seed=21, jitter=0.2),              # 4000 atoms, 5^3 cells
             mi.vacancy_box(1000, 0.8442, 1.44, rng),         # 1000 atoms, 3^3 cells
             mi.lj_melt(12, seed=22, jitter=0.3)]             # 6912 atoms, 7^3 cells
    for s in cases:
        rs = s.rc + s.skin
        got = noalloc_perm(s.box, s.x, rs, stream)
        perm_o, _, _ = oracle.bin_sort(s.x, s.box, rs)
        assert np.array_equal(got, perm_o)
        assert np.array_equal(got, existing_path_perm(s))


def test_noalloc_dense_cell_equals_oracle():
    """96 atoms packed into one cell of a 4^3-cell box beside a sparse gas (and
    positions outside [0, L) that must wrap): the same permutation as the
    oracle, on two calls in a row."""
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(5)
    L = np.array([12.0, 12.0, 12.0])
    dense = rng.uniform(3.05, 5.95, size=(96, 3))             # cell (1, 1, 1), edge 3.0
    gas = rng.uniform(-12.0, 24.0, size=(150, 3))
    x = np.concatenate([gas[:70], dense, gas[70:]])
    perm_o, _, cell_o = oracle.bin_sort(x, L, 2.8)
    assert np.bincount(cell_o).max() >= 96
    for _ in range(2):
        assert np.array_equal(noalloc_perm(L, x, 2.8, stream), perm_o)


def test_noalloc_rejects_oversize_and_host_memory():
    stream = torch.cuda.Stream()
    box = [40.0, 40.0, 40.0]
    big = torch.zeros((262145, 3), dtype=torch.float64, device="cuda")
    perm = torch.zeros(262145, dtype=torch.int32, device="cuda")
    with pytest.raises(MDError) as e:
        md_bin_sort_noalloc(box, big, 2.8, perm, stream=stream)
    assert "MD_ERR_ARG" in str(e.value)
    huge_box = [200.0, 200.0, 200.0]                          # 71^3 cells > 131072
    x = torch.rand((100, 3), dtype=torch.float64, device="cuda") * 200.0
    with pytest.raises(MDError):
        md_bin_sort_noalloc(huge_box, x, 2.8, perm[:100], stream=stream)
    # an edge whose L/rs does not fit an int32 (checked before any conversion)
    with pytest.raises(MDError) as e:
        md_bin_sort_noalloc([1e300, 40.0, 40.0], x, 2.8, perm[:100], stream=stream)
    assert "MD_ERR_ARG" in str(e.value)
    xh = torch.rand((100, 3), dtype=torch.float64) * 40.0      # host memory
    with pytest.raises(MDError):
        md_bin_sort_noalloc(box, xh, 2.8, perm[:100], stream=stream)


def test_noalloc_wrapper_rejects_wrong_tensors_without_calling():
    """Wrong dtype, shape, layout or a short perm raise MDError before any
    kernel runs, and the caller's perm is left as it was."""
    stream = torch.cuda.Stream()
    box = [12.0, 12.0, 12.0]
    x = torch.rand((64, 3), dtype=torch.float64, device="cuda") * 12.0
    perm = torch.full((64,), -7, dtype=torch.int32, device="cuda")
    bad = [(x.float(), perm), (x.t().contiguous(), perm), (x.t(), perm),
           (x, perm.long()), (x, perm[:63]), (x, perm[::2]), (x.cpu(), perm)]
    for xb, pb in bad:
        with pytest.raises(MDError):
            md_bin_sort_noalloc(box, xb, 2.8, pb, stream=stream)
    assert bool((perm == -7).all())
