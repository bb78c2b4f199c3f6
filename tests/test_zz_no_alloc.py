"""md_bin_sort_noalloc: the binning + stable cell-order permutation for callers
that may not allocate device memory (code running under an allocator that
owns the device's memory, or a loop that must not pay the device-wide
synchronisation cudaMalloc/cudaFree can cause).  Its intermediates live in a
fixed array inside the library, shared by every call.

Checked through the C ABI against the existing path (md_create bins and
re-sorts its input; md_get_permutation returns that permutation): integer
results, so the two must be identical, on consecutive calls of different sizes
(the second call must not see the first call's leftovers).  This file is
collected last on purpose.
"""
import numpy as np
import pytest

import md_inputs as mi

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


def test_noalloc_permutation_equals_md_create_on_consecutive_calls():
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(31)
    cases = [mi.lj_melt(10, seed=21, jitter=0.2),              # 4000 atoms, 5^3 cells
             mi.vacancy_box(1000, 0.8442, 1.44, rng),         # 1000 atoms, 3^3 cells
             mi.lj_melt(12, seed=22, jitter=0.3)]             # 6912 atoms, 7^3 cells
    for s in cases:
        x = torch.from_numpy(s.x).cuda()
        perm = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
        md_bin_sort_noalloc(s.box, x, s.rc + s.skin, perm, stream=stream)
        stream.synchronize()
        assert np.array_equal(perm.cpu().numpy(), existing_path_perm(s))


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
    xh = torch.rand((100, 3), dtype=torch.float64) * 40.0      # host memory
    with pytest.raises(MDError):
        md_bin_sort_noalloc(box, xh, 2.8, perm[:100], stream=stream)
