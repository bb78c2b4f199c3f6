"""The mixed force kernel's bounded wait for a list copy: when it runs out the
kernel abandons the step, the call returns MD_ERR_TIMEOUT, and the CUDA
context stays usable.  The wait is made to run out by the md_debug_expire_waits
hook (the copy barrier expects 16 bytes that never arrive), so nothing faults
and nothing waits without a bound."""
import time

import numpy as np
import pytest

import md_inputs as mi

pytestmark = pytest.mark.gpu


def test_list_copy_wait_runs_out_and_context_survives():
    import torch
    from paper_2109_09056_b300 import MDError, md_debug_expire_waits
    from gpu_util import make
    s = mi.lj_melt(6, seed=3, jitter=0.05)       # 864 atoms
    sysm = make(s, "mixed")
    md_debug_expire_waits(sysm.ctx, True)
    t0 = time.perf_counter()
    with pytest.raises(MDError) as e:
        sysm.step(1)
    waited = time.perf_counter() - t0
    assert "MD_ERR_TIMEOUT" in str(e.value)
    assert 0.9 < waited < 30.0                   # ~1 s per bounded wait, a few in sequence
    sysm.close()
    torch.cuda.synchronize()
    # a fresh context on the same device runs normally
    a = make(s, "mixed")
    b = make(s, "mixed")
    a.step(5)
    b.step(5)
    fa = a.state()["f"]
    fb = b.state()["f"]
    assert np.array_equal(fa, fb) and np.all(np.isfinite(fa))
    a.close()
    b.close()
