"""Asynchronous state download (md_state_stream_*): each push's snapshot
equals md_get_state of the same state bit for bit, while the context keeps
stepping between the push and the wait (pinned host and device outputs)."""
import numpy as np
import pytest

import md_inputs as mi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import make  # noqa: E402


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_state_stream_snapshots_match_get_state(precision):
    s = mi.lj_melt(8, seed=4, jitter=0.05)
    sysm = make(s, precision)
    ss = sysm.state_stream()
    outs, refs = [], []
    for k in range(5):                      # 5 pushes: both slots reused
        xo = torch.empty((s.n, 3), dtype=torch.float64).pin_memory()
        vo = torch.empty((s.n, 3), dtype=torch.float64).pin_memory() if k % 2 == 0 else None
        st = sysm.state(forces=False)
        refs.append((st["x"].copy(), st["v"].copy()))
        ss.push(xo, vo)
        outs.append((xo, vo))
        sysm.step(7)                        # the context moves on meanwhile
    xd = torch.empty((s.n, 3), dtype=torch.float64, device="cuda")
    vd = torch.empty((s.n, 3), dtype=torch.float64, device="cuda")
    st = sysm.state(forces=False)
    ss.push(xd, vd)
    ss.wait()
    for (xo, vo), (xr, vr) in zip(outs, refs):
        assert np.array_equal(xo.numpy(), xr)
        if vo is not None:
            assert np.array_equal(vo.numpy(), vr)
    assert np.array_equal(xd.cpu().numpy(), st["x"]) and np.array_equal(vd.cpu().numpy(), st["v"])
    ss.close()
    sysm.close()
