"""GPU force-matching adjoint (md_force_backward) through the C ABI.

Workload: the 32,000-atom two-type FCC box (20^3 cells, types 50/50, per-pair
eps, sigma in U[0.8, 1.2]); targets are the oracle's FP64 forces at parameters
shifted by +5%; L = sum |F - F_target|^2 + c * PE.  Bars: the GPU gradient
equals the FP64 oracle's to relative L2 1e-10 (dL/dx and the six pair
parameters); central finite differences (h = 1e-6) of L through the GPU's own
FP64 forward agree to 1e-6 relative on all six parameters and 64 sampled
coordinates (atoms with a pair within 10 h of rc skipped, since the FD would
cross the cutoff); dE/dx = -F; the autograd Function gives the same numbers.
"""
import numpy as np
import pytest

import md_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import make, rel_l2  # noqa: E402

H = 1e-6
C_E = 0.37


@pytest.fixture(scope="module")
def fm():
    s = mi.workload("lj_2type_fcc20_32000")
    xw = oracle.wrap(s.x, s.box)[0]
    ft, _, _ = oracle.lj_forces(xw, s.types, s.box, eps=1.05 * s.eps, sigma=1.05 * s.sigma)
    sysm = make(s, "fp64")
    return s, xw, ft, sysm


def gpu_loss(sysm, ft, x=None, eps=None, sig=None):
    if eps is not None:
        sysm.set_params(eps, sig)
    if x is not None:
        sysm.set_positions(x)
    pe = sysm.compute_forces()
    f = sysm.state()["f"]
    return float(((f - ft) ** 2).sum() + C_E * pe)


def test_gradient_equals_oracle(fm):
    s, xw, ft, sysm = fm
    sysm.set_params(s.eps, s.sigma)
    sysm.set_positions(xw)
    sysm.compute_forces()
    f = sysm.state()["f"]
    G = 2.0 * (f - ft)
    dx, de, ds = sysm.force_backward(G, C_E)
    dx_o, de_o, ds_o = oracle.lj_adjoint(xw, s.types, s.box, G, C_E, eps=s.eps, sigma=s.sigma)
    assert rel_l2(dx, dx_o) <= 1e-10
    assert rel_l2(de, de_o) <= 1e-10
    assert rel_l2(ds, ds_o) <= 1e-10
    assert np.allclose(de, de.T) and np.allclose(ds, ds.T)


def test_parameter_gradient_matches_finite_differences(fm):
    s, xw, ft, sysm = fm
    sysm.set_params(s.eps, s.sigma)
    sysm.set_positions(xw)
    sysm.compute_forces()
    G = 2.0 * (sysm.state()["f"] - ft)
    _, de, ds = sysm.force_backward(G, C_E)
    for name, grad in (("eps", de), ("sig", ds)):
        for a, b in [(0, 0), (0, 1), (1, 1)]:
            vals = []
            for sgn in (+1, -1):
                e, sg = s.eps.copy(), s.sigma.copy()
                t = e if name == "eps" else sg
                t[a, b] += sgn * H
                if a != b:
                    t[b, a] += sgn * H
                vals.append(gpu_loss(sysm, ft, eps=e, sig=sg))
            fd = (vals[0] - vals[1]) / (2 * H)
            assert grad[a, b] == pytest.approx(fd, rel=1e-6), (name, a, b)
    sysm.set_params(s.eps, s.sigma)


def test_position_gradient_matches_finite_differences(fm):
    s, xw, ft, sysm = fm
    sysm.set_params(s.eps, s.sigma)
    sysm.set_positions(xw)
    sysm.compute_forces()
    G = 2.0 * (sysm.state()["f"] - ft)
    dx, _, _ = sysm.force_backward(G, C_E)
    rng = np.random.default_rng(17)
    checked = 0
    for flat in rng.choice(s.n * 3, 200, replace=False):
        i, a = divmod(int(flat), 3)
        d = xw - xw[i]
        d -= s.box * np.round(d / s.box)
        r = np.sqrt((d * d).sum(1))
        r[i] = 0.0
        if np.any(np.abs(r - 2.5) < 10 * H):
            continue
        xp = xw.copy(); xp[i, a] += H
        xm = xw.copy(); xm[i, a] -= H
        fd = (gpu_loss(sysm, ft, x=xp) - gpu_loss(sysm, ft, x=xm)) / (2 * H)
        assert dx[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(dx).mean())
        checked += 1
        if checked == 64:
            break
    assert checked == 64
    sysm.set_positions(xw)


def test_energy_gradient_is_minus_force(fm):
    s, xw, ft, sysm = fm
    sysm.set_params(s.eps, s.sigma)
    sysm.set_positions(xw)
    sysm.compute_forces()
    f = sysm.state()["f"]
    dx, _, _ = sysm.force_backward(np.zeros_like(f), 1.0)
    assert rel_l2(dx, -f) <= 1e-12


def test_autograd_function_matches_backward_and_gradcheck():
    from paper_2109_09056_b300 import LJForce
    s = mi.two_type_melt(5, seed=23)                  # 500 atoms
    sysm = make(s, "fp64")
    x = torch.from_numpy(oracle.wrap(s.x, s.box)[0]).cuda().requires_grad_(True)
    E0 = torch.from_numpy(s.eps).cuda().requires_grad_(True)
    S0 = torch.from_numpy(s.sigma).cuda().requires_grad_(True)
    ft = torch.from_numpy(oracle.lj_forces(s.x, s.types, s.box, eps=1.05 * s.eps,
                                           sigma=1.05 * s.sigma)[0]).cuda()

    def loss_fn(x, E, S):
        eps = 0.5 * (E + E.T)                           # a symmetric parameterisation
        sig = 0.5 * (S + S.T)
        F, pe = LJForce.apply(x, eps, sig, sysm)
        return ((F - ft) ** 2).sum() + C_E * pe

    L = loss_fn(x, E0, S0)
    L.backward()
    # the autograd result against the C-ABI backward on the same state
    G = 2.0 * (LJForce.apply(x.detach(), E0.detach(), S0.detach(), sysm)[0] - ft)
    dx, de, ds = sysm.force_backward(G, C_E)
    assert rel_l2(x.grad.cpu().numpy(), dx.cpu().numpy() if torch.is_tensor(dx) else dx) <= 1e-12
    assert np.allclose(E0.grad.cpu().numpy(), np.where(np.eye(2, dtype=bool), de, 0.5 * de),
                       rtol=1e-12, atol=0)
    # central differences through the symmetric parameterisation (parameters only)
    for M, grad in ((E0, E0.grad), (S0, S0.grad)):
        for a, b in [(0, 0), (0, 1), (1, 0), (1, 1)]:
            vals = []
            for sgn in (+1, -1):
                with torch.no_grad():
                    M[a, b] += sgn * H
                vals.append(float(loss_fn(x.detach(), E0.detach(), S0.detach())))
                with torch.no_grad():
                    M[a, b] -= sgn * H
            fd = (vals[0] - vals[1]) / (2 * H)
            assert float(grad[a, b]) == pytest.approx(fd, rel=1e-6)
