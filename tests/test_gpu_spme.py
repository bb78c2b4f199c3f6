"""SPME long-range Coulomb solver (include/md_spme.h) against the FP64 Ewald /
SPME oracle (oracle/ewald.py), through the C ABI, on a B300.

An FP64 context computes everything in FP64 and must match the oracle's SPME
at the same grid and order, and its brute-force real-space erfc sum, to 1e-10
(energies and forces).  A mixed context (FP32 splines, grid, FFTs and gather;
FP32 real-space pairs with Kahan sums; FP64 energy totals) must match to 1e-5.
Cases: the three spline orders, ragged non-power-of-two grids, an orthorhombic box, positions after steps (drift and a re-sort), a charged box
(background term), degenerate charge sets, host and device output buffers, the
argument checks, half Verlet lists, and sampled atoms of the 4M-atom workload.
"""
import numpy as np
import pytest

import md_inputs as mi
from oracle import ewald as ew

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import make, rel_l2  # noqa: E402
from paper_2109_09056_b300 import SPME, MDError  # noqa: E402


def tol(precision):
    return 1e-10 if precision == "fp64" else 1e-5


def oracle_parts(x, q, box, alpha, rc, K, order, sample=None):
    Ek, Fk = ew.spme_reciprocal(x, q, box, alpha, K, order, sample=sample)
    if sample is None:
        Er, Fr = ew.ewald_real(x, q, box, alpha, rc)
    else:
        Er, Fr = None, ew.ewald_real_sample(x, q, box, alpha, rc, sample)
    Ec = ew.ewald_self(q, alpha) + ew.ewald_background(q, box, alpha)
    return Er, Fr, Ek, Fk, Ec


def check_against_oracle(sysm, solver, q, box, alpha, rc, K, order, precision, device=None):
    e, f = solver.compute(device=device)
    f = f.cpu().numpy() if torch.is_tensor(f) else f
    x = sysm.state(forces=False)["x"]
    Er, Fr, Ek, Fk, Ec = oracle_parts(x, q, box, alpha, rc, K, order)
    assert abs(e["recip"] - Ek) <= tol(precision) * abs(Ek)
    assert abs(e["real"] - Er) <= tol(precision) * abs(Er)
    assert abs(e["self"] - Ec) <= 1e-12 * abs(Ec)
    assert abs(e["total"] - (e["real"] + e["recip"] + e["self"])) <= 1e-12 * abs(e["total"])
    assert rel_l2(f, Fr + Fk) <= tol(precision)
    return e, f


@pytest.mark.parametrize("order", [4, 6, 8])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_parity_orders(precision, order):
    cs = mi.charged_workload("coulomb_fcc10_4000")
    s = cs.lj
    K = (40, 36, 45)                      # ragged, non-power-of-two grid
    sysm = make(s, precision)
    sp = SPME(sysm, cs.q, alpha=cs.alpha, rc=cs.rc, K=K, order=order)
    check_against_oracle(sysm, sp, cs.q, s.box, cs.alpha, cs.rc, K, order, precision)
    sp.close()
    sysm.close()


@pytest.mark.parametrize("K", [(45, 42, 35), (49, 28, 30), (16, 64, 27)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_fft_radices(precision, K):
    """Every FFT radix on every axis: an odd K_x (the half spectrum's last
    element then stands for a conjugate pair), radix 7 (45 = 3 3 5, 42 = 2 3 7,
    35 = 5 7, 49 = 7 7, 28 = 4 7, 30 = 2 3 5) and pure radix 8 / 4 / 3 axes."""
    cs = mi.charged_workload("coulomb_fcc10_4000")
    s = cs.lj
    order = 4
    sysm = make(s, precision)
    sp = SPME(sysm, cs.q, alpha=cs.alpha, rc=cs.rc, K=K, order=order)
    check_against_oracle(sysm, sp, cs.q, s.box, cs.alpha, cs.rc, K, order, precision)
    sp.close()
    sysm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_after_steps_and_device_output(precision):
    cs = mi.charged_workload("coulomb_fcc10_4000")
    s = cs.lj
    sysm = make(s, precision)
    sp = SPME(sysm, cs.q, alpha=cs.alpha, rc=cs.rc, K=cs.K, order=cs.order)
    sysm.step(27)                         # drift, one re-sort + rebuild at step 20
    e_h, f_h = check_against_oracle(sysm, sp, cs.q, s.box, cs.alpha, cs.rc, cs.K, cs.order,
                                    precision)
    e_d, f_d = check_against_oracle(sysm, sp, cs.q, s.box, cs.alpha, cs.rc, cs.K, cs.order,
                                    precision, device=torch.device("cuda"))
    # host and device outputs agree (the grid's atomic adds may round in another order)
    assert rel_l2(f_d, f_h) <= (1e-12 if precision == "fp64" else 1e-6)
    sp.close()
    sysm.close()


def test_spme_orthorhombic_charged_box():
    rng = np.random.default_rng(31)
    a = mi.fcc_lattice_constant(mi.RHO_MELT)
    x = mi.fcc_sites(10, 8, 12, a) + rng.uniform(-0.05, 0.05, size=(4 * 10 * 8 * 12, 3))
    n = x.shape[0]
    box = np.array([10 * a, 8 * a, 12 * a])
    s = mi.LJSystem(x=x, v=mi.maxwell_velocities(n, 1.0, rng), types=np.zeros(n, np.int32),
                    box=box)
    q = mi.neutral_charges(n, rng) + 0.05          # net charge: background term
    K = (40, 32, 48)
    for precision in ("fp64", "mixed"):
        sysm = make(s, precision)
        sp = SPME(sysm, q, alpha=1.25, rc=2.5, K=K, order=6)
        check_against_oracle(sysm, sp, q, box, 1.25, 2.5, K, 6, precision)
        sp.close()
        sysm.close()


def test_spme_degenerate_charges():
    cs = mi.charged_workload("coulomb_fcc10_4000")
    s = cs.lj
    sysm = make(s, "fp64")
    zero = np.zeros(s.n)
    sp = SPME(sysm, zero, alpha=cs.alpha, rc=cs.rc, K=cs.K, order=4)
    e, f = sp.compute()
    assert e == {"real": 0.0, "recip": 0.0, "self": 0.0, "total": 0.0}
    assert np.all(f == 0.0)
    # one charge alone: no real-space pair, only its periodic images and the background
    one = zero.copy()
    one[123] = 1.0
    sp.set_charges(one)
    check_against_oracle(sysm, sp, one, s.box, cs.alpha, cs.rc, cs.K, 4, "fp64")
    sp.close()
    sysm.close()


def test_spme_argument_checks():
    cs = mi.charged_workload("coulomb_fcc10_4000")
    s = cs.lj
    sysm = make(s, "fp64")
    bad = [dict(alpha=cs.alpha, rc=cs.rc, K=40, order=5),
           dict(alpha=cs.alpha, rc=3.0, K=40, order=4),          # rc above the pair cutoff
           dict(alpha=0.0, rc=cs.rc, K=40, order=4),
           dict(alpha=cs.alpha, rc=cs.rc, K=(40, 3, 40), order=4),
           dict(alpha=cs.alpha, rc=cs.rc, K=(40, 40, 5000), order=4),
           dict(alpha=cs.alpha, rc=cs.rc, K=(40, 41, 40), order=4),  # 41: no radix
           dict(alpha=cs.alpha, rc=cs.rc, K=(40, 40, 44), order=4)]  # 44 = 4 11
    for kw in bad:
        with pytest.raises(MDError) as ei:
            SPME(sysm, cs.q, **kw)
        assert ei.value.status == 1, kw
    q = cs.q.copy()
    q[7] = np.nan
    with pytest.raises(MDError) as ei:
        SPME(sysm, q, alpha=cs.alpha, rc=cs.rc, K=40, order=4)
    assert ei.value.status == 5
    # a grid too large for the device (4096^3 FP64, 550 GB): the allocation
    # fails, MD_ERR_NOMEM, and the context stays usable
    with pytest.raises(MDError) as ei:
        SPME(sysm, cs.q, alpha=cs.alpha, rc=cs.rc, K=4096, order=4)
    assert ei.value.status == 8
    sp = SPME(sysm, cs.q, alpha=cs.alpha, rc=cs.rc, K=cs.K, order=cs.order)
    assert np.isfinite(sp.compute()[0]["total"])
    sp.close()
    sysm.close()
    # a batched context is refused
    boxes = mi.ensemble(nbox=2, seed=3, n_lo=300, n_hi=400)
    from paper_2109_09056_b300 import MDSystem
    bx = np.stack([b.box for b in boxes])
    bs = MDSystem(np.vstack([b.x for b in boxes]), np.vstack([b.v for b in boxes]),
                  np.concatenate([b.types for b in boxes]), None,
                  n_per_box=[b.n for b in boxes], boxes=bx, stream=torch.cuda.Stream())
    with pytest.raises(MDError):
        SPME(bs, np.zeros(bs.n), alpha=1.0, rc=2.5, K=16, order=4)
    bs.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_spme_fullsize_sampled(precision):
    """The 4M-atom charged workload (K = 384^3, order 4) in the configuration
    the benchmark times: energies against the oracle's full SPME grid, forces
    of sampled atoms against the oracle's sampled gather + brute-force real
    space."""
    cs = mi.charged_workload("coulomb_fcc100_4m")
    s = cs.lj
    sysm = make(s, precision)
    sp = SPME(sysm, cs.q, alpha=cs.alpha, rc=cs.rc, K=cs.K, order=cs.order)
    e, f = sp.compute()
    x = sysm.state(forces=False)["x"]
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([rng.choice(s.n, 48, replace=False), [0, s.n - 1]]))
    Er, Fr, Ek, Fk, Ec = oracle_parts(x, cs.q, s.box, cs.alpha, cs.rc, cs.K, cs.order,
                                      sample=idx)
    assert abs(e["recip"] - Ek) <= tol(precision) * abs(Ek)
    assert abs(e["self"] - Ec) <= 1e-12 * abs(Ec)
    assert rel_l2(f[idx], Fr + Fk) <= tol(precision)
    sp.close()
    sysm.close()


@pytest.mark.parametrize("lanes", [1, 2, 8])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_lanes_per_atom(precision, lanes):
    """The real-space pass walks the context's list layout: every lanes-per-atom
    layout (1, 2, 8 besides the default 4) gives the oracle's forces."""
    cs = mi.charged_workload("coulomb_fcc10_4000")
    s = cs.lj
    sysm = make(s, precision, lanes_per_atom=lanes)
    sp = SPME(sysm, cs.q, alpha=cs.alpha, rc=cs.rc, K=cs.K, order=cs.order)
    check_against_oracle(sysm, sp, cs.q, s.box, cs.alpha, cs.rc, cs.K, cs.order, precision)
    sysm.step(21)                          # a rebuild in between
    check_against_oracle(sysm, sp, cs.q, s.box, cs.alpha, cs.rc, cs.K, cs.order, precision)
    sp.close()
    sysm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_half_lists(precision):
    """Half Verlet lists (each pair once, its reaction added to the partner):
    the real-space pass gives the oracle's energies and forces, before and
    after a rebuild."""
    cs = mi.charged_workload("coulomb_fcc10_4000")
    s = cs.lj
    sysm = make(s, precision, half_list=True)
    sp = SPME(sysm, cs.q, alpha=cs.alpha, rc=cs.rc, K=cs.K, order=cs.order)
    check_against_oracle(sysm, sp, cs.q, s.box, cs.alpha, cs.rc, cs.K, cs.order, precision)
    sysm.step(21)                          # a rebuild in between
    check_against_oracle(sysm, sp, cs.q, s.box, cs.alpha, cs.rc, cs.K, cs.order, precision)
    sp.close()
    sysm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_grid_as_small_as_the_stencil(precision):
    """K_d = order..order+2: every stencil row wraps around the grid (several
    of an atom's points coincide modulo K), the spread's scalar path."""
    cs = mi.charged_workload("coulomb_fcc10_4000")
    s = cs.lj
    sysm = make(s, precision)
    for order, K in ((8, (8, 9, 10)), (4, (4, 5, 6))):
        sp = SPME(sysm, cs.q, alpha=0.6, rc=cs.rc, K=K, order=order)
        check_against_oracle(sysm, sp, cs.q, s.box, 0.6, cs.rc, K, order, precision)
        sp.close()
    sysm.close()


def test_spme_after_set_state():
    """Positions replaced through md_set_state: the solver sees the new state
    (re-sorted, list rebuilt) at its next call."""
    cs = mi.charged_workload("coulomb_fcc10_4000")
    s = cs.lj
    sysm = make(s, "fp64")
    sp = SPME(sysm, cs.q, alpha=cs.alpha, rc=cs.rc, K=cs.K, order=cs.order)
    sp.compute()
    x2 = s.x + np.random.default_rng(9).uniform(-0.2, 0.2, size=s.x.shape)
    sysm.set_state(x2, s.v)
    check_against_oracle(sysm, sp, cs.q, s.box, cs.alpha, cs.rc, cs.K, cs.order, "fp64")
    x_now = sysm.state(forces=False)["x"]
    d = x_now - x2
    assert np.abs(d - s.box * np.round(d / s.box)).max() <= 1e-12
    sp.close()
    sysm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_real_space_pair_function_sweep(precision):
    """The real-space pair terms across [0, rc): a +-1 dimer at 24 separations
    from 0.05 to just below the cutoff (LJ off, eps = 0), energy and force of
    the real-space part against erfc evaluated by the oracle (scipy): relative
    1e-12 (FP64) / 2e-6 (mixed)."""
    from paper_2109_09056_b300 import MDSystem
    L, alpha, rc = 10.0, 1.25, 2.5
    tol = 1e-12 if precision == "fp64" else 2e-6
    q = np.array([1.0, -1.0])
    # 24 separations: the mixed pass's erfc is a fitted polynomial form on
    # [0, alpha rc], so its interior is sampled too, not only the ends
    for r in sorted(set(np.round(np.linspace(0.05, 2.45, 22), 6)) | {2.499, 1.37}):
        x = np.array([[3.0, 4.0, 5.0], [3.0 + r * 0.6, 4.0 + r * 0.8, 5.0]])
        sysm = MDSystem(x, np.zeros((2, 3)), np.zeros(2, np.int32), np.full(3, L),
                        eps=np.zeros((1, 1)), precision=precision, stream=torch.cuda.Stream())
        sp = SPME(sysm, q, alpha=alpha, rc=rc, K=16, order=4)
        e, f = sp.compute()
        Er, Fr = ew.ewald_real(x, q, np.full(3, L), alpha, rc)
        Ek, Fk = ew.spme_reciprocal(x, q, np.full(3, L), alpha, (16, 16, 16), 4)
        assert abs(e["real"] - Er) <= tol * abs(Er), (r, e["real"], Er)
        # the force holds the reciprocal part too: the bar scales with the total
        assert np.abs(f - (Fr + Fk)).max() <= tol * (np.abs(Fr).max() + np.abs(Fk).max()), r
        sp.close()
        sysm.close()


def test_spme_destroy_after_its_context():
    """Closing the system before its solver is safe (the solver's destroy
    touches only its own buffers and stream handles)."""
    cs = mi.charged_workload("coulomb_fcc10_4000")
    s = cs.lj
    sysm = make(s, "mixed")
    sp = SPME(sysm, cs.q, alpha=cs.alpha, rc=cs.rc, K=cs.K, order=cs.order)
    sp.compute()
    sysm.close()
    sp.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_rocksalt_madelung_on_gpu(precision):
    """The whole GPU solver against the rock-salt Madelung constant: 216 ions
    (nearest-neighbor distance 1, LJ off), alpha 1.8 (erfc(alpha rc) = 2e-10),
    order 8 on a 64^3 grid: the total energy per ion pair is -1.7475645946
    to 1e-8 (FP64) / 1e-5 (mixed), and the forces vanish by symmetry up to the
    grid's own symmetry breaking (the oracle's SPME at these settings: 9e-9)."""
    from paper_2109_09056_b300 import MDSystem
    x, q, box = mi.rocksalt(6)
    sysm = MDSystem(x, np.zeros_like(x), np.zeros(len(q), np.int32), box, eps=np.zeros((1, 1)),
                    precision=precision, stream=torch.cuda.Stream())
    sp = SPME(sysm, q, alpha=1.8, rc=2.5, K=64, order=8)
    e, f = sp.compute()
    tol = 1e-8 if precision == "fp64" else 1e-5
    assert abs(e["total"] / (len(q) / 2) + 1.7475645946331822) <= tol
    assert np.abs(f).max() <= (1e-7 if precision == "fp64" else 1e-4)
    sp.close()
    sysm.close()
