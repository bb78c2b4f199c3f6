"""FP64 CPU oracle for Ewald-split Coulomb interactions: the direct Ewald sum
and the smooth particle mesh Ewald (SPME) approximation of its
reciprocal-space part.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and by ``bench.py``'s CPU
baseline; the product package never imports it.  Plain numpy in FP64 (the FFT
is ``numpy.fft``, the error function ``scipy.special.erfc``); it shares no code
with the CUDA library.

What it follows.  The paper's CabanaMD section names the long-range solver's
three grid steps -- B-spline spreading of the charges onto a uniform grid, 3-D
FFTs for the reciprocal-space energy and forces, and a gradient gather of the
grid forces back onto the atoms -- and evaluates real-space pairs with the same
neighbor iteration as the short-range forces.  It takes the method from
Essmann et al., "A smooth particle mesh Ewald method", J. Chem. Phys. 103, 8577
(1995), whose definitions are written out below (unit Coulomb constant: the
pair energy is q_i q_j / r).

* Ewald split (SPME paper, Sec. 2):  E = E_real + E_recip + E_self + E_bg,
    E_real  = sum_{i<j, r_ij < rc} q_i q_j erfc(alpha r_ij) / r_ij,
    E_recip = 1/(2 pi V) sum_{m != 0} exp(-pi^2 |m|^2 / alpha^2) / |m|^2 |S(m)|^2,
    S(m)    = sum_j q_j exp(2 pi i m . x_j),  m = (k1/L1, k2/L2, k3/L3), k integer,
    E_self  = -alpha / sqrt(pi) sum_i q_i^2,
    E_bg    = -pi (sum_i q_i)^2 / (2 V alpha^2)  (uniform neutralising background;
              zero for a neutral box).
* SPME (SPME paper, Secs. 3-4): scaled fractional coordinates u_d = K_d x_d / L_d;
  cardinal B-splines M_n by their recursion; the charge array
    Q(k) = sum_i q_i prod_d M_n(u_id - k_d)    (k_d taken mod K_d);
  E_recip ~ 1/2 sum_m theta(m) |Qhat(m)|^2 with Qhat the DFT of Q and
    theta(m) = B(m) exp(-pi^2 |m|^2 / alpha^2) / (pi V |m|^2),  theta(0) = 0,
    B(m) = prod_d |b_d(m_d)|^2,
    b_d(m) = exp(2 pi i (n-1) m / K_d) / sum_{k=0}^{n-2} M_n(k+1) exp(2 pi i m k / K_d);
  forces F_i = -dE/dx_i = -sum_k dQ(k)/dx_i (theta * Q)(k), where
  (theta * Q)(k) = dE/dQ(k) is the inverse DFT (unnormalised) of theta Qhat.

Pinned by ``tests/test_oracle_ewald.py``: the B-spline recursion against the
exact truncated-power form in rational arithmetic; partition of unity; the
Euler-spline moduli for n = 4 and 6 against hand-derived closed forms; the
rock-salt Madelung constant; independence of the total energy and forces from
alpha (neutral and charged boxes); forces against central finite differences;
SPME converging to the direct Ewald sum as the grid and order grow.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

__all__ = ["bspline", "bspline_deriv", "bspline_moduli", "spme_reciprocal",
           "ewald_reciprocal", "ewald_real", "ewald_real_sample", "ewald_self",
           "ewald_background", "ewald_total", "wrap"]


def wrap(x, box):
    """Periodic images into [0, L) per axis (x - L floor(x / L); L itself -> 0)."""
    x = np.asarray(x, dtype=np.float64)
    L = np.asarray(box, dtype=np.float64)
    xw = x - L * np.floor(x / L)
    return np.where(xw >= L, 0.0, xw)


def bspline(n: int, x):
    """Cardinal B-spline M_n(x), n >= 2, by its recursion (SPME paper, Sec. 4):
    M_2(x) = 1 - |x - 1| on [0, 2] and 0 elsewhere;
    M_n(x) = x/(n-1) M_{n-1}(x) + (n-x)/(n-1) M_{n-1}(x-1)."""
    if n < 2:
        raise ValueError("B-spline order must be >= 2")
    x = np.asarray(x, dtype=np.float64)
    if n == 2:
        return np.where((x >= 0.0) & (x <= 2.0), 1.0 - np.abs(x - 1.0), 0.0)
    return (x * bspline(n - 1, x) + (n - x) * bspline(n - 1, x - 1.0)) / (n - 1)


def bspline_deriv(n: int, x):
    """dM_n/dx = M_{n-1}(x) - M_{n-1}(x - 1), n >= 3 (SPME paper, Sec. 4)."""
    if n < 3:
        raise ValueError("derivative needs order >= 3")
    return bspline(n - 1, x) - bspline(n - 1, np.asarray(x, dtype=np.float64) - 1.0)


def bspline_moduli(n: int, K: int) -> np.ndarray:
    """|b(m)|^2 for m = 0 .. K-1 (SPME paper, Sec. 4): the numerator of b has
    modulus 1, so |b(m)|^2 = 1 / |sum_{k=0}^{n-2} M_n(k+1) exp(2 pi i m k / K)|^2.
    Odd n can make the sum vanish at m = K/2; such a grid is rejected."""
    m = np.arange(K, dtype=np.float64)
    k = np.arange(n - 1, dtype=np.float64)
    den = (bspline(n, k + 1.0)[None, :]
           * np.exp(2j * np.pi * np.outer(m, k) / K)).sum(axis=1)
    a2 = np.abs(den) ** 2
    if np.any(a2 < 1e-30):
        raise ValueError("Euler spline modulus vanishes (odd order with even K)")
    return 1.0 / a2


def _influence(box, alpha: float, K, n: int) -> np.ndarray:
    """theta(m) on the full K3 x K2 x K1 grid (axis order z, y, x), theta(0) = 0."""
    L = np.asarray(box, dtype=np.float64)
    V = float(np.prod(L))
    # signed integer wave numbers 0, 1, .., -1 per axis, then m_d = k_d / L_d
    m = [np.fft.fftfreq(K[d], d=1.0 / K[d]) / L[d] for d in range(3)]
    msq = (m[2][:, None, None] ** 2 + m[1][None, :, None] ** 2 + m[0][None, None, :] ** 2)
    B = (bspline_moduli(n, K[2])[:, None, None] * bspline_moduli(n, K[1])[None, :, None]
         * bspline_moduli(n, K[0])[None, None, :])
    with np.errstate(divide="ignore", invalid="ignore"):
        C = np.exp(-math.pi ** 2 * msq / alpha ** 2) / (math.pi * V * msq)
    C[0, 0, 0] = 0.0
    return B * C


def _stencil(x, box, K, n: int):
    """Per atom and axis: the n grid indices k = floor(u) - a (mod K), a = 0..n-1,
    and M_n(u - k), dM_n/du at them (u - k = frac(u) + a)."""
    L = np.asarray(box, dtype=np.float64)
    Kf = np.asarray(K, dtype=np.float64)
    u = np.asarray(x, dtype=np.float64) * (Kf / L)
    u = u - Kf * np.floor(u / Kf)
    k0 = np.floor(u)
    t = (u - k0)[:, :, None] + np.arange(n, dtype=np.float64)
    idx = (k0.astype(np.int64)[:, :, None] - np.arange(n)) % np.asarray(K, dtype=np.int64)[None, :, None]
    return idx, bspline(n, t), bspline_deriv(n, t)


def spme_reciprocal(x, q, box, alpha: float, K, n: int, chunk: int = 65536, sample=None):
    """SPME reciprocal-space energy and forces (SPME paper, Secs. 3-4), in
    the order the paper's CabanaMD section lists the steps: spread the charges
    onto Q with the order-n B-splines, forward 3-D FFT, multiply by theta and
    sum the energy, inverse FFT to dE/dQ, gather the spline gradients.

    x (n_atoms, 3) positions (any periodic image), q (n_atoms,) charges,
    box (3,) edges, K (3,) grid points per axis (K_x, K_y, K_z).
    Returns (E_recip, F (n_atoms, 3)); with `sample` (atom indices) the forces
    of those atoms only (the grid always holds every charge)."""
    q = np.asarray(q, dtype=np.float64)
    K = [int(k) for k in K]
    L = np.asarray(box, dtype=np.float64)
    N = q.shape[0]
    ntot = K[0] * K[1] * K[2]
    Q = np.zeros(ntot)
    for s in range(0, N, chunk):
        idx, W, _ = _stencil(np.asarray(x)[s:s + chunk], L, K, n)
        flat = ((idx[:, 2, :, None, None] * K[1] + idx[:, 1, None, :, None]) * K[0]
                + idx[:, 0, None, None, :])
        w = (q[s:s + chunk, None, None, None] * W[:, 2, :, None, None]
             * W[:, 1, None, :, None] * W[:, 0, None, None, :])
        Q += np.bincount(flat.ravel(), weights=w.ravel(), minlength=ntot)
    Q = Q.reshape(K[2], K[1], K[0])
    theta = _influence(L, alpha, K, n)
    Qh = np.fft.fftn(Q)
    E = 0.5 * float(np.sum(theta * (Qh.real ** 2 + Qh.imag ** 2)))
    dEdQ = (np.fft.ifftn(theta * Qh).real * ntot).ravel()
    rows = np.arange(N) if sample is None else np.asarray(sample, dtype=np.int64)
    xr = np.asarray(x, dtype=np.float64)[rows]
    qr = q[rows]
    F = np.empty((len(rows), 3))
    for s in range(0, len(rows), chunk):
        idx, W, D = _stencil(xr[s:s + chunk], L, K, n)
        flat = ((idx[:, 2, :, None, None] * K[1] + idx[:, 1, None, :, None]) * K[0]
                + idx[:, 0, None, None, :])
        ph = dEdQ[flat]
        gx = (W[:, 2, :, None, None] * W[:, 1, None, :, None] * D[:, 0, None, None, :] * ph).sum((1, 2, 3))
        gy = (W[:, 2, :, None, None] * D[:, 1, None, :, None] * W[:, 0, None, None, :] * ph).sum((1, 2, 3))
        gz = (D[:, 2, :, None, None] * W[:, 1, None, :, None] * W[:, 0, None, None, :] * ph).sum((1, 2, 3))
        F[s:s + chunk] = -qr[s:s + chunk, None] * np.stack(
            [gx * (K[0] / L[0]), gy * (K[1] / L[1]), gz * (K[2] / L[2])], axis=1)
    return E, F


def ewald_reciprocal(x, q, box, alpha: float, kmax, chunk: int = 2048):
    """Direct Ewald reciprocal sum over all integer k with |k_d| <= kmax_d,
    k != 0 (SPME paper, Sec. 2).  Forces:
    F_i = (2 q_i / V) sum_m f(m) m Im(conj(S(m)) exp(2 pi i m . x_i)),
    f(m) = exp(-pi^2 |m|^2 / alpha^2) / |m|^2."""
    x = np.asarray(x, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    L = np.asarray(box, dtype=np.float64)
    V = float(np.prod(L))
    km = np.broadcast_to(np.asarray(kmax, dtype=np.int64), (3,))
    g = np.stack(np.meshgrid(*[np.arange(-km[d], km[d] + 1) for d in range(3)], indexing="ij"),
                 axis=-1).reshape(-1, 3)
    g = g[np.any(g != 0, axis=1)]
    E = 0.0
    F = np.zeros_like(x)
    for s in range(0, g.shape[0], chunk):
        m = g[s:s + chunk] / L
        msq = (m * m).sum(axis=1)
        f = np.exp(-math.pi ** 2 * msq / alpha ** 2) / msq
        e = np.exp(2j * math.pi * (x @ m.T))            # (N, M)
        S = q @ e                                       # (M,)
        E += float(np.sum(f * (S.real ** 2 + S.imag ** 2))) / (2.0 * math.pi * V)
        im = (np.conj(S)[None, :] * e).imag             # (N, M)
        F += (2.0 / V) * q[:, None] * ((im * f[None, :]) @ m)
    return E, F


def _min_image(d, L):
    """Separations of wrapped positions folded once: d > L/2 -> d - L,
    d < -L/2 -> d + L."""
    return np.where(d > 0.5 * L, d - L, np.where(d < -0.5 * L, d + L, d))


def _real_rows(xw, q, L, alpha: float, rc: float, rows):
    """Real-space forces and half-energies of atoms `rows` against every other
    atom, minimum image on wrapped positions (a separation d > L/2 is taken
    as d - L, d < -L/2 as d + L), pairs with r^2 < rc^2."""
    xi = xw[rows]
    d = _min_image(xw[None, :, :] - xi[:, None, :], L)  # x_j - x_i
    r2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    mask = r2 < rc * rc
    mask[np.arange(len(rows)), rows] = False
    r2s = np.where(mask, r2, 1.0)
    r = np.sqrt(r2s)
    qq = q[rows][:, None] * q[None, :]
    er = erfc(alpha * r)
    g = np.where(mask, qq * (er / r + 2.0 * alpha / math.sqrt(math.pi)
                             * np.exp(-alpha * alpha * r2s)) / r2s, 0.0)
    F = -(g[..., None] * d).sum(axis=1)
    e = 0.5 * np.where(mask, qq * er / r, 0.0).sum(axis=1)
    return F, e


def ewald_real(x, q, box, alpha: float, rc: float, block: int = 256):
    """Real-space Ewald sum by brute force over all pairs (SPME paper, Sec. 2):
    F_i = sum_{j != i, r < rc} q_i q_j [erfc(alpha r)/r + 2 alpha/sqrt(pi)
    exp(-alpha^2 r^2)] (x_i - x_j) / r^2.  Needs rc < L/2 (one image per pair).
    Returns (E_real, F)."""
    L = np.asarray(box, dtype=np.float64)
    if rc >= 0.5 * L.min():
        raise ValueError("rc must be below half the box")
    xw = wrap(x, L)
    q = np.asarray(q, dtype=np.float64)
    N = q.shape[0]
    F = np.zeros((N, 3))
    E = 0.0
    for s in range(0, N, block):
        rows = np.arange(s, min(N, s + block))
        f, e = _real_rows(xw, q, L, alpha, rc, rows)
        F[rows] = f
        E += float(e.sum())
    return E, F


def ewald_real_sample(x, q, box, alpha: float, rc: float, sample):
    """Real-space forces of the atoms in `sample` only: for each, the same
    minimum-image rule and pair terms as ewald_real over every other atom
    (atoms farther than rc along some axis are skipped first)."""
    L = np.asarray(box, dtype=np.float64)
    xw = wrap(x, L)
    q = np.asarray(q, dtype=np.float64)
    sample = np.asarray(sample, dtype=np.int64)
    F = np.zeros((len(sample), 3))
    for k, i in enumerate(sample):
        d = _min_image(xw - xw[i], L)
        near = np.flatnonzero(np.all(np.abs(d) < rc, axis=1))
        near = near[near != i]
        F[k], _ = _real_rows(np.vstack([xw[i:i + 1], xw[near]]),
                             np.concatenate([q[i:i + 1], q[near]]), L, alpha, rc, np.array([0]))
    return F


def ewald_self(q, alpha: float) -> float:
    """E_self = -alpha/sqrt(pi) sum q_i^2 (SPME paper, Sec. 2)."""
    q = np.asarray(q, dtype=np.float64)
    return -alpha / math.sqrt(math.pi) * float(np.dot(q, q))


def ewald_background(q, box, alpha: float) -> float:
    """E_bg = -pi Q^2 / (2 V alpha^2), Q = sum q_i: the energy of a uniform
    neutralising background (the k = 0 limit of the reciprocal sum)."""
    Qt = float(np.sum(np.asarray(q, dtype=np.float64)))
    V = float(np.prod(np.asarray(box, dtype=np.float64)))
    return -math.pi * Qt * Qt / (2.0 * V * alpha * alpha)


def ewald_total(x, q, box, alpha: float, rc: float, kmax=None, K=None, n: int = 0):
    """Total Coulomb energy and forces, real + reciprocal + self + background.
    The reciprocal part is the direct sum (kmax) or SPME (K, n)."""
    Er, Fr = ewald_real(x, q, box, alpha, rc)
    if kmax is not None:
        Ek, Fk = ewald_reciprocal(x, q, box, alpha, kmax)
    else:
        Ek, Fk = spme_reciprocal(x, q, box, alpha, K, n)
    return Er + Ek + ewald_self(q, alpha) + ewald_background(q, box, alpha), Fr + Fk
