"""Python binding of the C ABI (include/md.h, include/md_spme.h), one function
per C entry point with the same name, plus the ``MDSystem`` and ``SPME``
convenience wrappers.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); device
tensors are passed to the library as device pointers, so no copy happens on
the Python side.  Outputs are allocated as torch CUDA tensors when ``device``
is a CUDA device, else as numpy arrays.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import _native as N
from ._native import check, check_io, check_spme, lib

try:
    import torch
except ImportError:  # pragma: no cover - torch is part of the image
    torch = None


def _is_torch(a) -> bool:
    return torch is not None and isinstance(a, torch.Tensor)


def _arr(a, dtype, shape=None):
    """(pointer, keepalive) for a numpy array or torch tensor of `dtype`."""
    if a is None:
        return None, None
    if _is_torch(a):
        tdt = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        t = a.detach()
        if t.dtype != tdt:
            t = t.to(tdt)
        t = t.contiguous()
        if shape is not None and tuple(t.shape) != tuple(shape):
            t = t.reshape(shape)
        return C.c_void_p(t.data_ptr()), t
    n = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None:
        n = n.reshape(shape)
    return n.ctypes.data_as(C.c_void_p), n


def _stream_handle(stream) -> C.c_void_p:
    if stream is None:
        if torch is not None and torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _alloc(shape, dtype, device):
    if device is not None and torch is not None and torch.device(device).type == "cuda":
        tdt = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        t = torch.empty(shape, dtype=tdt, device=device)
        return C.c_void_p(t.data_ptr()), t
    a = np.empty(shape, dtype=dtype)
    return a.ctypes.data_as(C.c_void_p), a


class Ctx:
    """Owns an md_ctx*; destroyed with md_destroy."""

    def __init__(self, handle: C.c_void_p, n: int, nbox: int, ntypes: int, keep=()):
        self.handle = handle
        self.n = n
        self.nbox = nbox
        self.ntypes = ntypes
        self._keep = keep

    def __del__(self):
        try:
            md_destroy(self)
        except Exception:
            pass


def md_params_default() -> N.md_params:
    p = N.md_params()
    lib.md_params_default(C.byref(p))
    return p


def make_params(ntypes=1, eps=None, sigma=None, mass=None, rc=2.5, skin=0.3, dt=0.005,
                rebuild_every=20, precision="mixed", shift_energy=False,
                check_displacement=False, thermo_every=0, neigh_pad=0, lanes_per_atom=0,
                block_threads=0, use_graphs=True, half_list=False, shadow_vl=0):
    """md_params plus the arrays it points to (keep both alive together)."""
    eps = np.ascontiguousarray(np.ones((ntypes, ntypes)) if eps is None else eps, dtype=np.float64)
    sigma = np.ascontiguousarray(np.ones((ntypes, ntypes)) if sigma is None else sigma,
                                 dtype=np.float64)
    mass = np.ascontiguousarray(np.ones(ntypes) if mass is None else mass, dtype=np.float64)
    p = N.md_params()
    p.ntypes = int(ntypes)
    p.eps = eps.ctypes.data_as(C.POINTER(C.c_double))
    p.sigma = sigma.ctypes.data_as(C.POINTER(C.c_double))
    p.mass = mass.ctypes.data_as(C.POINTER(C.c_double))
    p.rc, p.skin, p.dt = float(rc), float(skin), float(dt)
    p.rebuild_every = int(rebuild_every)
    p.precision = {"mixed": N.MD_MIXED, "fp64": N.MD_FP64, N.MD_MIXED: N.MD_MIXED,
                   N.MD_FP64: N.MD_FP64}[precision]
    p.shift_energy = int(bool(shift_energy))
    p.check_displacement = int(bool(check_displacement))
    p.thermo_every = int(thermo_every)
    p.neigh_pad = int(neigh_pad)
    p.lanes_per_atom = int(lanes_per_atom)
    p.block_threads = int(block_threads)
    p.use_graphs = int(bool(use_graphs))
    p.half_list = int(bool(half_list))
    p.shadow_vl = int(shadow_vl)
    return p, (eps, sigma, mass)


def md_create(box, x, v, types, params, stream=None) -> Ctx:
    b = N.md_box()
    for d in range(3):
        b.L[d] = float(box[d])
    n = int(x.shape[0])
    px, kx = _arr(x, np.float64, (n, 3))
    pv, kv = _arr(v, np.float64, (n, 3))
    pt, kt = _arr(types, np.int32, (n,))
    h = C.c_void_p()
    check(lib.md_create(C.byref(b), n, px, pv, pt, C.byref(params), _stream_handle(stream),
                        C.byref(h)))
    return Ctx(h, n, 1, params.ntypes)


def md_batch_create(n_per_box, boxes, x, v, types, params, stream=None) -> Ctx:
    nb = len(n_per_box)
    counts = np.ascontiguousarray(n_per_box, dtype=np.int64)
    bx = (N.md_box * nb)()
    for k in range(nb):
        for d in range(3):
            bx[k].L[d] = float(boxes[k][d])
    n = int(counts.sum())
    px, kx = _arr(x, np.float64, (n, 3))
    pv, kv = _arr(v, np.float64, (n, 3))
    pt, kt = _arr(types, np.int32, (n,))
    h = C.c_void_p()
    check(lib.md_batch_create(nb, counts.ctypes.data_as(C.c_void_p), C.cast(bx, C.c_void_p), px, pv,
                              pt, C.byref(params), _stream_handle(stream), C.byref(h)))
    return Ctx(h, n, nb, params.ntypes)


def md_bin_sort(ctx: Ctx) -> None:
    check(lib.md_bin_sort(ctx.handle), ctx.handle)


def md_build_neighbors(ctx: Ctx) -> None:
    check(lib.md_build_neighbors(ctx.handle), ctx.handle)


def md_compute_forces(ctx: Ctx) -> float:
    e = C.c_double()
    check(lib.md_compute_forces(ctx.handle, C.byref(e)), ctx.handle)
    return e.value


def md_step(ctx: Ctx, nsteps: int) -> dict:
    t = N.md_thermo()
    check(lib.md_step(ctx.handle, int(nsteps), C.byref(t)), ctx.handle)
    return t.as_dict()


def md_force_backward(ctx: Ctx, dL_dF, dL_dE: float, device=None):
    """(dL/dx (n,3), dL/deps (nt,nt), dL/dsigma (nt,nt))."""
    pg, kg = _arr(dL_dF, np.float64, (ctx.n, 3))
    dev = device if device is not None else (dL_dF.device if _is_torch(dL_dF) else None)
    pdx, dx = _alloc((ctx.n, 3), np.float64, dev)
    de = np.zeros((ctx.ntypes, ctx.ntypes))
    ds = np.zeros((ctx.ntypes, ctx.ntypes))
    check(lib.md_force_backward(ctx.handle, pg, float(dL_dE), pdx, de.ctypes.data_as(C.c_void_p),
                                ds.ctypes.data_as(C.c_void_p)), ctx.handle)
    return dx, de, ds


def md_set_positions(ctx: Ctx, x) -> None:
    px, kx = _arr(x, np.float64, (ctx.n, 3))
    check(lib.md_set_positions(ctx.handle, px), ctx.handle)


def md_set_state(ctx: Ctx, x=None, v=None) -> None:
    px, kx = _arr(x, np.float64, (ctx.n, 3))
    pv, kv = _arr(v, np.float64, (ctx.n, 3))
    check(lib.md_set_state(ctx.handle, px, pv), ctx.handle)


def md_set_params(ctx: Ctx, eps=None, sigma=None) -> None:
    pe, ke = _arr(None if eps is None else np.asarray(eps), np.float64)
    ps, ks = _arr(None if sigma is None else np.asarray(sigma), np.float64)
    check(lib.md_set_params(ctx.handle, pe, ps), ctx.handle)


def md_get_state(ctx: Ctx, device=None, forces: bool = True) -> dict:
    n = ctx.n
    px, x = _alloc((n, 3), np.float64, device)
    pv, v = _alloc((n, 3), np.float64, device)
    pf, f = _alloc((n, 3), np.float64, device) if forces else (None, None)
    pi, img = _alloc((n, 3), np.int32, device)
    pd, ids = _alloc((n,), np.int32, device)
    check(lib.md_get_state(ctx.handle, px, pv, pf, pi, pd), ctx.handle)
    return {"x": x, "v": v, "f": f, "img": img, "ids": ids}


def md_get_permutation(ctx: Ctx, device=None):
    pp, perm = _alloc((ctx.n,), np.int32, device)
    check(lib.md_get_permutation(ctx.handle, pp), ctx.handle)
    return perm


def md_get_neighbors(ctx: Ctx, device=None):
    """(nn (n,), rows (n, pad)) in internal order; row i valid up to nn[i]."""
    pad = C.c_int32()
    check(lib.md_get_neighbors(ctx.handle, None, None, C.byref(pad)), ctx.handle)
    pn, nn = _alloc((ctx.n,), np.int32, device)
    pb, nbr = _alloc((ctx.n, pad.value), np.int32, device)
    check(lib.md_get_neighbors(ctx.handle, pn, pb, C.byref(pad)), ctx.handle)
    return nn, nbr


def md_get_thermo(ctx: Ctx) -> dict:
    t = N.md_thermo()
    check(lib.md_get_thermo(ctx.handle, C.byref(t)), ctx.handle)
    return t.as_dict()


def md_batch_thermo(ctx: Ctx) -> list:
    ts = (N.md_thermo * ctx.nbox)()
    check(lib.md_batch_thermo(ctx.handle, C.cast(ts, C.c_void_p)), ctx.handle)
    return [t.as_dict() for t in ts]


def md_get_thermo_log(ctx: Ctx, capacity: int = 4096) -> np.ndarray:
    rows = np.zeros((capacity, 4))
    cnt = C.c_int32(capacity)
    check(lib.md_get_thermo_log(ctx.handle, rows.ctypes.data_as(C.c_void_p), C.byref(cnt)),
          ctx.handle)
    return rows[: cnt.value].copy()


def md_profile(ctx: Ctx, on: bool) -> None:
    check(lib.md_profile(ctx.handle, int(bool(on))), ctx.handle)


def md_profile_read(ctx: Ctx) -> tuple:
    """(force launches, summed device ms, algorithmic bytes per launch)."""
    k = C.c_int64()
    ms = C.c_double()
    by = C.c_double()
    check(lib.md_profile_read(ctx.handle, C.byref(k), C.byref(ms), C.byref(by)), ctx.handle)
    return k.value, ms.value, by.value


def md_profile_rebuild(ctx: Ctx) -> tuple:
    """(rebuilds, summed re-sort ms, summed list-build ms) since the last call."""
    k = C.c_int64()
    ms_s = C.c_double()
    ms_b = C.c_double()
    check(lib.md_profile_rebuild(ctx.handle, C.byref(k), C.byref(ms_s), C.byref(ms_b)), ctx.handle)
    return k.value, ms_s.value, ms_b.value


def md_launch_count(ctx: Ctx) -> int:
    k = C.c_int64()
    check(lib.md_launch_count(ctx.handle, C.byref(k)), ctx.handle)
    return k.value


def md_debug_expire_waits(ctx: Ctx, on: bool = True) -> None:
    """Test hook: make the mixed force kernel's bounded list-copy waits run out."""
    check(lib.md_debug_expire_waits(ctx.handle, 1 if on else 0), ctx.handle)


def md_bin_sort_noalloc(box, x, rs: float, perm, stream=None) -> None:
    """Binning + stable cell-order permutation into the caller's device array
    `perm` without any device allocation.  x must be a contiguous CUDA float64
    tensor of shape (n, 3) and perm a contiguous CUDA int32 tensor with at
    least n elements on the same device; nothing is converted (a converted copy
    would leave the caller's perm unwritten), anything else raises MDError."""
    def bad(msg):
        raise N.MDError(N.MD_ERR_ARG, "md_bin_sort_noalloc: " + msg)
    if not (_is_torch(x) and _is_torch(perm)):
        bad("x and perm must be torch tensors")
    if not (x.is_cuda and perm.is_cuda):
        bad("x and perm must be CUDA tensors")
    if x.device != perm.device:
        bad("x and perm must be on the same device")
    if x.dtype != torch.float64 or x.dim() != 2 or x.shape[1] != 3 or not x.is_contiguous():
        bad("x must be a contiguous float64 tensor of shape (n, 3)")
    if perm.dtype != torch.int32 or not perm.is_contiguous() or perm.numel() < x.shape[0]:
        bad("perm must be a contiguous int32 tensor with at least n elements")
    b = N.md_box()
    for d in range(3):
        b.L[d] = float(box[d])
    check(lib.md_bin_sort_noalloc(C.byref(b), int(x.shape[0]), C.c_void_p(x.data_ptr()),
                                  float(rs), C.c_void_p(perm.data_ptr()), _stream_handle(stream)))


def md_info(ctx: Ctx) -> tuple:
    nb = C.c_int32()
    n = C.c_int64()
    check(lib.md_info(ctx.handle, C.byref(nb), C.byref(n)), ctx.handle)
    return nb.value, n.value


def md_destroy(ctx: Ctx) -> None:
    if ctx.handle is not None and ctx.handle.value:
        lib.md_destroy(ctx.handle)
        ctx.handle = C.c_void_p()


class StateStream:
    """Owns an md_state_stream* (asynchronous state download)."""

    def __init__(self, handle: C.c_void_p, ctx: Ctx):
        self.handle = handle
        self.ctx = ctx

    def push(self, x=None, v=None) -> None:
        md_state_stream_push(self, x, v)

    def wait(self) -> None:
        md_state_stream_wait(self)

    def close(self) -> None:
        md_state_stream_destroy(self)

    def __del__(self):
        try:
            md_state_stream_destroy(self)
        except Exception:
            pass


def md_state_stream_create(ctx: Ctx) -> StateStream:
    h = C.c_void_p()
    check_io(lib.md_state_stream_create(ctx.handle, C.byref(h)))
    return StateStream(h, ctx)


def _out_ptr(a, shape):
    """Pointer of a caller-owned float64 output (numpy or torch, contiguous)."""
    if a is None:
        return None
    if _is_torch(a):
        assert a.dtype == torch.float64 and a.is_contiguous() and tuple(a.shape) == shape
        return C.c_void_p(a.data_ptr())
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"] and a.shape == shape
    return a.ctypes.data_as(C.c_void_p)


def md_state_stream_push(s: StateStream, x=None, v=None) -> None:
    """Snapshot x and v now and copy them into the given (n, 3) float64 host
    (pinned for overlap) or device buffers in the background; they hold the
    snapshot after md_state_stream_wait."""
    n = s.ctx.n
    check_io(lib.md_state_stream_push(s.handle, _out_ptr(x, (n, 3)), _out_ptr(v, (n, 3))), s.handle)


def md_state_stream_wait(s: StateStream) -> None:
    check_io(lib.md_state_stream_wait(s.handle), s.handle)


def md_state_stream_destroy(s: StateStream) -> None:
    if s.handle is not None and s.handle.value:
        lib.md_state_stream_destroy(s.handle)
        s.handle = C.c_void_p()


class MDSystem:
    """One context (one box, or a batch of boxes) with its parameters."""

    def __init__(self, x, v, types, box, *, ntypes=1, eps=None, sigma=None, mass=None, rc=2.5,
                 skin=0.3, dt=0.005, rebuild_every=20, precision="mixed", shift_energy=False,
                 check_displacement=False, thermo_every=0, neigh_pad=0, lanes_per_atom=0,
                 block_threads=0, use_graphs=True, half_list=False, shadow_vl=0, stream=None,
                 n_per_box=None, boxes=None):
        self.params, self._arrays = make_params(
            ntypes, eps, sigma, mass, rc, skin, dt, rebuild_every, precision, shift_energy,
            check_displacement, thermo_every, neigh_pad, lanes_per_atom, block_threads, use_graphs,
            half_list, shadow_vl)
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream()
        self.stream = stream
        if n_per_box is None:
            self.ctx = md_create(box, x, v, types, self.params, stream)
        else:
            self.ctx = md_batch_create(n_per_box, boxes, x, v, types, self.params, stream)

    @property
    def n(self) -> int:
        return self.ctx.n

    def bin_sort(self):
        md_bin_sort(self.ctx)

    def build_neighbors(self):
        md_build_neighbors(self.ctx)

    def compute_forces(self) -> float:
        return md_compute_forces(self.ctx)

    def step(self, nsteps: int) -> dict:
        return md_step(self.ctx, nsteps)

    def force_backward(self, dL_dF, dL_dE=0.0, device=None):
        return md_force_backward(self.ctx, dL_dF, dL_dE, device)

    def set_positions(self, x):
        md_set_positions(self.ctx, x)

    def set_state(self, x=None, v=None):
        md_set_state(self.ctx, x, v)

    def launch_count(self) -> int:
        return md_launch_count(self.ctx)

    def profile_rebuild(self) -> tuple:
        return md_profile_rebuild(self.ctx)

    def set_params(self, eps=None, sigma=None):
        md_set_params(self.ctx, eps, sigma)

    def state(self, device=None, forces=True) -> dict:
        return md_get_state(self.ctx, device, forces)

    def permutation(self, device=None):
        return md_get_permutation(self.ctx, device)

    def neighbors(self, device=None):
        return md_get_neighbors(self.ctx, device)

    def thermo(self) -> dict:
        return md_get_thermo(self.ctx)

    def batch_thermo(self) -> list:
        return md_batch_thermo(self.ctx)

    def thermo_log(self) -> np.ndarray:
        return md_get_thermo_log(self.ctx)

    def profile(self, on: bool = True):
        md_profile(self.ctx, on)

    def profile_read(self):
        return md_profile_read(self.ctx)

    def state_stream(self) -> StateStream:
        """Asynchronous state download object for this system."""
        return md_state_stream_create(self.ctx)

    def close(self):
        md_destroy(self.ctx)


# ---- long-range Coulomb (include/md_spme.h) ----------------------------------

class Spme:
    """Owns an md_spme*; destroyed with md_spme_destroy.  Holds the context
    (which must outlive the solver)."""

    def __init__(self, handle: C.c_void_p, ctx: Ctx):
        self.handle = handle
        self.ctx = ctx

    def __del__(self):
        try:
            md_spme_destroy(self)
        except Exception:
            pass


def md_spme_create(ctx: Ctx, q, alpha: float, rc: float, K, order: int = 4) -> Spme:
    p = N.md_spme_params()
    p.alpha, p.rc = float(alpha), float(rc)
    Kt = (int(K),) * 3 if np.isscalar(K) else tuple(int(k) for k in K)
    for d in range(3):
        p.K[d] = Kt[d]
    p.order = int(order)
    pq, kq = _arr(q, np.float64, (ctx.n,))
    h = C.c_void_p()
    check_spme(lib.md_spme_create(ctx.handle, pq, C.byref(p), C.byref(h)))
    return Spme(h, ctx)


def md_spme_set_charges(s: Spme, q) -> None:
    pq, kq = _arr(q, np.float64, (s.ctx.n,))
    check_spme(lib.md_spme_set_charges(s.handle, pq), s.handle)


def md_spme_compute(s: Spme, device=None, forces: bool = True) -> tuple:
    """(energies, f): energies = {"real", "recip", "self", "total"} ("self"
    includes the neutralising-background term), f (n, 3) in original atom
    order (None if forces is False)."""
    pf, f = _alloc((s.ctx.n, 3), np.float64, device) if forces else (None, None)
    e = (C.c_double * 4)()
    check_spme(lib.md_spme_compute(s.handle, pf, e), s.handle)
    return {"real": e[0], "recip": e[1], "self": e[2], "total": e[3]}, f


def md_spme_step(s: Spme, nsteps: int) -> dict:
    """nsteps of Coulomb + LJ velocity Verlet; energies of the final state
    {"pe_lj", "coulomb", "ke", "total"}."""
    e = (C.c_double * 4)()
    check_spme(lib.md_spme_step(s.handle, int(nsteps), e), s.handle)
    return {"pe_lj": e[0], "coulomb": e[1], "ke": e[2], "total": e[3]}


def md_spme_profile(s: Spme, on: bool = True) -> None:
    check_spme(lib.md_spme_profile(s.handle, int(bool(on))), s.handle)


def md_spme_profile_read(s: Spme) -> dict:
    """Device ms of the last md_spme_compute per stage (profiling on)."""
    ms = (C.c_double * 6)()
    check_spme(lib.md_spme_profile_read(s.handle, ms), s.handle)
    return dict(zip(("spread", "fft_forward", "influence", "fft_inverse", "gather", "real"),
                    list(ms)))


def md_spme_destroy(s: Spme) -> None:
    if s.handle is not None and s.handle.value:
        lib.md_spme_destroy(s.handle)
        s.handle = C.c_void_p()


class SPME:
    """Smooth particle mesh Ewald Coulomb solver attached to an MDSystem
    (one box): ``compute()`` returns the energies and forces at the system's
    current positions."""

    def __init__(self, system: "MDSystem", q, *, alpha: float, rc: float, K, order: int = 4):
        self.system = system
        self.solver = md_spme_create(system.ctx, q, alpha, rc, K, order)

    def set_charges(self, q):
        md_spme_set_charges(self.solver, q)

    def compute(self, device=None, forces: bool = True) -> tuple:
        return md_spme_compute(self.solver, device, forces)

    def step(self, nsteps: int) -> dict:
        return md_spme_step(self.solver, nsteps)

    def profile(self, on: bool = True):
        md_spme_profile(self.solver, on)

    def profile_read(self) -> dict:
        return md_spme_profile_read(self.solver)

    def close(self):
        md_spme_destroy(self.solver)
