"""ctypes marshalling for libmd_b300.so (the C ABI declared in include/md.h and
include/md_spme.h).

Argument marshalling only: every step of the MD path runs in the library's
CUDA kernels.  There is no CPU fallback: importing this module raises if the
shared library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmd_b300.so")

MD_OK = 0
MD_ERR_ARG = 1
MD_ERR_BOX_TOO_SMALL = 2
MD_ERR_NEIGH_OVERFLOW = 3
MD_ERR_DANGEROUS_BUILD = 4
MD_ERR_NONFINITE = 5
MD_ERR_TIMEOUT = 6
MD_ERR_CUDA = 7
MD_ERR_NOMEM = 8
STATUS_NAMES = {0: "MD_OK", 1: "MD_ERR_ARG", 2: "MD_ERR_BOX_TOO_SMALL", 3: "MD_ERR_NEIGH_OVERFLOW",
                4: "MD_ERR_DANGEROUS_BUILD", 5: "MD_ERR_NONFINITE", 6: "MD_ERR_TIMEOUT",
                7: "MD_ERR_CUDA", 8: "MD_ERR_NOMEM"}
MD_FP64 = 0
MD_MIXED = 1


class md_box(C.Structure):
    _fields_ = [("L", C.c_double * 3)]


class md_params(C.Structure):
    _fields_ = [("ntypes", C.c_int32),
                ("eps", C.POINTER(C.c_double)),
                ("sigma", C.POINTER(C.c_double)),
                ("mass", C.POINTER(C.c_double)),
                ("rc", C.c_double), ("skin", C.c_double), ("dt", C.c_double),
                ("rebuild_every", C.c_int32), ("precision", C.c_int32),
                ("shift_energy", C.c_int32), ("check_displacement", C.c_int32),
                ("thermo_every", C.c_int32), ("neigh_pad", C.c_int32),
                ("lanes_per_atom", C.c_int32), ("block_threads", C.c_int32),
                ("use_graphs", C.c_int32), ("half_list", C.c_int32),
                ("shadow_vl", C.c_int32)]


class md_thermo(C.Structure):
    _fields_ = [("step", C.c_int64), ("pe", C.c_double), ("ke", C.c_double),
                ("etot", C.c_double), ("temperature", C.c_double),
                ("momentum", C.c_double * 3), ("max_displacement", C.c_double),
                ("nn_max", C.c_int32), ("pad", C.c_int32), ("builds", C.c_int64),
                ("dangerous_builds", C.c_int64)]

    def as_dict(self):
        return {"step": self.step, "pe": self.pe, "ke": self.ke, "etot": self.etot,
                "temperature": self.temperature, "momentum": list(self.momentum),
                "max_displacement": self.max_displacement, "nn_max": self.nn_max,
                "pad": self.pad, "builds": self.builds, "dangerous_builds": self.dangerous_builds}


class md_spme_params(C.Structure):
    _fields_ = [("alpha", C.c_double), ("rc", C.c_double), ("K", C.c_int32 * 3),
                ("order", C.c_int32)]


# Exported symbols and their signatures (kept in the order of include/md.h,
# then include/md_spme.h).
P = C.c_void_p
SIGNATURES = {
    "md_params_default": ([C.POINTER(md_params)], None),
    "md_create": ([C.POINTER(md_box), C.c_int64, P, P, P, C.POINTER(md_params), P, C.POINTER(P)], C.c_int),
    "md_bin_sort": ([P], C.c_int),
    "md_build_neighbors": ([P], C.c_int),
    "md_compute_forces": ([P, C.POINTER(C.c_double)], C.c_int),
    "md_step": ([P, C.c_int32, C.POINTER(md_thermo)], C.c_int),
    "md_force_backward": ([P, P, C.c_double, P, P, P], C.c_int),
    "md_set_positions": ([P, P], C.c_int),
    "md_set_state": ([P, P, P], C.c_int),
    "md_set_params": ([P, P, P], C.c_int),
    "md_get_state": ([P, P, P, P, P, P], C.c_int),
    "md_get_permutation": ([P, P], C.c_int),
    "md_get_neighbors": ([P, P, P, C.POINTER(C.c_int32)], C.c_int),
    "md_get_thermo": ([P, C.POINTER(md_thermo)], C.c_int),
    "md_get_thermo_log": ([P, P, C.POINTER(C.c_int32)], C.c_int),
    "md_profile": ([P, C.c_int32], C.c_int),
    "md_profile_read": ([P, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "md_launch_count": ([P, C.POINTER(C.c_int64)], C.c_int),
    "md_profile_rebuild": ([P, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_double)],
                           C.c_int),
    "md_debug_expire_waits": ([P, C.c_int32], C.c_int),
    "md_last_error": ([P], C.c_char_p),
    "md_destroy": ([P], None),
    "md_batch_create": ([C.c_int32, P, P, P, P, P, C.POINTER(md_params), P, C.POINTER(P)], C.c_int),
    "md_batch_thermo": ([P, P], C.c_int),
    "md_info": ([P, C.POINTER(C.c_int32), C.POINTER(C.c_int64)], C.c_int),
    "md_bin_sort_noalloc": ([C.POINTER(md_box), C.c_int64, P, C.c_double, P, P], C.c_int),
    "md_state_stream_create": ([P, C.POINTER(P)], C.c_int),
    "md_state_stream_push": ([P, P, P], C.c_int),
    "md_state_stream_wait": ([P], C.c_int),
    "md_state_stream_last_error": ([P], C.c_char_p),
    "md_state_stream_destroy": ([P], None),
    # include/md_spme.h
    "md_spme_create": ([P, P, C.POINTER(md_spme_params), C.POINTER(P)], C.c_int),
    "md_spme_set_charges": ([P, P], C.c_int),
    "md_spme_compute": ([P, P, P], C.c_int),
    "md_spme_step": ([P, C.c_int32, P], C.c_int),
    "md_spme_profile": ([P, C.c_int32], C.c_int),
    "md_spme_profile_read": ([P, P], C.c_int),
    "md_spme_last_error": ([P], C.c_char_p),
    "md_spme_destroy": ([P], None),
}


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load the library and attach signatures; raises if it is missing."""
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -m paper_2109_09056_b300.build` "
            "(there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


# MD_B300_LIB may name another build of the same library (the tests' checked
# build, for instance); the default is the in-tree one
LIB_PATH_USED = os.environ.get("MD_B300_LIB") or LIB_PATH
lib = load(LIB_PATH_USED)


class MDError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status: int, ctx=None) -> None:
    if status != MD_OK:
        msg = lib.md_last_error(ctx)
        raise MDError(status, msg.decode() if msg else "")


def check_io(status: int, obj=None) -> None:
    if status != MD_OK:
        msg = lib.md_state_stream_last_error(obj)
        raise MDError(status, msg.decode() if msg else "")


def check_spme(status: int, solver=None) -> None:
    if status != MD_OK:
        msg = lib.md_spme_last_error(solver)
        raise MDError(status, msg.decode() if msg else "")
