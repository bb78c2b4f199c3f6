"""B300-native short-range Lennard-Jones MD timestep (bin, re-sort, Verlet
list, LJ 12-6 forces, velocity Verlet, force-matching adjoint), and the
long-range Coulomb solver (smooth particle mesh Ewald) on the same context.

The compute lives in libmd_b300.so (hand-written sm_103a CUDA behind the C ABI
in include/md.h).  This package is the thin Python binding: the functions
below carry the C names and only marshal arguments; ``MDSystem`` bundles them
for one context, and ``LJForce`` is the torch.autograd.Function whose backward
is ``md_force_backward``.  PyTorch provides device memory and streams.
"""
from .api import (MDSystem, md_batch_create, md_bin_sort_noalloc, md_batch_thermo, md_bin_sort, md_build_neighbors,
                  md_compute_forces, md_create, md_destroy, md_force_backward, md_get_neighbors,
                  md_get_permutation, md_get_state, md_get_thermo, md_get_thermo_log, md_info,
                  md_debug_expire_waits, md_launch_count, md_params_default, md_profile, md_profile_read, md_profile_rebuild, md_set_params,
                  md_set_positions, md_set_state, md_step, SPME, md_spme_create, md_spme_set_charges,
                  md_spme_compute, md_spme_step, md_spme_profile, md_spme_profile_read, md_spme_destroy,
                  StateStream, md_state_stream_create, md_state_stream_push, md_state_stream_wait,
                  md_state_stream_destroy)
from ._native import LIB_PATH, MD_FP64, MD_MIXED, MDError

__all__ = [
    "MDSystem", "MDError", "LIB_PATH", "MD_FP64", "MD_MIXED", "md_create", "md_bin_sort",
    "md_build_neighbors", "md_compute_forces", "md_step", "md_force_backward", "md_set_positions",
    "md_set_state", "md_launch_count", "md_debug_expire_waits", "md_bin_sort_noalloc", "md_set_params", "md_get_state", "md_get_permutation", "md_get_neighbors", "md_get_thermo",
    "md_get_thermo_log", "md_profile", "md_profile_read", "md_profile_rebuild", "md_destroy", "md_batch_create",
    "md_batch_thermo", "md_info", "md_params_default", "LJForce", "SPME", "md_spme_create",
    "md_spme_set_charges", "md_spme_compute", "md_spme_step", "md_spme_profile", "md_spme_profile_read",
    "md_spme_destroy", "StateStream", "md_state_stream_create", "md_state_stream_push",
    "md_state_stream_wait", "md_state_stream_destroy",
]


def __getattr__(name):
    if name == "LJForce":
        from .autograd import LJForce
        return LJForce
    raise AttributeError(name)
