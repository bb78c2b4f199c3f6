#!/usr/bin/env python3
"""Benchmark of the short-range LJ MD timestep on B300.

One bench "step" = one rebuild period: 20 MD timesteps of the whole hot path
(wrap + bin + stable re-sort + Verlet-list build once, then 20 x LJ forces
with the fused velocity-Verlet update).  Default workload: the 4,000,000-atom
FCC 100^3 LJ melt (rho* 0.8442, +-0.05 sigma jitter, T* 1.44, rc 2.5, skin 0.3,
dt 0.005, rebuild every 20), mixed precision.  Synthetic, seeded inputs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is device-timed (inputs resident in HBM, CUDA
events on the library's stream); `e2e` goes through the C ABI with pinned HOST
buffers (state uploaded and read back every step: each step's inputs are
copied from pinned host memory one step ahead on an upload stream and passed to
md_set_state as device buffers, each step's result is an md_state_stream
snapshot copied while the next step runs, and the last one is waited for
inside the timed region); `roofline` is for the
dominant kernel (the mixed force kernel) timed live with per-launch CUDA
events; `cpu_baseline` is the FP64 oracle on the host cores (bounded sample).
The reference arm (`--impl reference`) times the oracle itself.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
# the mixed force kernel's sources (the traffic record is keyed by their hash)
FORCE_SOURCES = [os.path.join(ROOT, "paper_2109_09056_b300", "csrc", f)
                 for f in ("md_force.cu", "md_common.cuh")]
sys.path.insert(0, ROOT)

METRIC = "atom-steps/s LJ 4M atoms, mixed vs FP64 on 1 B300; pair-force % of roofline"
UNIT = "atom-steps/s"
MD_PER_STEP = 20
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lj_fcc100_4m")
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-drift", action="store_true")
    ap.add_argument("--no-spme", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--spme-workload", default="coulomb_fcc100_4m")
    return ap.parse_args()


class Dist:
    """Replicas: one independent system per rank; only timing is collective."""

    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
            self.pg = dist

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if self.pg is None:
            return x
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


class Clocks:
    """nvidia-smi sampler (every 50 ms) running during the timed region; the
    constructor returns once the first sample is in, so the region is covered."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        import threading
        self.lines = []
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50",
                                       "-i", str(index)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.p = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 5.0 and self.p.poll() is None:
            time.sleep(0.005)
        self.skip = len(self.lines)  # samples taken before the timed region starts

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line)

    def stop(self):
        if self.p is None:
            return None
        n_in = len(self.lines)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            self.p.wait()
        self.t.join(timeout=5)
        # the samples taken while the region ran, else the one just before it
        taken = self.lines[self.skip:n_in] or self.lines[max(0, n_in - 1):n_in]
        rows = [[f.strip() for f in r.split(",")] for r in taken if r.count(",") >= 8]
        if not rows:
            return None

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [v for v in (num(r[1]) for r in rows) if v is not None]
        mx = [v for v in (num(r[2]) for r in rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({nm for r in rows for k, nm in enumerate(names) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# Algorithmic bytes per atom of one re-sort (non-raw): k_bin reads r, the packed
# cell and r_build, writes the wrapped x, cell and rank (84 B); k_scatter 16 B;
# the per-cell ordering 8 B; k_permute gathers perm, cell, x, v, type, id, images
# (76 B) and writes r, r_build, x, v, type, id, images, cell, shadow, count (140 B).
SORT_BYTES_PER_ATOM = 84.0 + 16.0 + 8.0 + 76.0 + 140.0
# The list build writes every slot of its rows (4 B x pad) and reads each atom's
# shadow once from DRAM plus its count and cell bookkeeping.
BUILD_BYTES_PER_ATOM = 16.0 + 4.0

# FP64 operations per list entry in the adjoint pair term (k_adjoint): within rc
# (distance, one reciprocal, phi, psi, the Jacobian-vector product, the forces
# and the two parameter partials) and beyond rc (distance and test only).
ADJ_FLOPS_IN, ADJ_FLOPS_OUT = 86, 11
FP64_NOMINAL_TFLOPS = 1.25


# Algorithmic bytes of the SPME kernels (R = grid real size: 4 mixed, 8 FP64).
# Spread, per atom: r, packed cell, id, gathered charge (40 B) in, the slot's
# charge in FP64 and FP32 (12 B) out; per grid point the zeroing write and one
# read-modify-write (3 R).  Gather, per atom: r, cell, id, charge, real-space
# force in (64 B), force out (24 B); per grid point one read (R).  Influence,
# per half-spectrum element: Qhat read and written (4 R), theta read (R).
# FFTs (the forward x and y passes; the inverse y and x passes): the grid read
# and the half spectrum written, or back, once (R per grid point + 2 R per
# half-spectrum element; the passes move each element twice).  Influence (the
# fused z pass: forward z, theta, inverse z): Qhat read and written, theta read.  Real space:
# 4 B per list entry, and per atom its shadow or FP64 position, charge and
# count in, its force out.
SPME_SPREAD_ATOM, SPME_GATHER_ATOM = 52.0, 88.0


def spme_bytes(stage, n, n_list, ngrid, nhalf, rb, mixed):
    if stage == "spread":
        return SPME_SPREAD_ATOM * n + 3 * rb * ngrid
    if stage == "gather":
        return SPME_GATHER_ATOM * n + rb * ngrid
    if stage == "influence":
        return 5 * rb * nhalf
    if stage in ("fft_forward", "fft_inverse"):
        return rb * ngrid + 2 * rb * nhalf
    per_atom = (16 + 4 + 4 + 24) if mixed else (24 + 8 + 4 + 24)
    return 4.0 * n_list + per_atom * n


def spme_leg(args, stream, hbm_peak):
    """Long-range Coulomb by SPME (md_spme_compute) on a charged melt: the
    LJ-melt positions with neutral random +-1 charges, alpha 1.25, real-space
    cutoff 2.5, order-4 splines on a K^3 grid of ~0.44 sigma spacing.  Whole
    calls timed with CUDA events (each call returns its energies to the host);
    per-stage device times from md_spme_profile; the HBM view per stage; and
    the Coulomb + LJ timestep (md_spme_step) in atom-steps/s."""
    import numpy as np
    import torch

    import md_inputs as mi
    from paper_2109_09056_b300 import SPME, MDSystem
    from paper_2109_09056_b300 import api as A
    cs = mi.charged_workload(args.spme_workload)
    s = cs.lj
    K = cs.K
    ngrid = K[0] * K[1] * K[2]
    nhalf = (K[0] // 2 + 1) * K[1] * K[2]
    res = {"workload": args.spme_workload, "atoms": s.n, "alpha": cs.alpha, "rc": cs.rc,
           "grid": list(K), "order": cs.order, "unit": "atoms/s (one md_spme_compute)"}
    reps = max(args.steps // 3, 5)
    for prec in ("mixed", "fp64"):
        m = MDSystem(s.x, s.v, s.types, s.box, precision=prec, stream=stream)
        sp = SPME(m, cs.q, alpha=cs.alpha, rc=cs.rc, K=K, order=cs.order)
        dev = torch.device("cuda")
        for _ in range(3):
            sp.compute(device=dev)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            energies, _ = sp.compute(device=dev)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        sp.profile(True)
        stages = []
        for _ in range(3):
            sp.compute(device=dev)
            stages.append(sp.profile_read())
        sp.profile(False)
        stage_ms = {k: float(np.median([d[k] for d in stages])) for k in stages[0]}
        nn = torch.empty(s.n, dtype=torch.int32, device=dev)      # row lengths only
        pad = A.C.c_int32()
        A.check(A.lib.md_get_neighbors(m.ctx.handle, A.C.c_void_p(nn.data_ptr()), None,
                                       A.C.byref(pad)), m.ctx.handle)
        n_list = int(nn.sum().item())
        rb = 4 if prec == "mixed" else 8
        hbm = {}
        for k, t in stage_ms.items():
            b = spme_bytes(k, s.n, n_list, ngrid, nhalf, rb, prec == "mixed")
            hbm[k] = {"bytes": b, "achieved_gbs": b / (t * 1e-3) / 1e9,
                      "frac": b / (t * 1e-3) / 1e9 / hbm_peak}
        # Coulomb + LJ dynamics: md_spme_step over whole rebuild periods
        nstep = 20 if prec == "mixed" else 5
        sp.step(nstep)
        torch.cuda.synchronize()
        e0.record(stream)
        sp.step(nstep)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / nstep
        res[prec] = {"ms_per_call": ms, "value": s.n / (ms * 1e-3), "stage_ms": stage_ms,
                     "hbm_view": hbm, "energy": energies,
                     "md_step": {"steps_timed": nstep, "ms_per_step": step_ms,
                                 "atom_steps_per_s": s.n / (step_ms * 1e-3),
                                 "note": "LJ + SPME Coulomb velocity Verlet (md_spme_step), "
                                         "one re-sort + list rebuild per 20 steps"}}
        sp.close()
        m.close()
    res["mixed_over_fp64"] = res["mixed"]["value"] / res["fp64"]["value"]
    res["hbm_peak_gbs"] = hbm_peak
    # half Verlet lists (4 lanes per atom; each pair once, reactions by FP64
    # atomics): whole calls and the real-space stage, each precision
    half = {}
    for prec in ("mixed", "fp64"):
        m = MDSystem(s.x, s.v, s.types, s.box, precision=prec, half_list=True, stream=stream)
        sp = SPME(m, cs.q, alpha=cs.alpha, rc=cs.rc, K=K, order=cs.order)
        dev = torch.device("cuda")
        for _ in range(3):
            sp.compute(device=dev)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            sp.compute(device=dev)
        e1.record(stream)
        torch.cuda.synchronize()
        sp.profile(True)
        sp.compute(device=dev)
        real_ms = float(sp.profile_read()["real"])
        sp.profile(False)
        half[prec] = {"ms_per_call": e0.elapsed_time(e1) / reps, "real_ms": real_ms}
        sp.close()
        m.close()
    res["half_lists"] = half
    if not args.no_cpu:
        # the oracle (numpy FP64: SPME reciprocal part + brute-force real space)
        # on the small charged box, for scale
        from oracle import ewald
        cc = mi.charged_workload("coulomb_fcc10_4000")
        t = time.perf_counter()
        ewald.spme_reciprocal(cc.lj.x, cc.q, cc.lj.box, cc.alpha, cc.K, cc.order)
        ewald.ewald_real(cc.lj.x, cc.q, cc.lj.box, cc.alpha, cc.rc)
        el = time.perf_counter() - t
        res["cpu_baseline"] = {"value": cc.lj.n / el, "unit": res["unit"], "kind": "oracle",
                               "cores": os.cpu_count(),
                               "sample": "one oracle evaluation of coulomb_fcc10_4000 (4,000 "
                                         "atoms, 40^3 grid, order 4; numpy)"}
    return res


def variants_leg(sysd, stream, hbm_peak):
    """Traversal / list-layout variants of the LJ step on the benchmark
    workload: the team size of the hierarchical traversal (lanes per atom,
    which also fixes the list's warp-transposed layout) at 1, 2, 4 and 8, half
    lists (each pair once, reactions by atomics; 4 lanes), and the particle
    layout of the neighbor gathers (AoSoA of vector length 8 and 32 against
    the float4 shadow; 4 lanes; the AoSoA copy's refresh counted); and the FP64
    path with full lists (its automatic lanes) and with half lists (FP64
    atomics, 4 lanes).  Per variant:
    the force evaluation's device ms per launch (profiled launches, CUDA
    events; with half lists the force kernel and its epilogue kernel), its HBM
    fraction over its own algorithmic bytes, and the whole step's throughput
    over two rebuild periods."""
    import torch

    from paper_2109_09056_b300 import MDSystem
    res = {"workload": "see config",
           "axis": "lanes_per_atom; half: 4 lanes, half lists; aosoaV: 4 lanes, neighbor "
                   "gathers from an AoSoA shadow copy of vector length V; fp64: the FP64 path, "
                   "automatic lanes; fp64_half: the FP64 path, 4 lanes, half lists",
           "md_steps": 2 * MD_PER_STEP}
    for lanes in (1, 2, 4, 8, "half", "aosoa8", "aosoa32", "fp64", "fp64_half"):
        named = isinstance(lanes, str)
        fp64 = named and lanes.startswith("fp64")
        m = MDSystem(sysd.x, sysd.v, sysd.types, sysd.box, precision="fp64" if fp64 else "mixed",
                     rc=sysd.rc, skin=sysd.skin, dt=sysd.dt, rebuild_every=sysd.rebuild_every,
                     lanes_per_atom=0 if lanes == "fp64" else (4 if named else lanes),
                     half_list=lanes in ("half", "fp64_half"),
                     shadow_vl=int(lanes[5:]) if named and lanes.startswith("aosoa") else 0,
                     stream=stream)
        m.step(MD_PER_STEP)
        m.profile(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        m.step(2 * MD_PER_STEP)
        e1.record(stream)
        torch.cuda.synchronize()
        n_force, force_ms, alg = m.profile_read()
        m.profile(False)
        m.close()
        per = force_ms / max(n_force, 1)
        res[str(lanes)] = {"force_ms_per_launch": per,
                           "force_hbm_frac": alg / (per * 1e-3) / 1e9 / hbm_peak,
                           "atom_steps_per_s": sysd.n * 2 * MD_PER_STEP / (e0.elapsed_time(e1) * 1e-3)}
    return res


def adjoint_leg(args, stream, dev):
    """md_force_backward on the two-type 32,000-atom force-matching workload:
    forward (md_compute_forces, FP64) and backward (the whole call: re-sort,
    list rebuild, adjoint kernel, reductions) timed with CUDA events."""
    import numpy as np
    import torch

    import md_inputs as mi
    from paper_2109_09056_b300 import MDSystem
    from paper_2109_09056_b300 import api as A
    sa = mi.workload("lj_2type_fcc20_32000")
    m = MDSystem(sa.x, sa.v, sa.types, sa.box, ntypes=sa.ntypes, eps=sa.eps, sigma=sa.sigma,
                 mass=sa.mass, rc=sa.rc, skin=sa.skin, dt=sa.dt, rebuild_every=sa.rebuild_every,
                 precision="fp64", stream=stream)
    G = torch.randn((sa.n, 3), dtype=torch.float64,
                    generator=torch.Generator().manual_seed(5)).to(dev)
    reps = max(args.steps, 5)
    for _ in range(3):
        m.compute_forces()
        A.md_force_backward(m.ctx, G, 0.5)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    for _ in range(reps):
        m.compute_forces()
    ev[1].record(stream)
    for _ in range(reps):
        A.md_force_backward(m.ctx, G, 0.5)
    ev[2].record(stream)
    torch.cuda.synchronize()
    fwd = ev[0].elapsed_time(ev[1]) / reps
    bwd = ev[1].elapsed_time(ev[2]) / reps
    # list entries and those within rc, from the GPU's own list and positions
    st = m.state(forces=False)
    x_int = st["x"][st["ids"]]
    nn, rows = m.neighbors()
    ii = np.repeat(np.arange(sa.n), nn)
    jj = np.concatenate([rows[k, : nn[k]] for k in range(sa.n)])
    d = x_int[jj] - x_int[ii]
    d -= sa.box * np.round(d / sa.box)
    within = int(np.count_nonzero((d * d).sum(1) < sa.rc ** 2))
    flops = within * ADJ_FLOPS_IN + (ii.size - within) * ADJ_FLOPS_OUT
    m.close()
    achieved = flops / (bwd * 1e-3) / 1e12
    return {"workload": "lj_2type_fcc20_32000", "atoms": sa.n, "precision": "fp64",
            "forward_ms": fwd, "backward_ms": bwd, "backward_over_forward": bwd / fwd,
            "value": sa.n / (bwd * 1e-3), "unit": "atoms/s (one md_force_backward)",
            "fp64_view": {"achieved_tflops": achieved, "peak_tflops": FP64_NOMINAL_TFLOPS,
                          "peak_source": "nominal", "frac": achieved / FP64_NOMINAL_TFLOPS,
                          "flops_per_call": flops, "list_entries": int(ii.size),
                          "entries_within_rc": within}}


def drift_leg(stream):
    """Energy conservation on the 131,072-atom melt (32^3 FCC cells, T* 1.44):
    1000 NVE steps, mixed and FP64, total energy logged every 50 steps (the
    run's device time gives the throughput at this size too)."""
    import numpy as np
    import torch

    import md_inputs as mi
    from paper_2109_09056_b300 import MDSystem
    s = mi.workload("lj_fcc32_131072")
    res = {"workload": "lj_fcc32_131072", "atoms": s.n, "md_steps": 1000, "thermo_every": 50}
    logs = {}
    for prec in ("mixed", "fp64"):
        m = MDSystem(s.x, s.v, s.types, s.box, precision=prec, rc=s.rc, skin=s.skin, dt=s.dt,
                     rebuild_every=s.rebuild_every, thermo_every=50, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m.step(1000)
        e1.record(stream)
        torch.cuda.synchronize()
        lg = m.thermo_log()
        m.close()
        res.setdefault("atom_steps_per_s", {})[prec] = s.n * 1000 / (e0.elapsed_time(e1) * 1e-3)
        e = lg[:, 3] / s.n                            # total energy per atom
        slope = float(np.polyfit(lg[:, 0], e, 1)[0])
        logs[prec] = e
        res[prec] = {"etot_per_atom_start": float(e[0]), "etot_per_atom_end": float(e[-1]),
                     "drift_per_atom": float(e[-1] - e[0]),
                     "slope_per_atom_per_1000_steps": slope * 1000.0,
                     "max_abs_dev_per_atom": float(np.abs(e - e[0]).max())}
    res["max_abs_etot_mixed_minus_fp64_per_atom"] = float(np.abs(logs["mixed"] - logs["fp64"]).max())
    return res


def small_leg(stream):
    """Throughput at the 4,000-atom size (10^3 FCC cells, 100 steps, rebuild
    every 20), mixed and FP64: launch-bound, reported for completeness."""
    import torch

    import md_inputs as mi
    from paper_2109_09056_b300 import MDSystem
    s = mi.workload("lj_fcc10_4000")
    res = {"workload": "lj_fcc10_4000", "atoms": s.n, "md_steps": 100}
    for prec in ("mixed", "fp64"):
        m = MDSystem(s.x, s.v, s.types, s.box, precision=prec, rc=s.rc, skin=s.skin, dt=s.dt,
                     rebuild_every=s.rebuild_every, stream=stream)
        m.step(100)                                   # warm-up (graphs captured)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        m.step(100)
        e1.record(stream)
        torch.cuda.synchronize()
        m.close()
        res[prec] = s.n * 100 / (e0.elapsed_time(e1) * 1e-3)
    res["unit"] = "atom-steps/s"
    return res


def kernel_sources_sha256(files) -> str:
    h = hashlib.sha256()
    for f in files:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def traffic_record(kernel_files):
    """DRAM bytes per launch of the force kernel from the committed ncu summary,
    valid only while the kernel's sources are unchanged since the capture."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "force_kernel_traffic.json")))
    except (OSError, ValueError):
        return None
    return rec if rec.get("kernel_sha256") == kernel_sources_sha256(kernel_files) else None


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_period(sysd, threads=None):
    """Wall seconds of one rebuild period of the oracle on `sysd`: its entry
    re-sort + list build and 20 force evaluations (oracle.md_run of 19
    velocity-Verlet steps, which builds the list once, at its start, and
    evaluates the forces there and after every step), with `threads` OpenMP
    threads (None: all)."""
    import oracle
    prev = oracle.num_threads()
    if threads:
        oracle.set_num_threads(threads)
    try:
        t = time.perf_counter()
        oracle.md_run(sysd.x, sysd.v, sysd.types, sysd.box, MD_PER_STEP - 1)
        return time.perf_counter() - t, oracle.num_threads()
    finally:
        oracle.set_num_threads(prev)


# The oracle runs on a bounded sample of the workload: the same recipe at 1/8
# the atoms for the 4M-atom melt (about 1-2 s of CPU per period on all cores).
REFERENCE_SAMPLE = {"lj_fcc100_4m": "lj_fcc50_500k"}
PERIOD_NOTE = ("oracle on {what}: each step one measured rebuild period (one re-sort + list "
               "build and 20 force evaluations, 19 velocity-Verlet steps), wall time, no scaling")


def workload_config(args, n):
    """The workload both arms run (the same dict in both lines)."""
    # per atom ~100 list entries of 4 B plus ~100 B of state
    gb = n * 500 / 1e9
    l2 = (f"inputs larger than L2 (list + state ~{gb:.1f} GB per replica)" if gb > 0.126 else
          f"inputs ~{gb * 1e3:.0f} MB, within L2 (not flushed)")
    return {"workload": args.workload, "atoms": n, "md_steps_per_step": MD_PER_STEP,
            "rebuild_every": 20, "l2": l2}


def run_reference(args, dist):
    """The reference arm: the FP64 oracle, as it stands, on the host cores;
    every step is one rebuild period on the sample, timed as it runs."""
    if dist.rank != 0:
        return 0
    import md_inputs as mi
    import oracle
    sysd = mi.workload(REFERENCE_SAMPLE.get(args.workload, args.workload))
    oracle.build()
    for _ in range(args.warmup):
        oracle_period(sysd)
    t0 = time.perf_counter()
    cores = 1
    for _ in range(args.steps):
        _, cores = oracle_period(sysd)
    total = time.perf_counter() - t0
    value = sysd.n * MD_PER_STEP * args.steps / total
    line_atoms = mi.workload(args.workload).n if args.workload in REFERENCE_SAMPLE else sysd.n
    what = (f"all {sysd.n} atoms" if sysd.n == line_atoms else
            f"a {sysd.n}-atom sample of the same recipe")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, line_atoms),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": PERIOD_NOTE.format(what=what), "sample_atoms": sysd.n,
                             "nproc": os.cpu_count(), "cpu_model": cpu_model(),
                             "timed_s": total},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, dist):
    import torch

    import md_inputs as mi
    from paper_2109_09056_b300 import MDSystem
    from paper_2109_09056_b300 import api as A

    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    sysd = mi.workload(args.workload)
    n = sysd.n
    stream = torch.cuda.Stream(device=dev)
    common = dict(rc=sysd.rc, skin=sysd.skin, dt=sysd.dt, rebuild_every=sysd.rebuild_every,
                  lanes_per_atom=args.lanes, block_threads=args.block, stream=stream)

    # ---- device-resident value (mixed) -------------------------------------
    sysm = MDSystem(sysd.x, sysd.v, sysd.types, sysd.box, precision="mixed", **common)
    sysm.step(MD_PER_STEP * args.warmup)
    sysm.profile(True)
    k0 = sysm.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    dist.barrier()
    clk = Clocks(dist.local)
    e0.record(stream)
    th = sysm.step(MD_PER_STEP * args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = sysm.launch_count() - k0
    n_force, force_ms, alg_bytes = sysm.profile_read()
    n_reb, sort_ms, build_ms = sysm.profile_rebuild()
    sysm.profile(False)
    ms_max = dist.max(ms)
    value = n * MD_PER_STEP * args.steps * dist.world / (ms_max * 1e-3)

    out = {}
    pk = peaks()
    # ---- the FP64 path on the same workload, and mixed-vs-FP64 accuracy -----
    if not args.no_fp64:
        s64 = MDSystem(sysd.x, sysd.v, sysd.types, sysd.box, precision="fp64", **common)
        s64.step(MD_PER_STEP)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64.step(MD_PER_STEP)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        v64 = n * MD_PER_STEP / (ms64 * 1e-3)
        st = sysm.state(device=dev)
        s64.set_state(st["x"], st["v"])
        pe_d = s64.compute_forces()
        pe_m = sysm.compute_forces()
        fm = sysm.state(device=dev)["f"]
        f64 = s64.state(device=dev)["f"]
        rel = float(torch.linalg.norm(fm - f64) / torch.linalg.norm(f64))
        out["fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": ms64,
                       "mixed_speedup": value / dist.world / v64}
        out["accuracy"] = {"force_rel_l2_mixed_vs_fp64": rel,
                           "pe_rel_mixed_vs_fp64": abs(pe_m - pe_d) / abs(pe_d)}
        s64.close()

    # ---- batched ensemble: 512 boxes in one context -------------------------
    if not args.no_batch:
        ens = mi.ensemble(nbox=512, seed=11)
        import numpy as np
        xb = np.concatenate([b.x for b in ens])
        vb = np.concatenate([b.v for b in ens])
        tb = np.concatenate([b.types for b in ens])
        nb = int(sum(b.n for b in ens))
        ens_kw = dict(rc=ens[0].rc, skin=ens[0].skin, dt=ens[0].dt, stream=stream)

        def factory(**kw):
            return MDSystem(xb, vb, tb, None, precision="mixed", n_per_box=[b.n for b in ens],
                            boxes=[b.box for b in ens], **dict(ens_kw, **kw))
        tuned = {"lanes_per_atom": 4, "block_threads": 128, "rebuild_every": 20}
        if not args.no_tune:
            from paper_2109_09056_b300.tune import autotune
            t_tune = time.perf_counter()
            res = autotune(factory, nb, key="lj_ensemble_512", periods=1, lanes=(2, 4, 8),
                           blocks=(128, 256, 768), pad_slack=(8, 16), cadences=(10, 15, 20),
                           skins=(None, 0.4))
            tuned = res["params"]
            tune_s = time.perf_counter() - t_tune
        sb = factory(**tuned)
        every = tuned["rebuild_every"]
        sb.step(every)
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        kb0 = sb.launch_count()
        b0.record(stream)
        sb.step(MD_PER_STEP * args.steps)
        b1.record(stream)
        torch.cuda.synchronize()
        msb = b0.elapsed_time(b1)
        out["batch"] = {"workload": "lj_ensemble_512", "boxes": len(ens), "atoms": nb,
                        "value": nb * MD_PER_STEP * args.steps / (msb * 1e-3), "unit": UNIT,
                        "ms_per_step": msb / args.steps, "md_steps_per_step": MD_PER_STEP,
                        "precision": "mixed", "gpu_launches": sb.launch_count() - kb0,
                        "tuned": tuned, "tune_seconds": None if args.no_tune else tune_s}
        sb.close()

    # ---- roofline of the dominant kernel -----------------------------------
    t_launch = force_ms / max(n_force, 1) * 1e-3
    hbm_peak = pk.get("hbm_gbs")
    peak_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6400.0
    achieved = alg_bytes / t_launch / 1e9
    rec = traffic_record(FORCE_SOURCES)
    traffic = rec["dram_bytes_per_launch"] * n / rec["atoms"] if rec and rec.get("atoms") else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "traffic": traffic, "kernel": "k_force_mixed (fused VV)",
            "peak_source": peak_src, "launch_ms": t_launch * 1e3, "alg_bytes_per_launch": alg_bytes}
    list_per_atom = (alg_bytes - n * (16 + 16 + 4 + 96 + 16)) / 4.0 / n
    if clocks and clocks.get("sm_mhz"):
        sm_mhz = clocks["sm_mhz"]
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        rc_per_atom = list_per_atom * (sysd.rc / (sysd.rc + sysd.skin)) ** 3
        ops_atom = 10.0 * list_per_atom + 22.0 * rc_per_atom
        issue = nsm * FP32_LANES_PER_SM * sm_mhz * 1e6
        roof["alu_view"] = {"achieved_tops": n * ops_atom / t_launch / 1e12,
                            "peak_tops": issue / 1e12, "frac": n * ops_atom / t_launch / issue,
                            "sm_mhz": sm_mhz, "ops_per_atom": ops_atom}

    # ---- the rebuild kernels of the timed region (re-sort, list build) ------
    rebuild = None
    if n_reb > 0:
        t_sort = sort_ms / n_reb * 1e-3
        t_build = build_ms / n_reb * 1e-3
        pad = sysm.thermo()["pad"]
        sort_bytes = n * SORT_BYTES_PER_ATOM
        build_bytes = n * (4.0 * pad + BUILD_BYTES_PER_ATOM)
        hbm = pk.get("hbm_gbs")
        rebuild = {"rebuilds": n_reb,
                   "sort_ms": t_sort * 1e3, "build_ms": t_build * 1e3,
                   "sort_hbm_view": {"bytes": sort_bytes, "achieved_gbs": sort_bytes / t_sort / 1e9,
                                     "peak_gbs": hbm, "frac": sort_bytes / t_sort / 1e9 / hbm if hbm else None},
                   "build_hbm_view": {"bytes": build_bytes, "achieved_gbs": build_bytes / t_build / 1e9,
                                      "peak_gbs": hbm, "frac": build_bytes / t_build / 1e9 / hbm if hbm else None,
                                      "note": "the build is issue-bound (candidate tests), not DRAM-bound"}}

    # ---- end to end through the C ABI with pinned host buffers ------------
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(sysd.x).pin_memory()
        vh = torch.from_numpy(sysd.v).pin_memory()
        xo = torch.empty_like(xh).pin_memory()
        vo = torch.empty_like(vh).pin_memory()
        se = MDSystem(sysd.x, sysd.v, sysd.types, sysd.box, precision="mixed", **common)
        ss = se.state_stream()
        # each step's inputs are copied from pinned host memory into one of two
        # device buffers on an upload stream, one step ahead, and handed to
        # md_set_state as device pointers; the context's stream waits for them
        up = torch.cuda.Stream(device=dev)
        xd = [torch.empty_like(xh, device=dev) for _ in range(2)]
        vd = [torch.empty_like(vh, device=dev) for _ in range(2)]
        ready = [torch.cuda.Event() for _ in range(2)]

        def upload(k):
            with torch.cuda.stream(up):
                xd[k % 2].copy_(xh, non_blocking=True)
                vd[k % 2].copy_(vh, non_blocking=True)
                ready[k % 2].record(up)

        def e2e_steps(nsteps):
            upload(0)
            for k in range(nsteps):
                stream.wait_event(ready[k % 2])       # the step's inputs are on the device
                se.set_state(xd[k % 2], vd[k % 2])    # (md_set_state copies them in and returns)
                if k + 1 < nsteps:
                    upload(k + 1)                     # H2D of the next step's inputs, meanwhile
                se.step(MD_PER_STEP)                  # thermo of the step back to the host
                ss.push(xo, vo)                       # D2H of the step's result (x, v), copied
                                                      # while the next step runs
            ss.wait()                                 # the last step's result is on the host

        e2e_steps(max(args.warmup, 2))                # warm-up: both staging buffers, every copy
        torch.cuda.synchronize()
        dist.barrier()
        t = time.perf_counter()
        e2e_steps(args.steps)
        torch.cuda.synchronize()
        el = dist.max(time.perf_counter() - t)
        dist.barrier()
        e2e = {"value": n * MD_PER_STEP * args.steps * dist.world / el, "unit": UNIT,
               "h2d_bytes_per_step": int(xh.numel() * 8 + vh.numel() * 8),
               "d2h_bytes_per_step": int(xo.numel() * 8 + vo.numel() * 8 + 112),
               "ms_per_step": 1e3 * el / args.steps}
        ss.close()
        se.close()

    # ---- energy drift, mixed vs FP64 ------------------------------------------
    if not args.no_drift:
        out["energy_drift"] = drift_leg(stream)

    # ---- the 4,000-atom configuration -----------------------------------------
    if not args.no_drift:
        out["small"] = small_leg(stream)

    # ---- force-matching adjoint (FP64) ---------------------------------------
    if not args.no_adjoint:
        out["adjoint"] = adjoint_leg(args, stream, dev)

    # ---- long-range Coulomb (SPME) ---------------------------------------------
    if not args.no_spme:
        out["spme"] = spme_leg(args, stream, hbm_peak)

    # ---- traversal / list-layout variants of the LJ step ------------------------
    if not args.no_variants:
        out["variants"] = variants_leg(sysd, stream, hbm_peak)

    # ---- CPU baseline (oracle) on rank 0 at N = 1 ---------------------------
    # Two measured rebuild periods on all cores and one on a single thread, on
    # the bounded sample of the workload (the same recipe at 1/8 the atoms).
    cpu = None
    if not args.no_cpu and dist.world == 1 and dist.rank == 0:
        import oracle
        oracle.build()
        samp = mi.workload(REFERENCE_SAMPLE.get(args.workload, args.workload))
        t_all = []
        for _ in range(2):
            t, cores = oracle_period(samp)
            t_all.append(t)
        t_one, _ = oracle_period(samp, threads=1)
        per = samp.n * MD_PER_STEP
        cpu = {"value": per / min(t_all), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": PERIOD_NOTE.format(what=f"a {samp.n}-atom sample of the same recipe")
                         + f"; best of {len(t_all)} periods on all cores",
               "sample_atoms": samp.n, "period_s": min(t_all),
               "single_thread": {"value": per / t_one, "unit": UNIT, "period_s": t_one},
               "nproc": os.cpu_count(), "cpu_model": cpu_model()}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": workload_config(args, n),
            "launch": {"precision": "mixed", "lanes_per_atom": args.lanes or 4,
                       "list_entries_per_atom": list_per_atom,
                       "parallelism": f"replicas x{dist.world}"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks,
            "final_thermo": {"pe_per_atom": th["pe"] / n, "temperature": th["temperature"],
                             "dangerous_builds": th["dangerous_builds"], "nn_max": th["nn_max"]}}
    if rebuild is not None:
        line["rebuild"] = rebuild
    line.update(out)
    # the figures a reader of the line's tail looks for, last
    summ = {"value": value, "force_launch_ms": roof["launch_ms"], "roofline_frac": roof["frac"]}
    if "fp64" in out:
        summ.update(fp64_value=out["fp64"]["value"], mixed_over_fp64=out["fp64"]["mixed_speedup"],
                    force_rel_l2_mixed_vs_fp64=out["accuracy"]["force_rel_l2_mixed_vs_fp64"])
    if "batch" in out:
        summ["batch_value"] = out["batch"]["value"]
    if e2e:
        summ["e2e_value"] = e2e["value"]
    if cpu:
        summ.update(cpu_value=cpu["value"], cpu_single_thread=cpu["single_thread"]["value"])
    summ["dangerous_builds"] = th["dangerous_builds"]
    line["summary"] = summ
    sysm.close()
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    dist = Dist()
    try:
        if args.impl == "reference":
            return run_reference(args, dist)
        return run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    sys.exit(main())
