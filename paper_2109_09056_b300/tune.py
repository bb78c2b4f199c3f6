"""Autotuner for the MD step: picks lanes per atom (which fixes the list
layout), the force kernel's CTA size, the list padding, and the rebuild
cadence with the list skin, by timing short runs of the real workload on the
current GPU.

    from paper_2109_09056_b300.tune import autotune
    best = autotune(factory, n_atoms, cache="~/.cache/md_b300_tune.json")
    sysm = factory(**best["params"])

`factory(**params)` must build an MDSystem (one box or a batch) with the
given keyword overrides; the tuner never looks inside it.

Search: (1) every (lanes_per_atom, block_threads) pair with the automatic
pad, timed over `periods` rebuild periods after a warm-up period; (2) for the
winner, list pads of max-row + {8, 16, 32} slots against the automatic pad;
(3) rebuild cadences, for each candidate skin (default: the factory's own):
a cadence is safe when no atom moved more than skin/2 between two builds
during the trial (the list then provably holds every pair closer than rc); the
fastest safe (skin, cadence) wins, and if none is safe the smallest cadence is
kept.  A larger skin lengthens every row (by ((rc + skin') / (rc + skin))^3)
but makes longer cadences safe; the forces are the same for any skin, so it is
a pure speed trade.  A trial with another skin goes back to the automatic pad.
Results are cached per (workload key, GPU name).
"""
from __future__ import annotations

import json
import os
import time
from typing import Callable, Iterable

LANES = (1, 2, 4, 8)
BLOCKS = (128, 256, 768)
PAD_SLACK = (8, 16, 32)
CADENCES = (5, 10, 15, 20, 25)


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:  # pragma: no cover - no GPU
        return "unknown"


def time_config(factory: Callable, params: dict, periods: int, steps_per_period: int,
                n_atoms: int) -> dict:
    """Build the system with `params`, run one warm-up period, time `periods`
    more with CUDA events; returns atom-steps/s and the run's thermo."""
    import torch
    sysm = factory(**params)
    stream = sysm.stream
    sysm.step(steps_per_period)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    th = sysm.step(steps_per_period * periods)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sysm.close()
    return {"rate": n_atoms * steps_per_period * periods / (ms * 1e-3), "ms": ms, "thermo": th}


def choose(results: Iterable[tuple[dict, dict]], safe: Callable[[dict], bool] = lambda r: True):
    """The fastest (params, result) among those `safe` accepts, else None."""
    best = None
    for params, res in results:
        if not safe(res):
            continue
        if best is None or res["rate"] > best[1]["rate"]:
            best = (params, res)
    return best


def cadence_safe(res: dict) -> bool:
    return res["thermo"].get("dangerous_builds", 0) == 0


def autotune(factory: Callable, n_atoms: int, key: str = "", cache: str | None = None,
             periods: int = 2, lanes: Iterable[int] = LANES, blocks: Iterable[int] = BLOCKS,
             pad_slack: Iterable[int] = PAD_SLACK, cadences: Iterable[int] = CADENCES,
             skins: Iterable = (None,), timer: Callable = time_config,
             log: Callable = lambda *a: None) -> dict:
    """Tune and return {"params": {...}, "rate": atom-steps/s, "trials": [...]}."""
    cache_key = f"{key}|n={n_atoms}|gpu={_gpu_name()}"
    if cache:
        path = os.path.expanduser(cache)
        try:
            hit = json.load(open(path)).get(cache_key)
            if hit:
                return hit
        except (OSError, ValueError):
            pass
    trials = []
    base_every = 20

    def run(params, every):
        p = dict(params, rebuild_every=every)
        r = timer(factory, p, periods, every, n_atoms)
        trials.append({"params": p, "rate": r["rate"], "dangerous_builds":
                       r["thermo"].get("dangerous_builds", 0), "nn_max": r["thermo"].get("nn_max")})
        log(p, r["rate"])
        return p, r

    # (1) lanes per atom x CTA size, automatic pad
    stage1 = [run({"lanes_per_atom": t, "block_threads": b}, base_every)
              for t in lanes for b in blocks]
    best_p, best_r = choose(stage1)
    # (2) list pad: just above the largest row seen, with some slack
    nn_max = best_r["thermo"].get("nn_max") or 0
    stage2 = [(best_p, best_r)]
    if nn_max:
        for s in pad_slack:
            stage2.append(run(dict(best_p, neigh_pad=nn_max + s), base_every))
    best_p, best_r = choose(stage2)
    # (3) cadence x skin: fastest among the safe ones, else the smallest cadence
    stage3 = []
    for sk in skins:
        p3 = dict(best_p)
        if sk is not None:
            p3["skin"] = sk
            p3.pop("neigh_pad", None)
        stage3 += [run(p3, e) for e in cadences]
    pick = choose(stage3, cadence_safe)
    if pick is None:
        pick = min(stage3, key=lambda pr: pr[0]["rebuild_every"])
    best_p, best_r = pick
    out = {"params": best_p, "rate": best_r["rate"], "trials": trials,
           "when": time.strftime("%Y-%m-%dT%H:%M:%S"), "key": cache_key}
    if cache:
        path = os.path.expanduser(cache)
        try:
            db = json.load(open(path))
        except (OSError, ValueError):
            db = {}
        db[cache_key] = out
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        with open(path, "w") as fh:
            json.dump(db, fh, indent=1)
    return out
