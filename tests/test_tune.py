"""The autotuner's search and selection rules (CPU, with a fake timer) and one
real tuning run on the GPU whose result must still match the oracle."""
import json

import numpy as np
import pytest

from paper_2109_09056_b300 import tune


def fake_timer(factory, params, periods, steps, n):
    # faster with 4 lanes and 128 threads, pad just above the max row best,
    # longer cadence faster, but cadences above 15 are "dangerous"
    rate = 1e9
    rate *= {1: 0.5, 2: 0.8, 4: 1.0, 8: 0.7}[params["lanes_per_atom"]]
    rate *= {64: 0.9, 128: 1.0, 256: 0.95, 384: 0.93, 768: 0.9}[params["block_threads"]]
    if "neigh_pad" in params:
        rate *= 1.05 if params["neigh_pad"] == 90 + 16 else 1.01
    rate *= 1.0 + 0.01 * params["rebuild_every"]
    danger = 1 if params["rebuild_every"] > 15 else 0
    return {"rate": rate, "ms": 1.0, "thermo": {"dangerous_builds": danger, "nn_max": 90}}


def test_search_picks_fastest_safe_configuration(tmp_path):
    out = tune.autotune(None, 1000, key="fake", cache=str(tmp_path / "c.json"), timer=fake_timer)
    p = out["params"]
    assert p["lanes_per_atom"] == 4 and p["block_threads"] == 128
    assert p["neigh_pad"] == 106
    assert p["rebuild_every"] == 15                  # fastest cadence without dangerous builds
    n_trials = len(tune.LANES) * len(tune.BLOCKS) + len(tune.PAD_SLACK) + len(tune.CADENCES)
    assert len(out["trials"]) == n_trials
    db = json.load(open(tmp_path / "c.json"))
    assert out["key"] in db


def test_cache_hit_skips_trials(tmp_path):
    path = str(tmp_path / "c.json")
    first = tune.autotune(None, 1000, key="fake", cache=path, timer=fake_timer)

    def boom(*a, **k):
        raise AssertionError("timer called despite a cache hit")
    again = tune.autotune(None, 1000, key="fake", cache=path, timer=boom)
    assert again["params"] == first["params"]


def test_skin_axis_trades_row_length_for_cadence():
    # a larger skin: every row longer (slower per step) but cadence 20 safe
    def timer(factory, params, periods, steps, n):
        skin = params.get("skin", 0.3)
        rate = 1e9 * (1.0 + 0.02 * params["rebuild_every"]) * (0.95 if skin > 0.3 else 1.0)
        danger = int(params["rebuild_every"] > (20 if skin > 0.3 else 15))
        return {"rate": rate, "ms": 1.0, "thermo": {"dangerous_builds": danger, "nn_max": 90}}
    out = tune.autotune(None, 1000, key="s", timer=timer, skins=(None, 0.4), cadences=(10, 15, 20))
    p = out["params"]
    assert p["skin"] == 0.4 and p["rebuild_every"] == 20 and "neigh_pad" not in p
    # when the longer rows cost more than the cadence saves, the default skin stays
    def slow(factory, params, periods, steps, n):
        r = timer(factory, params, periods, steps, n)
        r["rate"] *= 0.5 if params.get("skin", 0.3) > 0.3 else 1.0
        return r
    out = tune.autotune(None, 1000, key="s2", timer=slow, skins=(None, 0.4), cadences=(10, 15, 20))
    assert "skin" not in out["params"] and out["params"]["rebuild_every"] == 15


def test_no_safe_cadence_keeps_smallest():
    def always_danger(factory, params, periods, steps, n):
        r = fake_timer(factory, params, periods, steps, n)
        r["thermo"]["dangerous_builds"] = 3
        return r
    out = tune.autotune(None, 1000, key="x", timer=always_danger, cadences=(10, 5, 20))
    assert out["params"]["rebuild_every"] == 5


@pytest.mark.gpu
def test_tuned_batch_runs_and_matches_oracle():
    torch = pytest.importorskip("torch")
    import md_inputs as mi
    import oracle
    from paper_2109_09056_b300 import MDSystem
    boxes = mi.ensemble(nbox=8, seed=3, n_lo=256, n_hi=2000)
    x = np.concatenate([b.x for b in boxes])
    v = np.concatenate([b.v for b in boxes])
    t = np.concatenate([b.types for b in boxes])
    n = int(sum(b.n for b in boxes))

    def factory(**kw):
        return MDSystem(x, v, t, None, n_per_box=[b.n for b in boxes],
                        boxes=[b.box for b in boxes], stream=torch.cuda.Stream(), **kw)
    out = tune.autotune(factory, n, key="test-batch", periods=1, lanes=(2, 4), blocks=(64, 128),
                        pad_slack=(16,), cadences=(10, 20))
    sysm = factory(**out["params"])
    sysm.compute_forces()
    f = sysm.state()["f"]
    off = np.concatenate([[0], np.cumsum([b.n for b in boxes])])
    for k, b in enumerate(boxes):
        f_o, _, _ = oracle.lj_forces(oracle.wrap(b.x, b.box)[0], b.types, b.box)
        err = np.linalg.norm(f[off[k]:off[k + 1]] - f_o) / np.linalg.norm(f_o)
        assert err <= 1e-5
