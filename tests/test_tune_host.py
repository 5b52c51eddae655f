"""Host logic of the autotuner (no GPU): every grid point is timed once,
the fastest wins, a candidate the library rejects counts as infinitely slow,
and a cached result is returned without timing anything."""
import json

import pytest

from paper_2508_08702_gb300 import instances as I
from paper_2508_08702_gb300 import msp as M
from paper_2508_08702_gb300 import tune


@pytest.fixture
def fake_timer(monkeypatch):
    calls = []

    def time_step(instances, repeats=1, **opts):
        calls.append(dict(opts))
        if opts["lanes"] == 4:
            raise M.MspError(M.MSP_EINVAL, "does not fit")
        return 10.0 * opts["lanes"] + (1.0 if opts["split_target"] else 0.0)

    monkeypatch.setattr(tune, "time_step", time_step)
    monkeypatch.setattr(tune, "_key", lambda insts: f"fake|{len(insts)}")
    return calls


def test_grid_search_picks_the_fastest(fake_timer):
    insts = I.batch_m4_7(4)
    out = tune.tune(insts, grid={"lanes": (4, 8, 16), "split_target": (0, 4096)})
    assert len(fake_timer) == 6
    assert out["opts"] == {"lanes": 8, "split_target": 0}
    assert out["ms"] == 80.0
    bad = [r for r in out["table"] if r["opts"]["lanes"] == 4]
    assert len(bad) == 2 and all(r["ms"] == float("inf") and "error" in r["opts"] for r in bad)


def test_cached_result_is_reused(fake_timer, tmp_path):
    insts = I.batch_m4_7(4)
    cache = tmp_path / "tune.json"
    first = tune.tune(insts, grid={"lanes": (8, 16), "split_target": (0,)}, cache=str(cache))
    n = len(fake_timer)
    again = tune.tune(insts, grid={"lanes": (8, 16), "split_target": (0,)}, cache=str(cache))
    assert len(fake_timer) == n   # nothing timed the second time
    assert again == json.loads(json.dumps(first))
    saved = json.loads(cache.read_text())
    assert list(saved) == ["fake|4"]


def test_descent_moves_one_parameter_at_a_time(monkeypatch):
    """Coordinate descent on a separable fake cost: it reaches the optimum of
    every parameter and times far fewer candidates than the grid."""
    calls = []

    def time_step(instances, repeats=1, **opts):
        calls.append(dict(opts))
        if opts["warps_per_block"] == 16:
            raise M.MspError(M.MSP_EINVAL, "does not fit")
        return (abs(opts["lanes"] - 16) + abs(opts["warps_per_block"] - 4) + abs(opts["blocks_per_sm"] - 2)
                + abs(opts["split_target"] - 1024) / 256.0 + 100.0)

    monkeypatch.setattr(tune, "time_step", time_step)
    monkeypatch.setattr(tune, "_key", lambda insts: "fake")
    grid = {"lanes": (8, 16), "warps_per_block": (4, 8, 16), "blocks_per_sm": (0, 1, 2),
            "split_target": (0, 256, 1024, 4096)}
    out = tune.tune(I.batch_m4_7(2), grid=grid, strategy="descent")
    assert out["opts"] == {"lanes": 16, "warps_per_block": 4, "blocks_per_sm": 2, "split_target": 1024}
    assert out["strategy"] == "descent"
    assert len(calls) < 2 * 3 * 3 * 4
    assert len({tuple(sorted(c.items())) for c in calls}) == len(calls)   # nothing timed twice
    assert any(r["ms"] == float("inf") for r in out["table"])
