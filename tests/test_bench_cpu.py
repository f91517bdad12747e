"""The host-side legs of bench.py that run without a GPU: the CPU baseline (the oracle on a
bounded sample of the starfish workload, on all host cores) and the reference arm's JSON line
(`--impl reference`), whose timing comes from that baseline.  The reference arm is checked with
the baseline replaced by a fixed stand-in, so that the line's keys and arithmetic are tested
without minutes of oracle work; the baseline itself runs once on a small budget."""
import io
import json
import types
from contextlib import redirect_stdout

import bench
import mh_workloads as W


def test_cpu_baseline_reports_the_oracle_on_a_bounded_sample():
    r = bench.cpu_baseline(W.starfish_domain(), budget_s=2.0)
    assert r["kind"] == "oracle" and r["unit"] == "points*timesteps/s"
    assert r["cores"] >= 1 and r["value"] > 0.0
    assert r["seconds_per_step_extrapolated"] > 0.0
    # value is the points of one step over the extrapolated seconds of one step
    wl = W.starfish_domain()
    n_gamma = sum(len(c) for c in wl.curves)
    assert "volume targets" in r["sample"] and "Nystrom rows" in r["sample"] and str(n_gamma) in r["sample"]
    assert r["wall_s"] < 120.0


def test_reference_arm_line(monkeypatch):
    calls = []

    def stand_in(wl, budget_s=20.0, seed=11):
        calls.append((budget_s, seed))
        return {"value": 100.0 + len(calls), "unit": "points*timesteps/s", "cores": 4, "kind": "oracle",
                "sample": "stand-in"}

    monkeypatch.setattr(bench, "cpu_baseline", stand_in)
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    args = types.SimpleNamespace(steps=2, warmup=3)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert len(calls) == 5                                    # 3 warm-up samples, then 2 timed
    assert [s for _, s in calls] == [100, 100, 100, 200, 201]
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] == (104.0 + 105.0) / 2               # mean over the timed samples only
    assert line["unit"] == "points*timesteps/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"] == {"value": line["value"], "unit": "points*timesteps/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing(monkeypatch):
    monkeypatch.setattr(bench, "cpu_baseline", lambda *a, **k: (_ for _ in ()).throw(AssertionError("ran")))
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(types.SimpleNamespace(steps=2, warmup=3))
    assert buf.getvalue() == ""
