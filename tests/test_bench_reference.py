"""The reference arm of bench.py (the FP64 CPU oracle) measures whole oracle
steps until its time budget is used, at least one, and reports the count it
measured as `steps` beside the count requested, with the mean of the
measured steps as the value.  The oracle step and the clock are replaced by
fakes here (each fake step takes 40 s of fake time), so the test checks the
arm's bookkeeping, not the oracle."""
import argparse
import json
import types

import bench


def run_arm(monkeypatch, capsys, steps, step_s):
    clock = [0.0]

    def fake_step(w, lat, psi=None, t=None):
        clock[0] += step_s
        return step_s * 1e3, psi, t, "fake oracle step"

    monkeypatch.setattr(bench, "time", types.SimpleNamespace(perf_counter=lambda: clock[0]))
    monkeypatch.setattr(bench, "cpu_full_step", fake_step)
    monkeypatch.setattr(bench, "cpu_warmup", lambda w, lat: None)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    bench.reference_arm(argparse.Namespace(steps=steps, warmup=3, gpus=1))
    return json.loads(capsys.readouterr().out.strip().splitlines()[-1])


def test_reference_arm_stops_at_its_budget(monkeypatch, capsys):
    line = run_arm(monkeypatch, capsys, steps=20, step_s=40.0)
    assert line["impl"] == "reference"
    assert line["steps"] == 4 and line["steps_requested"] == 20   # 160 s >= 150 s
    assert line["value"] == line["ms_per_step"] == 40000.0
    assert line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["value"] == line["value"]
    assert "4 consecutive steps measured (20 requested" in line["cpu_baseline"]["sample"]


def test_reference_arm_runs_every_requested_step_within_budget(monkeypatch, capsys):
    line = run_arm(monkeypatch, capsys, steps=3, step_s=20.0)
    assert line["steps"] == 3 and line["steps_requested"] == 3


def test_reference_arm_measures_at_least_one_step(monkeypatch, capsys):
    line = run_arm(monkeypatch, capsys, steps=0, step_s=500.0)
    assert line["steps"] == 1
