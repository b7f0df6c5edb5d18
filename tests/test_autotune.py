"""The autotuner's selection and the committed table, on the CPU (the
timings themselves need a GB300)."""
import json

import paper_1511_07658_gb300.autotune as at
import paper_1511_07658_gb300.manager as mgr_mod


def test_autotune_keeps_the_fastest_setting_and_the_manager_reads_it(tmp_path, monkeypatch):
    copy_s = {4 << 20: 3.0, 16 << 20: 1.0, 64 << 20: 2.0}
    monkeypatch.setattr(at, "time_copy_run", lambda c: copy_s[c])
    monkeypatch.setattr(at, "time_vadd_tile", lambda v: 1.0 + abs(v - (1 << 18)) * 1e-9)
    monkeypatch.setattr(at.torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(at.torch.cuda, "get_device_name", lambda d: "stand-in")
    path = tmp_path / "tuning.json"
    out = at.run(str(path))
    assert out["choice"] == {"copy_run_bytes": 16 << 20, "vadd_tile": 1 << 18}
    assert json.loads(path.read_text())["step_s"]["copy_run_bytes"] == {str(k): v for k, v in copy_s.items()}
    monkeypatch.setattr(mgr_mod, "TUNING_FILE", str(path))
    assert mgr_mod.tuning() == out["choice"]
    monkeypatch.setattr(mgr_mod, "TUNING_FILE", str(tmp_path / "missing.json"))
    assert mgr_mod.tuning() == {}


def test_committed_table_is_its_own_argmin():
    with open(mgr_mod.TUNING_FILE) as f:
        t = json.load(f)
    for key, timings in t["step_s"].items():
        assert set(timings) == {str(x) for x in (at.COPY_RUNS if key == "copy_run_bytes" else at.VADD_TILES)}
        assert t["choice"][key] == int(min(timings, key=timings.get))
