"""The autotuner's selection and the committed table, on the CPU (the
timings themselves need a GB300)."""
import json

import paper_1511_07658_gb300.autotune as at
import paper_1511_07658_gb300.manager as mgr_mod


def test_autotune_keeps_the_fastest_setting_and_the_manager_reads_it(tmp_path, monkeypatch):
    copy_s = {4 << 20: 3.0, 16 << 20: 1.0, 64 << 20: 2.0}
    monkeypatch.setattr(at, "time_copy_run", lambda c: copy_s[c])
    monkeypatch.setattr(at, "time_vadd_tile", lambda v: 1.0 + abs(v - (1 << 18)) * 1e-9)
    # the wide form wins two of the three SGEMM workloads, the TMA form the
    # grouped mix, the prefetch all three
    form_s = {("512x512x512", "split3"): 1.0, ("512x512x512", "split3_wide"): 0.9,
              ("512x512x512", "split3_tma"): 1.2,
              ("512x768x512", "split3"): 1.0, ("512x768x512", "split3_wide"): 1.1,
              ("512x768x512", "split3_tma"): 1.05,
              ("2048x2048x2048", "split3"): 1.0, ("2048x2048x2048", "split3_wide"): 0.8,
              ("2048x2048x2048", "split3_tma"): 0.85}
    monkeypatch.setattr(at, "time_sgemm", lambda m, n, k, per_rank=16, path="split3", prefetch=False: (
        form_s[(f"{m}x{n}x{k}", path)] * (0.95 if prefetch else 1.0)))
    monkeypatch.setattr(at, "time_grouped", lambda path: {"split3": 1.0, "split3_wide": 0.9, "split3_tma": 0.85}[path])
    monkeypatch.setattr(at.torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(at.torch.cuda, "get_device_name", lambda d: "stand-in")
    path = tmp_path / "tuning.json"
    out = at.run(str(path))
    assert out["choice"]["copy_run_bytes"] == 16 << 20 and out["choice"]["vadd_tile"] == 1 << 18
    assert out["choice"]["sgemm_form"] == "split3_wide" and out["choice"]["l2_prefetch"] == 1
    assert out["choice"]["sgemm_form_by_class"] == {"512x512x512": "split3_wide", "512x768x512": "split3",
                                                    "2048x2048x2048": "split3_wide", "grouped": "split3_tma"}
    assert set(json.loads(path.read_text())["step_s"]["sgemm_form"]["grouped"]) == set(at.SGEMM_FORMS)
    assert json.loads(path.read_text())["step_s"]["copy_run_bytes"] == {str(k): v for k, v in copy_s.items()}
    monkeypatch.setattr(mgr_mod, "TUNING_FILE", str(path))
    assert mgr_mod.tuning() == out["choice"]
    monkeypatch.setattr(mgr_mod, "TUNING_FILE", str(tmp_path / "missing.json"))
    assert mgr_mod.tuning() == {}


def test_committed_table_is_its_own_argmin():
    with open(mgr_mod.TUNING_FILE) as f:
        t = json.load(f)
    for key in ("copy_run_bytes", "vadd_tile"):
        timings = t["step_s"][key]
        assert set(timings) == {str(x) for x in (at.COPY_RUNS if key == "copy_run_bytes" else at.VADD_TILES)}
        assert t["choice"][key] == int(min(timings, key=timings.get))
    assert {k: t["choice"][k] for k in ("sgemm_form", "sgemm_form_by_class", "l2_prefetch")} == at.choose_sgemm(
        t["step_s"]["sgemm_form"], t["step_s"]["l2_prefetch"])


def test_sgemm_choice_per_class_and_prefetch_needs_every_workload():
    form = {"512x512x512": {"split3": 1.0, "split3_wide": 1.5}, "b": {"split3": 1.0, "split3_wide": 0.5}}
    pf = {"a": {"0": 1.0, "1": 0.9}, "b": {"0": 1.0, "1": 0.99}}
    assert at.choose_sgemm(form, pf) == {"sgemm_form": "split3", "l2_prefetch": 1,
                                         "sgemm_form_by_class": {"512x512x512": "split3", "b": "split3_wide"}}
    form["512x512x512"]["split3_wide"] = 0.7
    pf["b"]["1"] = 1.01
    out = at.choose_sgemm(form, pf)
    assert out["sgemm_form"] == "split3_wide" and out["l2_prefetch"] == 0
