"""The autotuner's selection and the committed table, on the CPU (the
timings themselves need a GB300)."""
import json

import paper_1511_07658_gb300.autotune as at
import paper_1511_07658_gb300.manager as mgr_mod


def test_autotune_keeps_the_fastest_setting_and_the_manager_reads_it(tmp_path, monkeypatch):
    copy_s = {4 << 20: 3.0, 16 << 20: 1.0, 64 << 20: 2.0}
    monkeypatch.setattr(at, "time_copy_run", lambda c: copy_s[c])
    monkeypatch.setattr(at, "time_vadd_tile", lambda v: 1.0 + abs(v - (1 << 18)) * 1e-9)
    # per-tile cost 1.0 for 256-wide tiles, 0.6 for 128, 0.8 for 192: step time = tiles x cost
    tile_cost = {128: 0.6, 192: 0.8, 256: 1.0}
    monkeypatch.setattr(at, "time_sgemm", lambda m, n, k, per_rank=16, path="split3", tile_n=None: (
        16 * per_rank * (m // 128) * (n // (tile_n or 256)) * tile_cost[tile_n or 256]
        * (1.5 if path == "split3_wide" else 1.0)))
    monkeypatch.setattr(at.torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(at.torch.cuda, "get_device_name", lambda d: "stand-in")
    path = tmp_path / "tuning.json"
    out = at.run(str(path))
    assert out["choice"]["copy_run_bytes"] == 16 << 20 and out["choice"]["vadd_tile"] == 1 << 18
    cost = out["choice"]["sgemm_tile_cost"]
    assert {w: round(c, 9) for w, c in cost.items()} == {"128": 0.6, "192": 0.8, "256": 1.0}
    assert out["choice"]["sgemm_form"] == "split3"
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
    assert t["choice"]["sgemm_tile_cost"] == at.tile_costs(t["step_s"]["sgemm_tile_n"])
    f = t["step_s"]["sgemm_form"]
    wide = f["split3_wide 512x768x512"] < f["split3 512x768x512"] and f["split3_wide 512^3"] < f["split3 512^3"]
    assert t["choice"]["sgemm_form"] == ("split3_wide" if wide else "split3")


def test_tile_width_rule_hand_cases():
    # ceil(n / w) * cost(w), the wider on ties
    even = {"128": 0.5, "192": 0.75, "256": 1.0}  # cost proportional to width: padding decides
    assert at.choose_width(256, even) == 256
    assert at.choose_width(128, even) == 128
    assert at.choose_width(192, even) == 192
    assert at.choose_width(384, even) == 192  # 2 x 0.75 = 3 x 0.5 = 1.5 < 2 x 1.0: 192 wins the tie
    assert at.choose_width(320, even) == 192  # 2 x 0.75 = 1.5 against 3 x 0.5 and 2 x 1.0
    assert at.choose_width(512, even) == 256
    flat = {"128": 1.0, "192": 1.0, "256": 1.0}  # every tile costs the same: fewest tiles
    for n in range(1, 2049, 7):
        assert at.choose_width(n, flat) == 256 or -(-n // at.choose_width(n, flat)) < -(-n // 256)
    steep = {"128": 0.9, "192": 0.95, "256": 1.0}  # narrow tiles barely cheaper: 256 unless padding is large
    assert at.choose_width(2048, steep) == 256
    assert at.choose_width(129, steep) == 192


def test_tile_costs_from_unpadded_steps():
    # 256 tasks of 512 x 768: 4 row tiles x 6, 4 and 3 column tiles
    steps = {"128": 256 * 4 * 6 * 2.0, "192": 256 * 4 * 4 * 3.0, "256": 256 * 4 * 3 * 4.0}
    assert at.tile_costs(steps) == {"128": 0.5, "192": 0.75, "256": 1.0}
