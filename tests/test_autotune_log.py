"""The autotuner's log and the shape -> configuration model read from it (host logic only)."""
import json

from paper_1004_5059_gb300 import autotune


def _rec(nx, ny, cfg, t, velset=2, storage=4, form="tiled"):
    return {"nx": nx, "ny": ny, "velset": velset, "storage": storage, "form": form, "config": cfg,
            "tile": [32, 8 * (cfg + 1), 4], "s_per_step": t}


def test_predict_takes_the_nearest_grids_winner(tmp_path):
    log = tmp_path / "sub" / "log.jsonl"
    log.parent.mkdir()
    recs = [_rec(1024, 1024, 0, 30e-6), _rec(1024, 1024, 1, 27e-6), _rec(1024, 1024, 1, 40e-6),
            _rec(1024, 1024, 1, 26e-6),  # config 1: median 27 us beats config 0's 30
            _rec(4096, 512, 0, 110e-6), _rec(4096, 512, 2, 120e-6),
            _rec(4096, 4096, 3, 400e-6), _rec(4096, 4096, 0, 410e-6),
            _rec(1024, 1024, 3, 1e-6, storage=2),  # another storage: ignored
            _rec(1024, 1024, 2, 1e-6, form="flow")]  # another form: ignored
    with open(log, "w") as fh:
        for r in recs:
            fh.write(json.dumps(r) + "\n")
        fh.write("not json\n")
    got = autotune.read_log(str(log))
    assert len(got) == len(recs)
    p = autotune.predict(got, 1200, 1000, 2, 4, "tiled")
    assert p["config"] == 1 and p["from"] == [1024, 1024]
    p = autotune.predict(got, 8192, 1024, 2, 4, "tiled")  # same aspect as 4096 x 512
    assert p["config"] == 0 and p["from"] == [4096, 512]
    p = autotune.predict(got, 3000, 3000, 2, 4, "tiled")
    assert p["config"] == 3 and p["from"] == [4096, 4096]
    assert autotune.predict(got, 1024, 1024, 2, 4, "flow")["config"] == 2
    assert autotune.predict(got, 64, 64, 1, 4, "tiled") is None
    assert autotune.read_log(str(tmp_path / "missing.jsonl")) == []


def test_default_log_path_honours_the_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("TVLBM_AUTOTUNE_LOG", str(tmp_path / "a.jsonl"))
    assert autotune.default_log_path() == str(tmp_path / "a.jsonl")
    monkeypatch.delenv("TVLBM_AUTOTUNE_LOG")
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    assert autotune.default_log_path() == str(tmp_path / "tvlbm_gb300" / "autotune.jsonl")
