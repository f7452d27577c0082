"""The JSON-lines result record of bench.py (host logic only)."""
import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_emit_prints_the_line_and_appends_a_record(tmp_path, capsys):
    import bench

    path = tmp_path / "runs.jsonl"
    line = {"metric": "m", "value": 1.5, "unit": "applies/s", "config": {"workload": "w"}}
    for k in range(2):
        bench.emit(dict(line, value=1.5 + k), argparse.Namespace(jsonl=str(path)))
    printed = [json.loads(x) for x in capsys.readouterr().out.splitlines()]
    assert [p["value"] for p in printed] == [1.5, 2.5] and all("record" not in p for p in printed)
    recs = [json.loads(x) for x in path.read_text().splitlines()]
    assert [r["value"] for r in recs] == [1.5, 2.5]
    for r in recs:
        assert r["config"] == {"workload": "w"}
        assert set(r["record"]) == {"time_utc", "argv", "gpu", "host_cores"}
        assert r["record"]["host_cores"] == os.cpu_count()


def test_emit_without_a_path_writes_no_file(tmp_path, capsys, monkeypatch):
    import bench

    monkeypatch.chdir(tmp_path)
    bench.emit({"value": 1}, argparse.Namespace(jsonl=None))
    assert json.loads(capsys.readouterr().out) == {"value": 1}
    assert list(tmp_path.iterdir()) == []
