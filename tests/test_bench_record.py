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


class _Info:
    """The fields of gm_info that the roofline record reads (300 x 250 x 60 gravity, real even spectra)."""
    n_model, n_data = 360 * 300 * 60, 300 * 250
    fft_nx, fft_ny, spec_nx, nz = 672, 560, 337, 60
    spectrum_real = 1
    spectrum_bytes = 4 * 337 * 60 * 281


def test_roofline_picks_the_roof_the_intensity_selects():
    import math

    import bench

    inf = _Info()
    # column kernel dominant: ~25 flop per algorithmic byte, above the ridge of 80.5 TFLOP/s and
    # 6.79 TB/s (~11.9 flop/B), so the ALU roof bounds it
    kt = {"fwd_rows_r2c": (10, 0.25), "fwd_cols_mac": (10, 0.35), "tr_cols": (10, 0.30)}
    r = bench.roofline_of(kt, inf, 0.104, 6789.6, "measured")
    assert r["bound"] == "alu" and r["kernel"] == "fwd_cols_mac" and r["unit"] == "TFLOP/s"
    tf = 5.0 * 560 * math.log2(560)
    flops = 337 * 60 * tf + 4.0 * 337 * 60 * 560 + 337 * tf
    assert math.isclose(r["achieved"], flops / 35e-6 / 1e12, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["achieved"] / bench.FP32_PEAK_TFLOPS, rel_tol=1e-12)
    assert math.isclose(r["ridge_flop_per_byte"], bench.FP32_PEAK_TFLOPS * 1e3 / 6789.6, rel_tol=1e-12)
    assert r["intensity_flop_per_byte"] > r["ridge_flop_per_byte"]
    assert math.isclose(r["hbm_view"]["achieved_gbs"], inf.spectrum_bytes / 35e-6 / 1e9, rel_tol=1e-12)
    assert math.isclose(sum(r["kernel_share"].values()), 1.0, rel_tol=1e-12)
    # a row kernel dominant: no flop count, the HBM roof
    kt = {"fwd_rows_r2c": (10, 0.50), "fwd_cols_mac": (10, 0.35)}
    r = bench.roofline_of(kt, inf, 0.104, 6789.6, "measured")
    assert r["bound"] == "hbm" and r["kernel"] == "fwd_rows_r2c" and r["unit"] == "GB/s"
    assert math.isclose(r["achieved"], 4 * inf.n_model / 50e-6 / 1e9, rel_tol=1e-12)
    assert r["alu_view"] is None and r["traffic"] is None


def test_roofline_with_complex_spectra_stays_below_the_ridge():
    import bench

    class Complex(_Info):
        spectrum_real = 0
        spectrum_bytes = 8 * 337 * 60 * 560

    r = bench.roofline_of({"fwd_cols_mac": (4, 0.16)}, Complex(), 0.2, 6789.6, "measured")
    # the complex spectrum moves 8x the bytes of the real quarter form: ~7 flop/B, under the ridge
    assert r["bound"] == "hbm" and r["intensity_flop_per_byte"] < r["ridge_flop_per_byte"]
    assert r["alu_view"]["kernel"] == "fwd_cols_mac"
