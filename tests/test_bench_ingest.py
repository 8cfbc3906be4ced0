"""bench.py --ingest-ncu: an ncu launch list (CSV, one row per metric and
launch) is folded into per-kernel totals and per-family DRAM bytes per launch,
stamped with the kernel-source hash (no GPU needed)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

HDR = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
       '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')


def _row(i, name, metric, unit, value):
    return ('"%d","1","python3","h","%s","1","13","(128, 1, 1)","(64, 1, 1)","0","10.3","m","%s","%s","%s"'
            % (i, name, metric, unit, value))


def _launch(i, name, rd_gb, wr_gb, ms):
    return [_row(i, name, "dram__bytes_read.sum", "Gbyte", rd_gb),
            _row(i, name, "dram__bytes_write.sum", "Mbyte", "%.3f" % (wr_gb * 1e3)),
            _row(i, name, "gpu__time_duration.sum", "ms", ms)]


def test_ingest_folds_launches_into_families(tmp_path):
    lines = ["==PROF== Connected to process 1", HDR]
    fa = "void k_plaq_force_a<double>(Geo, const vec2_of<T1>::type *, T1)"
    fb = "void k_plaq_force_b<double>(Geo, const vec2_of<T1>::type *, T1)"
    ap = "void unnamed>::k_cool_apply_df(Geo, float4 *, const df64 *, const df64 *, const CoolState *)"
    i = 0
    for _ in range(2):
        for name, rd, wr, ms in ((fa, 3.0, 2.0, 11.0), (fb, 6.0, 4.0, 15.0), (ap, 0.75, 0.5, 0.35)):
            lines += _launch(i, name, rd, wr, ms)
            i += 1
    lines += _launch(i, fa, "1,000", 0.0, 1.0)  # thousands separators as ncu prints them
    csv_path = tmp_path / "launches.csv"
    csv_path.write_text("\n".join(lines) + "\n")
    out_json = tmp_path / "traffic.json"
    agg, out = bench.ingest_ncu(str(csv_path), str(out_json))
    assert agg["k_plaq_force_a<double>"]["n"] == 3
    assert abs(agg["k_plaq_force_a<double>"]["rd"] - 1006e9) < 1.0
    assert agg["k_cool_apply_df"]["n"] == 2 and abs(agg["k_cool_apply_df"]["ms"] - 0.7) < 1e-12
    # a family sums the per-launch averages of its kernels (force: a then b each step)
    f = out["fp64"]["force"]["bytes_per_launch"]
    assert abs(f - ((1006e9 + 4e9) / 3 + 10e9)) < 1.0
    assert abs(out["df64"]["cool_apply"]["bytes_per_launch"] - 1.25e9) < 1.0
    assert "fp32" not in out  # no kernel of that form in the list
    saved = json.loads(out_json.read_text())
    assert saved["source_hash"] == bench.kernel_source_hash() == out["fp64"]["force"]["source_hash"]


def test_ingest_scales_a_small_capture_to_the_bench_lattice(tmp_path):
    """Per-kernel captures run a smaller lattice; the bytes per launch are
    stored with the captured site count and scaled to the bench's sites."""
    lines = [HDR]
    up = "void k_update_gather<float, 0>(Geo, const vec2_of<T1>::type *, UpdArgs)"
    lines += _launch(0, up, 0.6, 0.1, 1.0)
    a = tmp_path / "a.csv"
    a.write_text("\n".join(lines) + "\n")
    lines = [HDR] + _launch(0, up, 0.8, 0.1, 1.0)  # a second file: its launch IDs restart
    b = tmp_path / "b.csv"
    b.write_text("\n".join(lines) + "\n")
    out_json = tmp_path / "traffic.json"
    agg, out = bench.ingest_ncu([str(a), str(b)], str(out_json), capture_sites=331776)
    assert agg["k_update_gather<float, 0>"]["n"] == 2
    per = out["fp32"]["update"]["bytes_per_launch"]
    assert abs(per - 0.8e9) < 1.0
    scaled = bench.dram_traffic("update", "fp32", 32 ** 4, path=str(out_json))
    assert abs(scaled - 0.8e9 * 32 ** 4 / 331776) < 1.0
