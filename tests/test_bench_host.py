"""Host-side logic of bench.py (no GPU): per-model launch options and the guard on the recorded ncu traffic,
which is reported only while the compositing sources and the launch options match the capture."""
import json

import pytest

import bench


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_2603_02887_gb300 import build

    build.build()  # the options come from ngs_default_options (no GPU needed)


def test_tuned_options_parse_for_every_model():
    opts = bench.parse_options()
    assert set(opts) == set(bench.MODELS)
    for o in opts.values():
        assert (o["tile_w"], o["tile_h"]) in ((8, 8), (16, 16), (16, 32))
        assert o["chunk"] in (o["tile_w"] * o["tile_h"] // 2, o["tile_w"] * o["tile_h"], 2 * o["tile_w"] * o["tile_h"])
        assert o["schedule"] in (0, 1)
        assert bench._options_key(o) in bench.TUNED_OPTIONS
    custom = bench.parse_options("exp=16x32/256/tiles")
    assert list(custom) == ["exp"] and custom["exp"]["schedule"] == 0 and custom["exp"]["tile_h"] == 32


def _record(tmp_path, sha, options, per_model):
    rec = {"code_sha256": sha, "options": options, "command": "ncu ...",
           "kernels": {"composite_bwd": {"bytes_per_launch": per_model}}}
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(rec))
    return str(p)


def _current_sha():
    return bench.code_digest(bench.TRAFFIC_SOURCES)


def test_code_digest_ignores_comments_only(tmp_path, monkeypatch):
    root = tmp_path
    (root / "a.cu").write_text("int f(int x) {\n  return x + 1;  // one\n}\n/* note */\n")
    (root / "b.cu").write_text("int f(int x) { return x + 1; }\n")
    (root / "c.cu").write_text("int f(int x) { return x + 2; }\n")
    (root / "d.cu").write_text("int f(int x) { return x+1; }\n")
    monkeypatch.setattr(bench, "__file__", str(root / "bench.py"))
    dig = {k: bench.code_digest([k + ".cu"]) for k in "abcd"}
    assert dig["a"] == dig["b"]  # comments and layout do not count
    assert dig["c"] != dig["b"]  # code does
    assert dig["d"] != dig["b"]  # nor is whitespace between tokens dropped entirely


@pytest.fixture
def opts():
    return bench.parse_options()


def test_traffic_reported_when_sources_and_options_match(tmp_path, monkeypatch, opts):
    per = {m: 100.0 + 10 * i for i, m in enumerate(bench.MODELS)}
    keys = {m: bench._options_key(o) for m, o in opts.items()}
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", _record(tmp_path, _current_sha(), keys, per))
    value, note = bench.measured_traffic("composite_bwd", opts)
    assert value == pytest.approx(sum(per.values()) / len(per))
    assert note == "ncu ..."


def test_traffic_null_when_sources_changed(tmp_path, monkeypatch, opts):
    keys = {m: bench._options_key(o) for m, o in opts.items()}
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", _record(tmp_path, "0" * 64, keys, {m: 1.0 for m in bench.MODELS}))
    value, note = bench.measured_traffic("composite_bwd", opts)
    assert value is None and "changed" in note


def test_traffic_null_for_other_options_or_kernel(tmp_path, monkeypatch, opts):
    keys = {m: bench._options_key(o) for m, o in opts.items()}
    keys["exp"] = "16x32/1024/tiles"
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", _record(tmp_path, _current_sha(), keys, {m: 1.0 for m in bench.MODELS}))
    assert bench.measured_traffic("composite_bwd", opts)[0] is None
    assert bench.measured_traffic("composite_fwd", opts)[0] is None
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(tmp_path / "absent.json"))
    assert bench.measured_traffic("composite_bwd", opts)[0] is None


def test_record_traffic_from_an_ncu_csv(tmp_path):
    rows = ['"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
            '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"']
    lid = 0
    for i, m in enumerate(bench.MODELS):
        for kind, base in (("composite_forward_kernel", 1000), ("composite_backward_kernel", 5000)):
            name = f"void <unnamed>::{kind}<16, 16, 1, 128, 1>(const float4 *)"
            for metric, val in (("dram__bytes_read.sum", base + i), ("dram__bytes_write.sum", 10 * (i + 1)),
                                ("gpu__time_duration.sum", 7)):
                rows.append(f'"{lid}","1","python","h","{name}","1","7","(128, 1, 1)","(9, 1, 1)","0","10.3",'
                            f'"Command line profiler metrics","{metric}","byte","{val:,}"')
            lid += 1
    csv_path = tmp_path / "launches.csv"
    csv_path.write_text("\n".join(rows) + "\n")
    out = tmp_path / "rec.json"
    rec = bench.record_traffic(str(csv_path), "ncu ...", bench.TUNED_OPTIONS, out=str(out))
    assert json.loads(out.read_text()) == rec
    for i, m in enumerate(bench.MODELS):
        assert rec["kernels"]["composite_fwd"]["bytes_per_launch"][m] == 1000 + i + 10 * (i + 1)
        assert rec["kernels"]["composite_bwd"]["bytes_per_launch"][m] == 5000 + i + 10 * (i + 1)
    assert rec["code_sha256"] == bench.code_digest(bench.TRAFFIC_SOURCES)
    assert set(rec["options"]) == set(bench.MODELS)
