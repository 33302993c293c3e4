"""The workload files (workloads/<name>.json) describe the workloads of bgk_inputs.CONFIGS
parameter for parameter, and an edited copy selects a variant through config()."""
import json
import os

import pytest

import bgk_inputs as bi


@pytest.mark.parametrize("name", sorted(bi.CONFIGS))
def test_workload_file_matches_the_workload(name):
    path = os.path.join(bi.WORKLOAD_DIR, name + ".json")
    got, over = bi.workload_from_file(path)
    assert got == name and over == {}
    with open(path) as fh:
        assert json.load(fh)["params"] == bi.CONFIGS[name]


def test_edited_workload_file_gives_its_variant(tmp_path):
    with open(os.path.join(bi.WORKLOAD_DIR, "cavity2d_ale_n201_v32_f32.json")) as fh:
        d = json.load(fh)
    d["params"]["kn"] = 0.01
    d["params"]["storage"] = "bf16"
    path = tmp_path / "variant.json"
    path.write_text(json.dumps(d))
    name, over = bi.workload_from_file(str(path))
    assert name == "cavity2d_ale_n201_v32_f32" and over == {"kn": 0.01, "storage": "bf16"}
    p = bi.config(name, **over)
    assert p["kn"] == 0.01 and p["storage"] == "bf16" and p["n"] == 201


def test_bad_workload_files_are_refused(tmp_path):
    bad_name = tmp_path / "a.json"
    bad_name.write_text(json.dumps({"workload": "nope", "params": {}}))
    with pytest.raises(ValueError):
        bi.workload_from_file(str(bad_name))
    bad_key = tmp_path / "b.json"
    bad_key.write_text(json.dumps({"workload": "cavity2d_n41_v16_f64", "params": {"knudsen": 1.0}}))
    with pytest.raises(ValueError):
        bi.workload_from_file(str(bad_key))


def test_bench_takes_a_workload_file(tmp_path):
    # the reference arm (CPU only) of bench.py on a small variant given as a file
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(bi.WORKLOAD_DIR, "cavity2d_n41_v16_f64.json")) as fh:
        d = json.load(fh)
    d["params"]["kn"] = 1.0
    path = tmp_path / "small.json"
    path.write_text(json.dumps(d))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config-file", str(path), "--n", "13",
                        "--steps", "1", "--warmup", "1"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["config"]["workload"] == "cavity2d_n41_v16_f64"
    assert line["config"]["kn"] == 1.0 and line["config"]["points"] == 13 * 13
