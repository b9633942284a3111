"""Host-side logic of bench.py (no GPU).

* The traffic figure of a row comes from profiles/traffic.json only while the
  row's kernel sources hash to the value recorded with it; ncu CSV logs are
  read in bytes whatever unit ncu printed.
* The pipelined end-to-end step's row chunks cover each batch exactly once.
* The reference arm (the FP64 oracle on the host cores) prints one JSON line
  with the contract's keys.
"""

import json
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


NCU_CSV = """==PROF== Connected to process 1
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","python","h","k","1","7","(256, 1, 1)","(152, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Gbyte","4.30"
"0","1","python","h","k","1","7","(256, 1, 1)","(152, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","Mbyte","4,290.5"
"1","1","python","h","k","1","7","(256, 1, 1)","(152, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Gbyte","9.00"
"""


def test_ncu_csv_launches_in_bytes(tmp_path):
    p = tmp_path / "log.csv"
    p.write_text(NCU_CSV.replace('"9.00"\n', '"9.00"\n"1","1","python","h","k","1","7","x","y","0",'
                                             '"10.3","s","dram__bytes_write.sum","byte","12"\n'))
    got = bench.ncu_dram_bytes(str(p))
    assert got[0] == (pytest.approx(4.30e9), pytest.approx(4290.5e6))
    assert got[1] == (pytest.approx(9.0e9), pytest.approx(12.0))


def test_traffic_ingest_and_lookup(tmp_path):
    p = tmp_path / "log.csv"
    p.write_text(NCU_CSV.replace('"9.00"\n', '"9.00"\n"1","1","python","h","k","1","7","x","y","0",'
                                             '"10.3","s","dram__bytes_write.sum","byte","12"\n'))
    out = tmp_path / "traffic.json"
    bench.ingest_traffic(str(p), ["chain_W", "c2_n1024_h10_SYM"], str(out), "ncu ... bench.py")
    data = json.loads(out.read_text())
    rows = {e["row"]: e for e in data["entries"]}
    assert rows["chain_W"]["units"] == bench.B_CHAIN
    assert rows["c2_n1024_h10_SYM"]["units"] == 1_048_576
    assert rows["c2_n1024_h10_SYM"]["dram_read_bytes"] == pytest.approx(9.0e9)
    full = 4.30e9 + 4290.5e6
    assert bench.profiled_traffic("chain_W", bench.B_CHAIN, str(out)) == pytest.approx(full)
    assert bench.profiled_traffic("chain_W", bench.B_CHAIN // 2, str(out)) == pytest.approx(full / 2)
    assert bench.profiled_traffic("chain_WT", 10, str(out)) is None       # no figure
    with pytest.raises(ValueError):                                       # too few launches
        bench.ingest_traffic(str(p), ["chain_W", "chain_WT", "chain_SYM"], str(out), "")
    # a figure recorded against other kernel sources is not used
    rows["chain_W"]["sources_sha256"] = "0000000000000000"
    out.write_text(json.dumps({"entries": list(rows.values())}))
    assert bench.profiled_traffic("chain_W", bench.B_CHAIN, str(out)) is None
    assert bench.profiled_traffic("chain_W", 1, str(tmp_path / "absent.json")) is None


def test_committed_traffic_file_parses():
    if not os.path.exists(bench.TRAFFIC_JSON):
        pytest.skip("no traffic figures recorded")
    data = json.load(open(bench.TRAFFIC_JSON))
    for e in data["entries"]:
        assert e["row"] in bench.ALL_ROWS
        assert e["dram_read_bytes"] > 0 and e["dram_write_bytes"] > 0 and e["units"] > 0
        assert re.fullmatch(r"[0-9a-f]{16}", e["sources_sha256"])
        assert "ncu" in e["command"] and "--clock-control none" in e["command"]


def test_c2_rows_have_shapes():
    for nm in bench.C2_ROWS:
        n, h, b, mode = bench.c2_shape(nm)
        assert mode in ("W", "WT", "SYM") and b in (1_048_576, 262_144)


@pytest.mark.parametrize("B", [1, 7, 16, 17, 1000, 262144])
@pytest.mark.parametrize("parts", [1, 3, 16])
def test_row_chunks_partition(B, parts):
    ch = bench.row_chunks(B, parts)
    assert 1 <= len(ch) <= parts
    assert ch[0][0] == 0 and ch[-1][1] == B
    for (a0, a1), (b0, _) in zip(ch, ch[1:]):
        assert a0 < a1 == b0


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--rows", "chain_W,mahalanobis"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["warmup"] >= 3  # the contract's minimum, whatever was asked
    assert "workload" in line["config"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
