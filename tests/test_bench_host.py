"""Host-side logic of bench.py (no GPU).

* The traffic figure of the roofline object comes from a committed ncu summary
  only while the kernel sources hash to the value recorded beside it.
* The committed summaries carry parseable per-vector traffic lines.
* The pipelined end-to-end step's row chunks cover each batch exactly once.
* The reference arm (the FP64 oracle on the host cores) prints one JSON line
  with the contract's keys.
"""

import hashlib
import json
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def test_profiled_traffic_lookup(tmp_path):
    sha = _sha(bench.KERNEL_SOURCES)
    p = tmp_path / "summary.md"
    p.write_text("text\n"
                 f"TRAFFIC mode=W bytes_per_vector=100.5 sources_sha256={sha}\n"
                 "TRAFFIC mode=WT bytes_per_vector=7 sources_sha256=0000000000000000\n")
    assert bench.profiled_traffic("W", 10, path=str(p)) == pytest.approx(1005.0)
    assert bench.profiled_traffic("WT", 10, path=str(p)) is None      # stale capture
    assert bench.profiled_traffic("SYM", 10, path=str(p)) is None     # no line for the mode
    assert bench.profiled_traffic("W", 10, path=str(tmp_path / "absent.md")) is None


@pytest.mark.parametrize("path,modes", [(bench.TRAFFIC_FILE, ("W", "WT", "SYM")),
                                        (bench.BATCHED_TRAFFIC_FILE, ("C5",))])
def test_committed_traffic_lines_parse(path, modes):
    lines = [ln for ln in open(path) if ln.startswith("TRAFFIC ")]
    seen = set()
    for ln in lines:
        kv = dict(t.split("=", 1) for t in ln.split()[1:])
        assert float(kv["bytes_per_vector"]) > 0
        assert re.fullmatch(r"[0-9a-f]{16}", kv["sources_sha256"])
        seen.add(kv["mode"])
    assert set(modes) <= seen


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
