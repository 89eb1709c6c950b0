"""The bench's reference arm (the CPU oracle timed on the default workload)
prints one JSON line with the keys the measurement contract needs (CPU only;
about half a minute: the 1.7e9 tids are generated in parallel)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "bern_m4m_n8192_p5"


def test_merge_micro_small():
    # the Sec. IV-B merging experiment at a small size: the count is exact and
    # the rates are positive
    sys.path.insert(0, ROOT)
    import bench
    import datagen
    import numpy as np
    r = bench.merge_micro(n=1 << 16, repeats=1)
    a, b = datagen.sorted_u32(1 << 16, 1), datagen.sorted_u32(1 << 16, 2)
    assert r["common"] == len(set(a.tolist()) & set(b.tolist()))
    assert np.all(np.diff(a.astype(np.int64)) > 0)
    assert r["elements_per_s_1core"] > 0 and r["elements_per_s_all_cores"] > 0 and r["cores"] >= 1
