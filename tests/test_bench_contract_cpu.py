"""bench.py's reference arm (the FP64 oracle timed on the host cores) prints one JSON line with
the keys the benchmark contract asks for; a tiny sample of the water workload keeps it to a few
seconds on the CPU."""
import json
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1", "--config", "0",
                        "--cpu-seconds", "0.5"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, str(ROOT))
    import bench

    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    for key in ("value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "points/s" and d["steps"] == 2 and d["warmup"] == 1
    assert d["higher_is_better"] is True and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["ms_per_step_kind"].startswith("extrapolated")
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_h_tile_area_against_brute_force():
    """The issued/useful MMA area that bench.py reports for the split H contraction: closed form
    against a cell-by-cell count of the 128 x TN tiles that reach the upper triangle."""
    sys.path.insert(0, str(ROOT))
    import numpy as np

    import bench

    rng = np.random.Generator(np.random.PCG64(8))
    n = rng.integers(0, 400, 40)
    k = 4 * rng.integers(1, 20, 40) * 16
    tw = rng.choice([32, 48], 40)
    issued = useful = 0
    for nb, kk, tn in zip(n, k, tw):
        for i0 in range(0, nb, 128):
            for j0 in range(0, nb, tn):
                cells = [(i, j) for i in range(i0, i0 + 128) for j in range(j0, j0 + tn)]
                if any(i <= j and i < nb and j < nb for i, j in cells):
                    issued += 128 * tn * kk
                    useful += kk * sum(1 for i, j in cells if i <= j and j < nb)
    assert bench.h_tile_area(n, k, tw) == (issued, useful)
