"""bench.py's reference arm (the FP64 CPU oracle on the host cores) prints one
JSON line with the keys the measurement contract names; run on the smallest
grid the three-vesicle workload fits (N = 256), so that it takes seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--N", "256",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["unit"] == line["unit"]
    assert line["config"]["workload"] == "three_vesicles_N256"


def test_source_hash_ignores_comments_and_whitespace():
    """The key of the committed ncu traffic file: what the compiler sees.
    Comment and layout edits keep it; a change of code changes it."""
    import bench
    a = "int f(int x) {  // the sum\n    return x + 1; /* one */\n}\n"
    b = "int f(int x) {\n  // a different comment\n  return x + 1;\n}"
    c = "int f(int x) {\n    return x + 2;\n}\n"
    assert bench.code_text(a) == bench.code_text(b)
    assert bench.code_text(a) != bench.code_text(c)
    assert "//" not in bench.code_text(a) and "/*" not in bench.code_text(a)


def test_phase_roofline_figures():
    """The bench line's roofline: the dominant phase of the 40-pass schedule
    (the one with the longest kernel time among phases that move field
    data), its algorithmic bytes over that time against the peak; with the
    per-kernel times of an N = 2048 FP32 step the stencil + row DCT phase
    (12 passes of 4-byte fields) dominates."""
    import bench
    per_launch = {"k_stencil": 0.0633, "k_rowdct_T": 0.06278, "k_coldct_gram": 0.06363, "k_solve": 0.01434,
                  "k_comb_icolT": 0.06049, "k_irow": 0.0409}
    NN = 2048 * 2048
    r = bench.phase_roofline(per_launch, NN, 4, 6783.8, "measured", "no_such_workload")
    assert bench.STEP_PASSES_MIN_SCHEDULE == 40
    assert r["phase"].startswith("K1") and r["kernels"] == ["k_stencil", "k_rowdct_T"]
    assert r["alg_bytes_per_launch"] == 48 * NN
    assert abs(r["achieved"] - 48 * NN / (0.12608e-3) / 1e9) < 0.1
    assert abs(r["frac"] - r["achieved"] / 6783.8) < 1e-4
    assert r["traffic"] is None and r["traffic_ratio_step"] is None    # no capture for that workload
    # a solve-only slowdown never makes the zero-pass phase dominant
    slow = dict(per_launch, k_solve=10.0)
    assert bench.phase_roofline(slow, NN, 4, 6783.8, "measured", "x")["phase"].startswith("K1")
    assert abs(r["phases"]["K5 inverse row DCT"]["frac"] - 16 * NN / 0.0409e-3 / 1e9 / 6783.8) < 1e-4
