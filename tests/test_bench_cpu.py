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
