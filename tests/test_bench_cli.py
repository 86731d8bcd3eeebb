"""bench.py's command line parses and documents every mode (no GPU): the
default line, the batched flames, the accuracy run with its history, the
oracle's legs and the reference arm."""
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def test_bench_help_lists_the_modes():
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--help"], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    for flag in ("--gpus", "--steps", "--warmup", "--impl", "--workload", "--accuracy-steps", "--accuracy-every",
                 "--cpu-legs", "--skip-flames", "--flames-steps", "--skip-adjoint", "--skip-cflame"):
        assert flag in r.stdout, flag
