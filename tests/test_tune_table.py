"""The launch-variant tuning table (csrc/st_tune.h) on the CPU.

`st_autotune` times the valid launch variants of a kernel shape and keeps the fastest; this checks the host side
of that: the round reduction (the warm-up round is discarded), the margin that keeps the built-in choice unless a
variant is clearly faster, invalid variants, and lookups while other threads add entries.
"""

import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def test_tune_table_and_selection_rule(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("needs g++")
    exe = tmp_path / "tune_check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-pthread", f"-I{ROOT / 'paper_1912_10082_gb300' / 'csrc'}",
                    str(ROOT / "tests" / "tune_check.cpp"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip().endswith("PASS"), out.stdout
