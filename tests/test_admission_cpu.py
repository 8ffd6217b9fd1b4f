"""The request server's admission policy (csrc/admission.h: per-detector order, two staging
slots, the memory budget, coalescing of consecutive inserts, detectors split among scheduler
threads) on the host alone: tests/admission_policy.cpp is compiled against the library's own
header and checks fixed scenarios and a randomised run step by step."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_admission_policy(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "admission_policy")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Wextra", "-Werror",
                    "-I", os.path.join(ROOT, "paper_1706_06664_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "admission_policy.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok "), out.stdout
    assert int(out.stdout.split()[1]) > 10000  # the randomised run's per-step checks ran
