"""The integer-pipe conversions between float and double used by the mixed path
(paper_2401_03008_gb300/csrc/echo_convert.cuh), compiled by the host compiler from
the same source and checked against the host's IEEE conversions: every float
below 2^24 and every fifth bit pattern above for widening, 45 million doubles of
every class (random bits, values across the float range, exact ties) for
round-to-nearest-even narrowing."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_conversions_match_ieee(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "convert_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I",
                    os.path.join(ROOT, "paper_2401_03008_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "convert_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 mismatches; narrowing" in r.stdout and r.stdout.strip().endswith("0 mismatches")
