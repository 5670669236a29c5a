"""The FP64/FP32 bit-pattern conversions of the kernels (csrc/bits.cuh),
compiled as plain C++ on the CPU and checked against the host's own
conversions: f2d_exact bit for bit against the exact FP32 -> FP64
conversion, d2f_trunc against truncation toward zero (from the rounded
conversion and nextafter) with its documented range handling, and mag_bits
against the order of |x|."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bit_conversions_match_host_references(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "bits_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I",
                    os.path.join(ROOT, "paper_1906_01632_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "bits_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout
