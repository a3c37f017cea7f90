"""The library's integer-only double operations (csrc/bc_rn.h: u53 -> double,
RN(s*y), RN(1+x), RN(x/s)) against the host's IEEE-754 arithmetic, bit for bit,
on a few million operands (tests/rn_check.cpp, compiled here with g++)."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_integer_double_ops_match_ieee():
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no C++ compiler")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "rn_check")
        subprocess.check_call([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-o", exe,
                               os.path.join(HERE, "rn_check.cpp")])
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
