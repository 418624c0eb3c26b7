"""The double-single arithmetic of the preprocessing kernels (csrc/dsfloat.cuh) against exact
rational arithmetic: every operation's result is within 2^-44 relative of the exact sum, product,
reciprocal or square root of its double-single operands, and is renormalised (|lo| at most half an
ulp of hi). The header is compiled for the host with the system C++ compiler."""
import os
import shutil
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2301_12796_gb300", "csrc")
BOUND = Fraction(1, 2 ** 44)


def _val(h, l):
    return Fraction(float.fromhex(h)) + Fraction(float.fromhex(l))


def _renormalised(h, l):
    hi, lo = float.fromhex(h), float.fromhex(l)
    if hi == 0.0:
        return lo == 0.0
    import numpy as np
    return abs(lo) <= np.spacing(np.float32(abs(hi))) / 2


@pytest.fixture(scope="module")
def lines(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("ds") / "dsfloat_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "dsfloat_check.cpp"), "-o", exe],
                   check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return [ln.split() for ln in out.splitlines()]


def test_double_single_operations_within_bound(lines):
    worst = {}
    for t in lines:
        op = t[0]
        if op == "add":
            exact, got = _val(t[1], t[2]) + _val(t[3], t[4]), t[5:7]
        elif op == "mul":
            exact, got = _val(t[1], t[2]) * _val(t[3], t[4]), t[5:7]
        elif op == "mulf":
            exact, got = _val(t[1], t[2]) * Fraction(float.fromhex(t[3])), t[4:6]
        elif op == "recip":
            exact, got = 1 / _val(t[1], t[2]), t[3:5]
        else:  # sqrt: compare the square of the result with the operand, |d(y^2)| = 2|y dy|
            x, y = _val(t[1], t[2]), _val(t[3], t[4])
            rel = abs(y * y - x) / (2 * x)
            worst[op] = max(worst.get(op, 0), rel)
            assert rel <= BOUND * (1 + BOUND), t
            assert _renormalised(t[3], t[4]), t
            continue
        g = _val(*got)
        rel = abs(g - exact) / abs(exact) if exact != 0 else abs(g)
        worst[op] = max(worst.get(op, 0), rel)
        assert rel <= BOUND, (op, t, float(rel))
        assert _renormalised(*got), (op, t)
    print({k: f"{float(v):.2e}" for k, v in worst.items()})
    assert set(worst) == {"add", "mul", "mulf", "sqrt", "recip"}
