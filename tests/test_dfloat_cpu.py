"""The double-float helpers of the FP32 delay kernel (paper_1410_3677_gb300/csrc/
dfloat.cuh), compiled for the host with contraction off and checked against
exact rational arithmetic on seeded inputs: the two-sum is exact, the product
and the sum of pairs are within their error bounds, and the floor split of a
pair returns the exact integer part and a fraction in [0, 1] within a float
rounding."""
import os
import shutil
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1410_3677_gb300", "csrc", "dfloat.cuh")
CUDA_INC = "/usr/local/cuda/include"

PROG = r"""
#include <cstdio>
#include "dfloat.cuh"
using namespace fstat;
int main() {
    char op[8];
    float a, b, c, d;
    while (scanf("%7s %a %a %a %a", op, &a, &b, &c, &d) == 5) {
        DF r{0.f, 0.f};
        const DF x{a, b}, y{c, d};
        if (op[0] == 's') r = df_two_sum(a, c);
        else if (op[0] == 'a') r = df_add(x, y);
        else if (op[0] == 'm') r = df_mul(x, y);
        else { float f; const float i = df_split_floor(x, &f); r = DF{i, f}; }
        printf("%a %a\n", r.hi, r.lo);
    }
}
"""


@pytest.fixture(scope="module")
def prog():
    cxx = shutil.which("g++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "df.cpp")
    with open(src, "w") as fh:
        fh.write(PROG)
    exe = os.path.join(d, "df")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", f"-I{os.path.dirname(HDR)}",
                    f"-I{CUDA_INC}", src, "-o", exe], check=True, capture_output=True)
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def run(exe, rows):
    inp = "".join(f"{op} {float(a).hex()} {float(b).hex()} {float(c).hex()} {float(d).hex()}\n"
                  for op, a, b, c, d in rows)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
    return [(float.fromhex(out[2 * i]), float.fromhex(out[2 * i + 1])) for i in range(len(rows))]


def pair(rng, scale):
    """A normalised double-float pair around `scale`: hi a float, lo below half its ulp."""
    x = rng.uniform(-1, 1) * scale
    hi = float(np.float32(x))
    lo = float(np.float32(x - hi))
    return hi, lo


def F(*vals):
    return sum((Fraction(v) for v in vals), Fraction(0))


def test_two_sum_is_exact(prog):
    rng = np.random.default_rng(1)
    rows = []
    for _ in range(2000):
        a = float(np.float32(rng.uniform(-1, 1) * 10 ** rng.uniform(-3, 3)))
        c = float(np.float32(rng.uniform(-1, 1) * 10 ** rng.uniform(-3, 3)))
        rows.append(("s", a, 0.0, c, 0.0))
    for (op, a, _, c, _), (s, e) in zip(rows, run(prog, rows)):
        assert F(s, e) == F(a, c)
        assert s == float(np.float32(a + c))


@pytest.mark.parametrize("op,bound", [("a", 2.0 ** -44), ("m", 2.0 ** -44)])
def test_sum_and_product_bounds(prog, op, bound):
    rng = np.random.default_rng(2 if op == "a" else 3)
    rows = []
    for _ in range(2000):
        x = pair(rng, 10 ** rng.uniform(-2, 3))
        y = pair(rng, 10 ** rng.uniform(-2, 3))
        if op == "a" and rng.uniform() < 0.3:          # near cancellation
            y = (-x[0] * (1 + 2.0 ** -20), -x[1])
            y = (float(np.float32(y[0])), float(np.float32(y[1])))
        rows.append((op, x[0], x[1], y[0], y[1]))
    for (_, a, b, c, d), (h, l) in zip(rows, run(prog, rows)):
        exact = F(a, b) + F(c, d) if op == "a" else F(a, b) * F(c, d)
        got = F(h, l)
        if op == "a":
            # relative to the larger operand: cancellation cannot be beaten
            ref = max(abs(F(a, b)), abs(F(c, d)))
        else:
            ref = abs(exact)
        assert abs(got - exact) <= Fraction(bound) * ref + Fraction(2.0 ** -149)
        assert abs(l) <= abs(h) * 2.0 ** -23 or h == 0.0     # normalised


def test_floor_split(prog):
    rng = np.random.default_rng(4)
    rows = []
    for _ in range(2000):
        x = pair(rng, 10 ** rng.uniform(-1, 5))
        if rng.uniform() < 0.2:                      # just below or above an integer
            k = float(np.float32(np.round(x[0])))
            x = (k, float(np.float32(rng.choice([-1, 1]) * 10 ** rng.uniform(-12, -6))))
        rows.append(("f", x[0], x[1], 0.0, 0.0))
    for (_, a, b, _, _), (i, f) in zip(rows, run(prog, rows)):
        exact = F(a, b)
        assert i == int(i)
        assert 0.0 <= f <= 1.0
        assert abs(F(i) + F(f) - exact) <= Fraction(2.0 ** -24)
