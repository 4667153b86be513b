"""The double-float arithmetic of the mixed-precision band (csrc/dfloat.cuh), built for the host and
checked against exact rational arithmetic (sums, products, reciprocals) and 60-digit 1/sqrt."""
import ctypes as C
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1209_6038_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("dfloat") / "libdfh.so")
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-I", CSRC, "-o", out,
                    os.path.join(HERE, "dfloat_host.cpp")], check=True)
    L = C.CDLL(out)
    fp = C.POINTER(C.c_float)
    L.dfh_from_double.argtypes = [C.c_double, fp]
    for n in ("dfh_add", "dfh_sub", "dfh_mul"):
        getattr(L, n).argtypes = [C.c_float] * 4 + [fp]
    L.dfh_mulf.argtypes = [C.c_float] * 3 + [fp]
    L.dfh_rcp.argtypes = [C.c_float] * 2 + [fp]
    L.dfh_rsqrt.argtypes = [C.c_float] * 2 + [fp]
    return L


def call(f, *args):
    o = (C.c_float * 2)()
    f(*args, o)
    return float(o[0]), float(o[1])


def exact(p):
    return Fraction(p[0]) + Fraction(p[1])


def sample(lib, rng, n, positive=False):
    mag = 2.0 ** rng.uniform(-20, 4, n)
    sgn = np.ones(n) if positive else np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    return [call(lib.dfh_from_double, float(v)) for v in sgn * mag * rng.uniform(1, 2, n)]


def normalised(p):
    return abs(p[1]) <= abs(p[0]) * 2.0 ** -24


def test_split_of_a_double_keeps_48_bits(lib):
    rng = np.random.default_rng(1)
    for d in rng.normal(size=500) * 2.0 ** rng.uniform(-30, 30, 500):
        p = call(lib.dfh_from_double, float(d))
        assert normalised(p)
        assert abs(exact(p) - Fraction(float(d))) <= abs(Fraction(float(d))) * Fraction(2) ** -48


@pytest.mark.parametrize("op", ["add", "sub", "mul"])
def test_sum_difference_product(lib, op):
    rng = np.random.default_rng({"add": 2, "sub": 3, "mul": 4}[op])
    a, b = sample(lib, rng, 1500), sample(lib, rng, 1500)
    # near-cancelling pairs as well: b = -a (1 + 2^-k)
    for k in range(1, 40, 3):
        x = a[k]
        a.append(x)
        b.append(call(lib.dfh_from_double, -float(exact(x)) * (1 + 2.0 ** -k)))
    f = getattr(lib, "dfh_" + op)
    for x, y in zip(a, b):
        got = call(f, *x, *y)
        X, Y = exact(x), exact(y)
        if op == "mul":
            ref, scale = X * Y, abs(X * Y)
            bound = scale * Fraction(3) * Fraction(2) ** -48
        else:
            ref = X + Y if op == "add" else X - Y
            scale = max(abs(X), abs(Y))
            bound = scale * Fraction(3) * Fraction(2) ** -48
        assert abs(exact(got) - ref) <= bound, (op, x, y, got)
        assert normalised(got) or got[0] == 0.0


def test_product_with_a_float(lib):
    rng = np.random.default_rng(5)
    a = sample(lib, rng, 1000)
    b = (rng.uniform(-4, 4, 1000)).astype(np.float32)
    for x, y in zip(a, b):
        got = call(lib.dfh_mulf, *x, float(y))
        ref = exact(x) * Fraction(float(y))
        assert abs(exact(got) - ref) <= abs(ref) * Fraction(3) * Fraction(2) ** -48


def test_reciprocal(lib):
    rng = np.random.default_rng(6)
    for x in sample(lib, rng, 1500):
        got = call(lib.dfh_rcp, *x)
        ref = 1 / exact(x)
        assert abs(exact(got) - ref) <= abs(ref) * Fraction(2) ** -45, (x, got)


def test_reciprocal_square_root(lib):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    rng = np.random.default_rng(7)
    for x in sample(lib, rng, 1500, positive=True):
        got = call(lib.dfh_rsqrt, *x)
        X = exact(x)
        ref = 1 / mp.sqrt(mp.mpf(X.numerator) / X.denominator)
        g = mp.mpf(got[0]) + mp.mpf(got[1])
        assert abs(g - ref) <= abs(ref) * mp.mpf(2) ** -44, (x, got)
