"""The double-float operations of the FP64-class stage against exact arithmetic.

The header paper_2510_07539_gb300/csrc/hsgn_dfloat.cuh is plain C++ outside
nvcc; tests/dfloat_ops.cpp exports its operations for the host (g++,
-ffp-contract=off) and every result is compared with the exact rational value
of the operation on the same float pairs (fractions.Fraction). Bounds: the
error-free transformations exactly (TwoSum inside a sum, the unrenormalised
forms equal in value to the renormalised ones), sums within 2^-46 of
|a| + |b|, the cancellation-accurate sum within 2^-45 of |a + b|, products,
reciprocals and quotients within 2^-44 relative, h^2 - m within 2^-45 of h^2 - m
plus 2^-70 h^2. The device's reciprocal (the hardware approximation refined once)
differs from the host's rounded quotient; the GPU parity tests cover it.
No GPU needed."""
import ctypes
import os
import random
import shutil
import subprocess
from fractions import Fraction as F

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
N = 4000


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    so = tmp_path_factory.mktemp("dfo") / "libdfo.so"
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-o", str(so),
                    os.path.join(HERE, "dfloat_ops.cpp")], check=True, capture_output=True,
                   timeout=300)
    L = ctypes.CDLL(str(so))
    f, P = ctypes.c_float, ctypes.POINTER(ctypes.c_float)
    for name, nf in (("dfo_add", 4), ("dfo_add_u", 4), ("dfo_add_acc", 4), ("dfo_add_f", 3),
                     ("dfo_mul", 4), ("dfo_mul_f", 3), ("dfo_fma", 6), ("dfo_fma_u", 6),
                     ("dfo_rcp", 2), ("dfo_div", 4), ("dfo_sq_minus", 4)):
        getattr(L, name).argtypes = [f] * nf + [P]
        getattr(L, name).restype = None
    L.dfo_of.argtypes = [ctypes.c_double, P]
    L.dfo_of.restype = None
    return L


def call(L, name, *args):
    o = (ctypes.c_float * 2)()
    getattr(L, name)(*[float(a) for a in args], o)
    return float(o[0]), float(o[1])


def pair(L, x):
    o = (ctypes.c_float * 2)()
    L.dfo_of(float(x), o)
    return float(o[0]), float(o[1])


def val(p):
    return F(p[0]) + F(p[1])


def rnd(rng, lo=-3.0, hi=3.0):
    # a double with a random sign and a magnitude spread over a few binades
    return rng.choice((-1.0, 1.0)) * rng.uniform(0.5, 2.0) * 2.0 ** rng.randint(int(lo), int(hi))


def test_pairs_of_doubles_are_normalised_and_near(lib):
    rng = random.Random(1)
    for _ in range(N):
        x = rnd(rng, -20, 20)
        p = pair(lib, x)
        assert abs(p[1]) <= abs(np.spacing(np.float32(p[0]))) / 2
        assert abs(val(p) - F(x)) <= F(abs(x)) * F(2) ** -48


def test_sums(lib):
    rng = random.Random(2)
    for _ in range(N):
        a, b = pair(lib, rnd(rng)), pair(lib, rnd(rng))
        exact = val(a) + val(b)
        r = call(lib, "dfo_add", *a, *b)
        ru = call(lib, "dfo_add_u", *a, *b)
        # the renormalisation is error-free: both forms hold the same value
        assert val(ru) == val(r)
        assert abs(val(r) - exact) <= (abs(val(a)) + abs(val(b))) * F(2) ** -46
        assert abs(r[1]) <= abs(np.spacing(np.float32(r[0]))) / 2 or r[0] == 0.0


def test_accurate_sum_of_close_values(lib):
    rng = random.Random(3)
    for _ in range(N):
        x = rnd(rng)
        a = pair(lib, x)
        b = pair(lib, -x * (1.0 + rng.uniform(-1e-6, 1e-6)))
        exact = val(a) + val(b)
        r = call(lib, "dfo_add_acc", *a, *b)
        assert abs(val(r) - exact) <= abs(exact) * F(2) ** -45
        # the plain sum carries the operands' rounding instead
        assert abs(val(call(lib, "dfo_add", *a, *b)) - exact) <= (abs(val(a)) + abs(val(b))) * F(2) ** -46


def test_products_fma_and_single_float_operands(lib):
    rng = random.Random(4)
    for _ in range(N):
        a, b, c = pair(lib, rnd(rng)), pair(lib, rnd(rng)), pair(lib, rnd(rng))
        r = call(lib, "dfo_mul", *a, *b)
        assert abs(val(r) - val(a) * val(b)) <= abs(val(a) * val(b)) * F(2) ** -44
        x = float(np.float32(rnd(rng)))
        r = call(lib, "dfo_mul_f", *a, x)
        assert abs(val(r) - val(a) * F(x)) <= abs(val(a) * F(x)) * F(2) ** -44
        r = call(lib, "dfo_add_f", *a, x)
        assert abs(val(r) - (val(a) + F(x))) <= (abs(val(a)) + abs(F(x))) * F(2) ** -46
        exact = val(a) * val(b) + val(c)
        r = call(lib, "dfo_fma", *a, *b, *c)
        ru = call(lib, "dfo_fma_u", *a, *b, *c)
        assert val(ru) == val(r)
        assert abs(val(r) - exact) <= (abs(val(a) * val(b)) + abs(val(c))) * F(2) ** -44


def test_reciprocal_and_quotient(lib):
    rng = random.Random(5)
    for _ in range(N):
        a, b = pair(lib, rnd(rng)), pair(lib, rnd(rng))
        r = call(lib, "dfo_rcp", *b)
        assert abs(val(r) * val(b) - 1) <= F(2) ** -44
        q = call(lib, "dfo_div", *a, *b)
        assert abs(val(q) - val(a) / val(b)) <= abs(val(a) / val(b)) * F(2) ** -44


def test_square_minus_close_value(lib):
    # h^2 - m for m within a factor 2 of h^2 (the relaxation residual): exact
    # products and Sterbenz differences leave an error of the result's order
    rng = random.Random(6)
    for _ in range(N):
        h = pair(lib, rng.uniform(0.2, 3.0))
        m = pair(lib, float(val(h) ** 2) * (1.0 + rng.uniform(-0.4, 0.4) * 10.0 ** -rng.randint(0, 9)))
        exact = val(h) ** 2 - val(m)
        r = call(lib, "dfo_sq_minus", *h, *m)
        assert abs(val(r) - exact) <= abs(exact) * F(2) ** -45 + val(h) ** 2 * F(2) ** -70


def test_unrenormalised_inputs_keep_the_operand_scale_accuracy(lib):
    # a sum whose high parts cancel leaves a pair whose low part dominates;
    # a product or quotient of it stays within 2^-44 of the operands' scale
    # (the absolute accuracy that the renormalised sum's value has as well), and
    # a later sum of such a result adds an error of the same scale (2^-46 of the
    # magnitudes the chain went through, not only of its last operands)
    rng = random.Random(7)
    for _ in range(N):
        x = rnd(rng)
        a = pair(lib, x)
        b = pair(lib, -x * (1.0 + rng.uniform(-1e-6, 1e-6)))
        s = call(lib, "dfo_add_u", *a, *b)
        scale = abs(val(a)) + abs(val(b))
        c = pair(lib, rnd(rng))
        p = call(lib, "dfo_mul", *s, *c)
        assert abs(val(p) - val(s) * val(c)) <= scale * abs(val(c)) * F(2) ** -44
        den = pair(lib, 1.0 + rng.random())
        d = call(lib, "dfo_div", *s, *den)
        assert abs(val(d) - val(s) / val(den)) <= scale / abs(val(den)) * F(2) ** -44
        r = call(lib, "dfo_fma_u", *s, *c, *pair(lib, rnd(rng)))
        f = call(lib, "dfo_add_u", *r, *c)
        assert abs(val(f) - (val(r) + val(c))) <= (abs(val(r)) + abs(val(c)) + scale * abs(val(c))) * F(2) ** -46
