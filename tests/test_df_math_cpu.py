"""The FP64 path's double-float pair function, checked on the host.

The FP64 short range evaluates the screened pair kernel of eq. (ewald_split) in double-float
arithmetic (pairs of FP32 numbers, ``paper_2103_02046_gb300/csrc/df_math.cuh``). The header is
plain float arithmetic, so the same code compiles here with g++ (FP contraction off, as the
device code's rounded intrinsics demand) and is compared with long-double erfc and exp over
rho in (0, 1]: the potential, the force coefficient and the adjoint's Hessian term must stay
within a few 1e-14 (kappa = 3, the default) to 2e-13 (kappa = 6, the largest the context uses
it for), far inside the FP64 path's 1e-12 parity bound.
"""
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path_factory.mktemp("dfm") / "df_math_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "paper_2103_02046_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "df_math_check.cpp"), "-o", exe], check=True)
    return exe


def run(exe, arg):
    out = subprocess.run([exe, str(arg) if isinstance(arg, str) else repr(arg)], check=True,
                         capture_output=True, text=True)
    return json.loads(out.stdout)


@pytest.mark.parametrize("kappa,bound", [(3.0, 1e-13), (1.0, 1e-13), (6.0, 3e-13)])
def test_pair_function_double_float_accuracy(checker, kappa, bound):
    r = run(checker, kappa)
    assert r["fit"]
    # the fitted erfc(x) e^{x^2} itself is at double precision
    assert r["fit_err"] < 3e-15
    assert r["intervals"] * 0.375 >= kappa - 1e-9
    for key in ("pot", "fco", "dfr"):
        assert r[key] < bound, (key, r)


def test_pair_function_fit_range(checker):
    # the exponential's table covers kappa^2 < 88
    assert run(checker, 9.0)["fit"]
    assert not run(checker, 9.5)["fit"]


def test_split_double_by_bits(checker):
    # the charge spectrum enters the FP64 path's fused z solve as double-float, split by integer
    # operations on each double's bits: hi the leading 24 significand bits, lo the other 29
    # rounded once, so |hi + lo - v| <= 2^-47 |v| and |lo| < ulp(hi)
    r = run(checker, "split")
    assert r["fast"] > 350000
    assert r["worst"] <= 2.0 ** -47, r
    assert r["bad_ulp"] == 0 and r["bad_sign"] == 0, r
    assert r["zero"] and r["neg_zero"] and r["one"] and r["subnormal"], r
    assert r["third_err"] <= 3 * 2.0 ** -47 and r["edge_err"] <= 2.0 ** -47, r
    # the FP64 conversion outside the fast path (FP32's rounding of hi, then of the rest)
    assert r["worst_slow"] < 1e-13, r
