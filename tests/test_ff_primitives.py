"""Host-side check of the double-float primitives that decide every T3, T5, pT3 and pT5 candidate
(csrc/lst_ff.cuh; the functions are __host__ __device__, so a host build runs the same source).

Each primitive is compared with the same operation in long double (C library) over the argument
ranges the kernels use, against error bounds of the ~48-bit format: products, quotients, square
roots, asin, sinh within a few 1e-14 relative; sums and a^2 - b^2 within ~1e-14 of the operand
magnitudes (the results may cancel); sin / cos of angles up to 4 rad within ~4e-14 absolute. Those
bounds are seven orders of magnitude inside the 1e-5 relative band in which a selection's outcome
is allowed to differ from the float64 oracle. Results must also be normalised pairs
(|lo| <= ulp(hi) / 2), which the comparisons of the decision code assume.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "ff_check.cpp")
HDR = os.path.join(ROOT, "paper_2207_08207_gb300", "csrc", "lst_ff.cuh")
LIB = os.path.join(ROOT, "_build", "libff_check.so")


@pytest.fixture(scope="module")
def ffc():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)):
        cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
        tmp = f"{LIB}.{os.getpid()}.tmp"
        # -ffp-contract=off: the header's host path relies on each product and sum being rounded on
        # its own, as its device path does through non-contractible intrinsics
        subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-I" + cuda_inc,
                        "-I" + os.path.dirname(HDR), "-o", tmp, SRC], check=True)
        os.replace(tmp, LIB)
    L = ctypes.CDLL(LIB)
    L.ffc_binary.argtypes = [ctypes.c_int, ctypes.c_int64] + [ctypes.c_void_p] * 5
    L.ffc_unary.argtypes = [ctypes.c_int, ctypes.c_int64] + [ctypes.c_void_p] * 2
    L.ffc_normalised.argtypes = [ctypes.c_int, ctypes.c_int64] + [ctypes.c_void_p] * 4
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _ff(rng, n, lo, hi, log=False):
    """Random double-float values: a float64 draw split into its float and the rounded rest."""
    d = np.exp(rng.uniform(np.log(lo), np.log(hi), n)) * rng.choice([-1.0, 1.0], n) if log else rng.uniform(lo, hi, n)
    h = d.astype(np.float32)
    return h, (d - h.astype(np.float64)).astype(np.float32)


OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "sqrt": 4, "asin": 5, "diff_prod": 6}
BOUND = {"add": 2e-14, "sub": 2e-14, "mul": 3e-14, "div": 6e-14, "sqrt": 3e-14, "asin": 1e-13, "diff_prod": 4e-14}


@pytest.mark.parametrize("name", list(OPS))
def test_arithmetic(ffc, name):
    rng = np.random.default_rng(OPS[name] + 10)
    n = 100_000
    ah, al = _ff(rng, n, 1e-3, 1e4, log=True)   # coordinates, radii, curvatures, chi2 terms
    bh, bl = _ff(rng, n, 1e-3, 1e4, log=True)
    if name == "sqrt":
        ah, al = np.abs(ah), np.where(ah < 0, -al, al)
    if name == "asin":
        ah, al = _ff(rng, n, -1.0, 1.0)
        ah2, al2 = _ff(rng, n // 4, 0.99, 1.0)   # the branch near 1
        ah, al = np.concatenate([ah, ah2, -ah2]), np.concatenate([al, al2, -al2])
        bh, bl = np.resize(bh, ah.size), np.resize(bl, ah.size)
    err = np.zeros(ah.size)
    assert ffc.ffc_binary(OPS[name], ah.size, _p(ah), _p(al), _p(bh), _p(bl), _p(err)) == 0
    assert err.max() <= BOUND[name], (name, err.max())
    if name == "add":
        # exact cancellation: a + (-a) differs from zero by nothing
        err = np.zeros(n)
        nh, nl = -ah, -al
        ffc.ffc_binary(0, n, _p(ah), _p(al), _p(nh), _p(nl), _p(err))
        assert err.max() == 0.0


@pytest.mark.parametrize("name,op,lo,hi,bound", [("sin", 0, -4.0, 4.0, 6e-14), ("cos", 1, -4.0, 4.0, 6e-14),
                                                 ("sinh_small", 2, -0.5, 0.5, 5e-14),
                                                 ("sinh", 2, -12.0, 12.0, 5e-14)])
def test_transcendental(ffc, name, op, lo, hi, bound):
    rng = np.random.default_rng(op + 40)
    x = rng.uniform(lo, hi, 100_000).astype(np.float32)
    # quadrant edges of the sin / cos reduction
    x = np.concatenate([x, (np.arange(-2, 3) * np.float32(np.pi / 2)).astype(np.float32)])
    err = np.zeros(x.size)
    assert ffc.ffc_unary(op, x.size, _p(x), _p(err)) == 0
    assert err.max() <= bound, (name, err.max())


@pytest.mark.parametrize("op", range(4))
def test_results_are_normalised(ffc, op):
    rng = np.random.default_rng(op + 70)
    n = 50_000
    ah, al = _ff(rng, n, 1e-3, 1e4, log=True)
    bh, bl = _ff(rng, n, 1e-3, 1e4, log=True)
    if op == 3:
        ah, al = np.abs(ah), np.where(ah < 0, -al, al)
    assert ffc.ffc_normalised(op, n, _p(ah), _p(al), _p(bh), _p(bl)) == 1
