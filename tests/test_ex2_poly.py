"""The FMA-pipe exp2 of the degree passes, pinned on the CPU against the mathematics.

The CUDA source evaluates 2^x as 2^round(x) * p(x - round(x)) with a degree-6 polynomial p
on [-1/2, 1/2]. Here the coefficients are read from that source and the same FP32 steps
(round-to-nearest Horner with fused multiply-adds, emulated in FP64 and rounded per step)
are checked against exp2 in FP64: the maximum relative error must stay within 1.5e-7
(about 2.5 ulp, the accuracy class of the hardware ex2.approx the other half of the entries
use), over the reduced range and over the arguments the degree pass produces (|x| <= 24).
"""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2311_06115_gb300", "csrc", "k_degrees.cu")


def _coeffs():
    src = open(SRC).read()
    body = src[src.index("float2 dm_ex2_fma2(float2 x)"):]
    body = body[:body.index("return make_float2")]
    vals = re.findall(r"make_float2\(([-0-9.e]+)f, \1f\)", body)
    # the first two are the rounding constants, then c6 .. c0
    nums = [float(v) for v in vals]
    assert nums[0] == 12582912.0 and nums[1] == -12582912.0
    poly = [v for v in nums[2:] if v != -1.0]
    assert len(poly) == 7
    return np.array(poly, dtype=np.float32)  # c6, c5, ..., c0


def _fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _ex2_emulated(x):
    x = x.astype(np.float32)
    big = np.float32(12582912.0)
    t = (x + big).astype(np.float32)
    r = (t - big).astype(np.float32)
    f = _fma32(r, np.float32(-1.0) * np.ones_like(r), x)
    c = _coeffs()
    p = np.full_like(f, c[0])
    for k in c[1:]:
        p = _fma32(p, f, np.full_like(f, k))
    bits = (p.view(np.int32).astype(np.int64) + (t.view(np.int32).astype(np.int64) << 23)) & 0xFFFFFFFF
    return bits.astype(np.uint32).view(np.float32)


def test_reduced_range_accuracy():
    x = np.linspace(-0.5, 0.5, 400001, dtype=np.float32)
    rel = np.abs(_ex2_emulated(x).astype(np.float64) / np.exp2(x.astype(np.float64)) - 1.0)
    assert rel.max() < 1.5e-7, rel.max()


def test_degree_pass_argument_range():
    x = np.random.default_rng(0).uniform(-24.0, 24.0, 200000).astype(np.float32)
    x = np.concatenate([x, np.arange(-24, 25, dtype=np.float32), np.float32([-0.0, 1e-30, -1e-30])])
    rel = np.abs(_ex2_emulated(x).astype(np.float64) / np.exp2(x.astype(np.float64)) - 1.0)
    assert rel.max() < 1.5e-7, rel.max()


def test_integer_arguments_are_exact():
    x = np.arange(-24, 25, dtype=np.float32)
    np.testing.assert_array_equal(_ex2_emulated(x), np.exp2(x.astype(np.float64)).astype(np.float32))
