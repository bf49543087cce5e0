"""CPU check of the inward box bounds used by the FP32 admissibility pre-test.

The node records keep only the outward-rounded FP32 box (lo rounded down, hi
rounded up).  The pre-test derives inward bounds from it (tp_inward_lo/hi in
csrc/tp_internal.cuh): lo' = fma(|olo|, k, olo) + e and hi' = fma(-|ohi|, k,
ohi) - e.  The pre-test may only conclude "the boxes overlap" from inward
bounds that lie inside the FP64 box, so lo' >= lo and hi' <= hi must hold for
every FP64 bound.  The constants are read from the header, and the FP32
arithmetic is emulated exactly: the product of two floats and the sum with a
float are exact in FP64 here, so one rounding to FP32 gives the fused result.
"""

import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2509_22110_gb300", "csrc", "tp_internal.cuh")


def constants():
    src = open(HDR).read()
    lo = re.search(r"tp_inward_lo\(float olo\)\s*\{\s*return fmaf\(fabsf\(olo\),\s*([0-9.eE+-]+)f,\s*olo\)\s*\+\s*([0-9.eE+-]+)f;", src)
    hi = re.search(r"tp_inward_hi\(float ohi\)\s*\{\s*return fmaf\(-fabsf\(ohi\),\s*([0-9.eE+-]+)f,\s*ohi\)\s*-\s*([0-9.eE+-]+)f;", src)
    assert lo and hi, "inward-bound helpers not found in tp_internal.cuh"
    k_lo, e_lo = np.float32(float(lo.group(1))), np.float32(float(lo.group(2)))
    k_hi, e_hi = np.float32(float(hi.group(1))), np.float32(float(hi.group(2)))
    return k_lo, e_lo, k_hi, e_hi


def f32_down(x):
    f = np.float32(x)
    return np.nextafter(f, np.float32(-np.inf)) if float(f) > x else f


def f32_up(x):
    f = np.float32(x)
    return np.nextafter(f, np.float32(np.inf)) if float(f) < x else f


def fmaf(a, b, c):
    # exact in FP64 (24 + 24 bit product, and the sum spans under 53 bits), one rounding to FP32
    return np.float32(float(a) * float(b) + float(c))


def inward_lo(olo, k, e):
    return np.float32(fmaf(np.abs(olo), k, olo) + e)


def inward_hi(ohi, k, e):
    return np.float32(fmaf(-np.abs(ohi), k, ohi) - e)


def samples(rng, n=20000):
    xs = list(rng.standard_normal(n) * 10.0 ** rng.uniform(-6, 6, n))
    # values on and next to float boundaries, powers of two of both signs, tiny and zero
    for p in range(-30, 31):
        for s in (1.0, -1.0):
            b = s * 2.0 ** p
            xs += [b, np.nextafter(b, np.inf), np.nextafter(b, -np.inf)]
            f = float(np.float32(b))
            xs += [float(np.nextafter(np.float32(f), np.float32(np.inf))), float(np.nextafter(np.float32(f), np.float32(-np.inf)))]
    xs += [0.0, -0.0, 1e-40, -1e-40, 1e-38, -1e-38, 3e-39, -3e-39]
    # doubles strictly between two adjacent floats
    for f in rng.standard_normal(2000).astype(np.float32):
        g = np.nextafter(f, np.float32(np.inf))
        xs.append(float(f) + (float(g) - float(f)) * 0.5)
        xs.append(float(f) + (float(g) - float(f)) * 0.999)
    return xs


def test_inward_bounds_lie_inside_the_fp64_box():
    k_lo, e_lo, k_hi, e_hi = constants()
    rng = np.random.default_rng(7)
    for x in samples(rng):
        x = float(x)
        lo_in = inward_lo(f32_down(x), k_lo, e_lo)
        hi_in = inward_hi(f32_up(x), k_hi, e_hi)
        assert float(lo_in) >= x, (x, float(lo_in))
        assert float(hi_in) <= x, (x, float(hi_in))


def test_inward_bounds_stay_within_a_few_spacings():
    # tighter than the correctly rounded inward bounds by a few float spacings at most, so the
    # pre-test leaves only borderline cases to the FP64 test
    k_lo, e_lo, k_hi, e_hi = constants()
    rng = np.random.default_rng(11)
    for x in rng.standard_normal(5000) * 10.0 ** rng.uniform(-4, 4, 5000):
        x = float(x)
        lo_in = inward_lo(f32_down(x), k_lo, e_lo)
        ref = f32_up(x)
        for _ in range(4):
            ref = np.nextafter(ref, np.float32(np.inf))
        assert float(lo_in) <= float(ref)
