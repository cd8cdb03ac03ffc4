"""The paired near-field arithmetic (h2_near_field H2_NEAR_F32PAIR) on the host.

The kernel carries every near-field entry and input value as an unevaluated
pair of FP32 numbers hi + lo (hi = fp32(v), lo = fp32(v - hi)) and forms a
row's sum with error-free transformations: the product of the high words as
its rounded value p plus the exact residual (Dekker's product, the residual
given by an FMA), the cross terms hi*lo + lo*hi and the residuals collected in
a low word, and the running high word kept by TwoSum (Knuth).  This file
restates those steps in numpy FP32 arithmetic and checks the accuracy claim
the library documents: the error of a row of n terms stays below n * 2^-48
times the sum of the magnitudes of its terms (the low word's own rounding grows
with the row; ~6e-13 measured at n = 1000), far below the 1e-5 of the reduced
forms and the FP64 path's 1e-8, while a plain FP32 sum of the same terms is off
by ~1e-7.  The exact value comes from rational arithmetic on the FP64 inputs.
"""
from fractions import Fraction

import numpy as np

f32 = np.float32
f64 = np.float64


def split(v):
    """v (FP64) as the pair hi = fp32(v), lo = fp32(v - hi)."""
    hi = v.astype(f32)
    lo = (v - hi.astype(f64)).astype(f32)
    return hi, lo


def fma32(a, b, c):
    """fp32(a*b + c): the FP32 product is exact in FP64, one final rounding."""
    return (a.astype(f64) * b.astype(f64) + c.astype(f64)).astype(f32)


def pair_row_sums(A, x):
    """sum_j A[i, j] x[j] per row i, in the paired arithmetic, step by step."""
    ah, al = split(A)
    xh, xl = split(x)
    hi = np.zeros(A.shape[0], f32)
    lo = np.zeros(A.shape[0], f32)
    for j in range(A.shape[1]):
        a_h, a_l, x_h, x_l = ah[:, j], al[:, j], xh[j], xl[j]
        p = a_h * x_h                                            # rounded product
        e = (a_h.astype(f64) * f64(x_h) - p.astype(f64)).astype(f32)   # its exact residual
        s = hi + p                                               # TwoSum(hi, p)
        bb = s - hi
        t = (hi - (s - bb)) + (p - bb)
        hi = s
        lo = fma32(a_h, np.full_like(a_h, x_l), lo)
        lo = fma32(a_l, np.full_like(a_l, x_h), lo)
        lo = lo + (e + t)
    return hi.astype(f64) + lo.astype(f64)


def exact_row_sums(A, x):
    xf = [Fraction(float(v)) for v in x]
    return np.array([float(sum(Fraction(float(a)) * xv for a, xv in zip(row, xf))) for row in A])


def near_like_rows(rows, cols, seed):
    """Entries spread over several binades with both signs (near-field blocks
    hold weights from ~1e-1 down to ~1e-6 and the diagonal near -1/2), inputs
    ~N(0, 1)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((rows, cols)) * 10.0 ** rng.uniform(-6, -1, (rows, cols))
    A[:, 0] = -0.5 + 0.01 * rng.standard_normal(rows)
    x = rng.standard_normal(cols)
    return A, x


def test_paired_sum_is_fp64_equivalent():
    A, x = near_like_rows(24, 1000, 5)
    ref = exact_row_sums(A, x)
    mag = np.abs(A) @ np.abs(x)
    err_pair = np.max(np.abs(pair_row_sums(A, x) - ref) / mag)
    assert err_pair < A.shape[1] * 2.0 ** -48, err_pair
    # the same sum in plain FP32 (what dropping the low words would give)
    plain = (A.astype(f32) * x.astype(f32)).astype(f32)
    s32 = np.zeros(A.shape[0], f32)
    for j in range(A.shape[1]):
        s32 = s32 + plain[:, j]
    err32 = np.max(np.abs(s32.astype(f64) - ref) / mag)
    assert err32 > 1e3 * err_pair


def test_pair_representation_keeps_48_bits():
    # magnitudes where the low word stays a normal FP32 number (near-field
    # entries and inputs lie far inside this range)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(10000) * 10.0 ** rng.uniform(-12, 12, 10000)
    hi, lo = split(v)
    rel = np.abs(hi.astype(f64) + lo.astype(f64) - v) / np.abs(v)
    assert np.max(rel) <= 2.0 ** -48
    assert np.all(np.abs(lo) <= np.abs(hi) * 2.0 ** -24)


def test_dropping_any_low_term_is_visible():
    """Each low-word contribution matters: leaving one out raises the error
    far above the paired result's (a pin against a dropped term)."""
    A, x = near_like_rows(8, 400, 9)
    ref = exact_row_sums(A, x)
    mag = np.abs(A) @ np.abs(x)
    good = np.max(np.abs(pair_row_sums(A, x) - ref) / mag)
    ah, al = split(A)
    xh, xl = split(x)
    for drop in ("e", "t", "xl", "al"):
        hi = np.zeros(A.shape[0], f32)
        lo = np.zeros(A.shape[0], f32)
        for j in range(A.shape[1]):
            p = ah[:, j] * xh[j]
            e = (ah[:, j].astype(f64) * f64(xh[j]) - p.astype(f64)).astype(f32)
            s = hi + p
            bb = s - hi
            t = (hi - (s - bb)) + (p - bb)
            hi = s
            if drop != "xl":
                lo = fma32(ah[:, j], np.full(A.shape[0], xl[j], f32), lo)
            if drop != "al":
                lo = fma32(al[:, j], np.full(A.shape[0], xh[j], f32), lo)
            lo = lo + ((f32(0) if drop == "e" else e) + (f32(0) if drop == "t" else t))
        bad = np.max(np.abs(hi.astype(f64) + lo.astype(f64) - ref) / mag)
        assert bad > 100 * good, (drop, bad, good)
