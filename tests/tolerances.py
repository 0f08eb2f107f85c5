"""Floating-point acceptance rules for the CUDA path against the oracle.

Integer, bitwise, logical and min/max results must match the serial oracle
bit for bit (any association of these operators gives the same bits).

Floating-point sums are compared with the exactly rounded truth
(``oracle.truth_sum``), not with the serial float program, whose rounding
order is one of many.  The relative error is taken against
max(|truth|, 0.1 * sqrt(n)) -- for N(0,1) data |truth| is of order sqrt(n), and
the floor keeps a near-zero total from turning a tiny absolute error into a
huge relative one.  Tolerances:

* plain float sums:        1e-3  (at n = 2^28; smaller n only tighter)
* compensated float sums:  1e-5
* double sums:             1e-12

The BF16x3 form of the Listing-1a nest (``bf16x3_tol``) is held to a bound
derived from its arithmetic; see that function.
"""
import math

import numpy as np

import oracle

TOL_F32 = 1e-3
TOL_F32_COMP = 1e-5
TOL_F64 = 1e-12


def sum_rel_err(got, x, init=None):
    truth = oracle.truth_sum(x) if init is None else \
        oracle.truth_sum(np.concatenate([np.array([init], dtype=x.dtype), x]))
    n = max(int(x.size), 1)
    return abs(float(got) - truth) / max(abs(truth), 0.1 * math.sqrt(n), 1e-300), truth


def assert_sum_close(got, x, tol, init=None):
    err, truth = sum_rel_err(got, x, init)
    assert err <= tol, "sum %r vs truth %r: rel err %.3g > %.3g (n=%d)" % (got, truth, err, tol, x.size)
    return err


def same_bits(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return a.dtype == b.dtype and a.shape == b.shape and a.tobytes() == b.tobytes()


U24 = 2.0 ** -24
BF16X3_LAMBDA = 6.0
BF16X3_CAP = 2e-5


def bf16x3_tol(a, b, s):
    """Componentwise error bound of the BF16x3 nest, |c - c_exact| <= tol.

    Each float x is split as x = hi + lo + r with hi = bf16(x),
    lo = bf16(x - hi): |x - hi| <= 2^-8 |x| and |r| <= 2^-16 |x|.  The nest
    keeps hi*hi + hi*lo + lo*hi, so the term dropped from each product
    a_l b_l is lo*lo plus the residuals' products, at most 3 * 2^-16 |a_l b_l|.
    Summed over l these give at most 3 * 2^-16 * S (S = sum_l |a_l b_l|,
    the array `s`) whatever the signs; with signs independent across l
    (symmetric inputs) Hoeffding's inequality bounds the sum by
    lambda * 3 * 2^-16 * sqrt(max_l |a_l b_l| * S) except with probability
    2 exp(-lambda^2 / 2); max_l |a_l b_l| <= max|a_i.| max|b_.j|.  The float
    accumulator rounds once per 16-deep MMA step per product, K = 3 ceil(n/16)
    roundings of at most 2^-24 S each: at most K 2^-24 S, or lambda sqrt(K)
    2^-24 S for independent rounding errors.  Each part takes the smaller of
    its worst case and its lambda = 6 bound.  At n = 3072 with U(-1,1) inputs
    this is about 1.9e-5 S; a dropped cross term (hi*lo) leaves errors near
    3e-4 S in the largest entries, far outside it.
    """
    n = a.shape[0]
    ra = np.max(np.abs(a), axis=1).astype(np.float64)[:, None]
    cb = np.max(np.abs(b), axis=0).astype(np.float64)[None, :]
    sp = np.maximum(s, 1e-300)
    split = np.minimum(3 * 2.0 ** -16 * sp, BF16X3_LAMBDA * 3 * 2.0 ** -16 * np.sqrt(ra * cb * sp))
    k = 3 * -(-n // 16)
    acc = min(k, BF16X3_LAMBDA * math.sqrt(k)) * U24 * sp
    return split + acc
