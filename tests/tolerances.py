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
