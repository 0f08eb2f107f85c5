"""Seeded synthetic inputs for accelerator regions.

This module only draws random numbers (numpy PCG64) and lays them out; it
holds none of the reduction arithmetic.  Tests, the smoke check and the
benchmark take their inputs from here, so the CUDA path and the serial oracle
see the same bytes.

The paper measures on Rodinia and the CUDA SDK (Methodology), whose sources and
data are not available; these generators stand in for them with the shapes and
distributions of the workloads this library is measured on:

* ``scalar_i32_small``   n = 2^20 int32 uniform in [-1000, 1000]
* ``full_range_i32``     int32 uniform over the whole range
* ``normal``             float32 / float64 N(0, 1)
* ``uniform_matrix``     dense float32 U(-1, 1) (row nest, Listing-1 nest)
* ``adversarial_i32``    int32 arrays whose reduction is not trivially 0 / -1
* ``log_uniform_lengths``  region lengths log-uniform on [lo, hi]
* ``poisson_arrivals``   open-loop arrival times for the served request loop
* ``batched_regions``    20,000 regions of log-uniform length, float and int64
"""
import numpy as np

BASE_SEED = 14121127


def rng(config_id=0, salt=0):
    """PCG64 generator seeded from the workload id (and an optional salt)."""
    return np.random.Generator(np.random.PCG64([BASE_SEED + int(config_id), int(salt)]))


def scalar_i32_small(n=1 << 20, seed=1):
    """Uniform int32 in [-1000, 1000] (the one-region sum + max workload)."""
    return rng(seed).integers(-1000, 1001, size=n, dtype=np.int32)


def full_range_i32(n, seed=2, salt=0):
    """Uniform int32 over [-2^31, 2^31)."""
    return rng(seed, salt).integers(-(1 << 31), 1 << 31, size=n, dtype=np.int64).astype(np.int32)


def normal(n, dtype=np.float32, seed=2, salt=1):
    """N(0, 1) in float32 or float64."""
    g = rng(seed, salt)
    if np.dtype(dtype) == np.float32:
        return g.standard_normal(n, dtype=np.float32)
    return g.standard_normal(n, dtype=np.float64)


def uniform_i64(n, lo, hi, seed=4, salt=0):
    """Uniform int64 in [lo, hi]."""
    return rng(seed, salt).integers(lo, hi + 1, size=n, dtype=np.int64)


def uniform_matrix(rows, cols, seed=3, salt=0, dtype=np.float32):
    """Dense row-major matrix, uniform in (-1, 1)."""
    g = rng(seed, salt)
    return (g.random((rows, cols), dtype=np.float32) * 2.0 - 1.0).astype(dtype)


def small_int_matrix(rows, cols, bound=16, seed=3, salt=7):
    """Integer-valued float32 matrix with |v| <= bound (exact in float and bf16)."""
    g = rng(seed, salt)
    return g.integers(-bound, bound + 1, size=(rows, cols)).astype(np.float32)


def adversarial_i32(n, op, seed=2, salt=11):
    """int32 arrays whose full reduction is informative for `op`.

    * mul:  odd values only, so the product modulo 2^32 stays odd;
    * band: all bits set except one cleared bit planted in one element;
    * land: all nonzero except a zero planted at the last index;
    * lor:  all zero except one nonzero planted at a random index;
    * max / min: uniform values with the extremum planted at the last index;
    * other ops: full-range uniform.
    """
    g = rng(seed, salt)
    if n == 0:
        return np.zeros(0, dtype=np.int32)
    if op == "mul":
        x = g.integers(-(1 << 31), 1 << 31, size=n, dtype=np.int64).astype(np.int32)
        return x | np.int32(1)
    if op == "band":
        x = np.full(n, -1, dtype=np.int32)
        bit = int(g.integers(0, 31))
        x[int(g.integers(0, n))] = np.int32(~(1 << bit))
        return x
    if op == "land":
        x = g.integers(1, 1 << 31, size=n, dtype=np.int64).astype(np.int32)
        x[-1] = 0
        return x
    if op == "lor":
        x = np.zeros(n, dtype=np.int32)
        x[int(g.integers(0, n))] = np.int32(int(g.integers(1, 1 << 31)))
        return x
    if op == "max":
        x = g.integers(-(1 << 30), 1 << 30, size=n, dtype=np.int64).astype(np.int32)
        x[-1] = np.int32((1 << 30) + 12345)
        return x
    if op == "min":
        x = g.integers(-(1 << 30), 1 << 30, size=n, dtype=np.int64).astype(np.int32)
        x[-1] = np.int32(-(1 << 30) - 12345)
        return x
    return full_range_i32(n, seed, salt)


def log_uniform_lengths(count, lo, hi, seed=4, salt=0):
    """Integer lengths ceil(exp(U(log lo, log hi))), clipped to [lo, hi]."""
    g = rng(seed, salt)
    v = np.exp(g.uniform(np.log(lo), np.log(hi), size=count))
    return np.clip(np.ceil(v).astype(np.int64), lo, hi)


def offsets_from_lengths(lengths):
    """CSR offsets (length count + 1, int64) for consecutive segments."""
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(np.asarray(lengths, dtype=np.int64), out=off[1:])
    return off


def poisson_arrivals(rate_per_s, count, seed=5, salt=0):
    """Arrival times (seconds from 0) of an open-loop Poisson process."""
    g = rng(seed, salt)
    return np.cumsum(g.exponential(1.0 / rate_per_s, size=count))


def batched_regions(count=20000, lo=1, hi=1 << 20, seed=4, salt=0):
    """The many-regions workload: `count` regions with lengths log-uniform on
    [lo, hi], in random order; even-numbered regions hold float32 N(0,1),
    odd-numbered int64 uniform in [-2^40, 2^40].  Returns (lengths, f32 pool,
    f32 offsets, i64 pool, i64 offsets): region 2k is segment k of the f32
    pool, region 2k+1 segment k of the i64 pool."""
    lengths = log_uniform_lengths(count, lo, hi, seed, salt)
    lf, li = lengths[0::2], lengths[1::2]
    off_f = offsets_from_lengths(lf)
    off_i = offsets_from_lengths(li)
    pool_f = normal(int(off_f[-1]), np.float32, seed=seed, salt=salt + 1)
    pool_i = uniform_i64(int(off_i[-1]), -(1 << 40), 1 << 40, seed=seed, salt=salt + 2)
    return lengths, pool_f, off_f, pool_i, off_i
