"""Readers of the stored expected values in tests/golden/ (written by
tests/golden/make_golden.py from the serial oracle and a closed form)."""
import os
import sys

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)
import make_golden  # noqa: E402  (the fixtures' input recipes)

ND = make_golden.ND


def _rows(name):
    with open(os.path.join(HERE, name)) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


def reduce_cases():
    """[(type, array, op, var_type, init or None, bits, value)]"""
    arrays = {t: x for t, _, x in make_golden.small_inputs()}
    out = []
    for t, salt, n, op, acc, init, hx, val in _rows("reduce_small.txt"):
        x = arrays[t]
        assert x.size == int(n)
        iv = None if init == "-" else (float(init) if acc in ("f32", "f64") else int(init))
        out.append((t, x, op, acc, iv, int(hx, 16), val))
    return out


def listing1():
    rows = _rows("listing1_len6.txt")
    return np.array([[float(v) for v in r] for r in rows], dtype=np.float32)


def nearest():
    pts, qx, qy = make_golden.nearest_inputs()
    rows = _rows("nearest_k5_40pts.txt")
    idx = np.array([int(r[1]) for r in rows], dtype=np.int64)
    dbits = np.array([int(r[2], 16) for r in rows], dtype=np.uint32)
    return pts, qx, qy, idx, dbits.view(np.float32)


def bfs():
    grid, src = make_golden.bfs_grid()
    rows = _rows("bfs_7x9.txt")
    levels = int(rows[0][1])
    r, c = grid.shape
    stored_open = np.array([[int(v) for v in row] for row in rows[1:1 + r]], dtype=np.uint8)
    assert np.array_equal(stored_open, grid)
    dist = np.array([[int(v) for v in row] for row in rows[1 + r:1 + 2 * r]], dtype=np.int32)
    return grid, src, dist, levels


def bits_of(v, t):
    return make_golden.bits(v, t)
