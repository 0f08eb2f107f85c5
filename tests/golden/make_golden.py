"""Writes the stored expected values of tests/golden/*.txt.

    python tests/golden/make_golden.py

Every stored value comes from the serial C oracle (oracle/), or, for
listing1_len6.txt, from an exact closed form that the oracle is checked
against here before the file is written; nothing comes from the CUDA path.
Inputs come from the seeded generators in paper_1412_1127_gb300/inputs.py
(which hold none of the method's arithmetic).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1412_1127_gb300 import inputs  # noqa: E402

ND = {"i32": np.int32, "i64": np.int64, "f32": np.float32, "f64": np.float64}


def small_inputs():
    """The seeded arrays of reduce_small.txt: (type, salt, array)."""
    g32 = inputs.full_range_i32(37, salt=701)
    g64 = inputs.uniform_i64(29, -(1 << 62), 1 << 62, salt=702)
    f32 = inputs.normal(33, np.float32, salt=703)
    f64 = inputs.normal(31, np.float64, salt=704)
    return [("i32", 701, g32), ("i64", 702, g64), ("f32", 703, f32), ("f64", 704, f64)]


REDUCE_CASES = {  # type -> [(op, variable type, init or None)]
    "i32": [(op, acc, init) for op in ["add", "mul", "max", "min", "band", "bor", "bxor", "land", "lor"]
            for acc, init in [("i32", None), ("i32", 5), ("i64", None)]],
    "i64": [(op, "i64", init) for op in ["add", "mul", "max", "min", "band", "bor", "bxor", "land", "lor"]
            for init in [None, -7]],
    "f32": [(op, acc, init) for op in ["add", "mul", "max", "min"] for acc, init in [("f32", None), ("f32", 0.5)]],
    "f64": [(op, "f64", init) for op in ["add", "mul", "max", "min"] for init in [None, 0.25]],
}


def bits(v, t):
    return int(np.asarray(v, dtype=ND[t]).reshape(1).view(np.uint32 if t in ("i32", "f32") else np.uint64)[0])


def write_reduce():
    lines = ["# Reductions of small seeded arrays: var = init (op) x[0] (op) ... (op) x[n-1], the",
             "# region's serial program with the directives ignored (IPMACC Sec. 1.3; the",
             "# reduction clause, Stage 3.4 (iii)), computed by the serial C oracle.",
             "# Arrays: paper_1412_1127_gb300.inputs with the salts below (i32: full_range_i32,",
             "# i64: uniform_i64 on [-2^62, 2^62], f32/f64: normal).  init '-' is the operator's identity.",
             "# fields: type salt n op var_type init result_bits_hex result"]
    for t, salt, x in small_inputs():
        for op, acc, init in REDUCE_CASES[t]:
            v = oracle.reduce(x, op, acc, init=init)
            lines.append("%s %d %d %s %s %s %x %r" % (t, salt, x.size, op, acc, "-" if init is None else repr(init),
                                                        bits(v, acc), v.item()))
    open(os.path.join(HERE, "reduce_small.txt"), "w").write("\n".join(lines) + "\n")


def listing1_closed_form(n):
    """a[i][l] = i + 2l - 3, b[l][j] = l j - 2: c[i][j] = sum_l (i + 2l - 3)(l j - 2)
    = (i - 3)(j S1 - 2n) + 2 (j S2 - 2 S1), S1 = sum l, S2 = sum l^2."""
    s1, s2 = n * (n - 1) // 2, (n - 1) * n * (2 * n - 1) // 6
    return [[(i - 3) * (j * s1 - 2 * n) + 2 * (j * s2 - 2 * s1) for j in range(n)] for i in range(n)]


def write_listing1():
    n = 6
    a = np.array([[i + 2 * l - 3 for l in range(n)] for i in range(n)], dtype=np.float32)
    b = np.array([[l * j - 2 for j in range(n)] for l in range(n)], dtype=np.float32)
    c = np.array(listing1_closed_form(n), dtype=np.float32)
    assert np.array_equal(oracle.matmul_listing1(a, b), c), "oracle disagrees with the closed form"
    lines = ["# Listing 1a (Sec. 1.3) at LEN = 6 with a[i][l] = i + 2l - 3 and b[l][j] = l j - 2:",
             "# c[i][j] = sum_l a[i][l] b[l][j] = (i - 3)(15 j - 12) + 110 j - 60 (closed form; small",
             "# integers, so every mode of the nest is exact).  One row of c per line."]
    lines += [" ".join("%d" % int(v) for v in row) for row in c]
    open(os.path.join(HERE, "listing1_len6.txt"), "w").write("\n".join(lines) + "\n")


def nearest_inputs():
    pts = (inputs.rng(24, 40).random((40, 2), dtype=np.float32) * 10).astype(np.float32)
    pts[31] = pts[7]  # an exact tie, broken by index
    return pts, np.float32(4.5), np.float32(5.25)


def write_nearest():
    pts, qx, qy = nearest_inputs()
    idx, d2 = oracle.nearest_k(pts, qx, qy, 5)
    lines = ["# Nearest Neighbor (Sec. 4.2): the 5 smallest d = (x - qx)^2 + (y - qy)^2 in float,",
             "# every operation rounded, ties by index; 40 points from inputs.rng(24, 40) x 10 with",
             "# point 31 = point 7; q = (4.5, 5.25).  Serial C oracle.",
             "# fields: rank index d_bits_hex d"]
    for r in range(5):
        lines.append("%d %d %x %r" % (r, int(idx[r]), bits(d2[r], "f32"), float(d2[r])))
    open(os.path.join(HERE, "nearest_k5_40pts.txt"), "w").write("\n".join(lines) + "\n")


def bfs_grid():
    g = inputs.rng(25, 1)
    grid = (g.random((7, 9)) < 0.7).astype(np.uint8)
    grid[3, 4] = 1
    return grid, 3 * 9 + 4


def write_bfs():
    grid, src = bfs_grid()
    dist, levels = oracle.grid_bfs(grid, src)
    lines = ["# BFS (Sec. 4.2) on a 7 x 9 grid (1 = open; inputs.rng(25, 1) < 0.7, source (3, 4)",
             "# forced open): steps from the source through open cells, -1 unreached; the loop",
             "# runs %d levels (the last finds nothing new).  Serial C oracle (queue BFS)." % levels,
             "levels %d" % levels, "# open cells:"]
    lines += [" ".join(str(int(v)) for v in row) for row in grid]
    lines.append("# distances:")
    lines += [" ".join(str(int(v)) for v in row) for row in dist]
    open(os.path.join(HERE, "bfs_7x9.txt"), "w").write("\n".join(lines) + "\n")


if __name__ == "__main__":
    write_reduce()
    write_listing1()
    write_nearest()
    write_bfs()
    print("wrote", sorted(f for f in os.listdir(HERE) if f.endswith(".txt")))
