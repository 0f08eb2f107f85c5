"""The stored expected values in tests/golden/: the oracle still produces
them, and the ones with a definition independent of the oracle are checked
against it (closed form, brute force, invariants)."""
import numpy as np

import oracle
import golden_data as G


def test_oracle_reproduces_stored_reductions():
    for t, x, op, acc, init, bits, _ in G.reduce_cases():
        assert G.bits_of(oracle.reduce(x, op, acc, init=init), acc) == bits, (t, op, acc, init)


def test_listing1_fixture_is_the_closed_form_and_the_oracle():
    c = G.listing1()
    n = c.shape[0]
    for i in range(n):
        for j in range(n):
            assert c[i, j] == sum((i + 2 * l - 3) * (l * j - 2) for l in range(n))  # the sum itself
    a = np.array([[i + 2 * l - 3 for l in range(n)] for i in range(n)], dtype=np.float32)
    b = np.array([[l * j - 2 for j in range(n)] for l in range(n)], dtype=np.float32)
    assert np.array_equal(oracle.matmul_listing1(a, b), c)


def test_nearest_fixture_by_brute_force():
    pts, qx, qy, idx, d = G.nearest()
    # float32 numpy arithmetic: each subtraction, product and sum rounded separately
    dx = pts[:, 0] - qx
    dy = pts[:, 1] - qy
    dd = dx * dx + dy * dy
    order = sorted(range(len(dd)), key=lambda i: (float(dd[i]), i))[:5]
    assert list(idx) == order
    assert np.array_equal(d, dd[order])
    wi, wd = oracle.nearest_k(pts, qx, qy, 5)
    assert np.array_equal(wi, idx) and np.array_equal(wd, d)


def test_bfs_fixture_satisfies_the_level_equations():
    grid, src, dist, levels = G.bfs()
    r, c = grid.shape
    nb = lambda i, j: [(i + di, j + dj) for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1))
                       if 0 <= i + di < r and 0 <= j + dj < c]
    assert dist.flat[src] == 0
    for i in range(r):
        for j in range(c):
            if (i * c + j) == src:
                continue
            reached = [dist[p] for p in nb(i, j) if grid[p] and dist[p] >= 0]
            if grid[i, j] and reached:      # an open cell next to a reached one is one step further
                assert dist[i, j] == 1 + min(reached)
            else:                           # closed, or no reached neighbour: unreached
                assert dist[i, j] == -1
    assert levels == dist.max() + 1
    od, ol = oracle.grid_bfs(grid, src)
    assert np.array_equal(od, dist) and ol == levels


def test_fixtures_are_what_the_writer_produces(tmp_path, monkeypatch):
    """The stored files are exactly what tests/golden/make_golden.py writes
    from the oracle and the closed form (so no stored value has another source)."""
    import os
    import make_golden
    monkeypatch.setattr(make_golden, "HERE", str(tmp_path))
    make_golden.write_reduce()
    make_golden.write_listing1()
    make_golden.write_nearest()
    make_golden.write_bfs()
    for name in sorted(os.listdir(tmp_path)):
        with open(os.path.join(tmp_path, name)) as a, open(os.path.join(G.HERE, name)) as b:
            assert a.read() == b.read(), name
