"""The seeded input generators produce what the benchmark and the tests say
they do (no GPU): shapes, symmetry, diagonals, value ranges, densities, the
grid metric, the ragged and served size ranges, and determinism."""

import numpy as np
import pytest

from paper_2605_24408_gb300 import instances as G


def _offdiag(M):
    return M[~np.eye(M.shape[0], dtype=bool)]


def test_named_workloads():
    D, F = G.named("n12")
    assert D.shape == F.shape == (12, 12)
    # 3 x 4 grid Manhattan distances: location r*4 + c
    for a in range(12):
        for b in range(12):
            assert D[a, b] == abs(a // 4 - b // 4) + abs(a % 4 - b % 4)
    assert np.array_equal(F, F.T) and not F.diagonal().any()
    assert set(np.unique(_offdiag(F))) <= set(range(0, 11))
    D, F = G.named("n30")
    assert D.shape == (30, 30) and D.max() == 4 + 5  # 5 x 6 grid diameter
    D, F = G.named("n100")
    for M in (D, F):
        assert np.array_equal(M, M.T) and not M.diagonal().any()
        assert _offdiag(M).min() >= 0 and _offdiag(M).max() <= 99
    D, F = G.named("n100a")
    assert not np.array_equal(D, D.T) and not np.array_equal(F, F.T)
    assert not D.diagonal().any() and not F.diagonal().any()
    D, F = G.named("n256")
    assert D.shape == (256, 256) and np.array_equal(D, D.T)


def test_flow_densities_are_close_to_their_targets():
    F = G.sparse_symmetric(200, 0.3, 1, 10, seed=1, tag=5)
    frac = np.count_nonzero(_offdiag(F)) / (200 * 199)
    assert abs(frac - 0.3) < 0.02
    assert set(np.unique(_offdiag(F))) <= set(range(0, 11))


def test_ragged_and_request_sizes_and_kinds():
    sizes = [G.ragged_size(k, 0) for k in range(256)]
    assert min(sizes) >= 12 and max(sizes) <= 256
    assert len(set(sizes)) > 100
    for k in (0, 1, 2, 3):
        n = sizes[k]
        D, F = G.ragged_instance(k, n, 0)
        assert D.shape == (n, n) and np.array_equal(D, D.T) and np.array_equal(F, F.T)
        if k % 2 == 0:  # grid D on the smallest near-square grid, first n cells
            rows, cols = G.near_square_grid(n)
            assert rows * cols >= n and cols * (rows - 1) < n
            assert D[0, 1] == 1
        else:  # dense 0..99
            assert _offdiag(D).max() <= 99 and _offdiag(F).max() <= 99
    ns = [G.request_instance(r)[0].shape[0] for r in range(200)]
    assert min(ns) >= 20 and max(ns) <= 200


def test_generators_are_deterministic_and_seed_dependent():
    a = G.dense_instance(40, seed=3)
    b = G.dense_instance(40, seed=3)
    c = G.dense_instance(40, seed=4)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0])
    h = G.hash_u64(7, 11, np.arange(5, dtype=np.uint64))
    assert h.dtype == np.uint64 and len(set(h.tolist())) == 5
    u = G.hash_unit(7, 11, np.arange(100000, dtype=np.uint64))
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


@pytest.mark.parametrize("n,k", [(10, 0), (10, 1), (10, 10), (256, 92)])
def test_flow_class_instances(n, k):
    D, F = G.flow_class_instance(n, k, seed=2, f0=1, f=3, fdiag=5)
    assert np.array_equal(D, D.T) and not D.diagonal().any()
    assert (F.diagonal() == 5).all()
    x = np.zeros(n, bool)
    if k > 1:
        x = np.array([(F[c, np.arange(n) != c] == 4).any() for c in range(n)])
    assert x.sum() == (k if k > 1 else 0)
    expect = 1 + 3 * np.outer(x, x)
    assert np.array_equal(_offdiag(F), _offdiag(expect))


def test_asymmetric_instances():
    D, F = G.asymmetric_instance(30, seed=5, diag=True)
    assert not np.array_equal(D, D.T) and not np.array_equal(F, F.T)
    assert (D.diagonal() >= 1).all()
    D0, _ = G.asymmetric_instance(30, seed=5)
    assert not D0.diagonal().any()
    rows, cols = G.near_square_grid(30)
    base = G.grid_manhattan(rows, cols, 30)
    surcharge = D0 - base
    assert surcharge[~np.eye(30, dtype=bool)].min() >= 0 and surcharge.max() <= 9
