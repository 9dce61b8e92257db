"""Seeded synthetic QAP instances (the D and F inputs of Eq. 1).

The paper's workloads are QAPLIB instances; none are shipped here. These
generators stand in for them with the same shapes: integer, symmetric
distance (D) and flow (F) matrices with zero diagonals, either distances on a
grid of locations (Manhattan metric) with a sparse random flow, or dense
uniform random matrices.

This module holds no arithmetic of the method itself. Both the CUDA path and
the CPU oracle receive what it produces, so the two always see identical
inputs. Randomness is a counter-based hash (SplitMix64 finaliser, Steele,
Lea and Flood, OOPSLA 2014) of (seed, tag, index), so values do not depend on
the numpy version or on the order in which they are drawn.
"""

from __future__ import annotations

import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _mix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = x + np.uint64(0x9E3779B97F4A7C15)
        x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        x = x ^ (x >> np.uint64(31))
    return x


def hash_u64(seed: int, tag: int, idx) -> np.ndarray:
    """Deterministic 64-bit value for (seed, tag, idx); idx may be an array."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h = _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(tag) * np.uint64(0xD1B54A32D192ED03)))
        return _mix64(h ^ _mix64(idx))


def hash_unit(seed: int, tag: int, idx) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of hash_u64."""
    return (hash_u64(seed, tag, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def hash_int(seed: int, tag: int, idx, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive); the modulo bias is below 2^-50."""
    span = np.uint64(hi - lo + 1)
    return (hash_u64(seed, tag, idx) % span).astype(np.int64) + lo


def grid_manhattan(rows: int, cols: int, n: int | None = None) -> np.ndarray:
    """Manhattan distances between the first n cells (row-major) of a rows x cols grid."""
    n = rows * cols if n is None else n
    if n > rows * cols:
        raise ValueError("grid too small for n locations")
    cell = np.arange(n)
    r, c = cell // cols, cell % cols
    d = np.abs(r[:, None] - r[None, :]) + np.abs(c[:, None] - c[None, :])
    return d.astype(np.int32)


def _upper_pairs(n: int):
    iu, ju = np.triu_indices(n, k=1)
    return iu, ju, (iu * n + ju).astype(np.uint64)


def sparse_symmetric(n: int, density: float, lo: int, hi: int, seed: int, tag: int) -> np.ndarray:
    """Symmetric, zero diagonal; each unordered pair is nonzero with probability
    `density`, its value uniform in lo..hi."""
    iu, ju, key = _upper_pairs(n)
    keep = hash_unit(seed, tag, key) < density
    val = hash_int(seed, tag + 1, key, lo, hi)
    m = np.zeros((n, n), dtype=np.int64)
    m[iu, ju] = np.where(keep, val, 0)
    m = m + m.T
    return m.astype(np.int32)


def dense_symmetric(n: int, lo: int, hi: int, seed: int, tag: int) -> np.ndarray:
    """Symmetric, zero diagonal, every off-diagonal pair uniform in lo..hi."""
    return sparse_symmetric(n, 1.0, lo, hi, seed, tag)


def near_square_grid(n: int) -> tuple[int, int]:
    """Smallest near-square grid holding n cells: ceil(sqrt(n)) columns."""
    cols = int(math.ceil(math.sqrt(n)))
    rows = int(math.ceil(n / cols))
    return rows, cols


# --- The workload shapes ---------------------------------------------------

def grid_instance(rows: int, cols: int, density: float, seed: int, n: int | None = None):
    """Grid-Manhattan D with a sparse flow F in 1..10 (the small plain instances)."""
    n = rows * cols if n is None else n
    D = grid_manhattan(rows, cols, n)
    F = sparse_symmetric(n, density, 1, 10, seed, tag=11)
    return D, F


def dense_instance(n: int, seed: int):
    """Dense D and F, off-diagonal entries uniform in 0..99."""
    D = dense_symmetric(n, 0, 99, seed, tag=21)
    F = dense_symmetric(n, 0, 99, seed, tag=31)
    return D, F


def ragged_size(k: int, seed: int, lo: int = 12, hi: int = 256) -> int:
    """Size of the k-th instance of a ragged batch: uniform in lo..hi."""
    return int(hash_int(seed, 41, np.uint64(k), lo, hi))


def ragged_instance(k: int, n: int, seed: int):
    """The k-th instance of a ragged batch. Even k: grid-Manhattan D on the
    smallest near-square grid (first n cells row-major) with a 30% dense flow in
    1..10; odd k: dense uniform 0..99. `seed` keys the values."""
    if k % 2 == 0:
        rows, cols = near_square_grid(n)
        D = grid_manhattan(rows, cols, n)
        F = sparse_symmetric(n, 0.3, 1, 10, seed ^ (k * 0x9E37), tag=51)
        return D, F
    D = dense_symmetric(n, 0, 99, seed ^ (k * 0x9E37), tag=61)
    F = dense_symmetric(n, 0, 99, seed ^ (k * 0x9E37), tag=71)
    return D, F


def named(name: str, seed: int = 0):
    """The named single-instance workloads:
    'n12'  : 3x4 grid, flow density 0.5 (with 'n9', its 3x3 brute-force sibling)
    'n30'  : 5x6 grid, flow density 0.4
    'n100' : dense 0..99
    'n100a': the general-form analogue of 'n100': every entry of D and F
             drawn independently, uniform 0..99, zero diagonals (asymmetric)
    'n256' : dense 0..99 at N = 256, the largest size (tables in global memory)
    'c256' : two-level flow at the size of the paper's tai256c: N = 256, flow
             1 between every pair of a 92-facility subset and 0 elsewhere, D
             dense symmetric uniform 1..99 (synthetic values)
    """
    if name == "n12":
        return grid_instance(3, 4, 0.5, seed)
    if name == "n9":
        return grid_instance(3, 3, 0.5, seed)
    if name == "n30":
        return grid_instance(5, 6, 0.4, seed)
    if name == "n100":
        return dense_instance(100, seed)
    if name == "n100a":
        return asymmetric(100, 0, 99, seed, 101), asymmetric(100, 0, 99, seed, 103)
    if name == "c256":
        return flow_class_instance(256, 92, seed)
    if name == "n256":
        return dense_instance(256, seed)
    raise KeyError(name)


def random_symmetric(n: int, lo: int, hi: int, seed: int, tag: int, diag: bool = False) -> np.ndarray:
    """Symmetric matrix with entries uniform in lo..hi (may be negative); the
    diagonal is zero unless `diag`. Used for edge-case tests."""
    m = dense_symmetric(n, lo, hi, seed, tag).astype(np.int64)
    if diag:
        m[np.arange(n), np.arange(n)] = hash_int(seed, tag + 7, np.arange(n, dtype=np.uint64), lo, hi)
    return m.astype(np.int32)


def asymmetric(n: int, lo: int, hi: int, seed: int, tag: int, diag: bool = False) -> np.ndarray:
    """n x n matrix with every entry drawn independently, uniform in lo..hi (no
    symmetry); the diagonal is zero unless `diag`."""
    M = hash_int(seed, tag, np.arange(n * n, dtype=np.uint64), lo, hi).reshape(n, n)
    if not diag:
        M[np.arange(n), np.arange(n)] = 0
    return M.astype(np.int32)


def asymmetric_instance(n: int, seed: int, diag: bool = False):
    """The general-QAP workload: directed distances (grid-Manhattan plus a
    one-way surcharge 0..9 per ordered pair) and a dense asymmetric flow in
    0..99; `diag` adds a nonzero diagonal to both."""
    rows, cols = near_square_grid(n)
    D = grid_manhattan(rows, cols, n).astype(np.int64) + asymmetric(n, 0, 9, seed, 91)
    F = asymmetric(n, 0, 99, seed, 95, diag)
    if diag:
        D[np.arange(n), np.arange(n)] = hash_int(seed, 93, np.arange(n, dtype=np.uint64), 1, 9)
    else:
        D[np.arange(n), np.arange(n)] = 0
    return D.astype(np.int32), F


def flow_class_instance(n: int, k: int, seed: int, lo: int = 1, hi: int = 99, f0: int = 0, f: int = 1,
                        fdiag: int = 0):
    """A two-level-flow instance (the structure of the paper's tai256c
    discussion, synthetic values): D dense symmetric, off-diagonal uniform
    lo..hi, zero diagonal; a subset K of k facilities (the k smallest hashes of
    the facility ids, so not the first k); F[c][d] = f0 + f when c and d are
    both in K, f0 otherwise (c != d), and fdiag on the diagonal."""
    D = dense_symmetric(n, lo, hi, seed, tag=111)
    order = np.argsort(hash_u64(seed, 113, np.arange(n, dtype=np.uint64)), kind="stable")
    x = np.zeros(n, dtype=np.int64)
    x[order[:k]] = 1
    F = f0 + f * np.outer(x, x)
    F[np.arange(n), np.arange(n)] = fdiag
    return D, F.astype(np.int32)


def request_instance(request_id: int, lo: int = 20, hi: int = 200):
    """The instance of a serving request: N uniform in lo..hi from the request
    id, then the ragged-batch generator keyed by the request id."""
    n = int(hash_int(request_id, 81, np.uint64(0), lo, hi))
    return ragged_instance(request_id, n, request_id)
