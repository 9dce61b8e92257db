"""The bytes-per-update figures behind the bench line's roofline fractions,
against hand-worked values (no GPU)."""

import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_method_bytes_per_update():
    # 4 (4 N) gathers + A (8 N^2 + 8 N): N = 100, A = 0.5 -> 1600 + 0.5 * 80800
    assert bench.method_bytes_per_update(100, 0.5) == pytest.approx(1600 + 40400)
    # general form: four factor vectors, 16 N per accepted swap
    assert bench.method_bytes_per_update(100, 0.5, general=True) == pytest.approx(1600 + 0.5 * 81600)
    assert bench.method_bytes_per_update(256, 0.0) == 16 * 256


def test_design_bytes_per_update():
    n, dt, a = 100, 1, 0.25
    # immediate: gather 16 N + 2 N dt; swap 8 N^2 + 4 N dt + 12 N
    assert bench.algorithmic_bytes_per_update(n, dt, a, 1) == pytest.approx(
        1600 + 200 + a * (80000 + 400 + 1200))
    # 4 pending terms (one packed word): gather 16 N + 8 N + 2 N dt;
    # swap 8 N^2 / 4 + 4 N dt + 16 N
    assert bench.algorithmic_bytes_per_update(n, dt, a, 4) == pytest.approx(
        1600 + 800 + 200 + a * (20000 + 400 + 1600))
    # 16 pending terms (four packed words)
    assert bench.algorithmic_bytes_per_update(n, dt, a, 16) == pytest.approx(
        1600 + 3200 + 200 + a * (5000 + 400 + 1600))


def test_flow_class_bytes_per_update():
    # (17 + dt) N + A (2 N dt + 8 N)
    assert bench.class_bytes_per_update(256, 1, 1.0) == pytest.approx(18 * 256 + 2 * 256 + 8 * 256)


def test_shared_memory_peak_derivation():
    # 152 SMs x 128 B/clk x 2070 MHz = 40.27 TB/s
    assert 152 * bench.SMEM_BYTES_PER_CLK * 2070e6 / 1e9 == pytest.approx(40273.92)


def test_product_bytes_and_dp4a_per_update():
    # N = 100: row stride 112 (16 x 7); 2 N S + 2 S + 2 N + 4 + A (12 N + 4 S + 16)
    assert bench.product_stride(100) == 112
    assert bench.product_stride(96) == 112   # 6 units -> 7
    assert bench.product_stride(256) == 272  # 16 units -> 17
    assert bench.product_stride(12) == 16
    assert bench.product_bytes_per_update(100, 0.5) == pytest.approx(
        22400 + 224 + 200 + 4 + 0.5 * (1200 + 448 + 16))
    # two dot products of 28 words per candidate
    assert bench.product_dp4a_per_update(100) == 2 * 100 * 28


def test_ragged_targets_respect_the_brute_force_optima():
    """The ragged benchmark's stored reference-run bests can be no lower than
    the brute-force optimum of the same instance (N <= 12), and the bench
    reads those optima as the targets of those sizes."""
    import json

    opt = bench.ragged_optima()
    assert opt, "tests/golden/ragged_optima.txt missing"
    with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                           "bench_targets", "ragged.json")) as fh:
        tr = {t["k"]: t for t in json.load(fh)["targets"]}
    for k, c in opt.items():
        assert tr[k]["n"] <= 12
        assert tr[k]["best"] >= c


def test_dot_kernel_name_follows_the_compiled_strides():
    assert bench.dot_kernel_name(4, 1, 100) == "dot_kernel<4,1,7,0>"
    assert bench.dot_kernel_name(4, 1, 97, parts=16) == "dot_kernel<4,1,7,1>"
    assert bench.dot_kernel_name(4, 1, 113) == "dot_kernel<4,1,0,0>"
    assert bench.dot_kernel_name(2, 1, 60) == "dot_kernel<2,1,0,0>"
    assert bench.dot_kernel_name(1, 8, 256) == "dot_kernel<1,8,0,0>"


def test_dot_parts_rule():
    # n100: 4096 replicas in 2432 slots, 10000 sweeps -> 16 parts
    assert bench.dot_parts(4096, 2432, 10000) == 16
    assert bench.dot_parts(4096, 2432, 20) == 2      # parts of at least 8 sweeps
    assert bench.dot_parts(4096, 2432, 7) == 1
    assert bench.dot_parts(2432, 2432, 10000) == 1   # one whole round
    assert bench.dot_parts(4864, 2432, 10000) == 1   # two whole rounds
    assert bench.dot_parts(100, 2432, 10000) == 1
    assert bench.dot_parts(4090, 2432, 4, pt=True) == 4  # one exchange period, parts of one sweep
    assert bench.dot_parts(4096, 2432, 100000) == 100    # parts of at most 1000 sweeps
