"""The QAPLIB text-layout reader and solution reader/writer of libpdit (host
code, no GPU). Files are written here from the seeded generators; no QAPLIB
instance is reproduced."""

import numpy as np
import pytest

import oracle as O
from paper_2605_24408_gb300 import instances as G
from paper_2605_24408_gb300 import pdit as P


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_24408_gb300 import build as B

    B.build()


def _write_instance(path, A, B, wrap=7, blank=True):
    """The layout: n, blank line, A, blank line, B; rows wrapped every `wrap` values."""
    n = A.shape[0]
    lines = [" %d" % n]
    for M in (A, B):
        if blank:
            lines.append("")
        for row in M:
            vals = ["%d" % v for v in row]
            for k in range(0, n, wrap):
                lines.append("  ".join(vals[k:k + wrap]))
    path.write_text("\n".join(lines) + "\n")


@pytest.mark.parametrize("n,asym", [(2, False), (12, False), (31, True), (100, True), (256, False)])
def test_read_round_trips_generated_instances(tmp_path, n, asym):
    A, B = G.asymmetric_instance(n, seed=n) if asym else G.dense_instance(n, seed=n)
    f = tmp_path / "inst.dat"
    _write_instance(f, A, B, wrap=7 if n > 7 else n)
    D, F = P.read_qaplib(str(f))
    assert np.array_equal(D, A) and np.array_equal(F, B)


def test_read_accepts_negative_values_tabs_and_no_trailing_newline(tmp_path):
    A = G.random_symmetric(5, -2000000000, 2000000000, seed=1, tag=2, diag=True)
    B = G.asymmetric(5, -9, 9, seed=3, tag=4)
    text = "5\t" + " ".join(str(v) for v in A.ravel()) + "\r\n" + "\t".join(str(v) for v in B.ravel())
    f = tmp_path / "t.dat"
    f.write_text(text)
    D, F = P.read_qaplib(str(f))
    assert np.array_equal(D, A) and np.array_equal(F, B)


@pytest.mark.parametrize("text", ["", "1\n0\n0\n", "257\n", "3\n1 2 3\n", "2\n1 2 3 4\n5 6 7 x\n",
                                  "2\n1 2 3 4\n5 6 7 8\n9\n", "2\n1 2 3 4 5 6 7 2147483648\n",
                                  "2\n1.5 2 3 4 5 6 7 8\n", "2\n1 2 3 4 5 6 7 -2147483649\n"])
def test_read_rejects_malformed_files(tmp_path, text):
    f = tmp_path / "bad.dat"
    f.write_text(text)
    with pytest.raises(P.PditError) as e:
        P.read_qaplib(str(f))
    assert e.value.code == P.PDIT_EINVAL


def test_read_errors_for_missing_file_and_small_buffers(tmp_path):
    with pytest.raises(P.PditError) as e:
        P.read_qaplib(str(tmp_path / "missing.dat"))
    assert e.value.code == P.PDIT_EIO
    A, B = G.dense_instance(6, seed=2)
    f = tmp_path / "i.dat"
    _write_instance(f, A, B)
    import ctypes

    L = P.lib()
    n = ctypes.c_int(0)
    small = np.zeros(35, np.int32)
    assert L.pdit_read_qaplib(str(f).encode(), ctypes.byref(n), small.ctypes.data, small.ctypes.data,
                              35) == P.PDIT_ENOMEM
    assert L.pdit_read_qaplib(str(f).encode(), ctypes.byref(n), small.ctypes.data, None, 36) == P.PDIT_EINVAL
    assert L.pdit_read_qaplib(None, ctypes.byref(n), None, None, 0) == P.PDIT_EINVAL
    assert L.pdit_read_qaplib(str(f).encode(), ctypes.byref(n), None, None, 0) == P.PDIT_OK and n.value == 6


def test_solution_write_read_round_trip_and_cost(tmp_path):
    opt, perm, _ = O.brute_force(*G.named("n9"))
    D9, F9 = G.named("n9")
    f = tmp_path / "n9.sln"
    P.write_qaplib_solution(str(f), perm, opt)
    first = f.read_text().split("\n")[0].split()
    assert first == ["9", str(opt)]
    assert sorted(int(t) for t in f.read_text().split()[2:]) == list(range(1, 10))  # 1-based
    cost, p = P.read_qaplib_solution(str(f))
    assert cost == opt and np.array_equal(p, perm)
    assert O.cost(D9, F9, p) == cost


@pytest.mark.parametrize("text", ["3 10\n1 2 2\n", "3 10\n1 2\n", "3 10\n0 1 2\n", "3 10\n1 2 4\n",
                                  "3 10\n1 2 3 4\n", "3 x\n1 2 3\n"])
def test_solution_reader_rejects_malformed(tmp_path, text):
    f = tmp_path / "bad.sln"
    f.write_text(text)
    with pytest.raises(P.PditError) as e:
        P.read_qaplib_solution(str(f))
    assert e.value.code == P.PDIT_EINVAL


def test_solution_writer_rejects_non_permutations(tmp_path):
    with pytest.raises(P.PditError):
        P.write_qaplib_solution(str(tmp_path / "x.sln"), [0, 0, 1], 5)
    with pytest.raises(P.PditError):
        P.write_qaplib_solution(str(tmp_path / "x.sln"), [0, 1, 3], 5)
    with pytest.raises(P.PditError) as e:
        P.write_qaplib_solution(str(tmp_path / "no_such_dir" / "x.sln"), [0, 1, 2], 5)
    assert e.value.code == P.PDIT_EIO
