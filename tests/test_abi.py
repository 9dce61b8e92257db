"""The C-ABI library loads, exports every function include/pdit.h declares,
and its host-only logic (argument checks, beta schedules) behaves. No GPU."""

import ctypes
import os

import numpy as np
import pytest

import oracle as O
from paper_2605_24408_gb300 import build as B
from paper_2605_24408_gb300 import instances as G
from paper_2605_24408_gb300 import pdit as P


@pytest.fixture(scope="module")
def L():
    B.build()
    return P.lib()


def test_exports_every_declared_symbol(L):
    names = P.header_functions()
    assert {"qap_create", "qap_destroy", "pdit_anneal", "pdit_anneal_ex", "pdit_strerror"} <= set(names)
    for name in names:
        assert hasattr(L, name), name


def test_strerror_and_opts_defaults(L):
    for code in [0, -1, -2, -3, -4, -5, -6]:
        assert P.strerror(code)
    assert P.strerror(-99) == "unknown error"
    o = P.opts()
    assert o.struct_size == ctypes.sizeof(P.pdit_opts)
    assert o.sweep_end == -1 and o.exchange_period == 4 and o.timeout_periods == 100
    assert o.mode == P.PDIT_MODE_ANNEAL


def test_qap_create_rejects_bad_instances_before_touching_the_gpu(L):
    D, F = G.named("n12")
    h = ctypes.c_void_p()
    D32, F32 = np.ascontiguousarray(D, np.int32), np.ascontiguousarray(F, np.int32)
    # size out of range
    assert L.qap_create(1, D32.ctypes.data, F32.ctypes.data, ctypes.byref(h)) == P.PDIT_EINVAL
    assert L.qap_create(P.PDIT_N_MAX + 1, D32.ctypes.data, F32.ctypes.data, ctypes.byref(h)) == P.PDIT_EINVAL
    assert h.value is None
    # NULL
    assert L.qap_create(12, None, F32.ctypes.data, ctypes.byref(h)) == P.PDIT_EINVAL
    # int32 overflow risk: 16 (n+2) maxD maxF >= 2^31, symmetric or not (the
    # general form's two-term table obeys the same bound)
    big = np.full((12, 12), 4000, np.int32)
    np.fill_diagonal(big, 0)
    assert L.qap_create(12, big.ctypes.data, big.ctypes.data, ctypes.byref(h)) == P.PDIT_ERANGE
    bigA = big.copy()
    bigA[0, 1] += 1
    assert L.qap_create(12, bigA.ctypes.data, big.ctypes.data, ctypes.byref(h)) == P.PDIT_ERANGE
    assert h.value is None
    L.qap_destroy(None)


def test_beta_schedule_matches_oracle(L):
    for kind in ["linear", "geometric"]:
        for S in [1, 2, 7, 1000]:
            got = P.pdit_beta_schedule(kind, S, 0.37)
            want = O.beta_schedule(kind, S, 0.37)
            assert np.array_equal(got, want)
    with pytest.raises(P.PditError):
        P.pdit_beta_schedule("linear", -1, 1.0)
    out = np.zeros(3, np.float32)
    assert L.pdit_beta_schedule(0, 3, float("nan"), out.ctypes.data) == P.PDIT_EINVAL


def test_workspace_and_anneal_reject_null_handle(L):
    o = P.opts(replicas=4, sweeps=1)
    assert L.pdit_workspace_bytes(None, ctypes.byref(o)) == 0
    assert L.pdit_anneal_ex(None, ctypes.byref(o)) == P.PDIT_EINVAL
    assert L.pdit_anneal(None, 4, None, 0, 0, None, None) == P.PDIT_EINVAL
    assert L.qap_n(None) == P.PDIT_EINVAL


def test_beta_ladder_is_multiplicative(L):
    lad = P.pdit_beta_ladder(0.01, 1.0, 10)
    want = np.float32([0.01 * (100.0 ** (q / 9)) for q in range(10)])
    assert np.array_equal(lad, want)
    with pytest.raises(P.PditError):
        P.pdit_beta_ladder(0.0, 1.0, 10)
    with pytest.raises(P.PditError):
        P.pdit_beta_ladder(1.0, 0.5, 10)


def test_header_compiles_as_c99_and_links(tmp_path, L):
    """include/pdit.h is a plain C header: a C99 program that takes the
    address of every declared function compiles and links against
    libpdit.so (it is not run: there may be no GPU)."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    names = P.header_functions()
    src = tmp_path / "use_header.c"
    body = "\n".join("    (void)&%s;" % n for n in names)
    src.write_text('#include "pdit.h"\n#include <stdio.h>\nint main(void) {\n%s\n'
                   '    printf("%%s\\n", pdit_strerror(PDIT_OK));\n    return 0;\n}\n' % body)
    inc = os.path.join(os.path.dirname(P.HEADER))
    libdir = os.path.dirname(P.LIB_PATH)
    out = tmp_path / "use_header"
    cmd = [gcc, "-std=c99", "-Wall", "-Werror", "-I", inc, str(src), "-o", str(out), "-L", libdir, "-lpdit",
           "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_binding_constants_match_the_header():
    """Every PDIT_* constant of the Python binding has the value the C header
    defines (the header is the ABI; the binding restates it)."""
    import re

    from paper_2605_24408_gb300 import pdit

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "include", "pdit.h")) as fh:
        text = fh.read()
    defs = {}
    for name, value in re.findall(r"^#define\s+(PDIT_[A-Z0-9_]+)\s+\(?(-?[0-9]+)u?\)?", text, re.M):
        defs[name] = int(value)
    names = [n for n in dir(pdit) if re.fullmatch(r"PDIT_[A-Z0-9_]+", n) and isinstance(getattr(pdit, n), int)]
    assert len(names) >= 20
    for n in names:
        assert n in defs, n
        assert getattr(pdit, n) == defs[n], n
